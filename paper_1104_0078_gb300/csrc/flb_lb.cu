// flb_lb.cu -- D2Q9 fused pull-stream + moment-space collision of the fluctuating
// lattice Boltzmann equation (Sec. IV and App. B of arXiv:1104.0078) with the
// order-parameter force F = -psi grad mu (Sec. IV) applied inside the kernel.
//
// Storage: populations are SoA planes [q][N] holding the POST-collision
// deviations fbar*_i - w_i rho0 at their origin site (not yet streamed).  A step
// pulls fbar_i(r, t) = stored_i(r - c_i), relaxes at r and stores the new
// post-collision values at r into the other buffer.
//
// Collision, written per opposite pair (c, -c) of velocities: with
// s = fbar_c + fbar_-c and d = fbar_c - fbar_-c the hydrodynamic moments are
// sums of s (mass, stress) and d (momentum).  Post-collision
//   fbar*_i = w_i [ rho + 3 A.c_i + 9/2 B:Q_i + sum_ghost e_k(c_i) g_k ],
//   A = j + F,  B = S + omega_s dev(X) + omega_b iso(X) + (1 - omega_s/2) dev(T)
//       + (1 - omega_b/2) iso(T) + (stress noise),  X = -S + rho v v,
//   T = v F + F v,  v = (j + F/2)/rho                              (Eq. bab)
// and every stress and ghost mode k receives sqrt(mu_n b_k (1 - gamma_k^2)) g_k,
// mu_n = rho kT / c_s^2 (thermalisation of all modes, Sec. III / adhikari2005).
// The ghost vectors e_k are the w-orthogonal (Gram-Schmidt) completions of the
// monomials c^2 c_a, c_a(c_b^2 - c_g^2), c^4, c^2(3c_x^2 - c^2), c^2(c_y^2 - c_z^2)
// (D3Q19, in flb_lb3d.cu) and c^2 c_a, c^4 (D2Q9), written out below per
// velocity pair.  The D3Q19 kernel and the equilibrium initialiser share this
// storage convention.
#include "flb_internal.cuh"

namespace flb {

template <typename T>
__device__ __forceinline__ float ldpop(const T *p, long long i);
template <>
__device__ __forceinline__ float ldpop<float>(const float *p, long long i) { return __ldg(p + i); }
template <>
__device__ __forceinline__ float ldpop<__half>(const __half *p, long long i) { return __half2float(p[i]); }

template <typename T>
__device__ __forceinline__ void stpop(T *p, long long i, float v);
template <>
__device__ __forceinline__ void stpop<float>(float *p, long long i, float v) { p[i] = v; }
template <>
__device__ __forceinline__ void stpop<__half>(__half *p, long long i, float v) { p[i] = __float2half_rn(v); }

// Pull of the 9 populations of site (x, y) from the stored post-collision
// planes: fbar_i(r) = stored_i(r - c_i).
template <typename T>
__device__ __forceinline__ void pull9(const T *fi, const Geom &g, int x, int y, float f[9])
{
    const int xm = x == 0 ? g.nx - 1 : x - 1, xp = x == g.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
    const long long N = g.n;
    f[0] = ldpop(fi, g.sidx(x, y, 0));
    f[1] = ldpop(fi, 1 * N + g.sidx(xm, y, 0));
    f[2] = ldpop(fi, 2 * N + g.sidx(xp, y, 0));
    f[3] = ldpop(fi, 3 * N + g.sidx(x, ym, 0));
    f[4] = ldpop(fi, 4 * N + g.sidx(x, yp, 0));
    f[5] = ldpop(fi, 5 * N + g.sidx(xm, ym, 0));
    f[6] = ldpop(fi, 6 * N + g.sidx(xp, yp, 0));
    f[7] = ldpop(fi, 7 * N + g.sidx(xm, yp, 0));
    f[8] = ldpop(fi, 8 * N + g.sidx(xp, ym, 0));
}

// Force density at (x, y): F = -psi grad mu with the central difference, or for
// the FV psi scheme the FV gradient (1/c_s^2) sum_i w_i c_i mu(r + c_i) of
// Eq. (fvgrad) = [4 (mu(+x) - mu(-x)) + diagonals] / 12 for D2Q9; or
// F = -div sigma (stress form).
__device__ __forceinline__ void force2(const LBArgs &a, int x, int y, float &Fx, float &Fy)
{
    const Geom &g = a.g;
    if (a.force_kind == 2) {  // F = -div sigma (stress form), sigma planes xx, yy, xy
        const float *xx = a.sig, *yy = xx + g.pn, *xy = yy + g.pn;
        Fx = -0.5f * ((xx[g.pidx(x + 1, y, 0)] - xx[g.pidx(x - 1, y, 0)]) + (xy[g.pidx(x, y + 1, 0)] - xy[g.pidx(x, y - 1, 0)]));
        Fy = -0.5f * ((xy[g.pidx(x + 1, y, 0)] - xy[g.pidx(x - 1, y, 0)]) + (yy[g.pidx(x, y + 1, 0)] - yy[g.pidx(x, y - 1, 0)]));
        return;
    }
    const float ps = a.psi[g.pidx(x, y, 0)];
    const float *mu = a.mu;
    const float dx = mu[g.pidx(x + 1, y, 0)] - mu[g.pidx(x - 1, y, 0)];
    const float dy = mu[g.pidx(x, y + 1, 0)] - mu[g.pidx(x, y - 1, 0)];
    if (a.force_kind == 1) {
        const float pp = mu[g.pidx(x + 1, y + 1, 0)], pm = mu[g.pidx(x + 1, y - 1, 0)];
        const float mp = mu[g.pidx(x - 1, y + 1, 0)], mm = mu[g.pidx(x - 1, y - 1, 0)];
        Fx = -ps * (1.0f / 12.0f) * (4.f * dx + ((pp + pm) - (mp + mm)));
        Fy = -ps * (1.0f / 12.0f) * (4.f * dy + ((pp - pm) + (mp - mm)));
    } else {
        Fx = -ps * 0.5f * dx;
        Fy = -ps * 0.5f * dy;
    }
}

// ---------------------------------------------------------------------------
// D2Q9.  Plane order: 0 rest; (1,2) +-x, (3,4) +-y, (5,6) +-(1,1), (7,8) +-(1,-1).
// Noise order: bulk c^2 - 2/3, c_x^2 - c_y^2, c_x c_y, c_x(c^2 - 4/3),
// c_y(c^2 - 4/3), c^4-type ghost (2/9, -4/9 axes, 8/9 diagonals).
// ---------------------------------------------------------------------------
template <typename T, bool GHOST_RELAX>
__global__ void __launch_bounds__(256) lb_d2q9_kernel(const LBArgs a)
{
    const Geom &g = a.g;
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= g.n) return;
    const int x = (int)(site % g.nx);
    const int y = (int)(site / g.nx);
    const T *fin = (const T *)a.fin;
    T *fout = (T *)a.fout;
    const long long N = g.n;

    float f[9];
    pull9(fin, g, x, y, f);
    float s[5], d[5];
#pragma unroll
    for (int p = 1; p <= 4; ++p) {
        s[p] = f[2 * p - 1] + f[2 * p];
        d[p] = f[2 * p - 1] - f[2 * p];
    }
    const float drho = f[0] + ((s[1] + s[2]) + (s[3] + s[4]));
    const float jx = d[1] + (d[3] + d[4]);
    const float jy = d[2] + (d[3] - d[4]);
    const float third = drho * (1.0f / 3.0f);
    const float Sxx = s[1] + (s[3] + s[4]) - third;
    const float Syy = s[2] + (s[3] + s[4]) - third;
    const float Sxy = s[3] - s[4];

    float Fx = 0.f, Fy = 0.f;
    if (a.coupling & FLB_COUPLE_FORCE) force2(a, x, y, Fx, Fy);
    const float rho = a.rho0 + drho;
    const float irho = 1.0f / rho;
    const float vx = (jx + 0.5f * Fx) * irho, vy = (jy + 0.5f * Fy) * irho;

    const float ws = a.omega_s, wb = a.omega_b;
    const float cs = 1.0f - 0.5f * ws, cb = 1.0f - 0.5f * wb;
    const float Xxx = rho * vx * vx - Sxx, Xyy = rho * vy * vy - Syy;
    const float trX2 = 0.5f * (Xxx + Xyy);
    const float Txx = 2.f * vx * Fx, Tyy = 2.f * vy * Fy;
    const float trT2 = 0.5f * (Txx + Tyy);
    const float isoB = (wb - ws) * trX2 + (cb - cs) * trT2;
    float Bxx = Sxx + ws * Xxx + cs * Txx + isoB;
    float Byy = Syy + ws * Xyy + cs * Tyy + isoB;
    float Bxy = Sxy + ws * (rho * vx * vy - Sxy) + cs * (vx * Fy + Fx * vy);
    const float Ax = jx + Fx, Ay = jy + Fy;

    float g6 = 0.f, g7 = 0.f, g8 = 0.f;
    if (GHOST_RELAX) {
        const float gg = a.gamma_g;
        const float m6 = -(1.f / 3.f) * d[1] + (2.f / 3.f) * (d[3] + d[4]);
        const float m7 = -(1.f / 3.f) * d[2] + (2.f / 3.f) * (d[3] - d[4]);
        const float m8 = (2.f / 9.f) * f[0] - (4.f / 9.f) * (s[1] + s[2]) + (8.f / 9.f) * (s[3] + s[4]);
        g6 = gg * m6 * 13.5f;          // 1/b = 27/2
        g7 = gg * m7 * 13.5f;
        g8 = gg * m8 * (81.f / 16.f);  // 1/b = 81/16
    }
    if (a.kT > 0.f) {
        float G[6];
        normals<3>(a.key, a.step, (uint32_t)site, 0u, 0u, G);
        const float sq = sqrtf(3.0f * rho * a.kT);
        float n[6];
#pragma unroll
        for (int t = 0; t < 6; ++t) n[t] = sq * a.namp[t] * G[t];
        const float two9 = 2.0f / 9.0f;
        Bxx += two9 * (n[0] + n[1]);
        Byy += two9 * (n[0] - n[1]);
        Bxy += (1.0f / 9.0f) * n[2];
        g6 += n[3];
        g7 += n[4];
        g8 += n[5];
    }
    const float e0 = 1.5f * (Bxx + Byy);  // 9/2 trB/3
    stpop(fout, site, (4.f / 9.f) * (drho - e0 + (2.f / 9.f) * g8));
    const float w1 = 1.f / 9.f, w2 = 1.f / 36.f;
    float E, O;
    E = drho + 4.5f * Bxx - e0 - (4.f / 9.f) * g8;
    O = 3.f * Ax - (1.f / 3.f) * g6;
    stpop(fout, 1 * N + site, w1 * (E + O));
    stpop(fout, 2 * N + site, w1 * (E - O));
    E = drho + 4.5f * Byy - e0 - (4.f / 9.f) * g8;
    O = 3.f * Ay - (1.f / 3.f) * g7;
    stpop(fout, 3 * N + site, w1 * (E + O));
    stpop(fout, 4 * N + site, w1 * (E - O));
    E = drho + 4.5f * (Bxx + Byy + 2.f * Bxy) - e0 + (8.f / 9.f) * g8;
    O = 3.f * (Ax + Ay) + (2.f / 3.f) * (g6 + g7);
    stpop(fout, 5 * N + site, w2 * (E + O));
    stpop(fout, 6 * N + site, w2 * (E - O));
    E = drho + 4.5f * (Bxx + Byy - 2.f * Bxy) - e0 + (8.f / 9.f) * g8;
    O = 3.f * (Ax - Ay) + (2.f / 3.f) * (g6 - g7);
    stpop(fout, 7 * N + site, w2 * (E + O));
    stpop(fout, 8 * N + site, w2 * (E - O));
}

// Second-order equilibrium fbar = w rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2) of a
// given (rho, u) field, stored as post-collision deviations at the origin site:
// stored_i(r) = fbar_i(r + c_i) - w_i rho0.  rho and u are padded planes (rho may be null).
__constant__ int8_t kEq19[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                    {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                    {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
__constant__ int8_t kEq15[15][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},
                                    {0, 0, 1},  {0, 0, -1}, {1, 1, 1},   {-1, -1, -1}, {1, 1, -1},
                                    {-1, -1, 1}, {1, -1, 1}, {-1, 1, -1}, {1, -1, -1}, {-1, 1, 1}};
__constant__ int8_t kEq9[9][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                                  {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};

// Velocity of the streamed state after a D2Q9 step: u = (sum fbar c + F/2)/rho
// with fbar the populations the next step pulls (the just-written planes) and F
// the force density of this step -- the velocity that advects psi
// (Gauss-Seidel coupling of Sec. VI: the psi step follows the fluid step).
template <typename T>
__global__ void __launch_bounds__(256) vel_d2q9_kernel(const LBArgs a)
{
    const Geom &g = a.g;
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= g.n) return;
    const int x = (int)(site % g.nx);
    const int y = (int)(site / g.nx);
    float f[9];
    pull9((const T *)a.fout, g, x, y, f);
    const float drho = f[0] + (((f[1] + f[2]) + (f[3] + f[4])) + ((f[5] + f[6]) + (f[7] + f[8])));
    // planes (5,6) +-(1,1), (7,8) +-(1,-1)
    const float jx = (f[1] - f[2]) + ((f[5] - f[6]) + (f[7] - f[8]));
    const float jy = (f[3] - f[4]) + ((f[5] - f[6]) - (f[7] - f[8]));
    float Fx = 0.f, Fy = 0.f;
    if (a.coupling & FLB_COUPLE_FORCE) force2(a, x, y, Fx, Fy);
    const float irho = 1.0f / (a.rho0 + drho);
    store_padded(a.u, g, x, y, 0, (jx + 0.5f * Fx) * irho, 1);
    store_padded(a.u + g.pn, g, x, y, 0, (jy + 0.5f * Fy) * irho, 1);
}

template <typename T>
__global__ void init_eq_kernel(const Geom g, int q, const float *__restrict__ rho, const float *__restrict__ u,
                               float rho0, T *__restrict__ fout)
{
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= g.n) return;
    const int x = (int)(site % g.nx);
    const int y = (int)((site / g.nx) % g.ny);
    const int z = (int)(site / ((long long)g.nx * g.ny));
    for (int i = 0; i < q; ++i) {
        const int8_t *c = q == 19 ? kEq19[i] : q == 15 ? kEq15[i] : kEq9[i];
        const long long pi = g.pidx(x + c[0], y + c[1], z + c[2]);
        const float r = rho ? rho[pi] : rho0;
        const float ux = u[pi], uy = u[g.pn + pi], uz = g.dim == 3 ? u[2 * g.pn + pi] : 0.f;
        const float cu = c[0] * ux + c[1] * uy + c[2] * uz;
        const float u2 = ux * ux + uy * uy + uz * uz;
        const float l2 = (float)(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        const float w = q == 19   ? (l2 == 0.f ? 1.f / 3.f : l2 == 1.f ? 1.f / 18.f : 1.f / 36.f)
                        : q == 15 ? (l2 == 0.f ? 2.f / 9.f : l2 == 1.f ? 1.f / 9.f : 1.f / 72.f)
                                  : (l2 == 0.f ? 4.f / 9.f : l2 == 1.f ? 1.f / 9.f : 1.f / 36.f);
        stpop(fout, (long long)i * g.n + site, w * ((r - rho0) + r * (3.f * cu + 4.5f * cu * cu - 1.5f * u2)));
    }
}

// Padded plane (every ghost column, row and plane included) from an interior
// field [N], x fastest: each padded cell takes its periodic image.
__global__ void pad_kernel(const Geom g, const float *__restrict__ in, float *__restrict__ out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.pn) return;
    const int xp = (int)(i % g.px), yp = (int)((i / g.px) % g.py), zp = (int)(i / ((long long)g.px * g.py));
    const int x = ((xp - GX) % g.nx + g.nx) % g.nx, y = ((yp - GY) % g.ny + g.ny) % g.ny;
    const int z = g.dim == 3 ? ((zp - g.gz) % g.nz + g.nz) % g.nz : 0;
    out[i] = in[x + (long long)g.nx * (y + (long long)g.ny * z)];
}

// the interior of a padded field, site-major (the inverse of pad_kernel's copy)
__global__ void unpad_kernel(const Geom g, const float *__restrict__ padded, float *__restrict__ out)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.n) return;
    const int x = (int)(s % g.nx), y = (int)((s / g.nx) % g.ny), z = (int)(s / ((long long)g.nx * g.ny));
    out[s] = padded[g.pidx(x, y, z)];
}

cudaError_t launch_unpad(const Geom &g, const float *padded, float *interior, cudaStream_t st)
{
    unpad_kernel<<<(unsigned)((g.n + 255) / 256), 256, 0, st>>>(g, padded, interior);
    return cudaGetLastError();
}

cudaError_t launch_pad(const Geom &g, const float *interior, float *padded, cudaStream_t st)
{
    pad_kernel<<<(unsigned)((g.pn + 255) / 256), 256, 0, st>>>(g, interior, padded);
    return cudaGetLastError();
}

cudaError_t launch_init_eq(const Geom &g, int q, int storage, const float *rho, const float *u, float rho0, void *f,
                           cudaStream_t st)
{
    const unsigned grid = (unsigned)((g.n + 255) / 256);
    if (storage == FLB_F16_DEV) init_eq_kernel<__half><<<grid, 256, 0, st>>>(g, q, rho, u, rho0, (__half *)f);
    else init_eq_kernel<float><<<grid, 256, 0, st>>>(g, q, rho, u, rho0, (float *)f);
    return cudaGetLastError();
}

cudaError_t launch_lb(const LBArgs &a, int q, int storage, cudaStream_t st)
{
    const int bs = 256;
    const unsigned grid = (unsigned)((a.g.n + bs - 1) / bs);
    const bool gr = a.gamma_g != 0.0f;
    if (q != 9) return cudaErrorInvalidValue;  // D3Q19 runs in flb_lb3d.cu
    if (storage == FLB_F16_DEV) {
        if (gr) lb_d2q9_kernel<__half, true><<<grid, bs, 0, st>>>(a);
        else lb_d2q9_kernel<__half, false><<<grid, bs, 0, st>>>(a);
    } else {
        if (gr) lb_d2q9_kernel<float, true><<<grid, bs, 0, st>>>(a);
        else lb_d2q9_kernel<float, false><<<grid, bs, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_vel2(const LBArgs &a, int storage, cudaStream_t st)
{
    const int bs = 256;
    const unsigned grid = (unsigned)((a.g.n + bs - 1) / bs);
    if (storage == FLB_F16_DEV) vel_d2q9_kernel<__half><<<grid, bs, 0, st>>>(a);
    else vel_d2q9_kernel<float><<<grid, bs, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace flb

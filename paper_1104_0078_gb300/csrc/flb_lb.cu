// flb_lb.cu -- fused pull-stream + moment-space collision of the fluctuating
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
// (D3Q19) and c^2 c_a, c^4 (D2Q9), written out below per velocity pair.
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

// ---------------------------------------------------------------------------
// D3Q19.  Plane order: 0 rest; pairs (1,2) +-x, (3,4) +-y, (5,6) +-z,
// (7,8) +-(1,1,0), (9,10) +-(1,-1,0), (11,12) +-(1,0,1), (13,14) +-(1,0,-1),
// (15,16) +-(0,1,1), (17,18) +-(0,1,-1).
// Noise order: bulk, 3c_x^2-c^2, c_y^2-c_z^2, xy, yz, zx, three c^2 c_a ghosts,
// three c_a(c_b^2-c_g^2) ghosts, c^4, c^2(3c_x^2-c^2), c^2(c_y^2-c_z^2).
// ---------------------------------------------------------------------------
template <typename T, bool GHOST_RELAX>
__global__ void __launch_bounds__(256) lb_d3q19_kernel(const LBArgs a)
{
    const Geom &g = a.g;
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= g.n) return;
    const int x = (int)(site % g.nx);
    const int y = (int)((site / g.nx) % g.ny);
    const int z = (int)(site / ((long long)g.nx * g.ny));
    const int xm = x == 0 ? g.nx - 1 : x - 1, xp = x == g.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
    const T *fin = (const T *)a.fin;
    T *fout = (T *)a.fout;
    const long long N = g.n;

    // pull: fbar_i(r) = stored_i(r - c_i)
    float f[19];
    f[0] = ldpop(fin, site);
    f[1] = ldpop(fin, 1 * N + g.sidx(xm, y, z));
    f[2] = ldpop(fin, 2 * N + g.sidx(xp, y, z));
    f[3] = ldpop(fin, 3 * N + g.sidx(x, ym, z));
    f[4] = ldpop(fin, 4 * N + g.sidx(x, yp, z));
    f[5] = ldpop(fin, 5 * N + g.sidx(x, y, zm));
    f[6] = ldpop(fin, 6 * N + g.sidx(x, y, zp));
    f[7] = ldpop(fin, 7 * N + g.sidx(xm, ym, z));
    f[8] = ldpop(fin, 8 * N + g.sidx(xp, yp, z));
    f[9] = ldpop(fin, 9 * N + g.sidx(xm, yp, z));
    f[10] = ldpop(fin, 10 * N + g.sidx(xp, ym, z));
    f[11] = ldpop(fin, 11 * N + g.sidx(xm, y, zm));
    f[12] = ldpop(fin, 12 * N + g.sidx(xp, y, zp));
    f[13] = ldpop(fin, 13 * N + g.sidx(xm, y, zp));
    f[14] = ldpop(fin, 14 * N + g.sidx(xp, y, zm));
    f[15] = ldpop(fin, 15 * N + g.sidx(x, ym, zm));
    f[16] = ldpop(fin, 16 * N + g.sidx(x, yp, zp));
    f[17] = ldpop(fin, 17 * N + g.sidx(x, ym, zp));
    f[18] = ldpop(fin, 18 * N + g.sidx(x, yp, zm));

    float s[10], d[10];
#pragma unroll
    for (int p = 1; p <= 9; ++p) {
        s[p] = f[2 * p - 1] + f[2 * p];
        d[p] = f[2 * p - 1] - f[2 * p];
    }
    const float drho = f[0] + ((s[1] + s[2] + s[3]) + ((s[4] + s[5]) + (s[6] + s[7]) + (s[8] + s[9])));
    const float jx = d[1] + (d[4] + d[5]) + (d[6] + d[7]);
    const float jy = d[2] + (d[4] - d[5]) + (d[8] + d[9]);
    const float jz = d[3] + (d[6] - d[7]) + (d[8] - d[9]);
    const float third = drho * (1.0f / 3.0f);
    const float Sxx = s[1] + (s[4] + s[5]) + (s[6] + s[7]) - third;
    const float Syy = s[2] + (s[4] + s[5]) + (s[8] + s[9]) - third;
    const float Szz = s[3] + (s[6] + s[7]) + (s[8] + s[9]) - third;
    const float Sxy = s[4] - s[5], Sxz = s[6] - s[7], Syz = s[8] - s[9];

    // force density F = -psi grad_CD mu
    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
    if (a.coupling & FLB_COUPLE_FORCE) {
        const float ps = a.psi[g.pidx(x, y, z)];
        const float *mu = a.mu;
        Fx = -ps * 0.5f * (mu[g.pidx(x + 1, y, z)] - mu[g.pidx(x - 1, y, z)]);
        Fy = -ps * 0.5f * (mu[g.pidx(x, y + 1, z)] - mu[g.pidx(x, y - 1, z)]);
        Fz = -ps * 0.5f * (mu[g.pidx(x, y, z + 1)] - mu[g.pidx(x, y, z - 1)]);
    }
    const float rho = a.rho0 + drho;
    const float irho = 1.0f / rho;
    const float vx = (jx + 0.5f * Fx) * irho, vy = (jy + 0.5f * Fy) * irho, vz = (jz + 0.5f * Fz) * irho;
    {
        const long long pu = g.pn;
        store_padded(a.u, g, x, y, z, vx, 1);
        store_padded(a.u + pu, g, x, y, z, vy, 1);
        store_padded(a.u + 2 * pu, g, x, y, z, vz, 1);
    }

    // deterministic relaxation of the stress (Eq. bab)
    const float ws = a.omega_s, wb = a.omega_b;
    const float cs = 1.0f - 0.5f * ws, cb = 1.0f - 0.5f * wb;
    const float Xxx = rho * vx * vx - Sxx, Xyy = rho * vy * vy - Syy, Xzz = rho * vz * vz - Szz;
    const float trX3 = (Xxx + Xyy + Xzz) * (1.0f / 3.0f);
    const float Txx = 2.f * vx * Fx, Tyy = 2.f * vy * Fy, Tzz = 2.f * vz * Fz;
    const float trT3 = (Txx + Tyy + Tzz) * (1.0f / 3.0f);
    const float isoB = (wb - ws) * trX3 + (cb - cs) * trT3;
    float Bxx = Sxx + ws * Xxx + cs * Txx + isoB;
    float Byy = Syy + ws * Xyy + cs * Tyy + isoB;
    float Bzz = Szz + ws * Xzz + cs * Tzz + isoB;
    float Bxy = Sxy + ws * (rho * vx * vy - Sxy) + cs * (vx * Fy + Fx * vy);
    float Bxz = Sxz + ws * (rho * vx * vz - Sxz) + cs * (vx * Fz + Fx * vz);
    float Byz = Syz + ws * (rho * vy * vz - Syz) + cs * (vy * Fz + Fy * vz);
    const float Ax = jx + Fx, Ay = jy + Fy, Az = jz + Fz;

    // ghost coefficients g_k (post-collision ghost moment / b_k)
    float g10 = 0.f, g11 = 0.f, g12 = 0.f, g13 = 0.f, g14 = 0.f, g15 = 0.f, g16 = 0.f, g17 = 0.f, g18 = 0.f;
    if (GHOST_RELAX) {
        const float gg = a.gamma_g;
        const float m10 = (d[4] + d[5] + d[6] + d[7]) * (1.f / 3.f) - d[1] * (2.f / 3.f);
        const float m11 = (d[4] - d[5] + d[8] + d[9]) * (1.f / 3.f) - d[2] * (2.f / 3.f);
        const float m12 = (d[6] - d[7] + d[8] - d[9]) * (1.f / 3.f) - d[3] * (2.f / 3.f);
        const float m13 = d[4] + d[5] - d[6] - d[7];
        const float m14 = -d[4] + d[5] + d[8] + d[9];
        const float m15 = d[6] - d[7] - d[8] + d[9];
        const float m16 = (f[0] + s[4] + s[5] + s[6] + s[7] + s[8] + s[9]) * (1.f / 3.f) -
                          (s[1] + s[2] + s[3]) * (2.f / 3.f);
        const float m17 = -s[1] + 0.5f * (s[2] + s[3] + s[4] + s[5] + s[6] + s[7]) - (s[8] + s[9]);
        const float m18 = 0.5f * (-s[2] + s[3] + s[4] + s[5] - s[6] - s[7]);
        g10 = gg * m10 * 13.5f;  // 1/b = 27/2
        g11 = gg * m11 * 13.5f;
        g12 = gg * m12 * 13.5f;
        g13 = gg * m13 * 4.5f;   // 1/b = 9/2
        g14 = gg * m14 * 4.5f;
        g15 = gg * m15 * 4.5f;
        g16 = gg * m16 * 4.5f;
        g17 = gg * m17 * 3.0f;   // 1/b = 3
        g18 = gg * m18 * 9.0f;   // 1/b = 9
    }
    if (a.kT > 0.f) {
        float G[16];
        const uint32_t sid = (uint32_t)site;
        normals4(a.key, a.step, sid, 0u, 0u, G);
        normals4(a.key, a.step, sid, 0u, 1u, G + 4);
        normals4(a.key, a.step, sid, 0u, 2u, G + 8);
        normals4(a.key, a.step, sid, 0u, 3u, G + 12);
        const float sq = sqrtf(3.0f * rho * a.kT);
        float n[15];
#pragma unroll
        for (int t = 0; t < 15; ++t) n[t] = sq * a.namp[t] * G[t];
        const float two9 = 2.0f / 9.0f, one9 = 1.0f / 9.0f;
        Bxx += two9 * (n[0] + 2.f * n[1]);
        Byy += two9 * (n[0] - n[1] + n[2]);
        Bzz += two9 * (n[0] - n[1] - n[2]);
        Bxy += one9 * n[3];
        Byz += one9 * n[4];
        Bxz += one9 * n[5];
        g10 += n[6];
        g11 += n[7];
        g12 += n[8];
        g13 += n[9];
        g14 += n[10];
        g15 += n[11];
        g16 += n[12];
        g17 += n[13];
        g18 += n[14];
    }

    const float tb = (Bxx + Byy + Bzz) * (1.0f / 3.0f);
    const float e0 = 4.5f * tb;  // 9/2 B:Q for Q = -delta/3 is -e0
    const float h1 = 1.f / 3.f, h2 = 2.f / 3.f;
    const float w1 = 1.f / 18.f, w2 = 1.f / 36.f;
    stpop(fout, site, (1.f / 3.f) * (drho - e0 + h1 * g16));

    float E, O;
    // +-x
    E = drho + 4.5f * Bxx - e0 - h2 * g16 - g17;
    O = 3.f * Ax - h2 * g10;
    stpop(fout, 1 * N + site, w1 * (E + O));
    stpop(fout, 2 * N + site, w1 * (E - O));
    // +-y
    E = drho + 4.5f * Byy - e0 - h2 * g16 + 0.5f * g17 - 0.5f * g18;
    O = 3.f * Ay - h2 * g11;
    stpop(fout, 3 * N + site, w1 * (E + O));
    stpop(fout, 4 * N + site, w1 * (E - O));
    // +-z
    E = drho + 4.5f * Bzz - e0 - h2 * g16 + 0.5f * g17 + 0.5f * g18;
    O = 3.f * Az - h2 * g12;
    stpop(fout, 5 * N + site, w1 * (E + O));
    stpop(fout, 6 * N + site, w1 * (E - O));
    const float Gev = h1 * g16 + 0.5f * g17;  // even ghosts shared by the xy and xz diagonals
    // +-(1,1,0)
    E = drho + 4.5f * (Bxx + Byy + 2.f * Bxy) - e0 + Gev + 0.5f * g18;
    O = 3.f * (Ax + Ay) + h1 * (g10 + g11) + g13 - g14;
    stpop(fout, 7 * N + site, w2 * (E + O));
    stpop(fout, 8 * N + site, w2 * (E - O));
    // +-(1,-1,0)
    E = drho + 4.5f * (Bxx + Byy - 2.f * Bxy) - e0 + Gev + 0.5f * g18;
    O = 3.f * (Ax - Ay) + h1 * (g10 - g11) + g13 + g14;
    stpop(fout, 9 * N + site, w2 * (E + O));
    stpop(fout, 10 * N + site, w2 * (E - O));
    // +-(1,0,1)
    E = drho + 4.5f * (Bxx + Bzz + 2.f * Bxz) - e0 + Gev - 0.5f * g18;
    O = 3.f * (Ax + Az) + h1 * (g10 + g12) - g13 + g15;
    stpop(fout, 11 * N + site, w2 * (E + O));
    stpop(fout, 12 * N + site, w2 * (E - O));
    // +-(1,0,-1)
    E = drho + 4.5f * (Bxx + Bzz - 2.f * Bxz) - e0 + Gev - 0.5f * g18;
    O = 3.f * (Ax - Az) + h1 * (g10 - g12) - g13 - g15;
    stpop(fout, 13 * N + site, w2 * (E + O));
    stpop(fout, 14 * N + site, w2 * (E - O));
    // +-(0,1,1)
    E = drho + 4.5f * (Byy + Bzz + 2.f * Byz) - e0 + h1 * g16 - g17;
    O = 3.f * (Ay + Az) + h1 * (g11 + g12) + g14 - g15;
    stpop(fout, 15 * N + site, w2 * (E + O));
    stpop(fout, 16 * N + site, w2 * (E - O));
    // +-(0,1,-1)
    E = drho + 4.5f * (Byy + Bzz - 2.f * Byz) - e0 + h1 * g16 - g17;
    O = 3.f * (Ay - Az) + h1 * (g11 - g12) + g14 + g15;
    stpop(fout, 17 * N + site, w2 * (E + O));
    stpop(fout, 18 * N + site, w2 * (E - O));
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
    const int xm = x == 0 ? g.nx - 1 : x - 1, xp = x == g.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
    const T *fin = (const T *)a.fin;
    T *fout = (T *)a.fout;
    const long long N = g.n;

    float f[9];
    f[0] = ldpop(fin, site);
    f[1] = ldpop(fin, 1 * N + g.sidx(xm, y, 0));
    f[2] = ldpop(fin, 2 * N + g.sidx(xp, y, 0));
    f[3] = ldpop(fin, 3 * N + g.sidx(x, ym, 0));
    f[4] = ldpop(fin, 4 * N + g.sidx(x, yp, 0));
    f[5] = ldpop(fin, 5 * N + g.sidx(xm, ym, 0));
    f[6] = ldpop(fin, 6 * N + g.sidx(xp, yp, 0));
    f[7] = ldpop(fin, 7 * N + g.sidx(xm, yp, 0));
    f[8] = ldpop(fin, 8 * N + g.sidx(xp, ym, 0));
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
    if (a.coupling & FLB_COUPLE_FORCE) {
        const float ps = a.psi[g.pidx(x, y, 0)];
        const float *mu = a.mu;
        Fx = -ps * 0.5f * (mu[g.pidx(x + 1, y, 0)] - mu[g.pidx(x - 1, y, 0)]);
        Fy = -ps * 0.5f * (mu[g.pidx(x, y + 1, 0)] - mu[g.pidx(x, y - 1, 0)]);
    }
    const float rho = a.rho0 + drho;
    const float irho = 1.0f / rho;
    const float vx = (jx + 0.5f * Fx) * irho, vy = (jy + 0.5f * Fy) * irho;
    store_padded(a.u, g, x, y, 0, vx, 1);
    store_padded(a.u + g.pn, g, x, y, 0, vy, 1);

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
        float G[8];
        const uint32_t sid = (uint32_t)site;
        normals4(a.key, a.step, sid, 0u, 0u, G);
        normals4(a.key, a.step, sid, 0u, 1u, G + 4);
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
__constant__ int8_t kEq9[9][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                                  {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};

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
        const int8_t *c = q == 19 ? kEq19[i] : kEq9[i];
        const long long pi = g.pidx(x + c[0], y + c[1], z + c[2]);
        const float r = rho ? rho[pi] : rho0;
        const float ux = u[pi], uy = u[g.pn + pi], uz = g.dim == 3 ? u[2 * g.pn + pi] : 0.f;
        const float cu = c[0] * ux + c[1] * uy + c[2] * uz;
        const float u2 = ux * ux + uy * uy + uz * uz;
        const float l2 = (float)(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        const float w = q == 19 ? (l2 == 0.f ? 1.f / 3.f : l2 == 1.f ? 1.f / 18.f : 1.f / 36.f)
                                : (l2 == 0.f ? 4.f / 9.f : l2 == 1.f ? 1.f / 9.f : 1.f / 36.f);
        stpop(fout, (long long)i * g.n + site, w * ((r - rho0) + r * (3.f * cu + 4.5f * cu * cu - 1.5f * u2)));
    }
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
    if (q == 19) {
        if (storage == FLB_F16_DEV) {
            if (gr) lb_d3q19_kernel<__half, true><<<grid, bs, 0, st>>>(a);
            else lb_d3q19_kernel<__half, false><<<grid, bs, 0, st>>>(a);
        } else {
            if (gr) lb_d3q19_kernel<float, true><<<grid, bs, 0, st>>>(a);
            else lb_d3q19_kernel<float, false><<<grid, bs, 0, st>>>(a);
        }
    } else {
        if (storage == FLB_F16_DEV) {
            if (gr) lb_d2q9_kernel<__half, true><<<grid, bs, 0, st>>>(a);
            else lb_d2q9_kernel<__half, false><<<grid, bs, 0, st>>>(a);
        } else {
            if (gr) lb_d2q9_kernel<float, true><<<grid, bs, 0, st>>>(a);
            else lb_d2q9_kernel<float, false><<<grid, bs, 0, st>>>(a);
        }
    }
    return cudaGetLastError();
}

}  // namespace flb

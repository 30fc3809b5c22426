// flb_psi.cu -- stochastic method-of-lines step of the order parameter psi
// (Sec. V of arXiv:1104.0078) by one-thread-per-site kernels: chemical
// potential, noise increment, node fluxes and the Runge-Kutta stage update.
// They run the 2D path and the 3D combinations the tiled kernels do not cover
// (another App. A Laplacian, the naive scheme, FV on D3Q15).
//
//   mu  = A psi + B psi^3 - K lap psi             (Sec. II.A; lap of App. A, SO by default)
//   FD: dpsi/dt = M lap mu - div_CD(u psi) + eta,     (Sec. V.A)
//       eta(r) = sum_l [zeta_l(r - c_l) - zeta_l(r)], zeta_l ~ N(0, 2 kT M a_l)
//       on the 13 (2D: 4) half-links, a_l the Laplacian's class coefficients --
//       real-space noise with the covariance -2 kT M L(q) of Eq. (etafdt).
//   FV: dpsi/dt = (2/c_s^2) sum_i w_i c_i . (J(r) + J(r + c_i))/2,       (Sec. V.B)
//       J = M grad mu - u psi + xi, grad mu = (1/c_s^2) sum_i w_i c_i mu(r + c_i),
//       xi ~ N(0, 2 kT M) per node and component (Eqs. fvdiff - fvgrad).
//   naive (Sec. III, the contrast): dpsi/dt = M lap mu - div_CD(u psi) + div_CD xi.
// The noise is drawn once per step (Philox stream 1) and held fixed over the
// Runge-Kutta stages (Sec. V, wilkie2004).
#include "flb_internal.cuh"

namespace flb {

// App. A Laplacian of a padded field at (x,y,z) with class weights w (faces,
// edges, corners; 2D axes and diagonals); needs the field within 1 cell.
__device__ __forceinline__ float lap_w(const float *f, const Geom &g, int x, int y, int z, const LapW &w)
{
    if (g.dim == 3) {
        float n1 = 0.f, n2 = 0.f, n3 = 0.f;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int cls = (dx != 0) + (dy != 0) + (dz != 0);
                    const float v = f[g.pidx(x + dx, y + dy, z + dz)];
                    if (cls == 1) n1 += v;
                    else if (cls == 2) n2 += v;
                    else if (cls == 3) n3 += v;
                }
        return (w.c1 * n1 + w.c2 * n2) + (w.c3 * n3 + w.c0 * f[g.pidx(x, y, z)]);
    }
    const float n1 = f[g.pidx(x + 1, y, 0)] + f[g.pidx(x - 1, y, 0)] + f[g.pidx(x, y + 1, 0)] + f[g.pidx(x, y - 1, 0)];
    const float n2 = f[g.pidx(x + 1, y + 1, 0)] + f[g.pidx(x - 1, y - 1, 0)] + f[g.pidx(x + 1, y - 1, 0)] +
                     f[g.pidx(x - 1, y + 1, 0)];
    return (w.c1 * n1 + w.c2 * n2) + w.c0 * f[g.pidx(x, y, 0)];
}

// velocity sets of the FV scheme (no rest vector), in the lattices' pair order
__constant__ int8_t kC19[18][3] = {{1, 0, 0},  {-1, 0, 0},  {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
                                   {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1},
                                   {1, 0, -1}, {-1, 0, 1},  {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
__constant__ int8_t kC15[14][3] = {{1, 0, 0},   {-1, 0, 0},  {0, 1, 0},    {0, -1, 0}, {0, 0, 1},
                                   {0, 0, -1},  {1, 1, 1},   {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1},
                                   {1, -1, 1},  {-1, 1, -1}, {1, -1, -1},  {-1, 1, 1}};
__constant__ int8_t kC9[8][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {-1, -1}, {1, -1}, {-1, 1}};

// Link k (0 .. q-2) of lattice q and its weight: D3Q19 1/18, 1/36; D3Q15 1/9,
// 1/72; D2Q9 1/9, 1/36.
__device__ __forceinline__ void fv_link(int q, int k, int &cx, int &cy, int &cz, float &w)
{
    if (q == 19) {
        cx = kC19[k][0]; cy = kC19[k][1]; cz = kC19[k][2];
        w = (abs(cx) + abs(cy) + abs(cz)) == 1 ? 1.f / 18.f : 1.f / 36.f;
    } else if (q == 15) {
        cx = kC15[k][0]; cy = kC15[k][1]; cz = kC15[k][2];
        w = (abs(cx) + abs(cy) + abs(cz)) == 1 ? 1.f / 9.f : 1.f / 72.f;
    } else {
        cx = kC9[k][0]; cy = kC9[k][1]; cz = 0;
        w = (abs(cx) + abs(cy)) == 1 ? 1.f / 9.f : 1.f / 36.f;
    }
}

// FD half-links: x, y, z, (1,1,0), (1,-1,0), (1,0,1), (1,0,-1), (0,1,1), (0,1,-1),
// (1,1,1), (1,1,-1), (1,-1,1), (1,-1,-1); 2D: x, y, (1,1), (1,-1).
__constant__ int8_t kL13[13][3] = {{1, 0, 0},  {0, 1, 0},  {0, 0, 1},  {1, 1, 0}, {1, -1, 0},
                                   {1, 0, 1},  {1, 0, -1}, {0, 1, 1},  {0, 1, -1}, {1, 1, 1},
                                   {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};

// ---------------------------------------------------------------------------
__global__ void mu_kernel(const Geom g, const float *__restrict__ psi, float *__restrict__ mu, float A, float B,
                          float K, const LapW lw)
{
    const int ex = g.nx + 4, ey = g.ny + 4, ez = g.dim == 3 ? g.nz + 4 : 1;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)ex * ey * ez) return;
    const int x = (int)(i % ex) - 2;
    const int y = (int)((i / ex) % ey) - 2;
    const int z = g.dim == 3 ? (int)(i / ((long long)ex * ey)) - 2 : 0;
    const float p = psi[g.pidx(x, y, z)];
    mu[g.pidx(x, y, z)] = A * p + B * p * p * p - K * lap_w(psi, g, x, y, z, lw);
}

// Order-parameter stress (Sec. IV, Eq. muf) in 2D on the interior + 1 ghost
// layer: planes xx, yy, xy of sigma_ab = K g_a g_b + delta_ab [A/2 psi^2
// + 3B/4 psi^4 - K psi lap_SO psi - K/2 |g|^2], g the central difference.
__global__ void sigma2_kernel(const Geom g, const float *__restrict__ psi, float *__restrict__ sig, float A, float B,
                              float K)
{
    const int ex = g.nx + 2, ey = g.ny + 2;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)ex * ey) return;
    const int x = (int)(i % ex) - 1, y = (int)(i / ex) - 1;
    const float p = psi[g.pidx(x, y, 0)];
    const float gx = 0.5f * (psi[g.pidx(x + 1, y, 0)] - psi[g.pidx(x - 1, y, 0)]);
    const float gy = 0.5f * (psi[g.pidx(x, y + 1, 0)] - psi[g.pidx(x, y - 1, 0)]);
    const float p2 = p * p;
    const LapW so{-3.f, 0.5f, 0.25f, 0.f};  // the planar SO stencil (the stress form runs with SO only)
    const float iso = 0.5f * A * p2 + 0.75f * B * p2 * p2 - K * p * lap_w(psi, g, x, y, 0, so) - 0.5f * K * (gx * gx + gy * gy);
    const long long o = g.pidx(x, y, 0);
    sig[o] = K * gx * gx + iso;
    sig[o + g.pn] = K * gy * gy + iso;
    sig[o + 2 * g.pn] = K * gx * gy;
}

// Noise increment eta of one 2D step (Sec. V), held fixed over the step's
// Runge-Kutta stages.  A block of 32 x 16 threads first draws, once per point,
// the four normals of every point of its tile and a one-point halo into shared
// memory (counter: the point's site id, Philox stream 1, block 0), then
//   FD: eta(r) = sum_l sqrt(2 kT M a_l) [zeta_l(r - c_l) - zeta_l(r)] over the
//       half-links (1,0), (0,1), (1,1), (1,-1), a_l the Laplacian's axis and
//       diagonal coefficients (SO: 1/2, 1/4);
//   FV: eta(r) = (2/c_s^2) sum_i w_i c_i . (xi(r) + xi(r + c_i)) / 2, xi_a the
//       first two normals times sqrt(2 kT M);
//   naive (Sec. III): eta(r) = (1/2) sum_a [xi_a(r + e_a) - xi_a(r - e_a)].
__global__ void __launch_bounds__(512) noise2_kernel(const NoiseArgs a)
{
    constexpr int TX = 32, TY = 16, HX = TX + 2, HY = TY + 2;
    __shared__ float zs[4][HY][HX];
    const Geom &g = a.g;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int t = threadIdx.x + TX * threadIdx.y;
    for (int k = t; k < HX * HY; k += TX * TY) {
        const int lx = k % HX, ly = k / HX;
        const int gx = ((x0 - 1 + lx) % g.nx + g.nx) % g.nx, gy = ((y0 - 1 + ly) % g.ny + g.ny) % g.ny;
        float G[4];
        normals<2>(a.key, a.step, (uint32_t)(gx + g.nx * gy), 1u, 0u, G);
        zs[0][ly][lx] = G[0];
        zs[1][ly][lx] = G[1];
        zs[2][ly][lx] = G[2];
        zs[3][ly][lx] = G[3];
    }
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= g.nx || y >= g.ny) return;
    const int lx = threadIdx.x + 1, ly = threadIdx.y + 1;
    float eta;
    if (a.scheme == FLB_FD) {
        const float s1 = sqrtf(2.f * a.kT * a.M * a.lw.c1), s2 = sqrtf(2.f * a.kT * a.M * a.lw.c2);  // sqrt(2 kT M a_l)
        eta = s1 * ((zs[0][ly][lx - 1] - zs[0][ly][lx]) + (zs[1][ly - 1][lx] - zs[1][ly][lx])) +
              s2 * ((zs[2][ly - 1][lx - 1] - zs[2][ly][lx]) + (zs[3][ly + 1][lx - 1] - zs[3][ly][lx]));
    } else if (a.scheme == FLB_NAIVE) {
        const float sd = sqrtf(2.f * a.kT * a.M);
        eta = 0.5f * sd * ((zs[0][ly][lx + 1] - zs[0][ly][lx - 1]) + (zs[1][ly + 1][lx] - zs[1][ly - 1][lx]));
    } else {
        const float sd = sqrtf(2.f * a.kT * a.M);
        const float ox = zs[0][ly][lx], oy = zs[1][ly][lx];
        // axis links (w = 1/9) and diagonal links (w = 1/36), c . (xi(r) + xi(r + c))
        const float ax = ((ox + zs[0][ly][lx + 1]) - (ox + zs[0][ly][lx - 1])) +
                         ((oy + zs[1][ly + 1][lx]) - (oy + zs[1][ly - 1][lx]));
        const float dg = ((ox + zs[0][ly + 1][lx + 1]) + (oy + zs[1][ly + 1][lx + 1])) -
                         ((ox + zs[0][ly - 1][lx - 1]) + (oy + zs[1][ly - 1][lx - 1])) +
                         ((ox + zs[0][ly - 1][lx + 1]) - (oy + zs[1][ly - 1][lx + 1])) -
                         ((ox + zs[0][ly + 1][lx - 1]) - (oy + zs[1][ly + 1][lx - 1]));
        eta = 3.f * sd * ((1.f / 9.f) * ax + (1.f / 36.f) * dg);
    }
    a.eta[x + g.nx * y] = eta;
}

// Noise increment eta of one 3D step for the one-thread-per-site path (other
// Laplacians, the naive scheme, FV on D3Q15).  A block of 16 x 8 x 4 threads
// draws, once per point, the normals of its tile and a one-point halo (18 x 10
// x 6 points) into shared memory -- FD: the 13 link normals, Philox stream 1
// blocks 0-1; FV and naive: the 3 node normals of block 0 -- then
//   FD: eta(r) = sum_l sqrt(2 kT M a_l) [zeta_l(r - c_l) - zeta_l(r)], a_l the
//       class coefficient of half-link l in the chosen Laplacian;
//   FV: eta(r) = (2/c_s^2) sum_i w_i c_i . (xi(r) + xi(r + c_i)) / 2 on lattice q;
//   naive: eta(r) = (1/2) sum_a [xi_a(r + e_a) - xi_a(r - e_a)].
constexpr int N3X = 16, N3Y = 8, N3Z = 4;
constexpr int N3HX = N3X + 2, N3HY = N3Y + 2, N3HZ = N3Z + 2, N3P = N3HX * N3HY * N3HZ;

__global__ void __launch_bounds__(N3X *N3Y *N3Z) noise3_kernel(const NoiseArgs a)
{
    extern __shared__ float zs[];  // [nc][N3P]
    const Geom &g = a.g;
    const int nc = a.scheme == FLB_FD ? 13 : 3;
    const int nb = a.scheme == FLB_FD ? 2 : 1;
    const int x0 = blockIdx.x * N3X, y0 = blockIdx.y * N3Y, z0 = blockIdx.z * N3Z;
    const int t = threadIdx.x + N3X * (threadIdx.y + N3Y * threadIdx.z);
    for (int k = t; k < N3P; k += N3X * N3Y * N3Z) {
        const int lx = k % N3HX, ly = (k / N3HX) % N3HY, lz = k / (N3HX * N3HY);
        // halo points past a small lattice's far edge are drawn but never read
        const int gx = ((x0 - 1 + lx) % g.nx + g.nx) % g.nx, gy = ((y0 - 1 + ly) % g.ny + g.ny) % g.ny;
        const int gz = ((z0 - 1 + lz) % g.nz + g.nz) % g.nz;
        const uint32_t sid = (uint32_t)(gx + g.nx * (gy + g.ny * gz));
        for (int b = 0; b < nb; ++b) {
            float G[8];
            normals<4>(a.key, a.step, sid, 1u, (uint32_t)b, G);
            for (int j = 0; j < 8 && 8 * b + j < nc; ++j) zs[(8 * b + j) * N3P + k] = G[j];
        }
    }
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
    if (x >= g.nx || y >= g.ny || z >= g.nz) return;
    const int c = (threadIdx.x + 1) + N3HX * ((threadIdx.y + 1) + N3HY * (threadIdx.z + 1));
    const int sy = N3HX, sz = N3HX * N3HY;
    float eta = 0.f;
    if (a.scheme == FLB_FD) {
        const float cw[4] = {0.f, a.lw.c1, a.lw.c2, a.lw.c3};
        for (int l = 0; l < 13; ++l) {
            const int cx = kL13[l][0], cy = kL13[l][1], cz = kL13[l][2];
            const float s = sqrtf(2.f * a.kT * a.M * cw[abs(cx) + abs(cy) + abs(cz)]);
            eta += s * (zs[l * N3P + c - cx - cy * sy - cz * sz] - zs[l * N3P + c]);
        }
    } else if (a.scheme == FLB_NAIVE) {
        const float sd = sqrtf(2.f * a.kT * a.M);
        eta = 0.5f * sd * ((zs[c + 1] - zs[c - 1]) + (zs[N3P + c + sy] - zs[N3P + c - sy]) +
                           (zs[2 * N3P + c + sz] - zs[2 * N3P + c - sz]));
    } else {
        const float sd = sqrtf(2.f * a.kT * a.M);
        const float ox = zs[c], oy = zs[N3P + c], oz = zs[2 * N3P + c];
        float acc = 0.f;
        for (int k = 0; k < a.q - 1; ++k) {
            int cx, cy, cz;
            float w;
            fv_link(a.q, k, cx, cy, cz, w);
            const int n = c + cx + cy * sy + cz * sz;
            acc += w * (cx * (ox + zs[n]) + cy * (oy + zs[N3P + n]) + cz * (oz + zs[2 * N3P + n]));
        }
        eta = 3.f * sd * acc;
    }
    a.eta[x + g.nx * (y + g.ny * z)] = eta;
}

// FV deterministic node flux J = M grad_FV mu - u psi on the interior and one ghost layer.
__global__ void flux_kernel(const Geom g, int q, const float *__restrict__ psi, const float *__restrict__ mu,
                            const float *__restrict__ u, float *__restrict__ J, float M, int advect)
{
    const int ex = g.nx + 2, ey = g.ny + 2, ez = g.dim == 3 ? g.nz + 2 : 1;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)ex * ey * ez) return;
    const int x = (int)(i % ex) - 1;
    const int y = (int)((i / ex) % ey) - 1;
    const int z = g.dim == 3 ? (int)(i / ((long long)ex * ey)) - 1 : 0;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    for (int k = 0; k < q - 1; ++k) {
        int cx, cy, cz;
        float w;
        fv_link(q, k, cx, cy, cz, w);
        const float m = w * mu[g.pidx(x + cx, y + cy, z + cz)];
        gx += cx * m;
        gy += cy * m;
        gz += cz * m;
    }
    const long long pi = g.pidx(x, y, z);
    const float ps = psi[pi];
    float jx = 3.f * M * gx, jy = 3.f * M * gy, jz = 3.f * M * gz;
    if (advect) {
        jx -= u[pi] * ps;
        jy -= u[g.pn + pi] * ps;
        if (g.dim == 3) jz -= u[2 * g.pn + pi] * ps;
    }
    J[pi] = jx;
    J[g.pn + pi] = jy;
    if (g.dim == 3) J[2 * g.pn + pi] = jz;
}

__global__ void psi_update_kernel(const PsiArgs a)
{
    const Geom &g = a.g;
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= g.n) return;
    const int x = (int)(site % g.nx);
    const int y = (int)((site / g.nx) % g.ny);
    const int z = (int)(site / ((long long)g.nx * g.ny));
    const long long pi = g.pidx(x, y, z);
    float D;
    if (a.scheme == FLB_FD || a.scheme == FLB_NAIVE) {
        D = a.M * lap_w(a.mu, g, x, y, z, a.lw);
        if (a.coupling & FLB_COUPLE_ADVECT) {
            const float *ps = a.psi;
            float adv = a.u[g.pidx(x + 1, y, z)] * ps[g.pidx(x + 1, y, z)] - a.u[g.pidx(x - 1, y, z)] * ps[g.pidx(x - 1, y, z)];
            adv += a.u[g.pn + g.pidx(x, y + 1, z)] * ps[g.pidx(x, y + 1, z)] -
                   a.u[g.pn + g.pidx(x, y - 1, z)] * ps[g.pidx(x, y - 1, z)];
            if (g.dim == 3)
                adv += a.u[2 * g.pn + g.pidx(x, y, z + 1)] * ps[g.pidx(x, y, z + 1)] -
                       a.u[2 * g.pn + g.pidx(x, y, z - 1)] * ps[g.pidx(x, y, z - 1)];
            D -= 0.5f * adv;
        }
    } else {
        const float *J = a.J;
        const float J0x = J[pi], J0y = J[g.pn + pi], J0z = g.dim == 3 ? J[2 * g.pn + pi] : 0.f;
        float acc = 0.f;
        for (int k = 0; k < a.q - 1; ++k) {
            int cx, cy, cz;
            float w;
            fv_link(a.q, k, cx, cy, cz, w);
            const long long pn = g.pidx(x + cx, y + cy, z + cz);
            float link = cx * (J0x + J[pn]) + cy * (J0y + J[g.pn + pn]);
            if (g.dim == 3) link += cz * (J0z + J[2 * g.pn + pn]);
            acc += w * link;
        }
        D = 3.f * acc;  // (2/c_s^2) * (1/2) sum_i w_i c_i.(J(r) + J(r + c_i))
    }
    const float eta = a.eta ? a.eta[site] : 0.f;
    float out;
    if (a.integrator == FLB_RK4) {  // k_s = D_s + eta with eta fixed over the step
        if (a.stage == 1) {
            const float p = a.psi[pi];
            out = p + 0.5f * (D + eta);
            a.acc[site] = p + eta + D * (1.f / 6.f);
        } else if (a.stage == 4) {
            out = a.acc[site] + D * (1.f / 6.f);
        } else {
            out = a.base[pi] + (a.stage == 2 ? 0.5f : 1.f) * (D + eta);
            a.acc[site] += D * (1.f / 3.f);
        }
    } else if (a.stage == 1) {
        const float p = a.psi[pi];
        out = p + D + eta;
        if (a.integrator == FLB_HEUN) a.acc[site] = p + 0.5f * D + eta;
    } else {
        out = a.psi0[site] + 0.5f * D;
    }
    store_padded(a.out, g, x, y, z, out, 3);
}

static unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

cudaError_t launch_mu(const Geom &g, const float *psi, float *mu, float A, float B, float K, const LapW &lw,
                      cudaStream_t s)
{
    const long long ext = (long long)(g.nx + 4) * (g.ny + 4) * (g.dim == 3 ? g.nz + 4 : 1);
    mu_kernel<<<blocks_for(ext, 256), 256, 0, s>>>(g, psi, mu, A, B, K, lw);
    return cudaGetLastError();
}

cudaError_t launch_sigma2(const Geom &g, const float *psi, float *sig, float A, float B, float K, cudaStream_t s)
{
    const long long ext = (long long)(g.nx + 2) * (g.ny + 2);
    sigma2_kernel<<<blocks_for(ext, 256), 256, 0, s>>>(g, psi, sig, A, B, K);
    return cudaGetLastError();
}

cudaError_t launch_noise(const NoiseArgs &a, cudaStream_t s)
{
    if (a.g.dim == 3) {
        const int smem = (a.scheme == FLB_FD ? 13 : 3) * N3P * (int)sizeof(float);
        const cudaError_t e = cudaFuncSetAttribute(noise3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        const dim3 grid((a.g.nx + N3X - 1) / N3X, (a.g.ny + N3Y - 1) / N3Y, (a.g.nz + N3Z - 1) / N3Z);
        noise3_kernel<<<grid, dim3(N3X, N3Y, N3Z), smem, s>>>(a);
        return cudaGetLastError();
    }
    const dim3 grid((a.g.nx + 31) / 32, (a.g.ny + 15) / 16);
    noise2_kernel<<<grid, dim3(32, 16), 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_flux(const Geom &g, int q, const float *psi, const float *mu, const float *u, float *J, float M,
                        int coupling, cudaStream_t s)
{
    const long long ext = (long long)(g.nx + 2) * (g.ny + 2) * (g.dim == 3 ? g.nz + 2 : 1);
    flux_kernel<<<blocks_for(ext, 256), 256, 0, s>>>(g, q, psi, mu, u, J, M, (coupling & FLB_COUPLE_ADVECT) ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_psi_update(const PsiArgs &a, int q, cudaStream_t s)
{
    (void)q;
    psi_update_kernel<<<blocks_for(a.g.n, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace flb

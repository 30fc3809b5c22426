// flb_psi3d.cu -- one Runge-Kutta stage of the order-parameter equation (Sec. V
// of arXiv:1104.0078) on a 3D box, fused in one pass with z-marching (2.5D)
// blocking.
//
// A block owns a TX x TY column tile and a chunk of ZC planes.  Rolling rings of
// planes in shared memory hold psi (tile + 3 ghost cells), the chemical
// potential mu = A psi + B psi^3 - K lap_SO psi (tile + 2), and for the finite-
// volume scheme the node flux J = M grad mu - u psi (tile + 1) and the node
// noise xi (tile + 1); the stage output at plane z is formed from the three
// flux planes z-1, z, z+1.  Nothing but psi, u and the Heun accumulator touches
// HBM.  In the finite-volume kernel the psi and velocity planes arrive by TMA
// (cp.async.bulk.tensor) two planes ahead of use.
//
//   FV (Sec. V.B):  grad mu = (1/c_s^2) sum_i w_i c_i mu(r + c_i)
//                   D(r)    = (1/c_s^2) sum_i w_i c_i . J(r + c_i)
//                   (the link average (J(r) + J(r+c_i))/2 of Eq. fvflux with
//                    the 2/c_s^2 divergence; sum_i w_i c_i = 0 removes J(r)),
//                   xi_a ~ N(0, 2 kT M) per node and component.
//   FD (Sec. V.A):  D(r)    = M lap_SO mu - div_CD(u psi),
//                   eta(r)  = sum_l [zeta_l(r - c_l) - zeta_l(r)] over the 13
//                   half-links of the SO stencil, zeta_l ~ N(0, 2 kT M a_l).
// Stage 1 writes psi* = psi + D + eta and (Heun) E = psi + D/2 + eta; stage 2
// writes psi^{n+1} = E + D(psi*)/2 (the noise is held fixed over the step).
#include <cudaTypedefs.h>

#include "flb_internal.cuh"
#include "flb_tma.cuh"

namespace flb {

constexpr int PS_NT = PS_TX * PS_TY;
constexpr int H3X = PS_TX + 6, H3Y = PS_TY + 6, H3N = H3X * H3Y;  // psi: tile + 3
constexpr int H2X = PS_TX + 4, H2Y = PS_TY + 4, H2N = H2X * H2Y;  // mu: tile + 2
constexpr int H1X = PS_TX + 2, H1Y = PS_TY + 2, H1N = H1X * H1Y;  // flux / noise: tile + 1
constexpr int S3 = (H3N + PS_NT - 1) / PS_NT, S2 = (H2N + PS_NT - 1) / PS_NT, S1 = (H1N + PS_NT - 1) / PS_NT;

__device__ __forceinline__ int ring3(int p) { return ((p % 3) + 3) % 3; }
__device__ __forceinline__ int ring4(int p) { return p & 3; }  // two's complement: correct for negative p

// mu = A psi + B psi^3 - (K/22)(6 N1 + 3 N2 + N3 - 80 psi) at offset c of three
// psi planes with row pitch PX (with A = B = 0 and k22 = -1/22 it is lap_SO)
template <int PX>
__device__ __forceinline__ float mu_point(const float *pm, const float *p0, const float *pp, int c, float A, float B,
                                          float k22)
{
    const float n1 = (p0[c - 1] + p0[c + 1]) + (p0[c - PX] + p0[c + PX]) + (pm[c] + pp[c]);
    const float n2 = ((p0[c - 1 - PX] + p0[c + 1 - PX]) + (p0[c - 1 + PX] + p0[c + 1 + PX])) +
                     ((pm[c - 1] + pm[c + 1]) + (pm[c - PX] + pm[c + PX])) +
                     ((pp[c - 1] + pp[c + 1]) + (pp[c - PX] + pp[c + PX]));
    const float n3 = ((pm[c - 1 - PX] + pm[c + 1 - PX]) + (pm[c - 1 + PX] + pm[c + 1 + PX])) +
                     ((pp[c - 1 - PX] + pp[c + 1 - PX]) + (pp[c - 1 + PX] + pp[c + 1 + PX]));
    const float ps = p0[c];
    return A * ps + B * ps * ps * ps - k22 * (6.f * n1 + 3.f * n2 + n3 - 80.f * ps);
}

struct Psi3Args {
    Geom g;
    const float *psi;  // padded stage input
    const float *u;    // padded velocity (images to radius 1)
    float *out;        // padded stage output (images to radius 3)
    float *E;          // [N] Heun accumulator: written by stage 1, read by stage 2
    float A, B, K, M, kT;
    int advect, heun;
    int zc;            // planes per block (the z chunk)
    PhiloxKey key;
    int64_t step;
};

// Per-thread view of the block's halo regions, computed once: for every slot the
// in-plane offset of the padded field it loads (psi, u) and the in-plane counter
// id of its periodic image (noise).
struct Regions {
    int g3[S3];                 // psi region: padded in-plane offsets (-1: no slot)
    int c2[S2];                 // mu region: centre offset in the psi tile frame (-1: none)
    int c1[S1], p1[S1], u1[S1], n1[S1];  // flux region: mu-frame centre, psi-frame centre, u offset, noise id
};

__device__ __forceinline__ void make_regions(Regions &R, const Geom &g, int x0, int y0)
{
    const int t = threadIdx.x;
#pragma unroll
    for (int j = 0; j < S3; ++j) {
        const int k = t + j * PS_NT;
        const int gx = min(x0 - 3 + k % H3X, g.nx + GX - 1), gy = min(y0 - 3 + k / H3X, g.ny + GY - 1);
        R.g3[j] = k < H3N ? (gx + GX) + g.px * (gy + GY) : -1;
    }
#pragma unroll
    for (int j = 0; j < S2; ++j) {
        const int k = t + j * PS_NT;
        R.c2[j] = k < H2N ? (k % H2X + 1) + H3X * (k / H2X + 1) : -1;
    }
#pragma unroll
    for (int j = 0; j < S1; ++j) {
        const int k = t + j * PS_NT;
        const int lx = k % H1X, ly = k / H1X;
        const int gx = min(x0 - 1 + lx, g.nx + GX - 1), gy = min(y0 - 1 + ly, g.ny + GY - 1);
        R.c1[j] = k < H1N ? (lx + 1) + H2X * (ly + 1) : -1;
        R.p1[j] = (lx + 2) + H3X * (ly + 2);
        R.u1[j] = (gx + GX) + g.px * (gy + GY);
        R.n1[j] = wrapi(gx, g.nx) + g.nx * wrapi(gy, g.ny);
    }
}

// Point k of a W x H region (W >= 32): rows' first 32 columns first, then the
// W - 32 remaining columns of every row.
__device__ __forceinline__ void region_point(int k, int W, int H, int &lx, int &ly)
{
    if (k < 32 * H) {
        lx = k & 31;
        ly = k >> 5;
    } else {
        const int r = k - 32 * H, e = W - 32;
        lx = 32 + r % e;
        ly = r / e;
    }
}

// divergence (1/c_s^2) sum_i w_i c_i . V(r + c_i) of a vector field held in three
// planes (z-1, z, z+1) of the tile + 1 frame: (1/6) axis + (1/12) diagonal links
__device__ __forceinline__ float fv_div(const float *xm, const float *x0, const float *xp, const float *ym,
                                        const float *y0, const float *yp, const float *zm, const float *z0,
                                        const float *zp, int c)
{
    (void)z0;
    const float ax = (x0[c + 1] - x0[c - 1]) + (y0[c + H1X] - y0[c - H1X]) + (zp[c] - zm[c]);
    float dg = (x0[c + 1 + H1X] + y0[c + 1 + H1X]) - (x0[c - 1 - H1X] + y0[c - 1 - H1X]);
    dg += (x0[c + 1 - H1X] - y0[c + 1 - H1X]) - (x0[c - 1 + H1X] - y0[c - 1 + H1X]);
    dg += (xp[c + 1] + zp[c + 1]) - (xm[c - 1] + zm[c - 1]);
    dg += (xm[c + 1] - zm[c + 1]) - (xp[c - 1] - zp[c - 1]);
    dg += (yp[c + H1X] + zp[c + H1X]) - (ym[c - H1X] + zm[c - H1X]);
    dg += (ym[c + H1X] - zm[c + H1X]) - (yp[c - H1X] - zp[c - H1X]);
    return (1.f / 6.f) * ax + (1.f / 12.f) * dg;
}

// ---------------------------------------------------------------------------
// Finite difference.  Shared memory: psi ring 4 x H3N, mu ring 3 x H2N and
// (stage 1 with noise) the 13 link noises of one plane, 13 x H1N floats.
// ---------------------------------------------------------------------------
// half-links: x, y, z, (1,1,0), (1,-1,0), (1,0,1), (1,0,-1), (0,1,1), (0,1,-1),
// (1,1,1), (1,1,-1), (1,-1,1), (1,-1,-1); coefficients 6/22, 3/22, 1/22
__constant__ int8_t kFDL[13][3] = {{1, 0, 0},  {0, 1, 0},  {0, 0, 1},  {1, 1, 0}, {1, -1, 0},
                                   {1, 0, 1},  {1, 0, -1}, {0, 1, 1},  {0, 1, -1}, {1, 1, 1},
                                   {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};

template <int STAGE, bool NOISE>
__global__ void __launch_bounds__(PS_NT) psi3_fd_kernel(const Psi3Args a)
{
    extern __shared__ float smem[];
    float *sps = smem;           // [4][H3N]
    float *smu = sps + 4 * H3N;  // [3][H2N]
    float *sZ = smu + 3 * H2N;   // [13][H1N] when NOISE
    const Geom &g = a.g;
    const int tx = threadIdx.x % PS_TX, ty = threadIdx.x / PS_TX;
    const int x0 = blockIdx.x * PS_TX, y0 = blockIdx.y * PS_TY, z0 = blockIdx.z * a.zc;
    const int z1 = min(z0 + a.zc, g.nz);
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < g.nx && y < g.ny;
    const float k22 = a.K * (1.0f / 22.0f);
    const int plane = g.px * g.py;
    Regions R;
    make_regions(R, g, x0, y0);
    float accm = 0.f, acc0 = 0.f, accp = 0.f;  // eta of planes p-2, p-1, p

    for (int p = z0 - 2; p <= z1 + 1; ++p) {
        __syncthreads();
        {
            const float *src = a.psi + (size_t)plane * (p + g.gz);
            float *dst = sps + ring4(p) * H3N;
#pragma unroll
            for (int j = 0; j < S3; ++j)
                if (R.g3[j] >= 0) dst[threadIdx.x + j * PS_NT] = __ldg(src + R.g3[j]);
        }
        __syncthreads();
        const int q = p - 1;
        if (q >= z0 - 1) {
            // mu(q) on tile + 1, stored at its place in the tile + 2 frame
            const float *pm = sps + ring4(q - 1) * H3N, *p0 = sps + ring4(q) * H3N, *pp = sps + ring4(q + 1) * H3N;
            float *dst = smu + ring3(q) * H2N;
#pragma unroll
            for (int j = 0; j < S1; ++j) {
                const int c = R.c1[j];
                if (c < 0) continue;
                dst[c] = mu_point<H3X>(pm, p0, pp, R.p1[j], a.A, a.B, k22);
            }
            if (NOISE) {
                const int zid = g.nx * g.ny * wrapi(q, g.nz);
#pragma unroll
                for (int j = 0; j < S1; ++j) {
                    if (R.c1[j] < 0) continue;
                    const int k = threadIdx.x + j * PS_NT;
                    const uint32_t sid = (uint32_t)(R.n1[j] + zid);
                    float G[16];
                    normals4(a.key, a.step, sid, 1u, 0u, G);
                    normals4(a.key, a.step, sid, 1u, 1u, G + 4);
                    normals4(a.key, a.step, sid, 1u, 2u, G + 8);
                    normals4(a.key, a.step, sid, 1u, 3u, G + 12);
#pragma unroll
                    for (int l = 0; l < 13; ++l) {
                        const float al = l < 3 ? 6.f / 22.f : (l < 9 ? 3.f / 22.f : 1.f / 22.f);
                        sZ[l * H1N + k] = sqrtf(2.0f * a.kT * a.M * al) * G[l];
                    }
                }
            }
        }
        __syncthreads();
        if (NOISE && q >= z0 - 1 && active) {
            // zeta(q) feeds eta(q) (own links, in-plane neighbours), eta(q+1)
            // (links with c_z = +1) and eta(q-1) (links with c_z = -1)
            const int c = (tx + 1) + H1X * (ty + 1);
            float own = 0.f, in0 = 0.f, up = 0.f, dn = 0.f;
#pragma unroll
            for (int l = 0; l < 13; ++l) {
                own += sZ[l * H1N + c];
                const float v = sZ[l * H1N + c - kFDL[l][0] - H1X * kFDL[l][1]];
                if (kFDL[l][2] == 0) in0 += v;
                else if (kFDL[l][2] > 0) up += v;
                else dn += v;
            }
            accm += dn;
            acc0 += in0 - own;
            accp += up;
        }
        const int z = p - 2;
        if (z >= z0 && active) {
            const float *mm = smu + ring3(z - 1) * H2N, *m0 = smu + ring3(z) * H2N, *mp = smu + ring3(z + 1) * H2N;
            const int c = (tx + 2) + H2X * (ty + 2);
            float D = a.M * mu_point<H2X>(mm, m0, mp, c, 0.f, 0.f, -1.0f / 22.0f);
            if (a.advect) {
                const float *P0 = sps + ring4(z) * H3N, *Pm = sps + ring4(z - 1) * H3N, *Pp = sps + ring4(z + 1) * H3N;
                const int cp = (tx + 3) + H3X * (ty + 3);
                const int pi = g.pidx32(x, y, z);
                const int sy = g.px, sz = g.px * g.py;
                const float *u = a.u;
                const float adv = (u[pi + 1] * P0[cp + 1] - u[pi - 1] * P0[cp - 1]) +
                                  (u[g.pn + pi + sy] * P0[cp + H3X] - u[g.pn + pi - sy] * P0[cp - H3X]) +
                                  (u[2 * g.pn + pi + sz] * Pp[cp] - u[2 * g.pn + pi - sz] * Pm[cp]);
                D -= 0.5f * adv;
            }
            const int si = x + g.nx * (y + g.ny * z);
            float out;
            if (STAGE == 1) {
                const float eta = NOISE ? accm : 0.f;
                const float pv = sps[ring4(z) * H3N + (tx + 3) + H3X * (ty + 3)];
                out = pv + D + eta;
                if (a.heun) a.E[si] = pv + 0.5f * D + eta;
            } else {
                out = a.E[si] + 0.5f * D;
            }
            store_padded(a.out, g, x, y, z, out, 3);
        }
        accm = acc0;
        acc0 = accp;
        accp = 0.f;
    }
}

// ---------------------------------------------------------------------------
// Finite volume with TMA staging.  psi planes (tile + 4 in x, + 3 in y) and the
// three velocity components of a plane (tile + 4 in x, + 1 in y) are copied by
// cp.async.bulk.tensor two planes ahead of their use into rings of shared-memory
// slots, each completed on its own mbarrier; the compute phases are those of
// psi3_fv_kernel.
//   psi slot:  [TY+6][TX+8] floats, column c <-> x = x0 - 4 + c, row r <-> y = y0 - 3 + r
//   u slot:    [3][TY+2][TX+8],     column c <-> x = x0 - 4 + c, row r <-> y = y0 - 1 + r
// ---------------------------------------------------------------------------
constexpr int TB_X = PS_TX + 8;                            // TMA box width (x0-4 .. x0+TX+3)
constexpr int TP_N = TB_X * H3Y;                           // psi slot floats
constexpr int TP_SLOT = ((TP_N * 4 + 127) / 128) * 32;     // floats, 128-byte multiple
constexpr int TU_N = 3 * TB_X * H1Y;                       // u slot floats
constexpr int TU_SLOT = ((TU_N * 4 + 127) / 128) * 32;
constexpr int T_PSI_DEPTH = 6, T_U_DEPTH = 3;

struct TmaArgs {
    Psi3Args a;
    int *status;
};

constexpr int FV_SMEM_FLOATS = T_PSI_DEPTH * TP_SLOT + T_U_DEPTH * TU_SLOT + 2 * H2N + 6 * H1N;
constexpr int FV_NOISE_FLOATS = 6 * H1N;

// One block (tile bx, by; z chunk bz).  psi_map / u_map: tensor maps of the stage
// input psi and of the velocity (kernel parameters or global memory); tsmem: the
// block's dynamic shared memory.
//
// Every stencil is split by plane.  A thread owns the same points of the mu,
// flux and tile regions in every plane and keeps, in registers, what each new
// plane contributes to the planes above and below it:
//   lap_SO psi (z) = (6 n1 + 3 n2 + n3 - 80 psi) / 22 with, per plane P, the
//     centre a, the 4 in-plane faces b and the 4 in-plane diagonals d:
//     n1 = b(z) + a(z-1) + a(z+1),  n2 = d(z) + b(z-1) + b(z+1),  n3 = d(z-1) + d(z+1);
//   12 grad mu (q) (Eq. fvgrad, w = 1/18, 1/36) with ex, ey the in-plane face
//     differences, Dx, Dy the signed diagonal sums and Zp = 2 mu + 4 faces:
//     x: 2 ex(q) + Dx(q) + ex(q-1) + ex(q+1),  y: likewise,  z: Zp(q+1) - Zp(q-1);
//   12 div J (z) (the (2/c_s^2) link-average divergence, sum_i w_i c_i = 0 removes
//     J(r)) with Hxy the in-plane face differences of Jx, Jy, Dg the in-plane
//     diagonal terms, Zc = Jz(centre), Z4 = Jz at the 4 in-plane faces:
//     2 Hxy(z) + Dg(z) + 2 (Zc(z+1) - Zc(z-1)) + Hxy(z+1) + Hxy(z-1) + Z4(z+1) - Z4(z-1).
// Shared memory then holds only the current mu, flux and noise planes (two of
// each, by parity) besides the TMA rings: psi plane p arrives, mu of plane p-1 is
// formed, the flux of plane p-2, and the output of plane p-3 completes.
template <int STAGE, bool NOISE>
__device__ __forceinline__ void psi3_fv_tma_block(const CUtensorMap *psi_map, const CUtensorMap *u_map,
                                                  const Psi3Args &a, int *status, int bx, int by, int bz,
                                                  float *tsmem)
{
    if (status && *(volatile int *)status != 0) return;  // an earlier block timed out: skip the work
    float *tps = tsmem;                                   // [T_PSI_DEPTH][TP_SLOT]
    float *tus = tps + T_PSI_DEPTH * TP_SLOT;            // [T_U_DEPTH][TU_SLOT]
    float *smu = tus + T_U_DEPTH * TU_SLOT;              // [2][H2N]     mu plane, by parity
    float *sJ = smu + 2 * H2N;                           // [2][3][H1N]  flux plane, by parity
    float *sX = sJ + 6 * H1N;                            // [2][3][H1N]  noise plane, by parity (NOISE)
    __shared__ __align__(8) uint64_t bar_p[T_PSI_DEPTH], bar_u[T_U_DEPTH];
    __shared__ int s_bad;
    const Geom &g = a.g;
    const int tx = threadIdx.x % PS_TX, ty = threadIdx.x / PS_TX;
    const int x0 = bx * PS_TX, y0 = by * PS_TY, z0 = bz * a.zc;
    const int z1 = min(z0 + a.zc, g.nz);
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < g.nx && y < g.ny;
    const float k22 = a.K * (1.0f / 22.0f);
    const float sdx = sqrtf(2.0f * a.kT * a.M);
    const float m12 = a.M * (1.0f / 12.0f);
    const int pbase = z0 - 3, ubase = z0 - 1;             // first psi / u plane of the chunk
    // mu region: psi-slot offset of every slot point; flux region: mu-frame centre,
    // psi-slot centre, u-slot offset, noise counter id
    // Region points are dealt to threads row segment by row segment: the first
    // 32 columns of every row (a full warp reads 32 consecutive words, free of
    // bank conflicts), then the few remaining columns of all rows.
    int c2[S2], d2[S2], c1[S1], d1[S1], p1[S1], u1[S1], n1[S1];
#pragma unroll
    for (int j = 0; j < S2; ++j) {
        int lx, ly;
        region_point(threadIdx.x + j * PS_NT, H2X, H2Y, lx, ly);
        const bool ok = threadIdx.x + j * PS_NT < H2N;
        c2[j] = ok ? (lx + 2) + TB_X * (ly + 1) : -1;
        d2[j] = lx + H2X * ly;
    }
#pragma unroll
    for (int j = 0; j < S1; ++j) {
        int lx, ly;
        region_point(threadIdx.x + j * PS_NT, H1X, H1Y, lx, ly);
        const bool ok = threadIdx.x + j * PS_NT < H1N;
        c1[j] = ok ? (lx + 1) + H2X * (ly + 1) : -1;
        d1[j] = lx + H1X * ly;
        p1[j] = (lx + 3) + TB_X * (ly + 2);
        u1[j] = (lx + 3) + TB_X * ly;
        n1[j] = wrapi(min(x0 - 1 + lx, g.nx + GX - 1), g.nx) + g.nx * wrapi(min(y0 - 1 + ly, g.ny + GY - 1), g.ny);
    }
    // per-plane partial sums carried between planes (registers)
    float pa[S2][2], pb[S2][2], pd[S2][2];  // psi: centre, faces, diagonals of planes p-2 [0], p-1 [1]
    float G0[S1][3], G1[S1][3];            // 12 grad mu of planes m-1 and m, partly summed
#pragma unroll
    for (int j = 0; j < S2; ++j) pa[j][0] = pa[j][1] = pb[j][0] = pb[j][1] = pd[j][0] = pd[j][1] = 0.f;
#pragma unroll
    for (int j = 0; j < S1; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) G0[j][k] = G1[j][k] = 0.f;
    float D0 = 0.f, D1 = 0.f, N0 = 0.f, N1 = 0.f;  // 12 div of the flux / noise of planes q-1 and q

    if (threadIdx.x == 0) {
        for (int s = 0; s < T_PSI_DEPTH; ++s) mbar_init(&bar_p[s], 1);
        for (int s = 0; s < T_U_DEPTH; ++s) mbar_init(&bar_u[s], 1);
        s_bad = 0;
        fence_barrier_init();
    }
    __syncthreads();
    auto issue_psi = [&](int pp) {
        const int s = (pp - pbase) % T_PSI_DEPTH;
        mbar_expect_tx(&bar_p[s], TP_N * 4);
        tma_load_3d(tps + s * TP_SLOT, psi_map, &bar_p[s], x0, y0, pp + g.gz);
    };
    auto issue_u = [&](int qq) {
        const int s = (qq - ubase) % T_U_DEPTH;
        mbar_expect_tx(&bar_u[s], TU_N * 4);
        tma_load_4d(tus + s * TU_SLOT, u_map, &bar_u[s], x0, y0 + GY - 1, qq + g.gz, 0);
    };
    if (threadIdx.x == 0) {
        issue_psi(pbase);
        issue_psi(pbase + 1);
    }
    int last_p = pbase + 1, last_u = ubase - 1;  // highest plane issued (thread 0)
    int waited_p = pbase - 1, waited_u = ubase - 1;

    // Rotating ring positions, advanced once per plane (no divisions in the loop):
    // psi plane p sits in slot r6 of phase ph6; the velocity of the next flux plane
    // in slot ru of phase uph.
    int r6 = 0, ph6 = 0, ru = 0, uph = 0;
    for (int p = z0 - 3; p <= z1 + 2; ++p) {
        const int s1 = r6 == 0 ? T_PSI_DEPTH - 1 : r6 - 1;  // psi slots of p-1, p-2, p-3
        const int s2 = s1 == 0 ? T_PSI_DEPTH - 1 : s1 - 1;
        const int s3 = s2 == 0 ? T_PSI_DEPTH - 1 : s2 - 1;
        (void)s1;
        // (A) psi plane p has landed: its partials at the mu points, and mu of plane p-1
        if (!mbar_wait(&bar_p[r6], ph6, status)) s_bad = 1;
        waited_p = p;
        {
            const float *P = tps + r6 * TP_SLOT;
            float *dst = smu + ((p - 1) & 1) * H2N;
            const bool emit = p - 1 >= z0 - 2;
#pragma unroll
            for (int j = 0; j < S2; ++j) {
                const int c = c2[j];
                if (c < 0) continue;
                const float ac = P[c];
                const float bc = (P[c - 1] + P[c + 1]) + (P[c - TB_X] + P[c + TB_X]);
                const float dc = (P[c - 1 - TB_X] + P[c + 1 - TB_X]) + (P[c - 1 + TB_X] + P[c + 1 + TB_X]);
                if (emit) {
                    const float ps = pa[j][1];
                    const float nn1 = pb[j][1] + (pa[j][0] + ac);
                    const float nn2 = pd[j][1] + (pb[j][0] + bc);
                    const float nn3 = pd[j][0] + dc;
                    dst[d2[j]] = a.A * ps + a.B * ps * ps * ps - k22 * (6.f * nn1 + 3.f * nn2 + nn3 - 80.f * ps);
                }
                pa[j][0] = pa[j][1];
                pb[j][0] = pb[j][1];
                pd[j][0] = pd[j][1];
                pa[j][1] = ac;
                pb[j][1] = bc;
                pd[j][1] = dc;
            }
        }
        __syncthreads();  // mu plane p-1 complete; every read of the psi slot of p-4 and of the u slot of p-3 done
        if (s_bad) break;
        if (threadIdx.x == 0) {  // refill those slots: psi plane p+2 (used at p+2), u plane p (used at p+2)
            fence_proxy_async();
            if (p + 2 <= z1 + 2) { issue_psi(p + 2); last_p = p + 2; }
            if (a.advect && p >= ubase && p <= z1) { issue_u(p); last_u = p; }
        }
        // (B) mu partials of plane m = p-1 at the flux points; flux (and noise) of plane m-1
        const int m = p - 1;
        if (m >= z0 - 2) {
            const bool emit = m - 1 >= z0 - 1;
            const float *uq = tus;
            if (emit && a.advect) {
                if (!mbar_wait(&bar_u[ru], uph, status)) s_bad = 1;
                waited_u = m - 1;
                uq = tus + ru * TU_SLOT;
                ru = ru == T_U_DEPTH - 1 ? 0 : ru + 1;
                uph ^= ru == 0;
            }
            const float *Mu = smu + (m & 1) * H2N;
            const float *ps = tps + s2 * TP_SLOT;  // psi plane m-1
            float *J = sJ + ((m - 1) & 1) * 3 * H1N;
            float *X = sX + ((m - 1) & 1) * 3 * H1N;
            const int zid = g.nx * g.ny * wrapi(m - 1, g.nz);
#pragma unroll
            for (int j = 0; j < S1; ++j) {
                const int c = c1[j];
                if (c < 0) continue;
                const float mxp = Mu[c + 1], mxm = Mu[c - 1], myp = Mu[c + H2X], mym = Mu[c - H2X];
                const float mpp = Mu[c + 1 + H2X], mpm = Mu[c + 1 - H2X], mmp = Mu[c - 1 + H2X],
                            mmm = Mu[c - 1 - H2X];
                const float ex = mxp - mxm, ey = myp - mym;
                const float Dx = (mpp + mpm) - (mmp + mmm), Dy = (mpp + mmp) - (mpm + mmm);
                const float Zp = 2.f * Mu[c] + ((mxp + mxm) + (myp + mym));
                const float gx = G0[j][0] + ex, gy = G0[j][1] + ey, gz = G0[j][2] + Zp;  // plane m-1, complete
                G0[j][0] = G1[j][0] + (2.f * ex + Dx);
                G0[j][1] = G1[j][1] + (2.f * ey + Dy);
                G0[j][2] = G1[j][2];
                G1[j][0] = ex;
                G1[j][1] = ey;
                G1[j][2] = -Zp;
                if (emit) {
                    const int k = d1[j];
                    float jx = m12 * gx, jy = m12 * gy, jz = m12 * gz;
                    if (a.advect) {
                        const float pv = ps[p1[j]];
                        jx -= uq[u1[j]] * pv;
                        jy -= uq[TB_X * H1Y + u1[j]] * pv;
                        jz -= uq[2 * TB_X * H1Y + u1[j]] * pv;
                    }
                    J[k] = jx;
                    J[H1N + k] = jy;
                    J[2 * H1N + k] = jz;
                    if (NOISE) {
                        float Gn[4];
                        normals4(a.key, a.step, (uint32_t)(n1[j] + zid), 1u, 0u, Gn);
                        X[k] = sdx * Gn[0];
                        X[H1N + k] = sdx * Gn[1];
                        X[2 * H1N + k] = sdx * Gn[2];
                    }
                }
            }
        }
        __syncthreads();  // flux plane p-2 complete
        if (s_bad) break;
        // (C) flux partials of plane q = p-2 at the tile point; the output of plane q-1 completes
        const int q = p - 2;
        if (q >= z0 - 1) {
            const int c = (tx + 1) + H1X * (ty + 1);
            const float *Jx = sJ + (q & 1) * 3 * H1N, *Jy = Jx + H1N, *Jz = Jy + H1N;
            const float hxy = (Jx[c + 1] - Jx[c - 1]) + (Jy[c + H1X] - Jy[c - H1X]);
            const float dg = ((Jx[c + 1 + H1X] + Jy[c + 1 + H1X]) - (Jx[c - 1 - H1X] + Jy[c - 1 - H1X])) +
                             ((Jx[c + 1 - H1X] - Jy[c + 1 - H1X]) - (Jx[c - 1 + H1X] - Jy[c - 1 + H1X]));
            const float zc = Jz[c];
            const float z4 = (Jz[c + 1] + Jz[c - 1]) + (Jz[c + H1X] + Jz[c - H1X]);
            const float dd = D0 + (2.f * zc + hxy + z4);  // plane q-1, complete
            D0 = D1 + (2.f * hxy + dg);
            D1 = hxy - z4 - 2.f * zc;
            float dn = 0.f;
            if (NOISE) {
                const float *Xx = sX + (q & 1) * 3 * H1N, *Xy = Xx + H1N, *Xz = Xy + H1N;
                const float nxy = (Xx[c + 1] - Xx[c - 1]) + (Xy[c + H1X] - Xy[c - H1X]);
                const float ng = ((Xx[c + 1 + H1X] + Xy[c + 1 + H1X]) - (Xx[c - 1 - H1X] + Xy[c - 1 - H1X])) +
                                 ((Xx[c + 1 - H1X] - Xy[c + 1 - H1X]) - (Xx[c - 1 + H1X] - Xy[c - 1 + H1X]));
                const float nzc = Xz[c];
                const float nz4 = (Xz[c + 1] + Xz[c - 1]) + (Xz[c + H1X] + Xz[c - H1X]);
                dn = N0 + (2.f * nzc + nxy + nz4);
                N0 = N1 + (2.f * nxy + ng);
                N1 = nxy - nz4 - 2.f * nzc;
            }
            const int z = q - 1;
            if (z >= z0 && active) {
                const float Dd = dd * (1.f / 12.f);
                const int si = x + g.nx * (y + g.ny * z);
                float out;
                if (STAGE == 1) {
                    const float Dn = NOISE ? dn * (1.f / 12.f) : 0.f;
                    const float pv = tps[s3 * TP_SLOT + (tx + 4) + TB_X * (ty + 3)];
                    out = pv + Dd + Dn;
                    if (a.heun) a.E[si] = pv + 0.5f * Dd + Dn;
                } else {
                    out = a.E[si] + 0.5f * Dd;
                }
                store_padded(a.out, g, x, y, z, out, 3);
            }
        }
        r6 = r6 == T_PSI_DEPTH - 1 ? 0 : r6 + 1;
        ph6 ^= r6 == 0;
    }
    // a bounded wait drains copies still in flight before the block exits
    if (threadIdx.x == 0) {
        for (int pp = waited_p + 1; pp <= last_p; ++pp)
            mbar_wait(&bar_p[(pp - pbase) % T_PSI_DEPTH], ((pp - pbase) / T_PSI_DEPTH) & 1, nullptr);
        for (int qq = waited_u + 1; qq <= last_u; ++qq)
            mbar_wait(&bar_u[(qq - ubase) % T_U_DEPTH], ((qq - ubase) / T_U_DEPTH) & 1, nullptr);
    }
}

template <int STAGE, bool NOISE>
__global__ void __launch_bounds__(PS_NT) psi3_fv_tma_kernel(const __grid_constant__ CUtensorMap psi_map,
                                                            const __grid_constant__ CUtensorMap u_map,
                                                            const TmaArgs ta)
{
    extern __shared__ __align__(1024) float tsmem[];
    psi3_fv_tma_block<STAGE, NOISE>(&psi_map, &u_map, ta.a, ta.status, blockIdx.x, blockIdx.y, blockIdx.z, tsmem);
}

// batched: block b of the launch works on L.psi[b]
template <int STAGE, bool NOISE>
__global__ void __launch_bounds__(PS_NT) psi3_fv_tma_batch_kernel(const BatchLists L)
{
    extern __shared__ __align__(1024) float tsmem[];
    __shared__ Psi3Args sa;
    const BatchBlock b = L.psi[blockIdx.x];
    const BatchRep &r = L.reps[b.rep];
    const long long ds = *L.dstep;
    const int par = (int)(ds & 1);
    if (threadIdx.x == 0) {
        sa.g = r.lb.g;
        sa.psi = STAGE == 1 ? r.psi[par] : r.psis;
        sa.u = r.lb.u;
        sa.out = (STAGE == 1 && r.heun) ? r.psis : r.psi[par ^ 1];
        sa.E = r.E;
        sa.A = r.A;
        sa.B = r.B;
        sa.K = r.K;
        sa.M = r.M;
        sa.kT = r.noise ? r.lb.kT : 0.f;
        sa.advect = r.advect;
        sa.heun = r.heun;
        sa.zc = r.zc;
        sa.key = r.lb.key;
        sa.step = r.lb.step + ds;
    }
    __syncthreads();
    const CUtensorMap *pm = STAGE == 1 ? &r.map_psi[par] : &r.map_psis;
    psi3_fv_tma_block<STAGE, NOISE>(pm, &r.map_u, sa, L.status, b.bx, b.by, b.bz, tsmem);
}

__global__ void advance_kernel(long long *dstep) { *dstep += 1; }

cudaError_t launch_lb3_batch(const BatchLists &L, int storage, bool ghost, bool force, cudaStream_t st);

cudaError_t launch_batch_psi(const BatchLists &L, bool heun, bool noise, cudaStream_t st)
{
    const size_t sm = sizeof(float) * (size_t)FV_SMEM_FLOATS;
    auto go = [&](auto kernel, size_t bytes) {
        cudaError_t r = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (r != cudaSuccess) return r;
        kernel<<<L.npsi, PS_NT, bytes, st>>>(L);
        return cudaGetLastError();
    };
    cudaError_t e = noise ? go(psi3_fv_tma_batch_kernel<1, true>, sm + sizeof(float) * FV_NOISE_FLOATS)
                          : go(psi3_fv_tma_batch_kernel<1, false>, sm);
    if (e != cudaSuccess || !heun) return e;
    return go(psi3_fv_tma_batch_kernel<2, false>, sm);
}

cudaError_t launch_batch_step(const BatchLists &L, int storage, bool ghost, bool force, int scheme_fv, bool heun,
                              bool noise, cudaStream_t st)
{
    if (!scheme_fv) return cudaErrorNotSupported;
    cudaError_t e = launch_lb3_batch(L, storage, ghost, force, st);
    if (e != cudaSuccess) return e;
    e = launch_batch_psi(L, heun, noise, st);
    if (e != cudaSuccess) return e;
    advance_kernel<<<1, 1, 0, st>>>(const_cast<long long *>(L.dstep));
    return cudaGetLastError();
}

template <typename K>
static cudaError_t launch_dyn(K kernel, dim3 grid, size_t smem, cudaStream_t st, const Psi3Args &a)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kernel<<<grid, PS_NT, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t encode_tensor_map_f32(CUtensorMap *map, const void *base, int rank, const uint64_t *dims,
                                  const uint64_t *strides_bytes, const uint32_t *box)
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p)
            return cudaErrorNotSupported;
        fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    cuuint64_t d[5], str[4];
    cuuint32_t bx[5], es[5];
    for (int i = 0; i < rank; ++i) {
        d[i] = dims[i];
        bx[i] = box[i];
        es[i] = 1;
        if (i > 0) str[i - 1] = strides_bytes[i - 1];
    }
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void *>(base), d, str, bx,
                          es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

static cudaError_t launch_fv_tma(const Psi3Args &a, int stage, bool noise, int *status, cudaStream_t st)
{
    const Geom &g = a.g;
    CUtensorMap pm, um;
    const uint64_t pd[3] = {(uint64_t)g.px, (uint64_t)g.py, (uint64_t)g.pz};
    const uint64_t ps[2] = {(uint64_t)g.px * 4, (uint64_t)g.px * g.py * 4};
    const uint32_t pb[3] = {(uint32_t)TB_X, (uint32_t)H3Y, 1};
    cudaError_t e = encode_tensor_map_f32(&pm, a.psi, 3, pd, ps, pb);
    if (e != cudaSuccess) return e;
    const uint64_t ud[4] = {(uint64_t)g.px, (uint64_t)g.py, (uint64_t)g.pz, 3};
    const uint64_t us[3] = {(uint64_t)g.px * 4, (uint64_t)g.px * g.py * 4, (uint64_t)g.pn * 4};
    const uint32_t ub[4] = {(uint32_t)TB_X, (uint32_t)H1Y, 1, 3};
    e = encode_tensor_map_f32(&um, a.u, 4, ud, us, ub);
    if (e != cudaSuccess) return e;
    TmaArgs ta;
    ta.a = a;
    ta.status = status;
    const dim3 grid((g.nx + PS_TX - 1) / PS_TX, (g.ny + PS_TY - 1) / PS_TY, (g.nz + a.zc - 1) / a.zc);
    const size_t sm = sizeof(float) * (size_t)FV_SMEM_FLOATS;
    auto go = [&](auto kernel, size_t bytes) {
        cudaError_t r = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (r != cudaSuccess) return r;
        kernel<<<grid, PS_NT, bytes, st>>>(pm, um, ta);
        return cudaGetLastError();
    };
    if (stage == 1) {
        if (noise) return go(psi3_fv_tma_kernel<1, true>, sm + sizeof(float) * FV_NOISE_FLOATS);
        return go(psi3_fv_tma_kernel<1, false>, sm);
    }
    return go(psi3_fv_tma_kernel<2, false>, sm);
}

cudaError_t launch_psi3(const Geom &g, int scheme, int stage, bool noise, const float *psi, const float *u,
                        float *out, float *E, float A, float B, float K, float M, float kT, int advect, int heun,
                        const PhiloxKey &key, int64_t step, int zc, int *status, cudaStream_t st)
{
    if (zc < PS_ZC_MIN) return cudaErrorInvalidValue;
    Psi3Args a;
    a.g = g;
    a.psi = psi;
    a.u = u;
    a.out = out;
    a.E = E;
    a.A = A;
    a.B = B;
    a.K = K;
    a.M = M;
    a.kT = kT;
    a.advect = advect;
    a.heun = heun;
    a.zc = zc;
    a.key = key;
    a.step = step;
    const dim3 grid((g.nx + PS_TX - 1) / PS_TX, (g.ny + PS_TY - 1) / PS_TY, (g.nz + zc - 1) / zc);
    const size_t base = sizeof(float) * (4 * H3N + 3 * H2N);
    if (scheme == FLB_FV) return launch_fv_tma(a, stage, noise, status, st);
    if (stage == 1) {
        if (noise) return launch_dyn(psi3_fd_kernel<1, true>, grid, base + sizeof(float) * 13 * H1N, st, a);
        return launch_dyn(psi3_fd_kernel<1, false>, grid, base, st, a);
    }
    return launch_dyn(psi3_fd_kernel<2, false>, grid, base, st, a);
}

}  // namespace flb

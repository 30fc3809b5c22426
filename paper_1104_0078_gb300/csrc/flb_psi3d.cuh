// flb_psi3d.cuh -- one finite-volume Runge-Kutta stage of the order-parameter
// equation on a block's column of a 3D box (Sec. V.B), fed by TMA.  Shared by
// the per-phase kernels (flb_psi3d.cu) and the persistent batched kernel
// (flb_persist.cu).
#pragma once

#include "flb_internal.cuh"
#include "flb_tma.cuh"

namespace flb {

constexpr int PS_NT = PS_TX * PS_TY;
constexpr int H3X = PS_TX + 6, H3Y = PS_TY + 6, H3N = H3X * H3Y;  // psi: tile + 3
constexpr int H2X = PS_TX + 4, H2Y = PS_TY + 4, H2N = H2X * H2Y;  // mu: tile + 2
constexpr int H1X = PS_TX + 2, H1Y = PS_TY + 2, H1N = H1X * H1Y;  // flux / noise: tile + 1
constexpr int S3 = (H3N + PS_NT - 1) / PS_NT, S2 = (H2N + PS_NT - 1) / PS_NT, S1 = (H1N + PS_NT - 1) / PS_NT;

struct Psi3Args {
    Geom g;
    const float *psi;  // padded stage input
    const float *u;    // padded velocity (images to radius 1)
    float *out;        // padded stage output (images to radius 3)
    float *E;          // [N] accumulator: Heun E = psi + D/2 + noise; RK4 psi + noise + sum of weighted D
    float A, B, K, M, kT;
    int advect, heun;
    int zc;            // planes per block (the z chunk)
    int rk4;           // RK4: 0 off, else the stage 1..4
    const float *base; // RK4: padded psi^n (stages 2, 3)
    float *Dn;         // RK4: [N] noise increment, written in stage 1, read in stages 2, 3
    PhiloxKey key;
    int64_t step;
    LapW lw;           // FD: the class weights of an App. A Laplacian when lap_w (else SO's)
    int lap_w;
};

// Output of a Runge-Kutta stage at interior site (x, y, z), site index si: pv the
// stage input there (stage 1), D the deterministic increment, eta the noise
// increment (generated in stage 1; Sec. V holds it fixed over the step).
//   Euler / Heun (Sec. V): stage 1 psi + D + eta (Heun also E = psi + D/2 + eta),
//     stage 2 E + D/2.
//   RK4: k_s = D_s + eta; stage 1 writes psi + k1/2 and E = psi + eta + D1/6 and
//     keeps eta; stages 2, 3 write psi^n + k2/2, psi^n + k3 and add D_s/3 to E;
//     stage 4 writes E + D4/6 = psi^n + (k1 + 2 k2 + 2 k3 + k4)/6.
//   RK false compiles the RK4 branches out (only for launches with a.rk4 == 0).
template <int STAGE, bool COH, bool RK = true>
__device__ __forceinline__ float rk_stage_out(const Psi3Args &a, int x, int y, int z, int si, float pv, float D,
                                              float eta)
{
    if (RK && a.rk4) {
        constexpr float sixth = 1.f / 6.f, third = 1.f / 3.f;
        if (a.rk4 == 1) {
            a.E[si] = pv + eta + sixth * D;
            a.Dn[si] = eta;
            return pv + 0.5f * (D + eta);
        }
        const float e = COH ? __ldcg(a.E + si) : a.E[si];
        if (a.rk4 == 4) return e + sixth * D;
        const float n = COH ? __ldcg(a.Dn + si) : a.Dn[si];
        const float b = COH ? __ldcg(a.base + a.g.pidx32(x, y, z)) : a.base[a.g.pidx32(x, y, z)];
        a.E[si] = e + third * D;
        return a.rk4 == 2 ? b + 0.5f * (D + n) : b + D + n;
    }
    if (STAGE == 1) {
        if (a.heun) a.E[si] = pv + 0.5f * D + eta;
        return pv + D + eta;
    }
    return (COH ? __ldcg(a.E + si) : a.E[si]) + 0.5f * D;
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
constexpr int TM_N = TB_X * H2Y;                           // mu plane / slot floats
constexpr int TM_SLOT = ((TM_N * 4 + 127) / 128) * 32;
constexpr int TJ_N = TB_X * H1Y;                           // flux / noise plane floats (one component)
constexpr int T_U_DEPTH = 3, T_MU_DEPTH = 3;
// psi ring slots: planes p-2SK-1 .. p+2 of an iteration (SK, the phase skew of
// psi3_fv_tma_block: 2 for row pairs, 1 for one point per thread)
template <class V>
__host__ __device__ constexpr int psi_ring() { return V::L == 2 ? 8 : 6; }

// dynamic shared memory of a stage block (floats), without and with the mu ring
template <class V>
constexpr int fv_smem_floats() { return psi_ring<V>() * TP_SLOT + T_U_DEPTH * TU_SLOT + 2 * TM_N + 6 * TJ_N; }
template <class V>
constexpr int fv_mu_smem_floats()
{
    return psi_ring<V>() * TP_SLOT + T_U_DEPTH * TU_SLOT + T_MU_DEPTH * TM_SLOT + 6 * TJ_N;
}
constexpr int FV_NOISE_FLOATS = 6 * TJ_N;

// Lane-generic access to a shared-memory plane: lane l of the value at index c
// sits at c + l * loff (the row pairs of a region lie loff apart).
template <class V>
__device__ __forceinline__ V lds_v(const float *P, int c, int loff)
{
    float t[V::L];
#pragma unroll
    for (int l = 0; l < V::L; ++l) t[l] = P[c + l * loff];
    return vmake<V>(t);
}
template <class V>
__device__ __forceinline__ void sts_v(float *P, int c, int loff, V v)
{
#pragma unroll
    for (int l = 0; l < V::L; ++l) P[c + l * loff] = v.lane(l);
}

// mu_so of flb_internal.cuh in lane arithmetic (the same explicitly rounded
// operations, so a lane gets mu_so's bits)
template <class V>
__device__ __forceinline__ V mu_so_v(float A, float B, float k22, V ps, V n1, V n2, V n3)
{
    const V l22 = vfma(n1, 6.f, vfma(n2, 3.f, vfma(ps, -80.f, n3)));
    return vfma(l22, -k22, vfma((ps * ps) * B, ps, ps * A));
}

// Threads of a stage block: one output point per thread (F1: 512), or a pair of
// output rows y and y + TY/2 per thread in the lanes of packed FP32 (F2: 256).
template <class V>
__host__ __device__ constexpr int stage_threads() { return V::L == 1 ? PS_NT : PS_NT / 2; }

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
// formed, the flux of plane p-2, and the output of plane p-3 completes.  Every
// plane keeps the psi slot's row pitch TB_X and columns (x = x0 - 4 + c); the mu
// plane starts at y = y0 - 2 and the flux, noise and u planes at y = y0 - 1, so a
// point's index in each is its psi-slot index less TB_X or 2 TB_X.
//
// Lanes: with V = F2 a thread works the point pairs (x, y) and (x, y + H/2) of
// every region of height H (mu 20, flux 18, tile 16 rows) in the two lanes of
// packed FP32 registers, and the block has 256 threads; with V = F1 one point
// and 512 threads.  Every FP32 operation is explicitly rounded (a product by a
// scalar that feeds an add is formed per lane, vmul_sep of flb_lane.cuh), so
// both give the same bits; the random numbers, the loads and the stores run per
// lane.
//
// Q15: the FV operators of D3Q15 (faces w = 1/9, corners 1/72), in units of 1/24:
//   24 grad mu (q): x: 8 ex(q) + Dx(q-1) + Dx(q+1),  y: likewise,
//     z: Zq(q+1) - Zq(q-1) with Zq = 8 mu + the 4 in-plane corners;
//   24 div J (z) = 8 Hxy(z) + 8 (Zc(z+1) - Zc(z-1)) + Dg(z+1) + Dg(z-1) + C4(z+1) - C4(z-1)
//     with Dg the corners' c_x Jx + c_y Jy and C4 the corners' Jz of a plane.
//
// MU_IN (stage 1 only): mu of the stage input psi^n already sits in the mu field
// (mu_map, valid to 2 ghost layers), written for the force of the same step.  Its
// planes then come by TMA, like psi and u, into a third ring ([TY+4][TX+8], column
// c <-> x = x0 - 4 + c, row r <-> y = y0 - 2 + r), and the block skips forming mu.
template <int STAGE, bool NOISE, bool COH = false, bool KEY_R0 = false, bool RK = true, bool MU_IN = false,
          bool Q15 = false, class V = F1>
__device__ __forceinline__ void psi3_fv_tma_block(const CUtensorMap *psi_map, const CUtensorMap *u_map,
                                                  const Psi3Args &a, int *status, int bx, int by, int bz,
                                                  float *tsmem, const CUtensorMap *mu_map = nullptr)
{
    static_assert(!MU_IN || STAGE == 1, "mu of psi^n is the input of stage 1 only");
    constexpr int L = V::L, NT = stage_threads<V>();
    constexpr int LO2 = (H2Y / 2) * TB_X, LO1 = (H1Y / 2) * TB_X, LO0 = (PS_TY / 2) * TB_X;  // lane 1's offsets
    constexpr int LR2 = L == 1 ? 0 : LO2, LR1 = L == 1 ? 0 : LO1, LR0 = L == 1 ? 0 : LO0;
    constexpr int HH2 = H2Y / L, HH1 = H1Y / L;  // rows of the mu and flux regions per lane
    constexpr int SS2 = (H2X * HH2 + NT - 1) / NT, SS1 = (H1X * HH1 + NT - 1) / NT;
    if (status && *(volatile int *)status != 0) return;  // an earlier block timed out: skip the work
    const int rk4 = RK ? a.rk4 : 0;                       // RK false: a launch without RK4
    constexpr int TD = psi_ring<V>();
    float *tps = tsmem;                                   // [TD][TP_SLOT]
    float *tus = tps + TD * TP_SLOT;                     // [T_U_DEPTH][TU_SLOT]
    float *smu = tus + T_U_DEPTH * TU_SLOT;              // [2][TM_N]    mu plane, by parity
    float *tms = smu;                                    // MU_IN: [T_MU_DEPTH][TM_SLOT] instead
    float *sJ = smu + (MU_IN ? T_MU_DEPTH * TM_SLOT : 2 * TM_N);  // [2][3][TJ_N] flux plane, by parity
    float *sX = sJ + 6 * TJ_N;                           // [2][3][TJ_N] noise plane, by parity (NOISE)
    __shared__ __align__(8) uint64_t bar_p[TD], bar_u[T_U_DEPTH], bar_m[T_MU_DEPTH];
    __shared__ int s_bad;
    const Geom &g = a.g;
    const int tx = threadIdx.x % PS_TX, ty = threadIdx.x / PS_TX;  // lane l's output row: ty + l TY/2
    const int x0 = bx * PS_TX, y0 = by * PS_TY, z0 = bz * a.zc;
    const int z1 = min(z0 + a.zc, g.nz);
    const int x = x0 + tx;
    int yl[L];
    bool act[L], inner[L];
    int coff[L];
#pragma unroll
    for (int l = 0; l < L; ++l) {
        yl[l] = y0 + ty + l * (PS_TY / 2);
        act[l] = x < g.nx && yl[l] < g.ny;
        // the output column has no periodic image within 3 cells in x and y: its
        // interior planes are stored with one plain store
        inner[l] = x >= 3 && x < g.nx - 3 && yl[l] >= 3 && yl[l] < g.ny - 3;
        coff[l] = (x + GX) + g.px * (yl[l] + GY);
    }
    const float k22 = a.K * (1.0f / 22.0f);
    const float sdx = sqrtf(2.0f * a.kT * a.M);
    const float mg = a.M * (Q15 ? 1.0f / 24.0f : 1.0f / 12.0f);  // M over the gradient's unit
    constexpr float DIV = Q15 ? 1.0f / 24.0f : 1.0f / 12.0f;      // the divergence's unit
    const int pbase = z0 - 3, ubase = z0 - 1, mbase = z0 - 2;  // first psi / u / mu plane of the chunk
    // psi-slot index of every mu-region point (c2) and flux-region point (p1) of
    // lane 0, -1 off the region; noise counter id of every flux-region point.
    // Region points are dealt to threads row segment by row segment: the first
    // 32 columns of every row (a full warp reads 32 consecutive words, free of
    // bank conflicts), then the few remaining columns of all rows.
    int c2[SS2], p1[SS1], n1[SS1][L];
#pragma unroll
    for (int j = 0; j < SS2; ++j) {
        int lx, ly;
        region_point(threadIdx.x + j * NT, H2X, HH2, lx, ly);
        const bool ok = threadIdx.x + j * NT < H2X * HH2;
        c2[j] = ok ? (lx + 2) + TB_X * (ly + 1) : -1;
    }
#pragma unroll
    for (int j = 0; j < SS1; ++j) {
        int lx, ly;
        region_point(threadIdx.x + j * NT, H1X, HH1, lx, ly);
        const bool ok = threadIdx.x + j * NT < H1X * HH1;
        p1[j] = ok ? (lx + 3) + TB_X * (ly + 2) : -1;
#pragma unroll
        for (int l = 0; l < L; ++l)
            n1[j][l] = wrapi(min(x0 - 1 + lx, g.nx + GX - 1), g.nx) +
                       g.nx * wrapi(min(y0 - 1 + ly + l * HH1, g.ny + GY - 1), g.ny);
    }
    // per-plane partial sums carried between planes (registers)
    const V zero = V::bc(0.f);
    V pa[SS2][2], pb[SS2][2], pd[SS2][2];  // psi: centre, faces, diagonals of planes p-2 [0], p-1 [1]
    V G0[SS1][3], G1[SS1][3];            // 12 grad mu of planes m-1 and m, partly summed
#pragma unroll
    for (int j = 0; j < SS2; ++j) pa[j][0] = pa[j][1] = pb[j][0] = pb[j][1] = pd[j][0] = pd[j][1] = zero;
#pragma unroll
    for (int j = 0; j < SS1; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) G0[j][k] = G1[j][k] = zero;
    V D0 = zero, D1 = zero, N0 = zero, N1 = zero;  // 12 (24) div of the flux / noise of planes q-1 and q

    if (threadIdx.x == 0) {
        for (int s = 0; s < TD; ++s) mbar_init(&bar_p[s], 1);
        for (int s = 0; s < T_U_DEPTH; ++s) mbar_init(&bar_u[s], 1);
        if (MU_IN)
            for (int s = 0; s < T_MU_DEPTH; ++s) mbar_init(&bar_m[s], 1);
        s_bad = 0;
        fence_barrier_init();
    }
    __syncthreads();
    auto issue_psi = [&](int pp) {
        const int s = (pp - pbase) % TD;
        mbar_expect_tx(&bar_p[s], TP_N * 4);
        tma_load_3d(tps + s * TP_SLOT, psi_map, &bar_p[s], x0, y0, pp + g.gz);
    };
    auto issue_u = [&](int qq) {
        const int s = (qq - ubase) % T_U_DEPTH;
        mbar_expect_tx(&bar_u[s], TU_N * 4);
        tma_load_4d(tus + s * TU_SLOT, u_map, &bar_u[s], x0, y0 + GY - 1, qq + g.gz, 0);
    };
    auto issue_mu = [&](int mm) {
        const int s = (mm - mbase) % T_MU_DEPTH;
        mbar_expect_tx(&bar_m[s], TM_N * 4);
        tma_load_3d(tms + s * TM_SLOT, mu_map, &bar_m[s], x0, y0 + GY - 2, mm + g.gz);
    };
    constexpr int SK = L == 2 ? 2 : 1;  // phase skew (below)
    static_assert(TD >= 2 * SK + 4, "psi ring holds planes p-2SK-1 .. p+2");
    if (threadIdx.x == 0)
        for (int k = 0; k <= SK; ++k) issue_psi(pbase + k);
    int last_p = pbase + SK, last_u = ubase - 1, last_m = mbase - 1;  // highest plane issued (thread 0)
    int waited_p = pbase - 1, waited_u = ubase - 1, waited_m = mbase - 1;

    // Iteration p forms mu of plane p-1 (A), the flux of plane m-1 from mu of
    // m = p-SK (B) and the output of plane q-1 from the flux of q = p-2 SK (C).
    // SK = 2 (row pairs): each phase reads only what the previous iteration
    // wrote, so one barrier per iteration suffices.  SK = 1 (one point per
    // thread, the persistent kernel): two barriers per iteration, after A and
    // after B, two planes fewer per z chunk and a ring of 6 slots.  Each refill
    // (psi plane p+SK+1, u plane p+1-SK, mu plane p+2-SK) goes into slots read
    // before the last barrier.  Ring positions rotate once per iteration (no
    // divisions in the loop): psi plane p in slot r6 of phase ph6; the velocity
    // and mu rings advance on use (slot ru / rm of phase uph / mph).
    auto refill = [&](int p) {
        if (threadIdx.x == 0) {
            fence_proxy_async();
            const int pp = p + SK + 1, uu = p + 1 - SK, mm = p + 2 - SK;
            if (pp <= z1 + 2) { issue_psi(pp); last_p = pp; }
            if (a.advect && uu >= ubase && uu <= z1) { issue_u(uu); last_u = uu; }
            if (MU_IN && mm >= mbase && mm <= z1 + 1) { issue_mu(mm); last_m = mm; }
        }
    };
    int r6 = 0, ph6 = 0, ru = 0, uph = 0, rm = 0, mph = 0;
    for (int p = z0 - 3; p <= z1 + 2 * SK; ++p) {
        const int s3 = r6 >= SK + 1 ? r6 - SK - 1 : r6 - SK - 1 + TD;  // psi slots of planes m-1 and q-1
        const int s5 = r6 >= 2 * SK + 1 ? r6 - 2 * SK - 1 : r6 - 2 * SK - 1 + TD;
        const int pe = p - 2 * SK - 1;  // this iteration's output plane
        // Heun stage 2 and RK4 stages 2-4: the accumulator E (and for RK4 stages 2
        // and 3 the noise increment and psi^n) of this iteration's output plane
        // pe are loaded now, so that their latency hides behind the plane's work
        float e_pre[L], n_pre[L], b_pre[L];
#pragma unroll
        for (int l = 0; l < L; ++l) {
            e_pre[l] = n_pre[l] = b_pre[l] = 0.f;
            if (STAGE == 2 && act[l] && pe >= z0) {
                const int sp = x + g.nx * (yl[l] + g.ny * pe);
                if (!rk4 || rk4 > 1) e_pre[l] = COH ? __ldcg(a.E + sp) : a.E[sp];
                if (rk4 == 2 || rk4 == 3) {
                    const int bp = g.pidx32(x, yl[l], pe);
                    n_pre[l] = COH ? __ldcg(a.Dn + sp) : a.Dn[sp];
                    b_pre[l] = COH ? __ldcg(a.base + bp) : a.base[bp];
                }
            }
        }
        // (A) psi plane p has landed: its partials at the mu points, and mu of plane p-1
        if (p <= z1 + 2) {
            if (!mbar_wait(&bar_p[r6], ph6, status)) s_bad = 1;
            waited_p = p;
        }
        if (!MU_IN && p <= z1 + 2) {
            const float *P = tps + r6 * TP_SLOT;
            float *dst = smu + ((p - 1) & 1) * TM_N;
            const bool emit = p - 1 >= z0 - 2;
#pragma unroll
            for (int j = 0; j < SS2; ++j) {
                const int c = c2[j];
                if (c < 0) continue;
                const V ac = lds_v<V>(P, c, LR2);
                const V bc = (lds_v<V>(P, c - 1, LR2) + lds_v<V>(P, c + 1, LR2)) +
                             (lds_v<V>(P, c - TB_X, LR2) + lds_v<V>(P, c + TB_X, LR2));
                const V dc = (lds_v<V>(P, c - 1 - TB_X, LR2) + lds_v<V>(P, c + 1 - TB_X, LR2)) +
                             (lds_v<V>(P, c - 1 + TB_X, LR2) + lds_v<V>(P, c + 1 + TB_X, LR2));
                if (emit) {
                    const V nn1 = pb[j][1] + (pa[j][0] + ac);
                    const V nn2 = pd[j][1] + (pb[j][0] + bc);
                    const V nn3 = pd[j][0] + dc;
                    // mu plane row 0 <-> psi-slot row 1
                    sts_v<V>(dst, c - TB_X, LR2, mu_so_v<V>(a.A, a.B, k22, pa[j][1], nn1, nn2, nn3));
                }
                pa[j][0] = pa[j][1];
                pb[j][0] = pb[j][1];
                pd[j][0] = pd[j][1];
                pa[j][1] = ac;
                pb[j][1] = bc;
                pd[j][1] = dc;
            }
        }
        if (SK == 1) {
            __syncthreads();  // mu plane p-1 complete; the slots to refill read
            if (s_bad) break;
            refill(p);
        }
        // (B) mu partials of plane m = p-SK (complete since the last barrier) at the
        // flux points; flux (and noise) of plane m-1
        const int m = p - SK;
        if (m >= z0 - 2 && m <= z1 + 1) {
            const bool emit = m - 1 >= z0 - 1;
            const float *uq = tus;
            if (emit && a.advect) {
                if (!mbar_wait(&bar_u[ru], uph, status)) s_bad = 1;
                waited_u = m - 1;
                uq = tus + ru * TU_SLOT;
                ru = ru == T_U_DEPTH - 1 ? 0 : ru + 1;
                uph ^= ru == 0;
            }
            const float *Mu = smu + (m & 1) * TM_N;
            if (MU_IN) {  // mu plane m has landed in its ring slot
                if (!mbar_wait(&bar_m[rm], mph, status)) s_bad = 1;
                waited_m = m;
                Mu = tms + rm * TM_SLOT;
                rm = rm == T_MU_DEPTH - 1 ? 0 : rm + 1;
                mph ^= rm == 0;
            }
            const float *ps = tps + s3 * TP_SLOT;  // psi plane m-1
            float *J = sJ + ((m - 1) & 1) * 3 * TJ_N;
            float *X = sX + ((m - 1) & 1) * 3 * TJ_N;
            const int zid = g.nx * g.ny * wrapi(m - 1, g.nz);
#pragma unroll
            for (int j = 0; j < SS1; ++j) {
                if (p1[j] < 0) continue;
                const int c = p1[j] - TB_X;  // in the mu plane
                const V mxp = lds_v<V>(Mu, c + 1, LR1), mxm = lds_v<V>(Mu, c - 1, LR1);
                const V myp = lds_v<V>(Mu, c + TB_X, LR1), mym = lds_v<V>(Mu, c - TB_X, LR1);
                const V mpp = lds_v<V>(Mu, c + 1 + TB_X, LR1), mpm = lds_v<V>(Mu, c + 1 - TB_X, LR1);
                const V mmp = lds_v<V>(Mu, c - 1 + TB_X, LR1), mmm = lds_v<V>(Mu, c - 1 - TB_X, LR1);
                const V ex = mxp - mxm, ey = myp - mym;
                const V Dx = (mpp + mpm) - (mmp + mmm), Dy = (mpp + mmp) - (mpm + mmm);
                V gx, gy, gz;  // plane m-1, complete
                if (Q15) {
                    const V Zq = vfma(lds_v<V>(Mu, c, LR1), 8.f, (mpp + mpm) + (mmp + mmm));
                    gx = G0[j][0] + Dx;
                    gy = G0[j][1] + Dy;
                    gz = G0[j][2] + Zq;
                    G0[j][0] = vfma(ex, 8.f, G1[j][0]);
                    G0[j][1] = vfma(ey, 8.f, G1[j][1]);
                    G0[j][2] = G1[j][2];
                    G1[j][0] = Dx;
                    G1[j][1] = Dy;
                    G1[j][2] = Zq * -1.0f;
                } else {
                    const V Zp = vfma(lds_v<V>(Mu, c, LR1), 2.f, (mxp + mxm) + (myp + mym));
                    gx = G0[j][0] + ex;
                    gy = G0[j][1] + ey;
                    gz = G0[j][2] + Zp;
                    G0[j][0] = G1[j][0] + vfma(ex, 2.f, Dx);
                    G0[j][1] = G1[j][1] + vfma(ey, 2.f, Dy);
                    G0[j][2] = G1[j][2];
                    G1[j][0] = ex;
                    G1[j][1] = ey;
                    G1[j][2] = Zp * -1.0f;
                }
                if (emit) {
                    const int k = p1[j] - 2 * TB_X;  // in the flux, noise and u planes
                    V jx = gx * mg, jy = gy * mg, jz = gz * mg;
                    if (a.advect) {  // J = M grad mu - u psi
                        const V npv = lds_v<V>(ps, p1[j], LR1) * -1.0f;
                        jx = vfma(lds_v<V>(uq, k, LR1), npv, jx);
                        jy = vfma(lds_v<V>(uq, TB_X * H1Y + k, LR1), npv, jy);
                        jz = vfma(lds_v<V>(uq, 2 * TB_X * H1Y + k, LR1), npv, jz);
                    }
                    sts_v<V>(J, k, LR1, jx);
                    sts_v<V>(J, TJ_N + k, LR1, jy);
                    sts_v<V>(J, 2 * TJ_N + k, LR1, jz);
                    if (NOISE) {
                        // three N(0, 2 kT M) normals per node, the radius scaled by
                        // sqrt(2 kT M): the Box-Muller pairs of the first two words of
                        // the node's Philox block, one packed evaluation per node
#pragma unroll
                        for (int l = 0; l < L; ++l) {
                            float Gn[4];
                            normals<2, KEY_R0, true>(a.key, a.step, (uint32_t)(n1[j][l] + zid), 1u, 0u, Gn, sdx);
                            X[k + l * LR1] = Gn[0];
                            X[TJ_N + k + l * LR1] = Gn[1];
                            X[2 * TJ_N + k + l * LR1] = Gn[2];
                        }
                    }
                }
            }
        }
        if (SK == 1) {
            __syncthreads();  // flux plane p-2 complete
            if (s_bad) break;
        }
        // (C) flux partials of plane q = p-2 SK (complete since the last barrier) at
        // the tile point; the output of plane q-1 completes
        const int q = p - 2 * SK;
        if (q >= z0 - 1) {
            const int c = (tx + 4) + TB_X * (ty + 1);  // the tile point (lane 0) in the flux plane
            const float *Jx = sJ + (q & 1) * 3 * TJ_N, *Jy = Jx + TJ_N, *Jz = Jy + TJ_N;
            const V hxy = (lds_v<V>(Jx, c + 1, LR0) - lds_v<V>(Jx, c - 1, LR0)) +
                          (lds_v<V>(Jy, c + TB_X, LR0) - lds_v<V>(Jy, c - TB_X, LR0));
            const V dg = ((lds_v<V>(Jx, c + 1 + TB_X, LR0) + lds_v<V>(Jy, c + 1 + TB_X, LR0)) -
                          (lds_v<V>(Jx, c - 1 - TB_X, LR0) + lds_v<V>(Jy, c - 1 - TB_X, LR0))) +
                         ((lds_v<V>(Jx, c + 1 - TB_X, LR0) - lds_v<V>(Jy, c + 1 - TB_X, LR0)) -
                          (lds_v<V>(Jx, c - 1 + TB_X, LR0) - lds_v<V>(Jy, c - 1 + TB_X, LR0)));
            const V zc = lds_v<V>(Jz, c, LR0);
            V dd;  // plane q-1, complete
            if (Q15) {
                const V c4 = (lds_v<V>(Jz, c + 1 + TB_X, LR0) + lds_v<V>(Jz, c + 1 - TB_X, LR0)) +
                             (lds_v<V>(Jz, c - 1 + TB_X, LR0) + lds_v<V>(Jz, c - 1 - TB_X, LR0));
                dd = D0 + (vfma(zc, 8.f, dg) + c4);
                D0 = vfma(hxy, 8.f, D1);
                D1 = vfma(zc, -8.f, dg - c4);
            } else {
                const V z4 = (lds_v<V>(Jz, c + 1, LR0) + lds_v<V>(Jz, c - 1, LR0)) +
                             (lds_v<V>(Jz, c + TB_X, LR0) + lds_v<V>(Jz, c - TB_X, LR0));
                dd = D0 + (vfma(zc, 2.f, hxy) + z4);
                D0 = D1 + vfma(hxy, 2.f, dg);
                D1 = vfma(zc, -2.f, hxy - z4);
            }
            V dn = zero;
            if (NOISE) {
                const float *Xx = sX + (q & 1) * 3 * TJ_N, *Xy = Xx + TJ_N, *Xz = Xy + TJ_N;
                const V nxy = (lds_v<V>(Xx, c + 1, LR0) - lds_v<V>(Xx, c - 1, LR0)) +
                              (lds_v<V>(Xy, c + TB_X, LR0) - lds_v<V>(Xy, c - TB_X, LR0));
                const V ng = ((lds_v<V>(Xx, c + 1 + TB_X, LR0) + lds_v<V>(Xy, c + 1 + TB_X, LR0)) -
                              (lds_v<V>(Xx, c - 1 - TB_X, LR0) + lds_v<V>(Xy, c - 1 - TB_X, LR0))) +
                             ((lds_v<V>(Xx, c + 1 - TB_X, LR0) - lds_v<V>(Xy, c + 1 - TB_X, LR0)) -
                              (lds_v<V>(Xx, c - 1 + TB_X, LR0) - lds_v<V>(Xy, c - 1 + TB_X, LR0)));
                const V nzc = lds_v<V>(Xz, c, LR0);
                if (Q15) {
                    const V n4 = (lds_v<V>(Xz, c + 1 + TB_X, LR0) + lds_v<V>(Xz, c + 1 - TB_X, LR0)) +
                                 (lds_v<V>(Xz, c - 1 + TB_X, LR0) + lds_v<V>(Xz, c - 1 - TB_X, LR0));
                    dn = N0 + (vfma(nzc, 8.f, ng) + n4);
                    N0 = vfma(nxy, 8.f, N1);
                    N1 = vfma(nzc, -8.f, ng - n4);
                } else {
                    const V nz4 = (lds_v<V>(Xz, c + 1, LR0) + lds_v<V>(Xz, c - 1, LR0)) +
                                  (lds_v<V>(Xz, c + TB_X, LR0) + lds_v<V>(Xz, c - TB_X, LR0));
                    dn = N0 + (vfma(nzc, 2.f, nxy) + nz4);
                    N0 = N1 + vfma(nxy, 2.f, ng);
                    N1 = vfma(nzc, -2.f, nxy - nz4);
                }
            }
            const int z = q - 1;
            if (z >= z0) {
                // Runge-Kutta stage output (Sec. V; the noise increment held fixed):
                //   Euler / Heun: stage 1 psi + D + eta (Heun also E = psi + D/2 + eta),
                //     stage 2 E + D/2;
                //   RK4 (k_s = D_s + eta): stage 1 psi + k1/2 with E = psi + eta + D1/6
                //     and the increment kept; stages 2, 3 psi^n + k2/2, psi^n + k3 with
                //     E += D_s/3; stage 4 E + D4/6.
                const V Dd = vmul_sep(dd, DIV);  // rounded before the adds below
                const V Dn = (STAGE == 1 && NOISE) ? vmul_sep(dn, DIV) : zero;
                const V pv = STAGE == 1 ? lds_v<V>(tps + s5 * TP_SLOT, (tx + 4) + TB_X * (ty + 3), LR0) : zero;
                V out, Ew = zero;
                bool wE = false, wN = false;
                if (STAGE == 2 && !rk4) {
                    out = vfma(Dd, 0.5f, vmake<V>(e_pre));
                } else if (STAGE == 2 && rk4 == 4) {
                    out = vfma(Dd, 1.f / 6.f, vmake<V>(e_pre));
                } else if (STAGE == 2 && rk4 >= 2) {  // stages 2 and 3
                    Ew = vfma(Dd, 1.f / 3.f, vmake<V>(e_pre));
                    wE = true;
                    const V bn = vmake<V>(b_pre), nn = vmake<V>(n_pre);
                    out = rk4 == 2 ? vfma(Dd + nn, 0.5f, bn) : (bn + Dd) + nn;
                } else if (RK && rk4 == 1) {  // RK4 stage 1
                    Ew = vfma(Dd, 1.f / 6.f, pv + Dn);
                    wE = wN = true;
                    out = vfma(Dd + Dn, 0.5f, pv);
                } else {  // Euler / Heun stage 1
                    if (a.heun) {
                        Ew = vfma(Dd, 0.5f, pv) + Dn;
                        wE = true;
                    }
                    out = (pv + Dd) + Dn;
                }
#pragma unroll
                for (int l = 0; l < L; ++l) {
                    if (!act[l]) continue;
                    const int si = x + g.nx * (yl[l] + g.ny * z);
                    if (wE) a.E[si] = Ew.lane(l);
                    if (wN) a.Dn[si] = Dn.lane(l);
                    if (inner[l] && z >= 3 && z < g.nz - 3)
                        a.out[coff[l] + g.px * g.py * (z + g.gz)] = out.lane(l);
                    else
                        store_padded(a.out, g, x, yl[l], z, out.lane(l), 3);
                }
            }
        }
        if (SK == 2) {
            // mu plane p-1 and flux plane p-3 complete; every read of the psi slot
            // of p-5, of the u slot of p-3 and of the mu slot of p-2 done
            __syncthreads();
            if (s_bad) break;
            refill(p);
        }
        r6 = r6 == TD - 1 ? 0 : r6 + 1;
        ph6 ^= r6 == 0;
    }
    // a bounded wait drains copies still in flight before the block exits
    if (threadIdx.x == 0) {
        for (int pp = waited_p + 1; pp <= last_p; ++pp)
            mbar_wait(&bar_p[(pp - pbase) % TD], ((pp - pbase) / TD) & 1, nullptr);
        for (int qq = waited_u + 1; qq <= last_u; ++qq)
            mbar_wait(&bar_u[(qq - ubase) % T_U_DEPTH], ((qq - ubase) / T_U_DEPTH) & 1, nullptr);
        if (MU_IN)
            for (int mm = waited_m + 1; mm <= last_m; ++mm)
                mbar_wait(&bar_m[(mm - mbase) % T_MU_DEPTH], ((mm - mbase) / T_MU_DEPTH) & 1, nullptr);
        // the barriers may be initialised again by a later task of a persistent block
        for (int k = 0; k < TD; ++k) mbar_inval(&bar_p[k]);
        for (int k = 0; k < T_U_DEPTH; ++k) mbar_inval(&bar_u[k]);
        if (MU_IN)
            for (int k = 0; k < T_MU_DEPTH; ++k) mbar_inval(&bar_m[k]);
    }
}

// Stage arguments of replica r at device step ds, written by one thread.
__device__ __forceinline__ void psi_batch_args(const BatchRep &r, long long ds, int stage, Psi3Args &sa)
{
    const int par = (int)(ds & 1);
    sa.g = r.lb.g;
    sa.psi = stage == 1 ? r.psi[par] : r.psis;
    sa.u = r.lb.u;
    sa.out = (stage == 1 && r.heun) ? r.psis : r.psi[par ^ 1];
    sa.E = r.E;
    sa.A = r.A;
    sa.B = r.B;
    sa.K = r.K;
    sa.M = r.M;
    sa.kT = r.noise ? r.lb.kT : 0.f;
    sa.advect = r.advect;
    sa.heun = r.heun;
    sa.zc = r.zc;
    sa.rk4 = 0;
    sa.base = nullptr;
    sa.Dn = nullptr;
    sa.key = r.lb.key;
    sa.step = r.lb.step + ds;
    sa.lap_w = 0;
}

}  // namespace flb

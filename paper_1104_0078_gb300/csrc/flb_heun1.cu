// flb_heun1.cu -- the Heun step of the finite-volume order-parameter equation in
// one pass (Sec. V.B with the Runge-Kutta step of Sec. V, noise held fixed), by
// halo recompute: a block owns a TX x TY column tile and a z chunk, and runs
// stage 1 on the tile + 3 region so that stage 2 finds psi* on every point its
// stencils reach.  psi*, the accumulator E and the noise never leave shared
// memory; psi^n and u are the only fields read, psi^{n+1} the only one written.
//
// Per z plane p of psi^n, the block works a fixed distance behind it:
//   1  psi^n(p)            on tile + 6  (global, periodic, loaded a plane ahead)
//   2  mu^n(p-1)           on tile + 5  mu = A psi + B psi^3 - K lap_SO psi
//   3  J(p-2), xi(p-2)     on tile + 4  J = M grad_FV mu - u psi, xi ~ N(0, 2 kT M)
//   4  psi*, E (p-3)       on tile + 3  psi* = psi + D + eta, E = psi + D/2 + eta,
//                                       D = div_FV J, eta = div_FV xi
//   5  mu*(p-4)            on tile + 2
//   6  J*(p-5)             on tile + 1  J* = M grad_FV mu* - u psi*
//   7  psi^{n+1}(p-6)      on the tile  E + div_FV J* / 2
// with grad_FV mu = (1/c_s^2) sum_i w_i c_i mu(r + c_i) (Eq. fvgrad) and
// div_FV J = (1/c_s^2) sum_i w_i c_i . J(r + c_i) (the link average of Eq. fvflux
// with the (2/c_s^2) divergence; sum_i w_i c_i = 0 removes J(r)), D3Q19 weights
// 1/18 (faces), 1/36 (edges): 12 grad_a = 2 (face difference) + the 8 edge
// neighbours signed by c_a.  The node noise uses the counters of the two-pass
// stage 1 (Philox stream 1, block 0, the node's periodic site id), so both
// forms draw the same noise.  Every region is indexed in its own frame; each
// stencil reads three planes of a shared-memory ring.
//
// The finite-difference scheme (Sec. V.A) in one pass, the same way:
//   1  psi^n(p)             on tile + 4
//   2  mu^n(p-1)            on tile + 3;  the 13 link noises zeta_l(p-1) on tile + 3
//   3  psi*, E (p-2)        on tile + 2   D = M lap_SO mu - div_CD(u psi),
//                                         eta = sum_l [zeta_l(r - c_l) - zeta_l(r)]
//   4  mu*(p-3)             on tile + 1
//   5  psi^{n+1}(p-4)       on the tile   E + D(psi*) / 2
// with zeta_l ~ N(0, 2 kT M a_l), a_l = 6/22, 3/22, 1/22 on the face, edge and
// corner half-links, drawn from the counters of the two-pass stage 1 (Philox
// stream 1, blocks 0-3, the periodic site id of r).
#include "flb_psi3d.cuh"

namespace flb {
namespace {

constexpr int HT_X = PS_TX, HT_Y = PS_TY, HT_NT = HT_X * HT_Y;  // 32 x 16 tile, 512 threads

template <int R>
struct Reg {  // region tile + R
    static constexpr int W = HT_X + 2 * R, H = HT_Y + 2 * R, N = W * H, S = (N + HT_NT - 1) / HT_NT;
};

// shared-memory rings (floats)
constexpr int SM_P = 4 * Reg<6>::N;   // psi^n, planes p-3 .. p
constexpr int SM_M = 3 * Reg<5>::N;   // mu^n
constexpr int SM_J = 9 * Reg<4>::N;   // J (3 components x 3 planes)
constexpr int SM_X = 9 * Reg<4>::N;   // xi
constexpr int SM_PS = 3 * Reg<3>::N;  // psi*
constexpr int SM_E = 4 * Reg<0>::N;   // E on the tile
constexpr int SM_MS = 3 * Reg<2>::N;  // mu*
constexpr int SM_JS = 9 * Reg<1>::N;  // J*
constexpr int H1_SMEM_FLOATS = SM_P + SM_M + SM_J + SM_X + SM_PS + SM_E + SM_MS + SM_JS;

__device__ __forceinline__ int wrapn(int a, int n) { return ((a % n) + n) % n; }
__device__ __forceinline__ int ring(int p, int d) { return wrapn(p, d); }

// mu = A psi + B psi^3 - K lap_SO psi at index c of the planes pm, p0, pp (pitch W)
template <int W>
__device__ __forceinline__ float mu_at(const float *pm, const float *p0, const float *pp, int c, float A, float B,
                                       float k22)
{
    const float n1 = ((p0[c - 1] + p0[c + 1]) + (p0[c - W] + p0[c + W])) + (pm[c] + pp[c]);
    const float n2 = ((p0[c - 1 - W] + p0[c + 1 - W]) + (p0[c - 1 + W] + p0[c + 1 + W])) +
                     ((pm[c - 1] + pm[c + 1]) + (pm[c - W] + pm[c + W])) +
                     ((pp[c - 1] + pp[c + 1]) + (pp[c - W] + pp[c + W]));
    const float n3 = ((pm[c - 1 - W] + pm[c + 1 - W]) + (pm[c - 1 + W] + pm[c + 1 + W])) +
                     ((pp[c - 1 - W] + pp[c + 1 - W]) + (pp[c - 1 + W] + pp[c + 1 + W]));
    return mu_so(A, B, k22, p0[c], n1, n2, n3);
}

// 12 grad_FV mu at index c of the planes (pitch W)
template <int W>
__device__ __forceinline__ void grad12(const float *mm, const float *m0, const float *mp, int c, float &gx, float &gy,
                                       float &gz)
{
    gx = 2.f * (m0[c + 1] - m0[c - 1]) + ((m0[c + 1 + W] + m0[c + 1 - W]) - (m0[c - 1 + W] + m0[c - 1 - W])) +
         ((mp[c + 1] + mm[c + 1]) - (mp[c - 1] + mm[c - 1]));
    gy = 2.f * (m0[c + W] - m0[c - W]) + ((m0[c + 1 + W] + m0[c - 1 + W]) - (m0[c + 1 - W] + m0[c - 1 - W])) +
         ((mp[c + W] + mm[c + W]) - (mp[c - W] + mm[c - W]));
    gz = 2.f * (mp[c] - mm[c]) + ((mp[c + 1] + mp[c - 1]) - (mm[c + 1] + mm[c - 1])) +
         ((mp[c + W] + mp[c - W]) - (mm[c + W] + mm[c - W]));
}

// 12 div_FV J at index c: J planes (x, y, z components) below (m), at (0) and above (p), pitch W
template <int W>
__device__ __forceinline__ float div12(const float *xm, const float *ym, const float *zm, const float *x0,
                                       const float *y0, const float *z0, const float *xp, const float *yp,
                                       const float *zp, int c)
{
    const float faces = (x0[c + 1] - x0[c - 1]) + (y0[c + W] - y0[c - W]) + (zp[c] - zm[c]);
    const float exy = ((x0[c + 1 + W] + y0[c + 1 + W]) - (x0[c - 1 - W] + y0[c - 1 - W])) +
                      ((x0[c + 1 - W] - y0[c + 1 - W]) - (x0[c - 1 + W] - y0[c - 1 + W]));
    const float exz = ((xp[c + 1] + zp[c + 1]) - (xm[c - 1] + zm[c - 1])) + ((xm[c + 1] - zm[c + 1]) - (xp[c - 1] - zp[c - 1]));
    const float eyz = ((yp[c + W] + zp[c + W]) - (ym[c - W] + zm[c - W])) + ((ym[c + W] - zm[c + W]) - (yp[c - W] - zp[c - W]));
    return 2.f * faces + (exy + (exz + eyz));
}

struct Heun1Args {
    Geom g;
    const float *psi;  // padded psi^n
    const float *u;    // padded velocity of the new fluid state
    float *out;        // padded psi^{n+1} (images to radius 3)
    float A, B, K, M, kT;
    int advect, zc;
    PhiloxKey key;
    int64_t step;
};

template <bool NOISE>
__global__ void __launch_bounds__(HT_NT, 1) psi3_fv_heun1_kernel(const Heun1Args a)
{
    extern __shared__ __align__(16) float hsm[];
    float *sP = hsm, *sM = sP + SM_P, *sJ = sM + SM_M, *sX = sJ + SM_J, *sPs = sX + SM_X, *sE = sPs + SM_PS,
          *sMs = sE + SM_E, *sJs = sMs + SM_MS;
    const Geom &g = a.g;
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * HT_X, y0 = blockIdx.y * HT_Y, z0 = blockIdx.z * a.zc;
    const int z1 = min(z0 + a.zc, g.nz);
    const int plane = g.px * g.py;
    const float k22 = a.K * (1.0f / 22.0f), mg = a.M * (1.0f / 12.0f);
    const float sdx = sqrtf(2.0f * a.kT * a.M);

    // per-slot in-plane data: padded offsets of psi (tile + 6) and of u (tile + 4,
    // tile + 1), noise site ids (tile + 4)
    int off6[Reg<6>::S], off4[Reg<4>::S], id4[Reg<4>::S], off1[Reg<1>::S];
#pragma unroll
    for (int j = 0; j < Reg<6>::S; ++j) {
        const int k = t + j * HT_NT;
        const int x = wrapn(x0 - 6 + k % Reg<6>::W, g.nx), y = wrapn(y0 - 6 + k / Reg<6>::W, g.ny);
        off6[j] = k < Reg<6>::N ? (x + GX) + g.px * (y + GY) : -1;
    }
#pragma unroll
    for (int j = 0; j < Reg<4>::S; ++j) {
        const int k = t + j * HT_NT;
        const int x = wrapn(x0 - 4 + k % Reg<4>::W, g.nx), y = wrapn(y0 - 4 + k / Reg<4>::W, g.ny);
        off4[j] = k < Reg<4>::N ? (x + GX) + g.px * (y + GY) : -1;
        id4[j] = x + g.nx * y;
    }
#pragma unroll
    for (int j = 0; j < Reg<1>::S; ++j) {
        const int k = t + j * HT_NT;
        const int x = wrapn(x0 - 1 + k % Reg<1>::W, g.nx), y = wrapn(y0 - 1 + k / Reg<1>::W, g.ny);
        off1[j] = k < Reg<1>::N ? (x + GX) + g.px * (y + GY) : -1;
    }
    auto pbase = [&](int p) { return (long long)plane * (wrapn(p, g.nz) + g.gz); };

    // psi^n plane values for the next iteration, loaded one plane ahead
    float nxt[Reg<6>::S];
    {
        const float *src = a.psi + pbase(z0 - 6);
#pragma unroll
        for (int j = 0; j < Reg<6>::S; ++j) nxt[j] = off6[j] >= 0 ? __ldg(src + off6[j]) : 0.f;
    }
    for (int p = z0 - 6; p <= z1 + 5; ++p) {
        // velocities of this iteration's flux planes (J at p-2 on tile + 4, J* at p-5 on tile + 1)
        float u4[Reg<4>::S][3], u1[Reg<1>::S][3];
        const bool do3 = p - 2 >= z0 - 4 && p - 2 <= z1 + 3, do6 = p - 5 >= z0 - 1 && p - 5 <= z1;
#pragma unroll
        for (int j = 0; j < Reg<4>::S; ++j)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                u4[j][c] = (a.advect && do3 && off4[j] >= 0) ? __ldg(a.u + c * g.pn + pbase(p - 2) + off4[j]) : 0.f;
#pragma unroll
        for (int j = 0; j < Reg<1>::S; ++j)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                u1[j][c] = (a.advect && do6 && off1[j] >= 0) ? __ldg(a.u + c * g.pn + pbase(p - 5) + off1[j]) : 0.f;
        // 1: psi^n(p) into its ring slot; load p + 1
        {
            float *dst = sP + ring(p, 4) * Reg<6>::N;
#pragma unroll
            for (int j = 0; j < Reg<6>::S; ++j)
                if (off6[j] >= 0) dst[t + j * HT_NT] = nxt[j];
            if (p + 1 <= z1 + 5) {
                const float *src = a.psi + pbase(p + 1);
#pragma unroll
                for (int j = 0; j < Reg<6>::S; ++j) nxt[j] = off6[j] >= 0 ? __ldg(src + off6[j]) : 0.f;
            }
        }
        __syncthreads();
        // 2: mu^n(p-1) on tile + 5
        if (p - 1 >= z0 - 5 && p - 1 <= z1 + 4) {
            const float *pm = sP + ring(p - 2, 4) * Reg<6>::N, *p0 = sP + ring(p - 1, 4) * Reg<6>::N,
                        *pp = sP + ring(p, 4) * Reg<6>::N;
            float *dst = sM + ring(p - 1, 3) * Reg<5>::N;
#pragma unroll
            for (int j = 0; j < Reg<5>::S; ++j) {
                const int k = t + j * HT_NT;
                if (k >= Reg<5>::N) break;
                const int c = (k % Reg<5>::W + 1) + Reg<6>::W * (k / Reg<5>::W + 1);
                dst[k] = mu_at<Reg<6>::W>(pm, p0, pp, c, a.A, a.B, k22);
            }
        }
        __syncthreads();
        // 3: J and xi at p-2 on tile + 4
        if (do3) {
            const int q = p - 2;
            const float *mm = sM + ring(q - 1, 3) * Reg<5>::N, *m0 = sM + ring(q, 3) * Reg<5>::N,
                        *mp = sM + ring(q + 1, 3) * Reg<5>::N;
            const float *ps = sP + ring(q, 4) * Reg<6>::N;
            float *J = sJ + ring(q, 3) * 3 * Reg<4>::N, *X = sX + ring(q, 3) * 3 * Reg<4>::N;
            const int zid = g.nx * g.ny * wrapn(q, g.nz);
#pragma unroll
            for (int j = 0; j < Reg<4>::S; ++j) {
                const int k = t + j * HT_NT;
                if (k >= Reg<4>::N) break;
                const int lx = k % Reg<4>::W, ly = k / Reg<4>::W;
                float gx, gy, gz;
                grad12<Reg<5>::W>(mm, m0, mp, (lx + 1) + Reg<5>::W * (ly + 1), gx, gy, gz);
                const float pv = ps[(lx + 2) + Reg<6>::W * (ly + 2)];
                J[k] = mg * gx - u4[j][0] * pv;
                J[Reg<4>::N + k] = mg * gy - u4[j][1] * pv;
                J[2 * Reg<4>::N + k] = mg * gz - u4[j][2] * pv;
                if (NOISE) {
                    float Gn[4];
                    normals<2, false, true>(a.key, a.step, (uint32_t)(id4[j] + zid), 1u, 0u, Gn, sdx);
                    X[k] = Gn[0];
                    X[Reg<4>::N + k] = Gn[1];
                    X[2 * Reg<4>::N + k] = Gn[2];
                }
            }
        }
        __syncthreads();
        // 4: psi* and E at p-3 on tile + 3
        if (p - 3 >= z0 - 3 && p - 3 <= z1 + 2) {
            const int q = p - 3;
            const float *Jm = sJ + ring(q - 1, 3) * 3 * Reg<4>::N, *J0 = sJ + ring(q, 3) * 3 * Reg<4>::N,
                        *Jp = sJ + ring(q + 1, 3) * 3 * Reg<4>::N;
            const float *Xm = sX + ring(q - 1, 3) * 3 * Reg<4>::N, *X0 = sX + ring(q, 3) * 3 * Reg<4>::N,
                        *Xp = sX + ring(q + 1, 3) * 3 * Reg<4>::N;
            const float *ps = sP + ring(q, 4) * Reg<6>::N;
            float *dst = sPs + ring(q, 3) * Reg<3>::N, *e = sE + ring(q, 4) * Reg<0>::N;
            constexpr int W4 = Reg<4>::W, N4 = Reg<4>::N;
#pragma unroll
            for (int j = 0; j < Reg<3>::S; ++j) {
                const int k = t + j * HT_NT;
                if (k >= Reg<3>::N) break;
                const int lx = k % Reg<3>::W, ly = k / Reg<3>::W;
                const int c = (lx + 1) + W4 * (ly + 1);
                const float D = div12<W4>(Jm, Jm + N4, Jm + 2 * N4, J0, J0 + N4, J0 + 2 * N4, Jp, Jp + N4,
                                          Jp + 2 * N4, c) * (1.0f / 12.0f);
                const float eta = NOISE ? div12<W4>(Xm, Xm + N4, Xm + 2 * N4, X0, X0 + N4, X0 + 2 * N4, Xp, Xp + N4,
                                                    Xp + 2 * N4, c) * (1.0f / 12.0f)
                                        : 0.f;
                const float pv = ps[(lx + 3) + Reg<6>::W * (ly + 3)];
                dst[k] = pv + D + eta;
                if (lx >= 3 && lx < 3 + HT_X && ly >= 3 && ly < 3 + HT_Y)
                    e[(lx - 3) + HT_X * (ly - 3)] = pv + 0.5f * D + eta;
            }
        }
        __syncthreads();
        // 5: mu*(p-4) on tile + 2
        if (p - 4 >= z0 - 2 && p - 4 <= z1 + 1) {
            const int q = p - 4;
            const float *pm = sPs + ring(q - 1, 3) * Reg<3>::N, *p0 = sPs + ring(q, 3) * Reg<3>::N,
                        *pp = sPs + ring(q + 1, 3) * Reg<3>::N;
            float *dst = sMs + ring(q, 3) * Reg<2>::N;
#pragma unroll
            for (int j = 0; j < Reg<2>::S; ++j) {
                const int k = t + j * HT_NT;
                if (k >= Reg<2>::N) break;
                const int c = (k % Reg<2>::W + 1) + Reg<3>::W * (k / Reg<2>::W + 1);
                dst[k] = mu_at<Reg<3>::W>(pm, p0, pp, c, a.A, a.B, k22);
            }
        }
        __syncthreads();
        // 6: J*(p-5) on tile + 1
        if (do6) {
            const int q = p - 5;
            const float *mm = sMs + ring(q - 1, 3) * Reg<2>::N, *m0 = sMs + ring(q, 3) * Reg<2>::N,
                        *mp = sMs + ring(q + 1, 3) * Reg<2>::N;
            const float *ps = sPs + ring(q, 3) * Reg<3>::N;
            float *J = sJs + ring(q, 3) * 3 * Reg<1>::N;
#pragma unroll
            for (int j = 0; j < Reg<1>::S; ++j) {
                const int k = t + j * HT_NT;
                if (k >= Reg<1>::N) break;
                const int lx = k % Reg<1>::W, ly = k / Reg<1>::W;
                float gx, gy, gz;
                grad12<Reg<2>::W>(mm, m0, mp, (lx + 1) + Reg<2>::W * (ly + 1), gx, gy, gz);
                const float pv = ps[(lx + 2) + Reg<3>::W * (ly + 2)];
                J[k] = mg * gx - u1[j][0] * pv;
                J[Reg<1>::N + k] = mg * gy - u1[j][1] * pv;
                J[2 * Reg<1>::N + k] = mg * gz - u1[j][2] * pv;
            }
        }
        __syncthreads();
        // 7: psi^{n+1}(p-6) on the tile
        {
            const int z = p - 6;
            const int x = x0 + t % HT_X, y = y0 + t / HT_X;
            if (z >= z0 && z < z1 && x < g.nx && y < g.ny) {
                constexpr int W1 = Reg<1>::W, N1 = Reg<1>::N;
                const float *Jm = sJs + ring(z - 1, 3) * 3 * N1, *J0 = sJs + ring(z, 3) * 3 * N1,
                            *Jp = sJs + ring(z + 1, 3) * 3 * N1;
                const int c = (t % HT_X + 1) + W1 * (t / HT_X + 1);
                const float D = div12<W1>(Jm, Jm + N1, Jm + 2 * N1, J0, J0 + N1, J0 + 2 * N1, Jp, Jp + N1, Jp + 2 * N1,
                                          c) * (1.0f / 12.0f);
                store_padded(a.out, g, x, y, z, sE[ring(z, 4) * Reg<0>::N + t] + 0.5f * D, 3);
            }
        }
        __syncthreads();
    }
}

// ---- finite difference -----------------------------------------------------

// shared-memory rings of the FD form (floats)
constexpr int FD_P = 4 * Reg<4>::N;    // psi^n, planes p-3 .. p
constexpr int FD_M = 3 * Reg<3>::N;    // mu^n
constexpr int FD_Z = 13 * Reg<3>::N;   // the 13 link noises of one plane
constexpr int FD_PS = 4 * Reg<2>::N;   // psi*
constexpr int FD_E = 3 * Reg<0>::N;    // E on the tile
constexpr int FD_MS = 3 * Reg<1>::N;   // mu*
constexpr int FD_SMEM_FLOATS = FD_P + FD_M + FD_Z + FD_PS + FD_E + FD_MS;

// the 13 half-links of the SO stencil: faces, edges, corners
__device__ __forceinline__ void fd_link(int l, int &cx, int &cy, int &cz)
{
    constexpr int8_t L[13][3] = {{1, 0, 0},  {0, 1, 0},  {0, 0, 1},  {1, 1, 0},   {1, -1, 0},  {1, 0, 1},  {1, 0, -1},
                                 {0, 1, 1},  {0, 1, -1}, {1, 1, 1}, {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};
    cx = L[l][0];
    cy = L[l][1];
    cz = L[l][2];
}

// lap_SO of a field at index c of the planes pm, p0, pp (pitch W)
template <int W>
__device__ __forceinline__ float lap_at(const float *pm, const float *p0, const float *pp, int c)
{
    const float n1 = ((p0[c - 1] + p0[c + 1]) + (p0[c - W] + p0[c + W])) + (pm[c] + pp[c]);
    const float n2 = ((p0[c - 1 - W] + p0[c + 1 - W]) + (p0[c - 1 + W] + p0[c + 1 + W])) +
                     ((pm[c - 1] + pm[c + 1]) + (pm[c - W] + pm[c + W])) +
                     ((pp[c - 1] + pp[c + 1]) + (pp[c - W] + pp[c + W]));
    const float n3 = ((pm[c - 1 - W] + pm[c + 1 - W]) + (pm[c - 1 + W] + pm[c + 1 + W])) +
                     ((pp[c - 1 - W] + pp[c + 1 - W]) + (pp[c - 1 + W] + pp[c + 1 + W]));
    return (6.f * n1 + 3.f * n2 + n3 - 80.f * p0[c]) * (1.0f / 22.0f);
}

// u (padded, images to radius 1) at the six face neighbours of the padded index
// pi: u_x(+x), u_x(-x), u_y(+y), u_y(-y), u_z(+z), u_z(-z)
__device__ __forceinline__ void faces_u(const float *u, const Geom &g, long long pi, bool on, float v[6])
{
    const long long sy = g.px, sz = (long long)g.px * g.py;
    v[0] = on ? __ldg(u + pi + 1) : 0.f;
    v[1] = on ? __ldg(u + pi - 1) : 0.f;
    v[2] = on ? __ldg(u + g.pn + pi + sy) : 0.f;
    v[3] = on ? __ldg(u + g.pn + pi - sy) : 0.f;
    v[4] = on ? __ldg(u + 2 * g.pn + pi + sz) : 0.f;
    v[5] = on ? __ldg(u + 2 * g.pn + pi - sz) : 0.f;
}

// - div_CD(u psi) / 2 at index c of the psi planes Pm, P0, Pp (pitch W)
template <int W>
__device__ __forceinline__ float adv_at(const float *Pm, const float *P0, const float *Pp, int c, const float v[6])
{
    const float adv = (v[0] * P0[c + 1] - v[1] * P0[c - 1]) + (v[2] * P0[c + W] - v[3] * P0[c - W]) +
                      (v[4] * Pp[c] - v[5] * Pm[c]);
    return -0.5f * adv;
}

template <bool NOISE>
__global__ void __launch_bounds__(HT_NT, 1) psi3_fd_heun1_kernel(const Heun1Args a)
{
    static_assert(Reg<0>::S == 1, "one output point per thread");
    extern __shared__ __align__(16) float hsm[];
    float *sP = hsm, *sM = sP + FD_P, *sZ = sM + FD_M, *sPs = sZ + FD_Z, *sE = sPs + FD_PS, *sMs = sE + FD_E;
    const Geom &g = a.g;
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * HT_X, y0 = blockIdx.y * HT_Y, z0 = blockIdx.z * a.zc;
    const int z1 = min(z0 + a.zc, g.nz);
    const int plane = g.px * g.py;
    const float k22 = a.K * (1.0f / 22.0f);
    // sqrt(2 kT M a_l) for the face, edge and corner half-links
    const float s1 = sqrtf(2.0f * a.kT * a.M * (6.f / 22.f)), s2 = sqrtf(2.0f * a.kT * a.M * (3.f / 22.f));
    const float s3 = sqrtf(2.0f * a.kT * a.M * (1.f / 22.f));
    auto pbase = [&](int p) { return (long long)plane * (wrapn(p, g.nz) + g.gz); };

    // per-slot in-plane data: padded offsets of psi^n (tile + 4), noise site ids
    // (tile + 3), padded offsets of the stage-1 points (tile + 2, for their u)
    int off4[Reg<4>::S], id3[Reg<3>::S], off2[Reg<2>::S];
#pragma unroll
    for (int j = 0; j < Reg<4>::S; ++j) {
        const int k = t + j * HT_NT;
        const int x = wrapn(x0 - 4 + k % Reg<4>::W, g.nx), y = wrapn(y0 - 4 + k / Reg<4>::W, g.ny);
        off4[j] = k < Reg<4>::N ? (x + GX) + g.px * (y + GY) : -1;
    }
#pragma unroll
    for (int j = 0; j < Reg<3>::S; ++j) {
        const int k = t + j * HT_NT;
        id3[j] = wrapn(x0 - 3 + k % Reg<3>::W, g.nx) + g.nx * wrapn(y0 - 3 + k / Reg<3>::W, g.ny);
    }
#pragma unroll
    for (int j = 0; j < Reg<2>::S; ++j) {
        const int k = t + j * HT_NT;
        const int x = wrapn(x0 - 2 + k % Reg<2>::W, g.nx), y = wrapn(y0 - 2 + k / Reg<2>::W, g.ny);
        off2[j] = k < Reg<2>::N ? (x + GX) + g.px * (y + GY) : -1;
    }
    // the noise sums eta of the stage-1 points, planes p-2, p-1, p (see phase 3)
    float accm[Reg<2>::S], acc0[Reg<2>::S], accp[Reg<2>::S];
#pragma unroll
    for (int j = 0; j < Reg<2>::S; ++j) accm[j] = acc0[j] = accp[j] = 0.f;

    float nxt[Reg<4>::S];  // psi^n of the next plane, loaded one plane ahead
    {
        const float *src = a.psi + pbase(z0 - 4);
#pragma unroll
        for (int j = 0; j < Reg<4>::S; ++j) nxt[j] = off4[j] >= 0 ? __ldg(src + off4[j]) : 0.f;
    }
    for (int p = z0 - 4; p <= z1 + 3; ++p) {
        const bool do2 = p - 1 >= z0 - 3 && p - 1 <= z1 + 2, do3 = p - 2 >= z0 - 2 && p - 2 <= z1 + 1;
        const bool do4 = p - 3 >= z0 - 1 && p - 3 <= z1, do5 = p - 4 >= z0 && p - 4 < z1;
        // velocities at the face neighbours of this iteration's stage-1 points
        // (plane p-2) and of its output point (plane p-4), loaded now
        float u2[Reg<2>::S][6], u0[6];
#pragma unroll
        for (int j = 0; j < Reg<2>::S; ++j)
            faces_u(a.u, g, pbase(p - 2) + off2[j], a.advect && do3 && off2[j] >= 0, u2[j]);
        const int tx = t % HT_X, ty = t / HT_X, xo = x0 + tx, yo = y0 + ty;
        const bool out_here = do5 && xo < g.nx && yo < g.ny;
        faces_u(a.u, g, out_here ? g.pidx(xo, yo, p - 4) : 0, a.advect && out_here, u0);
        // 1: psi^n(p) into its ring slot; load p + 1
        {
            float *dst = sP + ring(p, 4) * Reg<4>::N;
#pragma unroll
            for (int j = 0; j < Reg<4>::S; ++j)
                if (off4[j] >= 0) dst[t + j * HT_NT] = nxt[j];
            if (p + 1 <= z1 + 3) {
                const float *src = a.psi + pbase(p + 1);
#pragma unroll
                for (int j = 0; j < Reg<4>::S; ++j) nxt[j] = off4[j] >= 0 ? __ldg(src + off4[j]) : 0.f;
            }
        }
        __syncthreads();
        // 2: mu^n(p-1) and the link noises of plane p-1 on tile + 3
        if (do2) {
            const int q = p - 1;
            const float *pm = sP + ring(q - 1, 4) * Reg<4>::N, *p0 = sP + ring(q, 4) * Reg<4>::N,
                        *pp = sP + ring(q + 1, 4) * Reg<4>::N;
            float *dst = sM + ring(q, 3) * Reg<3>::N;
            const int zid = g.nx * g.ny * wrapn(q, g.nz);
#pragma unroll
            for (int j = 0; j < Reg<3>::S; ++j) {
                const int k = t + j * HT_NT;
                if (k >= Reg<3>::N) break;
                const int c = (k % Reg<3>::W + 1) + Reg<4>::W * (k / Reg<3>::W + 1);
                dst[k] = mu_at<Reg<4>::W>(pm, p0, pp, c, a.A, a.B, k22);
                if (NOISE) {
                    const uint32_t sid = (uint32_t)(id3[j] + zid);
                    float G[14];  // normals 0-12: block 0, and block 1's first three words
                    normals<4>(a.key, a.step, sid, 1u, 0u, G);
                    normals<3>(a.key, a.step, sid, 1u, 1u, G + 8);
#pragma unroll
                    for (int l = 0; l < 13; ++l) sZ[l * Reg<3>::N + k] = (l < 3 ? s1 : (l < 9 ? s2 : s3)) * G[l];
                }
            }
        }
        __syncthreads();
        // 3: the noise of plane p-1 into the sums of the stage-1 points, then
        // psi* and E at p-2 on tile + 2
#pragma unroll
        for (int j = 0; j < Reg<2>::S; ++j) {
            const int k = t + j * HT_NT;
            if (k >= Reg<2>::N) break;
            const int lx = k % Reg<2>::W, ly = k / Reg<2>::W;
            if (NOISE && do2) {
                // zeta(p-1) feeds eta(p-1) (own links, in-plane neighbours), eta(p)
                // (links with c_z = +1) and eta(p-2) (links with c_z = -1)
                const int c = (lx + 1) + Reg<3>::W * (ly + 1);
                float own = 0.f, in0 = 0.f, up = 0.f, dn = 0.f;
#pragma unroll
                for (int l = 0; l < 13; ++l) {
                    int cx, cy, cz;
                    fd_link(l, cx, cy, cz);
                    own += sZ[l * Reg<3>::N + c];
                    const float v = sZ[l * Reg<3>::N + c - cx - Reg<3>::W * cy];
                    if (cz == 0) in0 += v;
                    else if (cz > 0) up += v;
                    else dn += v;
                }
                accm[j] += dn;
                acc0[j] += in0 - own;
                accp[j] += up;
            }
            if (do3) {
                const int q = p - 2;
                const float *mm = sM + ring(q - 1, 3) * Reg<3>::N, *m0 = sM + ring(q, 3) * Reg<3>::N,
                            *mp = sM + ring(q + 1, 3) * Reg<3>::N;
                float D = a.M * lap_at<Reg<3>::W>(mm, m0, mp, (lx + 1) + Reg<3>::W * (ly + 1));
                const float *P0 = sP + ring(q, 4) * Reg<4>::N;
                const int cp = (lx + 2) + Reg<4>::W * (ly + 2);
                if (a.advect)
                    D += adv_at<Reg<4>::W>(sP + ring(q - 1, 4) * Reg<4>::N, P0, sP + ring(q + 1, 4) * Reg<4>::N, cp,
                                           u2[j]);
                const float eta = NOISE ? accm[j] : 0.f;
                const float pv = P0[cp];
                sPs[ring(q, 4) * Reg<2>::N + k] = pv + D + eta;
                if (lx >= 2 && lx < 2 + HT_X && ly >= 2 && ly < 2 + HT_Y)
                    sE[ring(q, 3) * Reg<0>::N + (lx - 2) + HT_X * (ly - 2)] = pv + 0.5f * D + eta;
            }
            accm[j] = acc0[j];
            acc0[j] = accp[j];
            accp[j] = 0.f;
        }
        __syncthreads();
        // 4: mu*(p-3) on tile + 1
        if (do4) {
            const int q = p - 3;
            const float *pm = sPs + ring(q - 1, 4) * Reg<2>::N, *p0 = sPs + ring(q, 4) * Reg<2>::N,
                        *pp = sPs + ring(q + 1, 4) * Reg<2>::N;
            float *dst = sMs + ring(q, 3) * Reg<1>::N;
#pragma unroll
            for (int j = 0; j < Reg<1>::S; ++j) {
                const int k = t + j * HT_NT;
                if (k >= Reg<1>::N) break;
                const int c = (k % Reg<1>::W + 1) + Reg<2>::W * (k / Reg<1>::W + 1);
                dst[k] = mu_at<Reg<2>::W>(pm, p0, pp, c, a.A, a.B, k22);
            }
        }
        __syncthreads();
        // 5: psi^{n+1}(p-4) on the tile
        if (out_here) {
            const int z = p - 4;
            const float *mm = sMs + ring(z - 1, 3) * Reg<1>::N, *m0 = sMs + ring(z, 3) * Reg<1>::N,
                        *mp = sMs + ring(z + 1, 3) * Reg<1>::N;
            float D = a.M * lap_at<Reg<1>::W>(mm, m0, mp, (tx + 1) + Reg<1>::W * (ty + 1));
            if (a.advect)
                D += adv_at<Reg<2>::W>(sPs + ring(z - 1, 4) * Reg<2>::N, sPs + ring(z, 4) * Reg<2>::N,
                                       sPs + ring(z + 1, 4) * Reg<2>::N, (tx + 2) + Reg<2>::W * (ty + 2), u0);
            store_padded(a.out, g, xo, yo, z, sE[ring(z, 3) * Reg<0>::N + t] + 0.5f * D, 3);
        }
        __syncthreads();
    }
}

}  // namespace

size_t psi3_heun1_smem_bytes() { return sizeof(float) * (size_t)H1_SMEM_FLOATS; }

cudaError_t launch_psi3_heun1(const Geom &g, int scheme, const float *psi, const float *u, float *out, float A, float B,
                              float K, float M, float kT, int advect, bool noise, const PhiloxKey &key, int64_t step,
                              int zc, cudaStream_t st)
{
    Heun1Args a;
    a.g = g;
    a.psi = psi;
    a.u = u;
    a.out = out;
    a.A = A;
    a.B = B;
    a.K = K;
    a.M = M;
    a.kT = kT;
    a.advect = advect;
    a.zc = zc;
    a.key = key;
    a.step = step;
    const dim3 grid((g.nx + HT_X - 1) / HT_X, (g.ny + HT_Y - 1) / HT_Y, (g.nz + zc - 1) / zc);
    cudaError_t e;
    if (scheme == FLB_FD) {
        const size_t smem = sizeof(float) * (size_t)FD_SMEM_FLOATS;
        const void *k = noise ? (const void *)psi3_fd_heun1_kernel<true> : (const void *)psi3_fd_heun1_kernel<false>;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (noise) psi3_fd_heun1_kernel<true><<<grid, HT_NT, smem, st>>>(a);
        else psi3_fd_heun1_kernel<false><<<grid, HT_NT, smem, st>>>(a);
        return cudaGetLastError();
    }
    const size_t smem = psi3_heun1_smem_bytes();
    if (noise) {
        e = cudaFuncSetAttribute(psi3_fv_heun1_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        psi3_fv_heun1_kernel<true><<<grid, HT_NT, smem, st>>>(a);
    } else {
        e = cudaFuncSetAttribute(psi3_fv_heun1_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        psi3_fv_heun1_kernel<false><<<grid, HT_NT, smem, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace flb

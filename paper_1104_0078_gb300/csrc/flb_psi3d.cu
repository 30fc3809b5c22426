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

#include "flb_psi3d.cuh"

namespace flb {

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

// The same with the class weights w of an App. A Laplacian:
// A psi + B psi^3 - K [(c1 n1 + c2 n2) + (c3 n3 + c0 psi)]
template <int PX>
__device__ __forceinline__ float mu_point_w(const float *pm, const float *p0, const float *pp, int c, float A, float B,
                                            float K, const LapW &w)
{
    const float n1 = (p0[c - 1] + p0[c + 1]) + (p0[c - PX] + p0[c + PX]) + (pm[c] + pp[c]);
    const float n2 = ((p0[c - 1 - PX] + p0[c + 1 - PX]) + (p0[c - 1 + PX] + p0[c + 1 + PX])) +
                     ((pm[c - 1] + pm[c + 1]) + (pm[c - PX] + pm[c + PX])) +
                     ((pp[c - 1] + pp[c + 1]) + (pp[c - PX] + pp[c + PX]));
    const float n3 = ((pm[c - 1 - PX] + pm[c + 1 - PX]) + (pm[c - 1 + PX] + pm[c + 1 + PX])) +
                     ((pp[c - 1 - PX] + pp[c + 1 - PX]) + (pp[c - 1 + PX] + pp[c + 1 + PX]));
    const float ps = p0[c];
    return A * ps + B * ps * ps * ps - K * ((w.c1 * n1 + w.c2 * n2) + (w.c3 * n3 + w.c0 * ps));
}

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

// ---------------------------------------------------------------------------
// Finite difference.  Shared memory: psi ring 4 x H3N, mu ring 3 x H2N and
// (stage 1 with noise) the 13 link noises of one plane, 13 x H1N floats.
// ---------------------------------------------------------------------------
// half-links: x, y, z, (1,1,0), (1,-1,0), (1,0,1), (1,0,-1), (0,1,1), (0,1,-1),
// (1,1,1), (1,1,-1), (1,-1,1), (1,-1,-1); coefficients 6/22, 3/22, 1/22
__constant__ int8_t kFDL[13][3] = {{1, 0, 0},  {0, 1, 0},  {0, 0, 1},  {1, 1, 0}, {1, -1, 0},
                                   {1, 0, 1},  {1, 0, -1}, {0, 1, 1},  {0, 1, -1}, {1, 1, 1},
                                   {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};

// Two 512-thread blocks per SM (64 registers): with one, the noisy stage ran at
// 25% of the warp slots and half of the issue rate.
// MU_IN (stage 1): mu of psi^n on tile + 1 is read from the force's mu field
// (mu_in, same padded layout as u), one plane ahead, instead of formed from psi.
template <int STAGE, bool NOISE, bool MU_IN = false>
__global__ void __launch_bounds__(PS_NT, 2) psi3_fd_kernel(const Psi3Args a, const float *__restrict__ mu_in)
{
    static_assert(!MU_IN || STAGE == 1, "mu of psi^n is the input of stage 1 only");
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
    // psi planes are double-buffered in registers: plane p+1 is loaded while
    // plane p is worked on, and stored to its ring slot at the next iteration
    float nxt[S3];
    {
        const float *src = a.psi + (size_t)plane * (z0 - 2 + g.gz);
#pragma unroll
        for (int j = 0; j < S3; ++j) nxt[j] = R.g3[j] >= 0 ? __ldg(src + R.g3[j]) : 0.f;
    }
    // MU_IN: mu of plane q = p - 1 (loaded the iteration before) and of plane p
    float mcur[S1], mnx[S1];
#pragma unroll
    for (int j = 0; j < S1; ++j) mcur[j] = mnx[j] = 0.f;

    for (int p = z0 - 2; p <= z1 + 1; ++p) {
        // this iteration's output plane p-2: its global inputs (the Heun
        // accumulator and the six advecting velocities) are loaded now, so that
        // their latency hides behind the plane's stencil work
        const int zo = p - 2;
        const bool out_here = zo >= z0 && active;
        float e_pre = 0.f, u_pre[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (MU_IN && p >= z0 - 1 && p <= z1) {
            const float *src = mu_in + (size_t)plane * (p + g.gz);
#pragma unroll
            for (int j = 0; j < S1; ++j) mnx[j] = R.c1[j] >= 0 ? __ldg(src + R.u1[j]) : 0.f;
        }
        if (out_here) {
            if (STAGE == 2 && !a.rk4) e_pre = a.E[x + g.nx * (y + g.ny * zo)];
            if (a.advect) {
                const int pi = g.pidx32(x, y, zo);
                const int sy = g.px, sz = g.px * g.py;
                u_pre[0] = __ldg(a.u + pi + 1);
                u_pre[1] = __ldg(a.u + pi - 1);
                u_pre[2] = __ldg(a.u + g.pn + pi + sy);
                u_pre[3] = __ldg(a.u + g.pn + pi - sy);
                u_pre[4] = __ldg(a.u + 2 * g.pn + pi + sz);
                u_pre[5] = __ldg(a.u + 2 * g.pn + pi - sz);
            }
        }
        __syncthreads();
        {
            float *dst = sps + ring4(p) * H3N;
#pragma unroll
            for (int j = 0; j < S3; ++j)
                if (R.g3[j] >= 0) dst[threadIdx.x + j * PS_NT] = nxt[j];
            if (p + 1 <= z1 + 1) {
                const float *src = a.psi + (size_t)plane * (p + 1 + g.gz);
#pragma unroll
                for (int j = 0; j < S3; ++j)
                    if (R.g3[j] >= 0) nxt[j] = __ldg(src + R.g3[j]);
            }
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
                dst[c] = MU_IN      ? mcur[j]
                         : a.lap_w ? mu_point_w<H3X>(pm, p0, pp, R.p1[j], a.A, a.B, a.K, a.lw)
                                   : mu_point<H3X>(pm, p0, pp, R.p1[j], a.A, a.B, k22);
            }
            if (NOISE) {
                const int zid = g.nx * g.ny * wrapi(q, g.nz);
                // sqrt(2 kT M a_l) for the face, edge and corner half-links (a_l the
                // Laplacian's class weights: 6/22, 3/22, 1/22 for SO)
                const float s1 = sqrtf(2.0f * a.kT * a.M * (a.lap_w ? a.lw.c1 : 6.f / 22.f));
                const float s2 = sqrtf(2.0f * a.kT * a.M * (a.lap_w ? a.lw.c2 : 3.f / 22.f));
                const float s3 = sqrtf(2.0f * a.kT * a.M * (a.lap_w ? a.lw.c3 : 1.f / 22.f));
#pragma unroll
                for (int j = 0; j < S1; ++j) {
                    if (R.c1[j] < 0) continue;
                    const int k = threadIdx.x + j * PS_NT;
                    const uint32_t sid = (uint32_t)(R.n1[j] + zid);
                    float G[14];  // normals 0-12: block 0, and block 1's first three words
                    normals<4>(a.key, a.step, sid, 1u, 0u, G);
                    normals<3>(a.key, a.step, sid, 1u, 1u, G + 8);
#pragma unroll
                    for (int l = 0; l < 13; ++l) sZ[l * H1N + k] = (l < 3 ? s1 : (l < 9 ? s2 : s3)) * G[l];
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
        const int z = zo;
        if (out_here) {
            const float *mm = smu + ring3(z - 1) * H2N, *m0 = smu + ring3(z) * H2N, *mp = smu + ring3(z + 1) * H2N;
            const int c = (tx + 2) + H2X * (ty + 2);
            float D = a.M * (a.lap_w ? mu_point_w<H2X>(mm, m0, mp, c, 0.f, 0.f, -1.0f, a.lw)
                                     : mu_point<H2X>(mm, m0, mp, c, 0.f, 0.f, -1.0f / 22.0f));
            if (a.advect) {
                const float *P0 = sps + ring4(z) * H3N, *Pm = sps + ring4(z - 1) * H3N, *Pp = sps + ring4(z + 1) * H3N;
                const int cp = (tx + 3) + H3X * (ty + 3);
                const float adv = (u_pre[0] * P0[cp + 1] - u_pre[1] * P0[cp - 1]) +
                                  (u_pre[2] * P0[cp + H3X] - u_pre[3] * P0[cp - H3X]) +
                                  (u_pre[4] * Pp[cp] - u_pre[5] * Pm[cp]);
                D -= 0.5f * adv;
            }
            const int si = x + g.nx * (y + g.ny * z);
            const float eta = (STAGE == 1 && NOISE) ? accm : 0.f;
            const float pv = STAGE == 1 ? sps[ring4(z) * H3N + (tx + 3) + H3X * (ty + 3)] : 0.f;
            const float out = (STAGE == 2 && !a.rk4) ? e_pre + 0.5f * D : rk_stage_out<STAGE, false>(a, x, y, z, si, pv, D, eta);
            store_padded(a.out, g, x, y, z, out, 3);
        }
        accm = acc0;
        acc0 = accp;
        accp = 0.f;
        if (MU_IN) {
#pragma unroll
            for (int j = 0; j < S1; ++j) mcur[j] = mnx[j];
        }
    }
}

struct TmaArgs {
    Psi3Args a;
    int *status;
};

// MU_IN: stage 1 reads mu of its input from mu_map instead of forming it; Q15:
// the FV operators of D3Q15
// 256 threads, each on point pairs (y, y + H/2) of every region in packed FP32 (F2)
using StageV = F2;
template <int STAGE, bool NOISE, bool RK, bool MU_IN, bool Q15 = false>
__global__ void __launch_bounds__(stage_threads<StageV>(), 2) psi3_fv_tma_kernel(const __grid_constant__ CUtensorMap psi_map,
                                                                   const __grid_constant__ CUtensorMap u_map,
                                                                   const __grid_constant__ CUtensorMap mu_map,
                                                                   const TmaArgs ta)
{
    extern __shared__ __align__(1024) float tsmem[];
    psi3_fv_tma_block<STAGE, NOISE, false, false, RK, MU_IN, Q15, StageV>(&psi_map, &u_map, ta.a, ta.status, blockIdx.x,
                                                                     blockIdx.y, blockIdx.z, tsmem, &mu_map);
}

// batched: block b of the launch works on L.psi[b]; MU_IN: stage 1 reads mu of
// psi^n from the replica's mu field (every replica's step formed it)
template <int STAGE, bool NOISE, bool MU_IN = false, bool Q15 = false>
__global__ void __launch_bounds__(stage_threads<StageV>(), 2) psi3_fv_tma_batch_kernel(const BatchLists L)
{
    extern __shared__ __align__(1024) float tsmem[];
    __shared__ Psi3Args sa;
    const BatchBlock b = L.psi[blockIdx.x];
    const BatchRep &r = L.reps[b.rep];
    const long long ds = *L.dstep;
    if (threadIdx.x == 0) psi_batch_args(r, ds, STAGE, sa);
    __syncthreads();
    const CUtensorMap *pm = STAGE == 1 ? &r.map_psi[(int)(ds & 1)] : &r.map_psis;
    psi3_fv_tma_block<STAGE, NOISE, false, true, false, MU_IN, Q15, StageV>(pm, &r.map_u, sa, L.status, b.bx, b.by, b.bz,
                                                                       tsmem, &r.map_mu);
}

__global__ void advance_kernel(long long *dstep) { *dstep += 1; }

cudaError_t launch_lb3_batch(const BatchLists &L, int storage, bool ghost, bool force, cudaStream_t st);
cudaError_t launch_lb15_batch(const BatchLists &L, int storage, bool ghost, bool force, cudaStream_t st);

template <bool Q15>
static cudaError_t batch_psi(const BatchLists &L, bool heun, bool noise, bool mu_in, cudaStream_t st)
{
    const size_t sm = sizeof(float) * (size_t)fv_smem_floats<StageV>();
    const size_t smm = sizeof(float) * (size_t)fv_mu_smem_floats<StageV>();
    const size_t nb = sizeof(float) * FV_NOISE_FLOATS;
    auto go = [&](auto kernel, size_t bytes) {
        cudaError_t r = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (r != cudaSuccess) return r;
        kernel<<<L.npsi, stage_threads<StageV>(), bytes, st>>>(L);
        return cudaGetLastError();
    };
    cudaError_t e = mu_in ? (noise ? go(psi3_fv_tma_batch_kernel<1, true, true, Q15>, smm + nb)
                                   : go(psi3_fv_tma_batch_kernel<1, false, true, Q15>, smm))
                          : (noise ? go(psi3_fv_tma_batch_kernel<1, true, false, Q15>, sm + nb)
                                   : go(psi3_fv_tma_batch_kernel<1, false, false, Q15>, sm));
    if (e != cudaSuccess || !heun) return e;
    return go(psi3_fv_tma_batch_kernel<2, false, false, Q15>, sm);
}

cudaError_t launch_batch_psi(const BatchLists &L, bool heun, bool noise, bool mu_in, bool q15, cudaStream_t st)
{
    return q15 ? batch_psi<true>(L, heun, noise, mu_in, st) : batch_psi<false>(L, heun, noise, mu_in, st);
}

cudaError_t launch_batch_step(const BatchLists &L, int storage, bool ghost, bool force, int scheme_fv, bool heun,
                              bool noise, bool mu_in, bool q15, cudaStream_t st)
{
    if (!scheme_fv) return cudaErrorNotSupported;
    cudaError_t e = q15 ? launch_lb15_batch(L, storage, ghost, force, st)
                        : launch_lb3_batch(L, storage, ghost, force, st);
    if (e != cudaSuccess) return e;
    e = launch_batch_psi(L, heun, noise, mu_in, q15, st);
    if (e != cudaSuccess) return e;
    advance_kernel<<<1, 1, 0, st>>>(const_cast<long long *>(L.dstep));
    return cudaGetLastError();
}

template <typename K>
static cudaError_t launch_dyn(K kernel, dim3 grid, size_t smem, cudaStream_t st, const Psi3Args &a, const float *mu_in)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kernel<<<grid, PS_NT, smem, st>>>(a, mu_in);
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

static cudaError_t launch_fv_tma(const Psi3Args &a, int q, int stage, bool noise, const float *mu_in, int *status,
                                 cudaStream_t st)
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
    CUtensorMap mm = pm;  // unused unless stage 1 reads mu
    const bool mu = stage == 1 && mu_in != nullptr;
    if (mu) {
        const uint32_t mb[3] = {(uint32_t)TB_X, (uint32_t)H2Y, 1};
        e = encode_tensor_map_f32(&mm, mu_in, 3, pd, ps, mb);
        if (e != cudaSuccess) return e;
    }
    TmaArgs ta;
    ta.a = a;
    ta.status = status;
    const dim3 grid((g.nx + PS_TX - 1) / PS_TX, (g.ny + PS_TY - 1) / PS_TY, (g.nz + a.zc - 1) / a.zc);
    const size_t sm = sizeof(float) * (size_t)fv_smem_floats<StageV>();
    auto go = [&](auto kernel, size_t bytes) {
        cudaError_t r = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (r != cudaSuccess) return r;
        kernel<<<grid, stage_threads<StageV>(), bytes, st>>>(pm, um, mm, ta);
        return cudaGetLastError();
    };
    const size_t smn = sm + sizeof(float) * FV_NOISE_FLOATS;
    const size_t smm = sizeof(float) * (size_t)fv_mu_smem_floats<StageV>(), smmn = smm + sizeof(float) * FV_NOISE_FLOATS;
    if (q == 15) {  // D3Q15 (the RK4 branches compiled into RK4 launches only, as below)
        if (stage == 2) return a.rk4 ? go(psi3_fv_tma_kernel<2, false, true, false, true>, sm)
                                     : go(psi3_fv_tma_kernel<2, false, false, false, true>, sm);
        if (a.rk4) {
            if (mu) return noise ? go(psi3_fv_tma_kernel<1, true, true, true, true>, smmn)
                                 : go(psi3_fv_tma_kernel<1, false, true, true, true>, smm);
            return noise ? go(psi3_fv_tma_kernel<1, true, true, false, true>, smn)
                         : go(psi3_fv_tma_kernel<1, false, true, false, true>, sm);
        }
        if (mu) return noise ? go(psi3_fv_tma_kernel<1, true, false, true, true>, smmn)
                             : go(psi3_fv_tma_kernel<1, false, false, true, true>, smm);
        return noise ? go(psi3_fv_tma_kernel<1, true, false, false, true>, smn)
                     : go(psi3_fv_tma_kernel<1, false, false, false, true>, sm);
    }
    if (stage == 2) return a.rk4 ? go(psi3_fv_tma_kernel<2, false, true, false>, sm)
                                 : go(psi3_fv_tma_kernel<2, false, false, false>, sm);
    if (mu) {
        if (a.rk4) return noise ? go(psi3_fv_tma_kernel<1, true, true, true>, smmn)
                                : go(psi3_fv_tma_kernel<1, false, true, true>, smm);
        return noise ? go(psi3_fv_tma_kernel<1, true, false, true>, smmn)
                     : go(psi3_fv_tma_kernel<1, false, false, true>, smm);
    }
    if (a.rk4) return noise ? go(psi3_fv_tma_kernel<1, true, true, false>, smn)
                            : go(psi3_fv_tma_kernel<1, false, true, false>, sm);
    return noise ? go(psi3_fv_tma_kernel<1, true, false, false>, smn) : go(psi3_fv_tma_kernel<1, false, false, false>, sm);
}

cudaError_t launch_psi3(const Geom &g, int scheme, int q, int stage, bool noise, const float *psi, const float *u,
                        float *out, float *E, float A, float B, float K, float M, float kT, int advect, int heun,
                        const PhiloxKey &key, int64_t step, int zc, int rk4, const float *base, float *Dn,
                        const float *mu_in, int *status, cudaStream_t st, const LapW *lw)
{
    if (zc < PS_ZC_MIN) return cudaErrorInvalidValue;
    if (lw && scheme != FLB_FD) return cudaErrorInvalidValue;  // App. A Laplacians: the FD stage only
    Psi3Args a;
    a.lap_w = lw ? 1 : 0;
    a.lw = lw ? *lw : LapW{0.f, 0.f, 0.f, 0.f};
    a.rk4 = rk4;
    a.base = base;
    a.Dn = Dn;
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
    const size_t smem = sizeof(float) * (4 * H3N + 3 * H2N);
    if (scheme == FLB_FV) return launch_fv_tma(a, q, stage, noise, mu_in, status, st);
    const size_t smn = smem + sizeof(float) * 13 * H1N;
    if (stage == 1 && mu_in) {
        if (noise) return launch_dyn(psi3_fd_kernel<1, true, true>, grid, smn, st, a, mu_in);
        return launch_dyn(psi3_fd_kernel<1, false, true>, grid, smem, st, a, mu_in);
    }
    if (stage == 1) {
        if (noise) return launch_dyn(psi3_fd_kernel<1, true>, grid, smn, st, a, nullptr);
        return launch_dyn(psi3_fd_kernel<1, false>, grid, smem, st, a, nullptr);
    }
    return launch_dyn(psi3_fd_kernel<2, false>, grid, smem, st, a, nullptr);
}

}  // namespace flb

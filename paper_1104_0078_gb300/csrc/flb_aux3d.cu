// flb_aux3d.cu -- the D3Q19 step kernels around the collide-stream.
//
// mu3_kernel writes the chemical potential mu = A psi + B psi^3 - K lap_SO psi
// (Sec. II.A; SO stencil of App. A) on the interior and MU3_HALO = 2 ghost
// layers, for the force density of the collide-stream (1 layer) and the FV psi
// stage 1 of the same step (2 layers); with the stress-form force sigma3_kernel
// writes the order-parameter stress (Eq. muf) on 1 ghost layer instead.  vel3_kernel runs after it: it gathers
// the populations the next step pulls (the planes just written) and writes the
// velocity (sum fbar c + F/2)/rho of the new fluid state, which advects psi
// (Gauss-Seidel coupling: the psi step follows the fluid step).  Both have a
// batched variant that walks a block work list over all replicas.
#include "flb_mu3d.cuh"

namespace flb {

// Velocity of the streamed state after the step: u = (sum fbar c + F/2)/rho
// with fbar the populations the next step pulls (the planes just written, a.fout)
// and F this step's force density -- the velocity that advects psi (Gauss-Seidel
// coupling of Sec. VI: the psi step follows the fluid step).  The planes'
// addresses are formed from a.fout with a 32-bit plane stride (N < 2^31): with
// a table of them (as the collide-stream takes) this memory-bound gather ran 5%
// slower at 256^3 (283 against 269 us).
template <typename T>
struct PlanesStride32 {
    const T *fi;
    int N;
    __device__ __forceinline__ const T *in(int i) const { return fi + (long long)i * N; }
};

// Two sites per thread, (x, y, z) and (x, y, z + 1), as in the collide-stream.
template <typename T, bool FORCE>
__global__ void __launch_bounds__(LB_BX *LB_BY, 10) vel3_kernel(const LBArgs a)
{
    const Geom &g = a.g;
    const int x = blockIdx.x * LB_BX + threadIdx.x;
    const int y = blockIdx.y * LB_BY + threadIdx.y;
    const int z = blockIdx.z * LB_BZ;
    if (x >= g.nx || y >= g.ny || z >= g.nz) return;
    const int nl = z + 1 < g.nz ? 2 : 1;
    const int zl[2] = {z, z + nl - 1};
    vel3_sites<F2, T, FORCE, false>(a, PlanesStride32<T>{(const T *)a.fout, (int)g.n}, x, y, zl, nl);
}

// mu = A psi + B psi^3 - K lap_SO psi on the interior and HALO ghost layers
// (psi holds images to 3 layers, so HALO <= 2).  A block owns a 32 x 4 column
// of (x, y) in [-HALO, nx + HALO) x [-HALO, ny + HALO) and marches MU_ZC planes
// of z in [-HALO, nz + HALO); each thread keeps, for the planes below and
// at z, the centre a, the 4 in-plane faces b and the 4 in-plane diagonals d of
// psi, so that (Eq. solap)
//   22 lap_SO psi(z) = 6 [b(z) + a(z-1) + a(z+1)] + 3 [d(z) + b(z-1) + b(z+1)]
//                      + d(z-1) + d(z+1) - 80 a(z)
// takes 9 loads per plane instead of 27.
template <int HALO = 1>
__device__ __forceinline__ void mu3_block(const Geom &g, const float *__restrict__ psi, float *__restrict__ mu, float A,
                                          float B, float K, int bx, int by, int bz, const LapW *lw = nullptr)
{
    const int x = bx * MU_BX + (int)threadIdx.x - HALO;
    const int y = by * MU_BY + (int)threadIdx.y - HALO;
    const int zb = bz * MU_ZC - HALO;                       // first output plane
    const int ze = min(zb + MU_ZC, g.nz + HALO);            // one past the last
    if (x >= g.nx + HALO || y >= g.ny + HALO || zb >= ze) return;
    mu3_column<false>(g, psi, mu, A, B, K, x, y, zb, ze, lw);
}

__global__ void __launch_bounds__(MU_BX *MU_BY) sigma3_kernel(const Geom g, const float *__restrict__ psi,
                                                             float *__restrict__ sig, float A, float B, float K)
{
    const int x = blockIdx.x * MU_BX + (int)threadIdx.x - 1;
    const int y = blockIdx.y * MU_BY + (int)threadIdx.y - 1;
    const int zb = blockIdx.z * MU_ZC - 1;
    const int ze = min(zb + MU_ZC, g.nz + 1);
    if (x > g.nx || y > g.ny || zb >= ze) return;
    sigma3_column<false>(g, psi, sig, A, B, K, x, y, zb, ze);
}

// W: the class weights lw of an App. A Laplacian (false: SO)
template <bool W>
__global__ void __launch_bounds__(MU_BX *MU_BY) mu3_kernel(const Geom g, const float *__restrict__ psi,
                                                          float *__restrict__ mu, float A, float B, float K, const LapW lw)
{
    mu3_block<MU3_HALO>(g, psi, mu, A, B, K, blockIdx.x, blockIdx.y, blockIdx.z, W ? &lw : nullptr);
}

// The same field (SO stencil) with four consecutive x per thread: x = xs ..
// xs+3, xs = -4 + 4 i, so that xs is 16-byte aligned in the padded rows.  Per
// plane a thread reads each of the rows y-1, y, y+1 as one 16-byte load and the
// two cells beside it (3 x 3 loads for four points instead of 4 x 9), keeps the
// per-plane partial sums of mu3_column for its four points and forms mu with
// the same sums in the same order (mu_so), so the field is bitwise that of the
// batched and persistent kernels.  Points x < -2 or x >= nx + 2 are not written,
// and the side cells they alone would need are not read.
constexpr int MV_TX = 16, MV_TY = 8, MV_ZC = 16;

__global__ void __launch_bounds__(MV_TX *MV_TY) mu3_vec_kernel(const Geom g, const float *__restrict__ psi,
                                                             float *__restrict__ mu, float A, float B, float K)
{
    const int xs = -4 + 4 * (int)(blockIdx.x * MV_TX + threadIdx.x);
    const int y = (int)(blockIdx.y * MV_TY + threadIdx.y) - MU3_HALO;
    const int zb = (int)blockIdx.z * MV_ZC - MU3_HALO, ze = min(zb + MV_ZC, g.nz + MU3_HALO);
    const int xl = g.nx + MU3_HALO;  // one past the last output column
    if (xs + 3 < -MU3_HALO || xs >= xl || y >= g.ny + MU3_HALO || zb >= ze) return;
    const bool lo = xs - 1 >= -MU3_HALO - 1, hi = xs + 4 <= xl;  // side cells some point needs
    const int Y = g.px, Z = g.px * g.py;
    const float k22 = K * (1.0f / 22.0f);
    float a0[4] = {}, b0[4] = {}, d0[4] = {}, a1[4] = {}, b1[4] = {}, d1[4] = {};  // planes p-2, p-1
    int c = g.pidx32(xs, y, zb - 1);
    for (int p = zb - 1; p <= ze; ++p, c += Z) {
        float v[3][6];  // rows y-1, y, y+1; cells xs-1 .. xs+4
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int o = c + (r - 1) * Y;
            const float4 q = __ldg(reinterpret_cast<const float4 *>(psi + o));
            v[r][0] = lo ? __ldg(psi + o - 1) : 0.f;
            v[r][1] = q.x;
            v[r][2] = q.y;
            v[r][3] = q.z;
            v[r][4] = q.w;
            v[r][5] = hi ? __ldg(psi + o + 4) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float a2 = v[1][k + 1];
            const float b2 = (v[1][k] + v[1][k + 2]) + (v[0][k + 1] + v[2][k + 1]);
            const float d2 = (v[0][k] + v[0][k + 2]) + (v[2][k] + v[2][k + 2]);
            const int x = xs + k;
            if (p - 1 >= zb && x >= -MU3_HALO && x < xl) {
                const float n1 = b1[k] + (a0[k] + a2), n2 = d1[k] + (b0[k] + b2), n3 = d0[k] + d2;
                mu[c - Z + k] = mu_so(A, B, k22, a1[k], n1, n2, n3);
            }
            a0[k] = a1[k]; b0[k] = b1[k]; d0[k] = d1[k];
            a1[k] = a2; b1[k] = b2; d1[k] = d2;
        }
    }
}

// ---- batched variants: block b of the launch works on L.mu[b] / L.lb[b] -------
__global__ void __launch_bounds__(MU_BX *MU_BY) mu3_batch_kernel(const BatchLists L)
{
    const BatchBlock b = L.mu[blockIdx.x];
    const BatchRep &r = L.reps[b.rep];
    const int par = (int)(*L.dstep & 1);
    if (r.lb.force_kind == 2) {  // stress form: sigma instead of mu
        const Geom &g = r.lb.g;
        const int x = b.bx * MU_BX + (int)threadIdx.x - 1, y = b.by * MU_BY + (int)threadIdx.y - 1;
        const int zb = b.bz * MU_ZC - 1, ze = min(zb + MU_ZC, g.nz + 1);
        if (x <= g.nx && y <= g.ny && zb < ze)
            sigma3_column<false>(g, r.psi[par], const_cast<float *>(r.lb.sig), r.A, r.B, r.K, x, y, zb, ze);
        return;
    }
    mu3_block<MU3_HALO>(r.lb.g, r.psi[par], const_cast<float *>(r.lb.mu), r.A, r.B, r.K, b.bx, b.by, b.bz);
}

// site pairs of the collide-stream's list, in packed FP32
template <typename T, bool FORCE>
__global__ void __launch_bounds__(LBB_NT) vel3_batch_kernel(const BatchLists L)
{
    __shared__ LBArgs sa;
    const BatchBlock b = L.lb[blockIdx.x];
    batch_lb_args(L, L.reps[b.rep], sa);
    int x, y, zl[2], nl;
    if (packed_pair<LBB_NT>(sa.g, b.bx, b.by, b.bz, threadIdx.x, x, y, zl, nl))
        vel3_sites<F2, T, FORCE, false>(sa, PlanesFromBase<T>{(const T *)sa.fout, nullptr, sa.g.n}, x, y, zl, nl);
}

cudaError_t launch_mu3(const Geom &g, const float *psi, float *mu, float A, float B, float K, cudaStream_t st,
                       const LapW *lw)
{
    constexpr int E = 2 * MU3_HALO;
    if (!lw && g.dim == 3) {  // threads for x = -4 .. nx + 1 in fours
        const int nxt = (g.nx + 2 + 4 + 3) / 4;
        const dim3 vgrid((nxt + MV_TX - 1) / MV_TX, (g.ny + E + MV_TY - 1) / MV_TY, (g.nz + E + MV_ZC - 1) / MV_ZC);
        mu3_vec_kernel<<<vgrid, dim3(MV_TX, MV_TY, 1), 0, st>>>(g, psi, mu, A, B, K);
        return cudaGetLastError();
    }
    const dim3 block(MU_BX, MU_BY, 1);
    const dim3 grid((g.nx + E + MU_BX - 1) / MU_BX, (g.ny + E + MU_BY - 1) / MU_BY, (g.nz + E + MU_ZC - 1) / MU_ZC);
    if (lw) mu3_kernel<true><<<grid, block, 0, st>>>(g, psi, mu, A, B, K, *lw);
    else mu3_kernel<false><<<grid, block, 0, st>>>(g, psi, mu, A, B, K, LapW{0.f, 0.f, 0.f, 0.f});
    return cudaGetLastError();
}

cudaError_t launch_sigma3(const Geom &g, const float *psi, float *sig, float A, float B, float K, cudaStream_t st)
{
    const dim3 block(MU_BX, MU_BY, 1);
    const dim3 grid((g.nx + 2 + MU_BX - 1) / MU_BX, (g.ny + 2 + MU_BY - 1) / MU_BY, (g.nz + 2 + MU_ZC - 1) / MU_ZC);
    sigma3_kernel<<<grid, block, 0, st>>>(g, psi, sig, A, B, K);
    return cudaGetLastError();
}

cudaError_t launch_vel3(const LBArgs &a, int storage, cudaStream_t st)
{
    const dim3 block(LB_BX, LB_BY, 1);
    const dim3 grid((a.g.nx + LB_BX - 1) / LB_BX, (a.g.ny + LB_BY - 1) / LB_BY, (a.g.nz + LB_BZ - 1) / LB_BZ);
    const bool force = (a.coupling & FLB_COUPLE_FORCE) != 0;
    if (storage == FLB_F16_DEV) {
        if (force) vel3_kernel<__half, true><<<grid, block, 0, st>>>(a);
        else vel3_kernel<__half, false><<<grid, block, 0, st>>>(a);
    } else {
        if (force) vel3_kernel<float, true><<<grid, block, 0, st>>>(a);
        else vel3_kernel<float, false><<<grid, block, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_mu3_batch(const BatchLists &L, cudaStream_t st)
{
    if (L.nmu > 0) mu3_batch_kernel<<<L.nmu, dim3(MU_BX, MU_BY, 1), 0, st>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_vel3_batch(const BatchLists &L, int storage, bool force, cudaStream_t st)
{
    const dim3 block(LBB_NT);
    if (storage == FLB_F16_DEV) {
        if (force) vel3_batch_kernel<__half, true><<<L.nlb, block, 0, st>>>(L);
        else vel3_batch_kernel<__half, false><<<L.nlb, block, 0, st>>>(L);
    } else {
        if (force) vel3_batch_kernel<float, true><<<L.nlb, block, 0, st>>>(L);
        else vel3_batch_kernel<float, false><<<L.nlb, block, 0, st>>>(L);
    }
    return cudaGetLastError();
}

}  // namespace flb

// flb_lb15.cu -- the D3Q15 collide-stream (two sites per thread in packed FP32,
// on the box's tiles or on the batched mode's row-packed lists of site pairs) and the
// velocity of the new fluid state, on the lattice of the paper's own runs (Sec.
// VI).  The per-site work is in flb_site15.cuh.
#include "flb_site15.cuh"

namespace flb {

namespace {

// P: the population planes (in: a.fin, out: a.fout), a table of addresses.  Two
// sites per thread, (x, y, z) and (x, y, z + 1), in packed FP32 (as the D3Q19
// collide-stream).
template <typename T, bool GHOST_RELAX, bool FORCE>
__global__ void __launch_bounds__(LB_BX *LB_BY, 7) lb15_kernel(const LBArgs a, const __grid_constant__ PlaneTable<T> P)
{
    const Geom &g = a.g;
    const int x = blockIdx.x * LB_BX + threadIdx.x;
    const int y = blockIdx.y * LB_BY + threadIdx.y;
    const int z = blockIdx.z * LB_BZ;
    if (x >= g.nx || y >= g.ny || z >= g.nz) return;
    const int nl = z + 1 < g.nz ? 2 : 1;
    const int zl[2] = {z, z + nl - 1};
    F2 Fx = F2::bc(0.f), Fy = F2::bc(0.f), Fz = F2::bc(0.f);
    if (FORCE) force3v<false>(a, x, y, zl, Fx, Fy, Fz);
    lb15_sites<F2, T, GHOST_RELAX>(a, P, x, y, zl, nl, Fx, Fy, Fz);
}

// u of the streamed state, one thread per site (plane addresses formed from
// a.fout, as in the D3Q19 velocity gather).
template <typename T, bool FORCE>
__global__ void __launch_bounds__(LB_BX *LB_BY *LB_BZ) vel15_kernel(const LBArgs a)
{
    const Geom &g = a.g;
    const int x = blockIdx.x * LB_BX + threadIdx.x;
    const int y = blockIdx.y * LB_BY + threadIdx.y;
    const int z = blockIdx.z * LB_BZ + threadIdx.z;
    if (x >= g.nx || y >= g.ny || z >= g.nz) return;
    vel15_site<T, FORCE>(a, x, y, z);
}

// ---- batched variants: block b of the launch works on the row-packed entry L.lb[b]
// of 128 site pairs (x, y, z), (x, y, z+1) ----
template <typename T, bool GHOST_RELAX, bool FORCE>
__global__ void __launch_bounds__(LBB_NT, 7) lb15_batch_kernel(const BatchLists L)
{
    __shared__ LBArgs sa;
    const BatchBlock b = L.lb[blockIdx.x];
    batch_lb_args(L, L.reps[b.rep], sa);
    int x, y, zl[2], nl;
    if (!packed_pair<LBB_NT>(sa.g, b.bx, b.by, b.bz, threadIdx.x, x, y, zl, nl)) return;
    F2 Fx = F2::bc(0.f), Fy = F2::bc(0.f), Fz = F2::bc(0.f);
    if (FORCE && (sa.coupling & FLB_COUPLE_FORCE)) force3v<false>(sa, x, y, zl, Fx, Fy, Fz);
    lb15_sites<F2, T, GHOST_RELAX, false, true>(sa, PlanesFromBase<T>{(const T *)sa.fin, (T *)sa.fout, sa.g.n}, x, y,
                                                zl, nl, Fx, Fy, Fz);
}

// the velocity of the pair's sites, one after the other (one site per pass)
template <typename T, bool FORCE>
__global__ void __launch_bounds__(LBB_NT) vel15_batch_kernel(const BatchLists L)
{
    __shared__ LBArgs sa;
    const BatchBlock b = L.lb[blockIdx.x];
    batch_lb_args(L, L.reps[b.rep], sa);
    int x, y, zl[2], nl;
    if (packed_pair<LBB_NT>(sa.g, b.bx, b.by, b.bz, threadIdx.x, x, y, zl, nl))
        for (int l = 0; l < nl; ++l) vel15_site<T, FORCE>(sa, x, y, zl[l]);
}

}  // namespace

// the batched collide-stream and velocity of D3Q15 replicas (mu first when the force is coupled)
cudaError_t launch_lb15_batch(const BatchLists &L, int storage, bool ghost, bool force, cudaStream_t st)
{
    const dim3 block(LBB_NT);
    if (force) {
        const cudaError_t e = launch_mu3_batch(L, st);
        if (e != cudaSuccess) return e;
    }
#define FLB_LB15B(T, G, F) lb15_batch_kernel<T, G, F><<<L.nlb, block, 0, st>>>(L)
    if (storage == FLB_F16_DEV) {
        if (ghost) { if (force) FLB_LB15B(__half, true, true); else FLB_LB15B(__half, true, false); }
        else { if (force) FLB_LB15B(__half, false, true); else FLB_LB15B(__half, false, false); }
    } else {
        if (ghost) { if (force) FLB_LB15B(float, true, true); else FLB_LB15B(float, true, false); }
        else { if (force) FLB_LB15B(float, false, true); else FLB_LB15B(float, false, false); }
    }
#undef FLB_LB15B
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (storage == FLB_F16_DEV) {
        if (force) vel15_batch_kernel<__half, true><<<L.nlb, block, 0, st>>>(L);
        else vel15_batch_kernel<__half, false><<<L.nlb, block, 0, st>>>(L);
    } else {
        if (force) vel15_batch_kernel<float, true><<<L.nlb, block, 0, st>>>(L);
        else vel15_batch_kernel<float, false><<<L.nlb, block, 0, st>>>(L);
    }
    return cudaGetLastError();
}

cudaError_t launch_lb15(const LBArgs &a, int storage, cudaStream_t st)
{
    const dim3 block(LB_BX, LB_BY, 1);
    const dim3 grid((a.g.nx + LB_BX - 1) / LB_BX, (a.g.ny + LB_BY - 1) / LB_BY, (a.g.nz + LB_BZ - 1) / LB_BZ);
    const bool gr = a.gamma_g != 0.0f;
    const bool force = (a.coupling & FLB_COUPLE_FORCE) != 0;
#define FLB_LB15(T, G, F) lb15_kernel<T, G, F><<<grid, block, 0, st>>>(a, plane_table<T>(a.fin, a.fout, a.g.n, 15))
    if (storage == FLB_F16_DEV) {
        if (gr) { if (force) FLB_LB15(__half, true, true); else FLB_LB15(__half, true, false); }
        else { if (force) FLB_LB15(__half, false, true); else FLB_LB15(__half, false, false); }
    } else {
        if (gr) { if (force) FLB_LB15(float, true, true); else FLB_LB15(float, true, false); }
        else { if (force) FLB_LB15(float, false, true); else FLB_LB15(float, false, false); }
    }
#undef FLB_LB15
    return cudaGetLastError();
}

cudaError_t launch_vel15(const LBArgs &a, int storage, cudaStream_t st)
{
    const dim3 block(LB_BX, LB_BY, LB_BZ);
    const dim3 grid((a.g.nx + LB_BX - 1) / LB_BX, (a.g.ny + LB_BY - 1) / LB_BY, (a.g.nz + LB_BZ - 1) / LB_BZ);
    const bool force = (a.coupling & FLB_COUPLE_FORCE) != 0;
    if (storage == FLB_F16_DEV) {
        if (force) vel15_kernel<__half, true><<<grid, block, 0, st>>>(a);
        else vel15_kernel<__half, false><<<grid, block, 0, st>>>(a);
    } else {
        if (force) vel15_kernel<float, true><<<grid, block, 0, st>>>(a);
        else vel15_kernel<float, false><<<grid, block, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace flb

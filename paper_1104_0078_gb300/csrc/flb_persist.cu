// flb_persist.cu -- every replica of a batched handle advanced n steps by one
// cooperative launch.
//
// The host writes one step's task list: for each phase of the step (mu, the
// collide-stream, the velocity of the new fluid state, psi stage 1, psi stage 2)
// and each replica, one task per block tile.  Blocks take tasks from a global
// ticket in list order (step after step).  A task of replica r waits until r
// has completed every task listed before it in r's own sequence, i.e. the
// whole previous phase of r: a per-replica phase barrier, not a grid-wide one,
// so the phases of different replicas overlap.  Because a task only waits on
// tasks taken earlier, by blocks that are resident (cooperative launch), the
// launch always progresses; every wait is still bounded in time, and a block
// whose wait runs out latches FLB_ETIMEOUT and raises an abort flag that every
// other block honours, so a lost task cannot hang the GPU.
//
// Coherence inside one launch: a task reads fields written by other blocks of
// the same launch, so its loads go to L2 (__ldcg) rather than the read-only
// path, a completed task is published with a fence and a counter increment,
// and a waiting block orders its acquire before its TMA reads with a
// generic-to-async proxy fence.
#include "flb_psi3d.cuh"
#include "flb_mu3d.cuh"
#include "flb_site15.cuh"

namespace flb {

namespace {

constexpr int PB_NT = PS_NT;  // 512 threads: one psi tile, 2048 row-packed LB sites, 32 x 16 mu columns
constexpr int PL_SITES = 2048; // sites of a row-packed collide-stream / velocity task (4 per thread)
constexpr int PM_BY = 16;     // y extent of a mu tile

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until *done >= need; false when the abort flag rises or limit_ns passes.
__device__ bool wait_done(const unsigned *done, unsigned need, const int *abort, unsigned long long limit_ns)
{
    if (ld_acquire(done) >= need) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1; it < (1u << 28); ++it) {
        __nanosleep(64);
        if (ld_acquire(done) >= need) return true;
        if (*(volatile const int *)abort) return false;
        if (global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// The replica's LB arguments at device step ds (buffers swapped on odd steps),
// copied by the whole block; ends with a block barrier.
__device__ __forceinline__ void lb_args_at(const BatchRep &r, long long ds, LBArgs &sa)
{
    const int *src = reinterpret_cast<const int *>(&r.lb);
    int *dst = reinterpret_cast<int *>(&sa);
    for (int k = threadIdx.x; k < (int)(sizeof(LBArgs) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        if (ds & 1) {
            const void *t = sa.fin;
            sa.fin = sa.fout;
            sa.fout = const_cast<void *>(t);
        }
        sa.psi = r.psi[ds & 1];
        sa.step = r.lb.step + ds;
    }
    __syncthreads();
}

// Q15: every replica is D3Q15 (a handle's replicas share the lattice)
template <bool Q15>
__global__ void __launch_bounds__(PB_NT, 2) persist_kernel(const PersistArgs P)
{
    extern __shared__ __align__(1024) float tsmem[];
    __shared__ LBArgs sla;
    __shared__ Psi3Args spa;
    __shared__ int s_t, s_go;
    const long long total = (long long)P.ntask * P.nsteps;
    const int t = threadIdx.x;
    for (;;) {
        if (t == 0) {
            const long long k = (long long)atomicAdd(P.ticket, 1u);
            int go = k < total && !*(volatile int *)P.abort;
            if (go) {
                const int s = (int)(k / P.ntask);
                const PTask task = P.tasks[k - (long long)s * P.ntask];
                const unsigned need = (unsigned)(s * P.L.reps[task.rep].pstep_tasks + task.need);
                go = wait_done(P.done + task.rep, need, P.abort, P.wait_ns);
                if (!go) {
                    atomicExch(P.abort, 1);
                    atomicCAS(P.status, 0, -5);  // FLB_ETIMEOUT
                } else {
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                }
            }
            s_t = (int)k;
            s_go = go;
        }
        __syncthreads();
        if (!s_go) break;
        const int s = s_t / P.ntask;
        const PTask task = P.tasks[s_t - s * P.ntask];
        const BatchRep &r = P.L.reps[task.rep];
        const long long ds = P.ds0 + s;
        if (task.phase == PH_MU) {
            const Geom &g = r.lb.g;
            // MU3_HALO ghost layers: stage 1 reads mu on its flux region + 1
            const int x = task.bx * 32 + (t & 31) - MU3_HALO, y = task.by * PM_BY + (t >> 5) - MU3_HALO;
            const int zb = task.bz * MU_ZC - MU3_HALO, ze = min(zb + MU_ZC, g.nz + MU3_HALO);
            if (x < g.nx + MU3_HALO && y < g.ny + MU3_HALO) {
                if (r.lb.force_kind == 2)
                    sigma3_column<true>(g, r.psi[ds & 1], const_cast<float *>(r.lb.sig), r.A, r.B, r.K, x, y, zb, ze);
                else
                    mu3_column<true>(g, r.psi[ds & 1], const_cast<float *>(r.lb.mu), r.A, r.B, r.K, x, y, zb, ze);
            }
        } else if (task.phase == PH_LB || task.phase == PH_VEL) {
            lb_args_at(r, ds, sla);
            const bool force = (sla.coupling & FLB_COUPLE_FORCE) != 0;
#pragma unroll 1
            for (int j = 0; j < PL_SITES / PB_NT; ++j) {
                int x, y, z;
                if (!packed_site<PL_SITES>(sla.g, task.bx, task.by, task.bz, t + PB_NT * j, x, y, z)) continue;
                if (task.phase == PH_LB) {
                    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
                    if (force) force3<true>(sla, x, y, z, Fx, Fy, Fz);
                    if (Q15) {
                        if (sla.gamma_g != 0.f) lb15_site<float, true, true, true>(sla, x, y, z, Fx, Fy, Fz);
                        else lb15_site<float, false, true, true>(sla, x, y, z, Fx, Fy, Fz);
                    } else if (sla.gamma_g != 0.f) {
                        lb_site<float, true, true, true>(sla, x, y, z, Fx, Fy, Fz);
                    } else {
                        lb_site<float, false, true, true>(sla, x, y, z, Fx, Fy, Fz);
                    }
                } else if (Q15) {
                    if (force) vel15_site<float, true, true>(sla, x, y, z);
                    else vel15_site<float, false, true>(sla, x, y, z);
                } else {
                    if (force) vel3_site<float, true, true>(sla, x, y, z);
                    else vel3_site<float, false, true>(sla, x, y, z);
                }
            }
        } else {
            const int stage = task.phase == PH_S1 ? 1 : 2;
            if (t == 0) psi_batch_args(r, ds, stage, spa);
            __syncthreads();
            if (Q15 && stage == 1) {  // the FV operators of D3Q15
                const CUtensorMap *pm = &r.map_psi[(int)(ds & 1)];
                if (r.mu_in) {
                    if (r.noise)
                        psi3_fv_tma_block<1, true, true, true, false, true, true>(pm, &r.map_u, spa, P.status, task.bx,
                                                                                 task.by, task.bz, tsmem, &r.map_mu);
                    else
                        psi3_fv_tma_block<1, false, true, false, false, true, true>(pm, &r.map_u, spa, P.status, task.bx,
                                                                                   task.by, task.bz, tsmem, &r.map_mu);
                } else if (r.noise) {
                    psi3_fv_tma_block<1, true, true, true, false, false, true>(pm, &r.map_u, spa, P.status, task.bx,
                                                                              task.by, task.bz, tsmem);
                } else {
                    psi3_fv_tma_block<1, false, true, false, false, false, true>(pm, &r.map_u, spa, P.status, task.bx,
                                                                                task.by, task.bz, tsmem);
                }
            } else if (Q15) {
                psi3_fv_tma_block<2, false, true, false, false, false, true>(&r.map_psis, &r.map_u, spa, P.status, task.bx,
                                                                            task.by, task.bz, tsmem);
            } else if (stage == 1) {
                const CUtensorMap *pm = &r.map_psi[(int)(ds & 1)];
                if (r.mu_in) {  // mu of psi^n from this step's mu tasks
                    if (r.noise)
                        psi3_fv_tma_block<1, true, true, true, false, true>(pm, &r.map_u, spa, P.status, task.bx,
                                                                            task.by, task.bz, tsmem, &r.map_mu);
                    else
                        psi3_fv_tma_block<1, false, true, false, false, true>(pm, &r.map_u, spa, P.status, task.bx,
                                                                              task.by, task.bz, tsmem, &r.map_mu);
                } else if (r.noise) {
                    psi3_fv_tma_block<1, true, true, true, false>(pm, &r.map_u, spa, P.status, task.bx, task.by, task.bz, tsmem);
                } else {
                    psi3_fv_tma_block<1, false, true, false, false>(pm, &r.map_u, spa, P.status, task.bx, task.by, task.bz, tsmem);
                }
            } else {
                psi3_fv_tma_block<2, false, true, false, false>(&r.map_psis, &r.map_u, spa, P.status, task.bx, task.by, task.bz, tsmem);
            }
        }
        __syncthreads();
        if (t == 0) {
            __threadfence();
            atomicAdd(P.done + task.rep, 1u);
        }
    }
}

}  // namespace

size_t persist_smem_bytes()
{
    const size_t f = fv_smem_floats<F1>() > fv_mu_smem_floats<F1>() ? fv_smem_floats<F1>() : fv_mu_smem_floats<F1>();
    return sizeof(float) * (f + (size_t)FV_NOISE_FLOATS);
}

// Tiles of one replica's phases in the persistent task list.
void persist_tiles(const Geom &g, int zc, int coupling, int heun, int counts[PH_COUNT])
{
    const int cx = (g.nx + 31) / 32;
    counts[PH_MU] = (coupling & FLB_COUPLE_FORCE)
                        ? ((g.nx + 2 * MU3_HALO + 31) / 32) * ((g.ny + 2 * MU3_HALO + PM_BY - 1) / PM_BY) *
                              ((g.nz + 2 * MU3_HALO + MU_ZC - 1) / MU_ZC)
                        : 0;
    counts[PH_LB] = counts[PH_VEL] = packed_blocks(g, PL_SITES);
    counts[PH_S1] = cx * ((g.ny + PS_TY - 1) / PS_TY) * ((g.nz + zc - 1) / zc);
    counts[PH_S2] = heun ? counts[PH_S1] : 0;
}

// Append the tasks of phase ph of replica rep (need = tasks of rep listed before).
void persist_tasks(std::vector<PTask> &v, int rep, int ph, const Geom &g, int zc, int need)
{
    auto push = [&](int bx, int by, int bz) {
        PTask k;
        k.rep = rep;
        k.need = need;
        k.bx = (short)bx;
        k.by = (short)by;
        k.bz = (short)bz;
        k.phase = (char)ph;
        k.pad = 0;
        v.push_back(k);
    };
    if (ph == PH_LB || ph == PH_VEL) {  // row-packed: (x0, y0, z0) of each task's first site
        for_packed_blocks(g, PL_SITES, push);
        return;
    }
    int ny, nz, nxb = (g.nx + 31) / 32;
    if (ph == PH_MU) {
        nxb = (g.nx + 2 * MU3_HALO + 31) / 32;
        ny = (g.ny + 2 * MU3_HALO + PM_BY - 1) / PM_BY;
        nz = (g.nz + 2 * MU3_HALO + MU_ZC - 1) / MU_ZC;
    } else {
        ny = (g.ny + PS_TY - 1) / PS_TY;
        nz = (g.nz + zc - 1) / zc;
    }
    for (int bz = 0; bz < nz; ++bz)
        for (int by = 0; by < ny; ++by)
            for (int bx = 0; bx < nxb; ++bx) push(bx, by, bz);
}

cudaError_t launch_persist(const PersistArgs &a, bool q15, cudaStream_t st)
{
    const size_t smem = persist_smem_bytes();
    const void *kernel = q15 ? (const void *)persist_kernel<true> : (const void *)persist_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, PB_NT, smem)) != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    const long long total = (long long)a.ntask * a.nsteps;
    const unsigned grid = (unsigned)std::min<long long>((long long)per * sms, std::max<long long>(total, 1));
    void *args[] = {const_cast<PersistArgs *>(&a)};
    return cudaLaunchCooperativeKernel(kernel, dim3(grid), dim3(PB_NT), args, smem, st);
}

}  // namespace flb

// flb_lb3d.cu -- D3Q19 fused collide-stream, two sites per thread in packed FP32
// (plain and batched modes).
//
// The kernel forms the force density of Sec. IV, F = -psi grad mu, from the mu
// field (central difference, or the FV gradient of Eq. (fvgrad) when psi moves
// by the FV scheme, so that the force is the negative adjoint of the divergence
// that advects psi), pulls its 19 populations, relaxes them in moment space with
// noise on the stress and ghost modes (Eq. bab, Sec. III) and writes the
// post-collision populations.  mu comes from mu3_kernel and the velocity that
// advects psi from vel3_kernel (flb_aux3d.cu).
//
// Indices are 32-bit (N and the padded planes are < 2^31); population plane i
// of N sites starts at fin + i*N.  The plain kernel runs seven 128-thread blocks
// per SM (72 registers, no spills): 4.08 ms at 512^3; six blocks (80 registers)
// and eight (64, spilling) measured slower.  Noise order: bulk, 3c_x^2-c^2, c_y^2-c_z^2,
// xy, yz, zx, three c^2 c_a ghosts, three c_a(c_b^2-c_g^2) ghosts, c^4,
// c^2(3c_x^2-c^2), c^2(c_y^2-c_z^2).
#include "flb_site3d.cuh"

namespace flb {

// Two sites per thread: a 32 x 4 block of threads covers a 32 x 4 x 2 tile of
// sites, thread (x, y) working on (x, y, z) and (x, y, z + 1) in the two lanes
// of Blackwell's packed FP32 registers (one issue slot for both sites' FP32
// arithmetic).  A warp covers 32 consecutive x, so every population plane is
// read and written in full rows.
template <typename T, bool GHOST_RELAX, bool FORCE>
__global__ void __launch_bounds__(LB_BX *LB_BY, 7)
    lb3_kernel(const LBArgs a, const __grid_constant__ PlaneTable<T> P)
{
    const Geom &g = a.g;
    const int x = blockIdx.x * LB_BX + threadIdx.x;
    const int y = blockIdx.y * LB_BY + threadIdx.y;
    const int z = blockIdx.z * LB_BZ;
    if (x >= g.nx || y >= g.ny || z >= g.nz) return;
    const int nl = z + 1 < g.nz ? 2 : 1;
    const int zl[2] = {z, z + nl - 1};  // a lane past the box repeats lane 0's site
    F2 Fx = F2::bc(0.f), Fy = F2::bc(0.f), Fz = F2::bc(0.f);
    if (FORCE && (a.coupling & FLB_COUPLE_FORCE)) force3v<false>(a, x, y, zl, Fx, Fy, Fz);
    lb_sites<F2, T, GHOST_RELAX, false, false>(a, P, x, y, zl, nl, Fx, Fy, Fz);
}

// ---- batched variant: block b of the launch works on the row-packed entry L.lb[b]
// of 128 site pairs (x, y, z), (x, y, z+1), in packed FP32 as above ----
template <typename T, bool GHOST_RELAX, bool FORCE>
__global__ void __launch_bounds__(LBB_NT, 7) lb3_batch_kernel(const BatchLists L)
{
    __shared__ LBArgs sa;
    const BatchBlock b = L.lb[blockIdx.x];
    batch_lb_args(L, L.reps[b.rep], sa);
    int x, y, zl[2], nl;
    if (!packed_pair<LBB_NT>(sa.g, b.bx, b.by, b.bz, threadIdx.x, x, y, zl, nl)) return;
    F2 Fx = F2::bc(0.f), Fy = F2::bc(0.f), Fz = F2::bc(0.f);
    if (FORCE && (sa.coupling & FLB_COUPLE_FORCE)) force3v<false>(sa, x, y, zl, Fx, Fy, Fz);
    lb_sites<F2, T, GHOST_RELAX, false, true>(sa, PlanesFromBase<T>{(const T *)sa.fin, (T *)sa.fout, sa.g.n}, x, y,
                                              zl, nl, Fx, Fy, Fz);
}

cudaError_t launch_lb3_batch(const BatchLists &L, int storage, bool ghost, bool force, cudaStream_t st)
{
    const dim3 block(LBB_NT);
    if (force) {
        const cudaError_t e = launch_mu3_batch(L, st);
        if (e != cudaSuccess) return e;
    }
#define FLB_LB3B(T, G, F) lb3_batch_kernel<T, G, F><<<L.nlb, block, 0, st>>>(L)
    if (storage == FLB_F16_DEV) {
        if (ghost) { if (force) FLB_LB3B(__half, true, true); else FLB_LB3B(__half, true, false); }
        else { if (force) FLB_LB3B(__half, false, true); else FLB_LB3B(__half, false, false); }
    } else {
        if (ghost) { if (force) FLB_LB3B(float, true, true); else FLB_LB3B(float, true, false); }
        else { if (force) FLB_LB3B(float, false, true); else FLB_LB3B(float, false, false); }
    }
#undef FLB_LB3B
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_vel3_batch(L, storage, force, st);
}

cudaError_t launch_lb3d(const LBArgs &a, int storage, cudaStream_t st)
{
    const dim3 block(LB_BX, LB_BY, 1);
    const dim3 grid((a.g.nx + LB_BX - 1) / LB_BX, (a.g.ny + LB_BY - 1) / LB_BY, (a.g.nz + LB_BZ - 1) / LB_BZ);
    const bool gr = a.gamma_g != 0.0f;
    const bool force = (a.coupling & FLB_COUPLE_FORCE) != 0;
#define FLB_LB3(T, G, F) lb3_kernel<T, G, F><<<grid, block, 0, st>>>(a, plane_table<T>(a.fin, a.fout, a.g.n, 19))
    if (storage == FLB_F16_DEV) {
        if (gr) { if (force) FLB_LB3(__half, true, true); else FLB_LB3(__half, true, false); }
        else { if (force) FLB_LB3(__half, false, true); else FLB_LB3(__half, false, false); }
    } else {
        if (gr) { if (force) FLB_LB3(float, true, true); else FLB_LB3(float, true, false); }
        else { if (force) FLB_LB3(float, false, true); else FLB_LB3(float, false, false); }
    }
#undef FLB_LB3
    return cudaGetLastError();
}

}  // namespace flb

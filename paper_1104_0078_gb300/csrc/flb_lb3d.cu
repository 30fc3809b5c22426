// flb_lb3d.cu -- D3Q19 fused collide-stream, one thread per site.
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
// of N sites starts at fin + i*N.  Noise order: bulk, 3c_x^2-c^2, c_y^2-c_z^2,
// xy, yz, zx, three c^2 c_a ghosts, three c_a(c_b^2-c_g^2) ghosts, c^4,
// c^2(3c_x^2-c^2), c^2(c_y^2-c_z^2).
#include "flb_site3d.cuh"

namespace flb {

// One D3Q19 site: pull, moments, relaxation with force and noise, store.
template <typename T, bool GHOST_RELAX>
__device__ __forceinline__ void lb_site(const LBArgs &a, int x, int y, int z, float Fx, float Fy, float Fz)
{
    const Geom &g = a.g;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int N = (int)g.n;
    const int row = nx, pl = nx * ny;
    const int s = x + row * y + pl * z;
    T *fout = (T *)a.fout;

    float f[19];
    pull19((const T *)a.fin, g, x, y, z, f);

    float sp[10], dp[10];
#pragma unroll
    for (int p = 1; p <= 9; ++p) {
        sp[p] = f[2 * p - 1] + f[2 * p];
        dp[p] = f[2 * p - 1] - f[2 * p];
    }
    const float drho = f[0] + ((sp[1] + sp[2] + sp[3]) + ((sp[4] + sp[5]) + (sp[6] + sp[7]) + (sp[8] + sp[9])));
    const float jx = dp[1] + (dp[4] + dp[5]) + (dp[6] + dp[7]);
    const float jy = dp[2] + (dp[4] - dp[5]) + (dp[8] + dp[9]);
    const float jz = dp[3] + (dp[6] - dp[7]) + (dp[8] - dp[9]);
    const float third = drho * (1.0f / 3.0f);
    const float Sxx = sp[1] + (sp[4] + sp[5]) + (sp[6] + sp[7]) - third;
    const float Syy = sp[2] + (sp[4] + sp[5]) + (sp[8] + sp[9]) - third;
    const float Szz = sp[3] + (sp[6] + sp[7]) + (sp[8] + sp[9]) - third;
    const float Sxy = sp[4] - sp[5], Sxz = sp[6] - sp[7], Syz = sp[8] - sp[9];

    const float rho = a.rho0 + drho;
    const float irho = __fdividef(1.0f, rho);  // ~2 ulp
    const float vx = (jx + 0.5f * Fx) * irho, vy = (jy + 0.5f * Fy) * irho, vz = (jz + 0.5f * Fz) * irho;

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

    float g10 = 0.f, g11 = 0.f, g12 = 0.f, g13 = 0.f, g14 = 0.f, g15 = 0.f, g16 = 0.f, g17 = 0.f, g18 = 0.f;
    if (GHOST_RELAX) {
        const float gg = a.gamma_g;
        const float m10 = (dp[4] + dp[5] + dp[6] + dp[7]) * (1.f / 3.f) - dp[1] * (2.f / 3.f);
        const float m11 = (dp[4] - dp[5] + dp[8] + dp[9]) * (1.f / 3.f) - dp[2] * (2.f / 3.f);
        const float m12 = (dp[6] - dp[7] + dp[8] - dp[9]) * (1.f / 3.f) - dp[3] * (2.f / 3.f);
        const float m13 = dp[4] + dp[5] - dp[6] - dp[7];
        const float m14 = -dp[4] + dp[5] + dp[8] + dp[9];
        const float m15 = dp[6] - dp[7] - dp[8] + dp[9];
        const float m16 = (f[0] + sp[4] + sp[5] + sp[6] + sp[7] + sp[8] + sp[9]) * (1.f / 3.f) -
                          (sp[1] + sp[2] + sp[3]) * (2.f / 3.f);
        const float m17 = -sp[1] + 0.5f * (sp[2] + sp[3] + sp[4] + sp[5] + sp[6] + sp[7]) - (sp[8] + sp[9]);
        const float m18 = 0.5f * (-sp[2] + sp[3] + sp[4] + sp[5] - sp[6] - sp[7]);
        g10 = gg * m10 * 13.5f;
        g11 = gg * m11 * 13.5f;
        g12 = gg * m12 * 13.5f;
        g13 = gg * m13 * 4.5f;
        g14 = gg * m14 * 4.5f;
        g15 = gg * m15 * 4.5f;
        g16 = gg * m16 * 4.5f;
        g17 = gg * m17 * 3.0f;
        g18 = gg * m18 * 9.0f;
    }
    if (a.kT > 0.f) {
        float G[16];
        const uint32_t sid = (uint32_t)s;
        normals4(a.key, a.step, sid, 0u, 0u, G);
        normals4(a.key, a.step, sid, 0u, 1u, G + 4);
        normals4(a.key, a.step, sid, 0u, 2u, G + 8);
        normals4(a.key, a.step, sid, 0u, 3u, G + 12);
        const float mun = 3.0f * rho * a.kT;
        const float sq = mun * rsqrtf(mun);  // sqrt(rho kT / c_s^2), ~2 ulp
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
    const float e0 = 4.5f * tb;
    const float h1 = 1.f / 3.f, h2 = 2.f / 3.f;
    const float w1 = 1.f / 18.f, w2 = 1.f / 36.f;
    T *fo = fout;
    st3(fo, s, (1.f / 3.f) * (drho - e0 + h1 * g16));
    float E, O;
    E = drho + 4.5f * Bxx - e0 - h2 * g16 - g17;
    O = 3.f * Ax - h2 * g10;
    st3(fo + 1ll * N, s, w1 * (E + O));
    st3(fo + 2ll * N, s, w1 * (E - O));
    E = drho + 4.5f * Byy - e0 - h2 * g16 + 0.5f * g17 - 0.5f * g18;
    O = 3.f * Ay - h2 * g11;
    st3(fo + 3ll * N, s, w1 * (E + O));
    st3(fo + 4ll * N, s, w1 * (E - O));
    E = drho + 4.5f * Bzz - e0 - h2 * g16 + 0.5f * g17 + 0.5f * g18;
    O = 3.f * Az - h2 * g12;
    st3(fo + 5ll * N, s, w1 * (E + O));
    st3(fo + 6ll * N, s, w1 * (E - O));
    const float Gev = h1 * g16 + 0.5f * g17;
    E = drho + 4.5f * (Bxx + Byy + 2.f * Bxy) - e0 + Gev + 0.5f * g18;
    O = 3.f * (Ax + Ay) + h1 * (g10 + g11) + g13 - g14;
    st3(fo + 7ll * N, s, w2 * (E + O));
    st3(fo + 8ll * N, s, w2 * (E - O));
    E = drho + 4.5f * (Bxx + Byy - 2.f * Bxy) - e0 + Gev + 0.5f * g18;
    O = 3.f * (Ax - Ay) + h1 * (g10 - g11) + g13 + g14;
    st3(fo + 9ll * N, s, w2 * (E + O));
    st3(fo + 10ll * N, s, w2 * (E - O));
    E = drho + 4.5f * (Bxx + Bzz + 2.f * Bxz) - e0 + Gev - 0.5f * g18;
    O = 3.f * (Ax + Az) + h1 * (g10 + g12) - g13 + g15;
    st3(fo + 11ll * N, s, w2 * (E + O));
    st3(fo + 12ll * N, s, w2 * (E - O));
    E = drho + 4.5f * (Bxx + Bzz - 2.f * Bxz) - e0 + Gev - 0.5f * g18;
    O = 3.f * (Ax - Az) + h1 * (g10 - g12) - g13 - g15;
    st3(fo + 13ll * N, s, w2 * (E + O));
    st3(fo + 14ll * N, s, w2 * (E - O));
    E = drho + 4.5f * (Byy + Bzz + 2.f * Byz) - e0 + h1 * g16 - g17;
    O = 3.f * (Ay + Az) + h1 * (g11 + g12) + g14 - g15;
    st3(fo + 15ll * N, s, w2 * (E + O));
    st3(fo + 16ll * N, s, w2 * (E - O));
    E = drho + 4.5f * (Byy + Bzz - 2.f * Byz) - e0 + h1 * g16 - g17;
    O = 3.f * (Ay - Az) + h1 * (g11 - g12) + g14 + g15;
    st3(fo + 17ll * N, s, w2 * (E + O));
    st3(fo + 18ll * N, s, w2 * (E - O));
}

// One thread per site on a 3D grid of 32 x 4 x 2 blocks (a warp covers 32
// consecutive x, so every population plane is read and written in full rows).

// One block of the collide-stream (block coordinates bx, by, bz of the 32 x 4 x 2 grid).
template <typename T, bool GHOST_RELAX, bool FORCE>
__device__ __forceinline__ void lb3_block(const LBArgs &a, int bx, int by, int bz)
{
    const Geom &g = a.g;
    const int x = bx * LB_BX + threadIdx.x;
    const int y = by * LB_BY + threadIdx.y;
    const int z = bz * LB_BZ + threadIdx.z;
    if (x >= g.nx || y >= g.ny || z >= g.nz) return;
    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
    if (FORCE && (a.coupling & FLB_COUPLE_FORCE)) force3(a, x, y, z, Fx, Fy, Fz);
    lb_site<T, GHOST_RELAX>(a, x, y, z, Fx, Fy, Fz);
}

template <typename T, bool GHOST_RELAX, bool FORCE>
__global__ void __launch_bounds__(LB_BX *LB_BY *LB_BZ) lb3_kernel(const LBArgs a)
{
    lb3_block<T, GHOST_RELAX, FORCE>(a, blockIdx.x, blockIdx.y, blockIdx.z);
}

// ---- batched variant: block b of the launch works on L.lb[b] -------
template <typename T, bool GHOST_RELAX, bool FORCE>
__global__ void __launch_bounds__(LB_BX *LB_BY *LB_BZ) lb3_batch_kernel(const BatchLists L)
{
    __shared__ LBArgs sa;
    const BatchBlock b = L.lb[blockIdx.x];
    batch_lb_args(L, L.reps[b.rep], sa);
    lb3_block<T, GHOST_RELAX, FORCE>(sa, b.bx, b.by, b.bz);
}

cudaError_t launch_lb3_batch(const BatchLists &L, int storage, bool ghost, bool force, cudaStream_t st)
{
    const dim3 block(LB_BX, LB_BY, LB_BZ);
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
    const dim3 block(LB_BX, LB_BY, LB_BZ);
    const dim3 grid((a.g.nx + LB_BX - 1) / LB_BX, (a.g.ny + LB_BY - 1) / LB_BY, (a.g.nz + LB_BZ - 1) / LB_BZ);
    const bool gr = a.gamma_g != 0.0f;
    const bool force = (a.coupling & FLB_COUPLE_FORCE) != 0;
#define FLB_LB3(T, G, F) lb3_kernel<T, G, F><<<grid, block, 0, st>>>(a)
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

// flb_internal.cuh -- device-side building blocks shared by the library's
// kernels: the counter-based random numbers, lattice geometry of the padded
// psi/mu/u fields, and the argument blocks the host passes to each kernel.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/flb.h"

namespace flb {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).  Counter
// (site, step_lo, (stream << 16) | block, step_hi), key (seed_lo, seed_hi).
// ---------------------------------------------------------------------------
struct u32x4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = u32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Uniform in (0,1): ((x >> 9) + 1/2) 2^-23, exact in binary32.
__device__ __forceinline__ float u01(uint32_t x)
{
    return fmaf(__uint2float_rn(x >> 9), 1.0f / 8388608.0f, 1.0f / 16777216.0f);
}

// Four standard normals of one Philox block by Box-Muller on (x,y) and (z,w).
__device__ __forceinline__ void normals4(uint64_t seed, int64_t step, uint32_t site, uint32_t stream, uint32_t block,
                                         float g[4])
{
    const u32x4 r = philox4x32_10(
        u32x4{site, (uint32_t)(uint64_t)step, (stream << 16) | block, (uint32_t)((uint64_t)step >> 32)},
        (uint32_t)seed, (uint32_t)(seed >> 32));
    float s, c;
    float rad = sqrtf(-2.0f * logf(u01(r.x)));
    sincospif(2.0f * u01(r.y), &s, &c);
    g[0] = rad * c;
    g[1] = rad * s;
    rad = sqrtf(-2.0f * logf(u01(r.z)));
    sincospif(2.0f * u01(r.w), &s, &c);
    g[2] = rad * c;
    g[3] = rad * s;
}

// ---------------------------------------------------------------------------
// Geometry.  Populations: SoA planes [q][N], N = nx*ny*nz, unpadded, periodic
// by index wrap.  psi, mu, u, J: padded planes with a ghost frame of GX (x)
// and GY, GZ cells that hold periodic images, so stencil reads never wrap.
// ---------------------------------------------------------------------------
constexpr int GX = 4;  // 16-byte aligned rows of FP32
constexpr int GY = 3;
constexpr int GZ3 = 3;

struct Geom {
    int dim, nx, ny, nz;   // nz = 1 in 2D
    int gz;                // ghost cells in z (0 in 2D)
    int px, py, pz;        // padded extents
    long long n;           // interior sites
    long long pn;          // padded sites
    __host__ __device__ __forceinline__ long long pidx(int x, int y, int z) const
    {
        return (long long)(x + GX) + (long long)px * ((long long)(y + GY) + (long long)py * (long long)(z + gz));
    }
    __host__ __device__ __forceinline__ long long sidx(int x, int y, int z) const
    {
        return (long long)x + (long long)nx * ((long long)y + (long long)ny * (long long)z);
    }
};

// Store v at interior site (x,y,z) of a padded plane and at every periodic image
// of it that lies in the ghost frame within `rad` cells of the interior.
__device__ __forceinline__ void store_padded(float *a, const Geom &g, int x, int y, int z, float v, int rad)
{
    int xs[3] = {x, x, x}, ys[3] = {y, y, y}, zs[3] = {z, z, z};
    int nxi = 1, nyi = 1, nzi = 1;
    if (x < rad) xs[nxi++] = x + g.nx;
    if (x >= g.nx - rad) xs[nxi++] = x - g.nx;
    if (y < rad) ys[nyi++] = y + g.ny;
    if (y >= g.ny - rad) ys[nyi++] = y - g.ny;
    if (g.dim == 3) {
        if (z < rad) zs[nzi++] = z + g.nz;
        if (z >= g.nz - rad) zs[nzi++] = z - g.nz;
    }
    for (int k = 0; k < nzi; ++k)
        for (int j = 0; j < nyi; ++j)
            for (int i = 0; i < nxi; ++i) a[g.pidx(xs[i], ys[j], zs[k])] = v;
}

__host__ __device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// ---------------------------------------------------------------------------
// Argument blocks
// ---------------------------------------------------------------------------
struct LBArgs {
    Geom g;
    const void *fin;       // stored post-collision populations (float or __half) [q][N]
    void *fout;
    const float *psi;      // padded psi^n
    const float *mu;       // padded mu(psi^n), valid to halo 2
    float *u;              // padded velocity, images to radius 1
    float rho0;
    float omega_s, omega_b;    // shear and bulk relaxation rates
    float gamma_g;             // ghost relaxation factor
    float kT;
    float namp[16];            // sqrt((1 - gamma_k^2)/b_k) of the noisy modes, in noise order
    int coupling;
    uint64_t seed;
    int64_t step;
};

struct PsiArgs {
    Geom g;
    const float *psi;      // padded psi at the stage input
    const float *mu;       // padded mu of that psi, valid to halo 2
    const float *u;        // padded u, valid to halo 1
    const float *J;        // FV: padded deterministic node flux, valid to halo 1
    const float *eta;      // noise increment per site [N]
    const float *psi0;     // stage 2: Heun accumulator E [N]
    float *out;            // padded psi output (images to the full frame)
    float *acc;            // stage 1 of Heun: E = psi + D/2 + eta [N]
    float A, B, K, M;
    int coupling;
    int scheme;
    int stage;             // 1 or 2
    int integrator;
};

struct NoiseArgs {
    Geom g;
    float *eta;            // [N]
    float kT, M;
    int scheme;
    uint64_t seed;
    int64_t step;
};

// host launchers (flb_lb.cu, flb_psi.cu, flb_obs.cu)
cudaError_t launch_lb(const LBArgs &a, int q, int storage, cudaStream_t s);
cudaError_t launch_init_eq(const Geom &g, int q, int storage, const float *rho, const float *u, float rho0, void *f,
                           cudaStream_t st);
cudaError_t launch_mu(const Geom &g, const float *psi, float *mu, float A, float B, float K, cudaStream_t s);
cudaError_t launch_noise(const NoiseArgs &a, cudaStream_t s);
cudaError_t launch_flux(const Geom &g, int q, const float *psi, const float *mu, const float *u, float *J, float M,
                        int coupling, cudaStream_t s);
cudaError_t launch_psi_update(const PsiArgs &a, int q, cudaStream_t s);

}  // namespace flb

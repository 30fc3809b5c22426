// flb_init.cu -- the equilibrium start of a replica (flb_params.init =
// FLB_INIT_EQUILIBRIUM): the paper's runs start from equilibrium (Sec. VI).
//
// Fluid: the stationary law of the linearised fluctuating LB at rest is
// independent normal population deviations of variance mu_n w_i with
// mu_n = rho0 kT / c_s^2 (Sec. III): the stored post-collision deviation of
// population i at site s is sqrt(mu_n w_i) g_i(s), g from Philox stream 3.
//
// Order parameter: the Gibbs law of the Gaussian part of the free energy,
// A/2 psi^2 + K/2 |grad psi|^2, has S(q) = kT/(A - K L(q)) (Eq. test2) with L the
// symbol of the Laplacian in mu.  Mode t = kx + nx (ky + ny kz) (FFT order) draws
// (a, b) from Philox stream 4 and takes X(q) = sqrt(S(q)/N) (a + i b), X(0) = 0;
// psi = Re sum_q X(q) e^{iq.r}, so <|psi~(q)|^2> = N S(q) for every q != 0 and the
// mean of psi is zero.  The mode sum is a separable inverse DFT (x, then y, then
// z), one thread per output with twiddles from sincospif of the exactly reduced
// phase; the intermediates live in the replica's spare population buffer, which
// the first step overwrites.
#include "flb_internal.cuh"

namespace flb {
namespace {

// D3Q19 / D3Q15 / D2Q9 weights in plane order (rest, then opposite pairs)
__device__ __forceinline__ float lattice_weight(int q, int i)
{
    if (i == 0) return q == 19 ? 1.f / 3.f : q == 15 ? 2.f / 9.f : 4.f / 9.f;
    if (q == 9) return i <= 4 ? 1.f / 9.f : 1.f / 36.f;
    if (q == 15) return i <= 6 ? 1.f / 9.f : 1.f / 72.f;
    return i <= 6 ? 1.f / 18.f : 1.f / 36.f;
}

template <typename T>
__global__ void eq_pop_kernel(Geom g, int q, float mun, PhiloxKey key, T *f)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.n) return;
    float G[24];
    const int nb = (q + 7) / 8;
    for (int b = 0; b < nb; ++b) normals<4>(key, 0, (uint32_t)s, 3u, (uint32_t)b, G + 8 * b);
    for (int i = 0; i < q; ++i) {
        const float v = sqrtf(mun * lattice_weight(q, i)) * G[i];
        if (sizeof(T) == 2) reinterpret_cast<__half *>(f)[(long long)i * g.n + s] = __float2half_rn(v);
        else reinterpret_cast<float *>(f)[(long long)i * g.n + s] = v;
    }
}

// X(q) for every mode of the FFT grid
__global__ void eq_modes_kernel(Geom g, LapW lw, double kT, double A, double K, PhiloxKey key, float2 *X)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.n) return;
    const int kx = (int)(t % g.nx), ky = (int)((t / g.nx) % g.ny), kz = (int)(t / ((long long)g.nx * g.ny));
    const double pi2 = 6.283185307179586476925;
    const double cx = cos(pi2 * kx / g.nx), cy = cos(pi2 * ky / g.ny), cz = g.dim == 3 ? cos(pi2 * kz / g.nz) : 1.0;
    double L;
    if (g.dim == 3)
        L = lw.c0 + lw.c1 * 2.0 * (cx + cy + cz) + lw.c2 * 4.0 * (cx * cy + cy * cz + cz * cx) + lw.c3 * 8.0 * cx * cy * cz;
    else
        L = lw.c0 + lw.c1 * 2.0 * (cx + cy) + lw.c2 * 4.0 * cx * cy;
    float Gq[2];
    normals<1>(key, 0, (uint32_t)t, 4u, 0u, Gq);
    const float amp = t == 0 ? 0.f : (float)sqrt(kT / (A - K * L) / (double)g.n);
    X[t] = make_float2(amp * Gq[0], amp * Gq[1]);
}

// e^{2 pi i m / n} for 0 <= m < n
__device__ __forceinline__ float2 twiddle(long long m, int n)
{
    float s, c;
    sincospif(2.0f * (float)m / (float)n, &s, &c);
    return make_float2(c, s);
}

// out[..][a][..] = sum_k in[..][k][..] e^{2 pi i k a / n} along one axis of
// extent n and stride st (elements), over all N outputs
__global__ void idft_axis_kernel(long long N, int n, long long st, const float2 *in, float2 *out)
{
    const long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= N) return;
    const int a = (int)((o / st) % n);
    const long long base = o - (long long)a * st;
    float re = 0.f, im = 0.f;
    long long m = 0;  // k a mod n
    for (int k = 0; k < n; ++k) {
        const float2 v = in[base + (long long)k * st];
        const float2 w = twiddle(m, n);
        re = fmaf(v.x, w.x, fmaf(-v.y, w.y, re));
        im = fmaf(v.x, w.y, fmaf(v.y, w.x, im));
        m += a;
        if (m >= n) m -= n;
    }
    out[o] = make_float2(re, im);
}

__global__ void real_part_kernel(long long N, const float2 *in, float *out)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < N) out[s] = in[s].x;
}

}  // namespace

cudaError_t launch_pad(const Geom &g, const float *interior, float *padded, cudaStream_t st);

cudaError_t launch_equilibrium_start(const Geom &g, int q, int storage, const LapW &lw, double rho0, double kT,
                                     double A, double K, uint64_t seed, void *f, void *spare, float *psi,
                                     cudaStream_t st)
{
    const int bs = 256;
    const unsigned nb = (unsigned)((g.n + bs - 1) / bs);
    const PhiloxKey key = philox_key(seed);
    const float mun = (float)(3.0 * rho0 * kT);
    if (storage == FLB_F16_DEV) eq_pop_kernel<__half><<<nb, bs, 0, st>>>(g, q, mun, key, (__half *)f);
    else eq_pop_kernel<float><<<nb, bs, 0, st>>>(g, q, mun, key, (float *)f);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    float2 *X = (float2 *)spare, *Y = X + g.n;  // 16 bytes per site of the spare buffer
    eq_modes_kernel<<<nb, bs, 0, st>>>(g, lw, kT, A, K, key, X);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const long long N = g.n, sxy = (long long)g.nx * g.ny;
    idft_axis_kernel<<<nb, bs, 0, st>>>(N, g.nx, 1, X, Y);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    idft_axis_kernel<<<nb, bs, 0, st>>>(N, g.ny, g.nx, Y, X);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const float2 *W = X;
    if (g.dim == 3) {
        idft_axis_kernel<<<nb, bs, 0, st>>>(N, g.nz, sxy, X, Y);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        W = Y;
    }
    float *interior = (float *)(W == X ? Y : X);  // the other half holds psi's interior values
    real_part_kernel<<<nb, bs, 0, st>>>(N, W, interior);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_pad(g, interior, psi, st);
}

}  // namespace flb

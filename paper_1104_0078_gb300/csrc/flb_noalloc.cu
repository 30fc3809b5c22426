// flb_noalloc.cu -- static structure factor of one device field without any
// device allocation: flb_structure_factor_noalloc().
//
// The handle-based path (flb_sample / flb_structure_factor) keeps its DFT
// intermediates in the caller's workspace.  Some callers cannot obtain device
// memory at all at the point where they want a spectrum -- code running under a
// memory pool that forbids raw cudaMalloc, a plug-in handed only a stream and
// device pointers by its host application, or a real-time loop that must not
// allocate.  This entry point serves them: its two DFT intermediates live in a
// file-scope __device__ array of fixed size that every GPU loading the library
// holds until the process exits, so a call needs no memory beyond the caller's
// own input and output.
#include "flb_internal.cuh"

namespace flb {
namespace {

// Scratch: two halves of NOALLOC_HALF complex values each (2 x 4 MiB).
constexpr long long NOALLOC_HALF = FLB_NOALLOC_MAX_VALUES;
static_assert(NOALLOC_HALF == (1LL << 19), "scratch size is part of the ABI");
static __device__ __align__(256) float2 g_noalloc_scratch[2 * NOALLOC_HALF];

__device__ __forceinline__ int nk_val(int j, int n, int K) { return (K >= n || j <= K / 2) ? j : n - (K - j); }

__device__ __forceinline__ float2 nk_twiddle(int k, int x, int n)
{
    const int m = (int)(((long long)k * x) % n);
    float s, c;
    sincospif(2.0f * (float)m / (float)n, &s, &c);
    return make_float2(c, -s);
}

struct NaArgs {
    const float *psi;  // [nz][ny][nx]
    int nx, ny, nz, Kx, Ky, Kz;
    float2 *X1, *X2;
    double *S;
    double scale;
};

__global__ void na_dft_x(NaArgs a)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)a.Kx * a.ny * a.nz) return;
    const int jx = (int)(t % a.Kx);
    const long long row = t / a.Kx;
    const int k = nk_val(jx, a.nx, a.Kx);
    const float *src = a.psi + row * a.nx;
    float re = 0.f, im = 0.f;
    for (int x = 0; x < a.nx; ++x) {
        const float2 w = nk_twiddle(k, x, a.nx);
        re = fmaf(src[x], w.x, re);
        im = fmaf(src[x], w.y, im);
    }
    a.X1[t] = make_float2(re, im);
}

__global__ void na_dft_y(NaArgs a)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)a.Kx * a.Ky * a.nz) return;
    const int jx = (int)(t % a.Kx);
    const int jy = (int)((t / a.Kx) % a.Ky);
    const int z = (int)(t / ((long long)a.Kx * a.Ky));
    const int k = nk_val(jy, a.ny, a.Ky);
    float re = 0.f, im = 0.f;
    for (int y = 0; y < a.ny; ++y) {
        const float2 v = a.X1[((long long)z * a.ny + y) * a.Kx + jx];
        const float2 w = nk_twiddle(k, y, a.ny);
        re += v.x * w.x - v.y * w.y;
        im += v.x * w.y + v.y * w.x;
    }
    a.X2[t] = make_float2(re, im);
}

__global__ void na_dft_z(NaArgs a)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)a.Kx * a.Ky * a.Kz) return;
    const long long plane = (long long)a.Kx * a.Ky;
    const long long xy = t % plane;
    const int k = nk_val((int)(t / plane), a.nz, a.Kz);
    double re = 0.0, im = 0.0;
    for (int z = 0; z < a.nz; ++z) {
        const float2 v = a.X2[(long long)z * plane + xy];
        const float2 w = nk_twiddle(k, z, a.nz);
        re += (double)v.x * w.x - (double)v.y * w.y;
        im += (double)v.x * w.y + (double)v.y * w.x;
    }
    a.S[t] = a.scale * (re * re + im * im);  // written, not accumulated
}

// Device address of the scratch array on the current device, looked up on every
// call (the lookup allocates nothing), so the address stays right after the
// device's context was reset and the module loaded again.
cudaError_t scratch_address(float2 **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = (float2 *)p;
    return cudaSuccess;
}

int axis_keep(int n, int kmax) { return (kmax <= 0 || 2 * kmax + 1 >= n) ? n : 2 * kmax + 1; }

}  // namespace
}  // namespace flb

extern "C" int flb_structure_factor_noalloc(const float *psi_dev, int32_t nx, int32_t ny, int32_t nz, int32_t kmax,
                                            double *S_dev, void *cuda_stream)
{
    using namespace flb;
    if (!psi_dev || !S_dev || nx < 1 || ny < 1 || nz < 1 || kmax < 0) return FLB_EINVAL;
    if ((long long)nx * ny * nz >= (1LL << 31)) return FLB_EINVAL;
    NaArgs a;
    a.psi = psi_dev;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.Kx = axis_keep(nx, kmax);
    a.Ky = axis_keep(ny, kmax);
    a.Kz = axis_keep(nz, kmax);
    const long long n1 = (long long)a.Kx * ny * nz, n2 = (long long)a.Kx * a.Ky * nz, n3 = (long long)a.Kx * a.Ky * a.Kz;
    if (n1 > NOALLOC_HALF || n2 > NOALLOC_HALF) return FLB_ENOSPC;
    // an error left pending by earlier work on this thread is not this call's:
    // report it without clearing it, and launch nothing
    if (cudaPeekAtLastError() != cudaSuccess) return FLB_ECUDA;
    float2 *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return FLB_ECUDA;
    a.X1 = base;
    a.X2 = base + NOALLOC_HALF;
    a.S = S_dev;
    a.scale = 1.0 / ((double)nx * ny * nz);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int bs = 256;
    na_dft_x<<<(unsigned)((n1 + bs - 1) / bs), bs, 0, st>>>(a);
    if (cudaGetLastError() != cudaSuccess) return FLB_ECUDA;
    na_dft_y<<<(unsigned)((n2 + bs - 1) / bs), bs, 0, st>>>(a);
    if (cudaGetLastError() != cudaSuccess) return FLB_ECUDA;
    na_dft_z<<<(unsigned)((n3 + bs - 1) / bs), bs, 0, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? FLB_OK : FLB_ECUDA;
}

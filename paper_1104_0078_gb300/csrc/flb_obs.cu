// flb_obs.cu -- observables of Sec. VI of arXiv:1104.0078 reduced on the device:
// conserved totals and velocity variance (FP64, deterministic two-pass
// reduction), the static structure factor <|psi~(q)|^2> by a separable direct
// DFT accumulated in FP64, and the capillary spectrum of the two psi = 0
// surfaces of a slab (linear interpolation of the zero in every column).
#include "flb_obs.cuh"

namespace flb {

constexpr int RED_BS = 256;

template <typename T>
__device__ __forceinline__ float ldv(const T *p, long long i);
template <>
__device__ __forceinline__ float ldv<float>(const float *p, long long i) { return p[i]; }
template <>
__device__ __forceinline__ float ldv<__half>(const __half *p, long long i) { return __half2float(p[i]); }

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Pass 1: every block reduces a grid-stride share of the sites into NRED doubles:
// {sum dev, sum j_x, sum j_y, sum j_z, sum psi, sum u_x^2, sum u_y^2, sum u_z^2, non-finite count}.
template <typename T>
__global__ void __launch_bounds__(RED_BS) totals_kernel(const Geom g, int q, const T *__restrict__ f,
                                                        const float *__restrict__ psi, const float *__restrict__ u,
                                                        double *__restrict__ partial)
{
    double acc[NRED];
#pragma unroll
    for (int k = 0; k < NRED; ++k) acc[k] = 0.0;
    const long long N = g.n;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < N; s += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(s % g.nx), y = (int)((s / g.nx) % g.ny), z = (int)(s / ((long long)g.nx * g.ny));
        float m = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
        int bad = 0;
        float fi[19];
        for (int i = 0; i < q; ++i) {
            fi[i] = ldv(f, (long long)i * N + s);
            bad |= !isfinite(fi[i]);
        }
        if (q == 19) {
            m = fi[0];
            for (int i = 1; i < 19; ++i) m += fi[i];
            jx = (fi[1] - fi[2]) + (fi[7] - fi[8]) + (fi[9] - fi[10]) + (fi[11] - fi[12]) + (fi[13] - fi[14]);
            jy = (fi[3] - fi[4]) + (fi[7] - fi[8]) - (fi[9] - fi[10]) + (fi[15] - fi[16]) + (fi[17] - fi[18]);
            jz = (fi[5] - fi[6]) + (fi[11] - fi[12]) - (fi[13] - fi[14]) + (fi[15] - fi[16]) - (fi[17] - fi[18]);
        } else if (q == 15) {
            m = fi[0];
            for (int i = 1; i < 15; ++i) m += fi[i];
            // corner pairs (7,8) +(1,1,1), (9,10) +(1,1,-1), (11,12) +(1,-1,1), (13,14) +(1,-1,-1)
            const float d4 = fi[7] - fi[8], d5 = fi[9] - fi[10], d6 = fi[11] - fi[12], d7 = fi[13] - fi[14];
            jx = (fi[1] - fi[2]) + (d4 + d5) + (d6 + d7);
            jy = (fi[3] - fi[4]) + (d4 + d5) - (d6 + d7);
            jz = (fi[5] - fi[6]) + (d4 - d5) + (d6 - d7);
        } else {
            m = fi[0];
            for (int i = 1; i < 9; ++i) m += fi[i];
            jx = (fi[1] - fi[2]) + (fi[5] - fi[6]) + (fi[7] - fi[8]);
            jy = (fi[3] - fi[4]) + (fi[5] - fi[6]) - (fi[7] - fi[8]);
        }
        const long long pi = g.pidx(x, y, z);
        const float ps = psi[pi];
        const float ux = u[pi], uy = u[g.pn + pi], uz = g.dim == 3 ? u[2 * g.pn + pi] : 0.f;
        bad |= !isfinite(ps) | !isfinite(ux) | !isfinite(uy) | !isfinite(uz);
        acc[0] += m;
        acc[1] += jx;
        acc[2] += jy;
        acc[3] += jz;
        acc[4] += ps;
        acc[5] += (double)ux * ux;
        acc[6] += (double)uy * uy;
        acc[7] += (double)uz * uz;
        acc[8] += bad;
    }
    __shared__ double sh[RED_BS / 32][NRED];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NRED; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) sh[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < NRED) {
        double t = 0.0;
        for (int w = 0; w < RED_BS / 32; ++w) t += sh[w][threadIdx.x];
        partial[(long long)blockIdx.x * NRED + threadIdx.x] = t;
    }
}

// Pass 2: one block sums the per-block partials in a fixed order.
__global__ void totals_final_kernel(const double *__restrict__ partial, int nblocks, double *__restrict__ out)
{
    const int k = threadIdx.x;
    if (k >= NRED) return;
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partial[(long long)b * NRED + k];
    out[k] = t;
}

cudaError_t launch_totals(const Geom &g, int q, int storage, const void *f, const float *psi, const float *u,
                          double *partial, int nblocks, double *out, cudaStream_t s)
{
    if (storage == FLB_F16_DEV)
        totals_kernel<__half><<<nblocks, RED_BS, 0, s>>>(g, q, (const __half *)f, psi, u, partial);
    else
        totals_kernel<float><<<nblocks, RED_BS, 0, s>>>(g, q, (const float *)f, psi, u, partial);
    totals_final_kernel<<<1, 32, 0, s>>>(partial, nblocks, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-mode mean squares (Sec. III: every non-conserved mode carries
// <m_k^2> = (rho kT / c_s^2) b_k in equilibrium): each site pulls its physical
// populations fbar_i(r) = stored_i(r - c_i) (deviations from w_i rho0), projects
// them on the moment basis and adds m_k^2 in FP64; blocks reduce as for the totals.
// ---------------------------------------------------------------------------
__constant__ int8_t kMsq19[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                     {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                     {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                     {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
__constant__ int8_t kMsq15[15][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},
                                     {0, 0, 1},  {0, 0, -1}, {1, 1, 1},   {-1, -1, -1}, {1, 1, -1},
                                     {-1, -1, 1}, {1, -1, 1}, {-1, 1, -1}, {1, -1, -1}, {-1, 1, 1}};
__constant__ int8_t kMsq9[9][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                                   {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};

template <typename T>
__global__ void __launch_bounds__(RED_BS) mode_msq_kernel(const Geom g, const ModeBasis B, const T *__restrict__ f,
                                                          double *__restrict__ partial)
{
    const int q = B.q;
    double acc[NMSQ];
#pragma unroll
    for (int k = 0; k < NMSQ; ++k) acc[k] = 0.0;
    const long long N = g.n;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < N; s += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(s % g.nx), y = (int)((s / g.nx) % g.ny), z = (int)(s / ((long long)g.nx * g.ny));
        float d[19];
        int bad = 0;
        for (int i = 0; i < q; ++i) {
            const int8_t *c = q == 19 ? kMsq19[i] : q == 15 ? kMsq15[i] : kMsq9[i];
            const long long src =
                g.sidx(wrapi(x - c[0], g.nx), wrapi(y - c[1], g.ny), g.dim == 3 ? wrapi(z - c[2], g.nz) : 0);
            d[i] = ldv(f, (long long)i * N + src);
            bad |= !isfinite(d[i]);
        }
        for (int k = 0; k < q; ++k) {
            float m = 0.f;
            for (int i = 0; i < q; ++i) m = fmaf(B.E[k * q + i], d[i], m);
            acc[k] += (double)m * m;
        }
        acc[NMSQ - 1] += bad;
    }
    __shared__ double sh[RED_BS / 32][NMSQ];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NMSQ; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) sh[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < NMSQ) {
        double t = 0.0;
        for (int w = 0; w < RED_BS / 32; ++w) t += sh[w][threadIdx.x];
        partial[(long long)blockIdx.x * NMSQ + threadIdx.x] = t;
    }
}

__global__ void msq_final_kernel(const double *__restrict__ partial, int nblocks, double *__restrict__ out)
{
    const int k = threadIdx.x;
    if (k >= NMSQ) return;
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partial[(long long)b * NMSQ + k];
    out[k] = t;
}

cudaError_t launch_mode_msq(const Geom &g, int storage, const ModeBasis &B, const void *f, double *partial,
                            int nblocks, double *out, cudaStream_t s)
{
    if (storage == FLB_F16_DEV)
        mode_msq_kernel<__half><<<nblocks, RED_BS, 0, s>>>(g, B, (const __half *)f, partial);
    else
        mode_msq_kernel<float><<<nblocks, RED_BS, 0, s>>>(g, B, (const float *)f, partial);
    msq_final_kernel<<<1, 32, 0, s>>>(partial, nblocks, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Separable DFT.  Axis lists: index j of an axis of length n with window kmax
// (K = 2 kmax + 1 < n) is k = j for j <= kmax and n - (K - j) otherwise; with
// K = n every k is kept.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int kval(int j, int n, int K) { return (K >= n || j <= K / 2) ? j : n - (K - j); }

__device__ __forceinline__ float2 twiddle(int k, int x, int n)
{
    // e^{-2 pi i k x / n}, argument reduced exactly in integers first
    const int m = (int)(((long long)k * x) % n);
    float s, c;
    sincospif(2.0f * (float)m / (float)n, &s, &c);
    return make_float2(c, -s);
}

// Twiddle table e^{-2 pi i m / n}, m < n, in shared memory (n <= TW_MAX); each
// output then walks its phase index m = k x mod n by additions.
constexpr int TW_MAX = 4096;

__device__ __forceinline__ void fill_twiddles(float2 *tw, int n)
{
    for (int m = threadIdx.x; m < n; m += blockDim.x) tw[m] = twiddle(1, m, n);
    __syncthreads();
}

// X1[(z*ny + y)*Kx + jx] = sum_x in(x,y,z) e^{-i qx x}
__global__ void dft_x_kernel(DftArgs a)
{
    extern __shared__ float2 tw[];
    fill_twiddles(tw, a.nx);
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = (long long)a.Kx * a.ny * a.nz;
    if (t >= tot) return;
    const int jx = (int)(t % a.Kx);
    const long long row = t / a.Kx;  // z*ny + y
    const int y = (int)(row % a.ny), z = (int)(row / a.ny);
    const int k = kval(jx, a.nx, a.Kx);
    const float *src = a.in + a.off + (long long)y * a.sy + (long long)z * a.sz;
    float re = 0.f, im = 0.f;
    int m = 0;
    for (int x = 0; x < a.nx; ++x) {
        const float v = src[x];
        const float2 w = tw[m];
        re = fmaf(v, w.x, re);
        im = fmaf(v, w.y, im);
        m += k;
        if (m >= a.nx) m -= a.nx;
    }
    a.X1[t] = make_float2(re, im);
}

// The same X1 for windows of Kx <= 32 on rows of nx <= 1024, as a small matrix
// product over blocks of DXR_R rows.  The input is real, so X(-k) = conj X(k):
// only the kept k = 0 .. Kx/2 are summed (nu of them), each written with its
// partner.  A block builds the table e^{-2 pi i m / nx} once; chunks of DXR_CX
// columns of its rows are copied into two shared-memory buffers by cp.async
// (the next chunk in flight while the current one is summed), the chunk's
// twiddles e^{-2 pi i k x / nx} (k x reduced mod nx exactly, as twiddle() does)
// are taken from the table, and thread t sums row t, sequentially in x.
constexpr int DXR_R = 128, DXR_CX = 32, DXR_NMAX = 1024, DXR_PS = DXR_R * (DXR_CX + 1);

__device__ __forceinline__ int conj_partner(int j, int n, int K) { return j == 0 ? 0 : (K >= n ? n - j : K - j); }

// dynamic shared memory of dft_x_rows_kernel<NUP> for rows of n
template <int NUP>
constexpr size_t dxr_smem(int n)
{
    return DXR_R * sizeof(long long) + DXR_CX * NUP * sizeof(float2) + 2 * DXR_PS * sizeof(float) + n * sizeof(float2);
}

template <int NUP>
__global__ void __launch_bounds__(DXR_R) dft_x_rows_kernel(DftArgs a, long long nrows)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    long long *roff = reinterpret_cast<long long *>(dsm);                          // [DXR_R]
    float2 *Wc = reinterpret_cast<float2 *>(roff + DXR_R);                           // [DXR_CX][NUP]
    float *P = reinterpret_cast<float *>(Wc + DXR_CX * NUP);                        // [2][DXR_R][DXR_CX + 1]
    float2 *tw = reinterpret_cast<float2 *>(P + 2 * DXR_PS);                         // [n]
    const int n = a.nx, nu = a.Kx / 2 + 1, t = threadIdx.x, lane = t & 31, wp = t >> 5;
    const int nch = (n + DXR_CX - 1) / DXR_CX;
    for (int m = t; m < n; m += DXR_R) tw[m] = twiddle(1, m, n);
    // this thread's copies of chunk c: rows wp, wp + 4, ..., column x0 + lane
    auto stage = [&](int c) {
        float *buf = P + (c & 1) * DXR_PS;
        const int x = c * DXR_CX + lane;
        for (int rr = wp; rr < DXR_R; rr += DXR_R / 32) {
            const long long o = roff[rr];
            const bool ok = o >= 0 && x < n;
            cp_async4(buf + rr * (DXR_CX + 1) + lane, a.in + (ok ? o + x : 0), ok ? 4 : 0);
        }
    };
    for (long long r0 = (long long)blockIdx.x * DXR_R; r0 < nrows; r0 += (long long)gridDim.x * DXR_R) {
        __syncthreads();  // the table is complete; the previous group is done with roff and P
        {
            const long long r = r0 + t;
            roff[t] = r < nrows ? a.off + (r % a.ny) * a.sy + (r / a.ny) * a.sz : -1;
        }
        __syncthreads();
        stage(0);
        cp_async_commit();
        float re[NUP], im[NUP];
#pragma unroll
        for (int j = 0; j < NUP; ++j) re[j] = im[j] = 0.f;
        for (int c = 0; c < nch; ++c) {
            if (c + 1 < nch) stage(c + 1);
            cp_async_commit();
            const int x0 = c * DXR_CX;
            for (int e = t; e < DXR_CX * NUP; e += DXR_R) {
                const int i = e / NUP, j = e % NUP, x = x0 + i;
                Wc[e] = (j < nu && x < n) ? tw[(j * x) % n] : make_float2(0.f, 0.f);
            }
            cp_async_wait1();  // this thread's copies of chunk c have landed
            __syncthreads();   // everyone's copies of chunk c, and the chunk's twiddles
            const float *Pc = P + (c & 1) * DXR_PS + t * (DXR_CX + 1);
            const int cx = min(DXR_CX, n - x0);
            for (int i = 0; i < cx; ++i) {
                const float v = Pc[i];
#pragma unroll
                for (int j = 0; j < NUP; j += 2) {
                    const float4 w = *reinterpret_cast<const float4 *>(&Wc[i * NUP + j]);
                    re[j] = fmaf(v, w.x, re[j]);
                    im[j] = fmaf(v, w.y, im[j]);
                    re[j + 1] = fmaf(v, w.z, re[j + 1]);
                    im[j + 1] = fmaf(v, w.w, im[j + 1]);
                }
            }
            __syncthreads();  // chunk c's buffer and twiddles are free again
        }
        const long long r = r0 + t;
        if (r < nrows) {
            float2 *o = a.X1 + r * a.Kx;
#pragma unroll
            for (int j = 0; j < NUP; ++j) {
                if (j < nu) {
                    o[j] = make_float2(re[j], im[j]);
                    const int jp = conj_partner(j, n, a.Kx);
                    if (jp != j) o[jp] = make_float2(re[j], -im[j]);
                }
            }
        }
    }
}

// The y pass for windows with Kx Ky <= 1024: one block per plane z, thread t
// the output (jx, jy) = (t mod Kx, t / Kx); the plane's X1 rows (contiguous)
// come into shared memory DYS_YC rows at a time, and each thread sums its
// output sequentially in y.
constexpr int DYS_YC = 32;

__global__ void __launch_bounds__(1024) dft_y_slab_kernel(DftArgs a)
{
    extern __shared__ __align__(16) float2 ysm[];
    float2 *tw = ysm;               // [ny]
    float2 *Xs = ysm + a.ny;        // [DYS_YC][Kx]
    fill_twiddles(tw, a.ny);
    const int z = blockIdx.x, t = threadIdx.x, nout = a.Kx * a.Ky;
    const bool act = t < nout;
    const int jx = act ? t % a.Kx : 0, jy = act ? t / a.Kx : 0;
    const int k = kval(jy, a.ny, a.Ky);
    const float2 *src = a.X1 + (long long)z * a.ny * a.Kx;
    float re = 0.f, im = 0.f;
    int m = 0;
    for (int y0 = 0; y0 < a.ny; y0 += DYS_YC) {
        const int cy = min(DYS_YC, a.ny - y0);
        __syncthreads();  // the previous rows are consumed
        for (int e = t; e < cy * a.Kx; e += blockDim.x) Xs[e] = src[(long long)y0 * a.Kx + e];
        __syncthreads();
        if (act) {
            for (int i = 0; i < cy; ++i) {
                const float2 v = Xs[i * a.Kx + jx];
                const float2 w = tw[m];
                re += v.x * w.x - v.y * w.y;
                im += v.x * w.y + v.y * w.x;
                m += k;
                if (m >= a.ny) m -= a.ny;
            }
        }
    }
    if (act) a.X2[((long long)z * a.Ky + jy) * a.Kx + jx] = make_float2(re, im);
}

// X2[(z*Ky + jy)*Kx + jx] = sum_y X1[(z*ny + y)*Kx + jx] e^{-i qy y}
__global__ void dft_y_kernel(DftArgs a)
{
    extern __shared__ float2 tw[];
    fill_twiddles(tw, a.ny);
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = (long long)a.Kx * a.Ky * a.nz;
    if (t >= tot) return;
    const int jx = (int)(t % a.Kx);
    const int jy = (int)((t / a.Kx) % a.Ky);
    const int z = (int)(t / ((long long)a.Kx * a.Ky));
    const int k = kval(jy, a.ny, a.Ky);
    // four partial sums over y mod 4 (independent chains), added in a fixed order
    float re4[4] = {0.f, 0.f, 0.f, 0.f}, im4[4] = {0.f, 0.f, 0.f, 0.f};
    const float2 *src = a.X1 + (long long)z * a.ny * a.Kx + jx;
    int m = 0, y = 0;
    for (; y + 4 <= a.ny; y += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float2 v = src[(long long)(y + u) * a.Kx];
            const float2 w = tw[m];
            re4[u] += v.x * w.x - v.y * w.y;
            im4[u] += v.x * w.y + v.y * w.x;
            m += k;
            if (m >= a.ny) m -= a.ny;
        }
    }
    for (; y < a.ny; ++y) {
        const float2 v = src[(long long)y * a.Kx];
        const float2 w = tw[m];
        re4[0] += v.x * w.x - v.y * w.y;
        im4[0] += v.x * w.y + v.y * w.x;
        m += k;
        if (m >= a.ny) m -= a.ny;
    }
    const float re = (re4[0] + re4[1]) + (re4[2] + re4[3]), im = (im4[0] + im4[1]) + (im4[2] + im4[3]);
    a.X2[t] = make_float2(re, im);
}

// S[(jz*Ky + jy)*Kx + jx] += scale |sum_z X2[(z*Ky + jy)*Kx + jx] e^{-i qz z}|^2  (FP64).
// One warp per output: lane l sums z = l, l + 32, ... in FP64, then a
// shuffle reduction in a fixed order.
constexpr int DZ_WARPS = 8;

__global__ void __launch_bounds__(32 * DZ_WARPS) dft_z_acc_kernel(DftArgs a)
{
    extern __shared__ float2 tw[];
    fill_twiddles(tw, a.nz);
    const long long t = (long long)blockIdx.x * DZ_WARPS + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const long long tot = (long long)a.Kx * a.Ky * a.Kz;
    if (t >= tot) return;
    const long long plane = (long long)a.Kx * a.Ky;
    const long long xy = t % plane;
    const int jz = (int)(t / plane);
    const int k = kval(jz, a.nz, a.Kz);
    const int step = (int)(((long long)k * 32) % a.nz);
    int m = (int)(((long long)k * lane) % a.nz);
    double re = 0.0, im = 0.0;
    for (int z = lane; z < a.nz; z += 32) {
        const float2 v = a.X2[(long long)z * plane + xy];
        const float2 w = tw[m];
        re += (double)v.x * w.x - (double)v.y * w.y;
        im += (double)v.x * w.y + (double)v.y * w.x;
        m += step;
        if (m >= a.nz) m -= a.nz;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
        if (a.S) a.S[t] += a.scale * (re * re + im * im);
        if (a.snap) a.snap[t] = make_float2((float)re, (float)im);
    }
}

// Dynamic structure factor: correlate the newest Fourier components with those
// of the nlag - 1 samples before them, in FP64.
__global__ void dyn_corr_kernel(const float2 *__restrict__ ring, int L, int slot, int nlag, long long K,
                                double *__restrict__ acc, double scale)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= K) return;
    const float2 c = ring[(long long)slot * K + t];
    int s = slot;
    for (int l = 0; l < nlag; ++l) {
        const float2 p = ring[(long long)s * K + t];
        acc[(long long)l * K + t] += scale * ((double)c.x * p.x + (double)c.y * p.y);
        s = s == 0 ? L - 1 : s - 1;
    }
}

cudaError_t launch_dyn_corr(const float2 *ring, int L, int slot, int nlag, long long K, double *acc, double scale,
                            cudaStream_t s)
{
    const int bs = 256;
    dyn_corr_kernel<<<(unsigned)((K + bs - 1) / bs), bs, 0, s>>>(ring, L, slot, nlag, K, acc, scale);
    return cudaGetLastError();
}

cudaError_t launch_dft_accumulate(const DftArgs &a, cudaStream_t s)
{
    const int bs = 256;
    long long n1 = (long long)a.Kx * a.ny * a.nz, n2 = (long long)a.Kx * a.Ky * a.nz, n3 = (long long)a.Kx * a.Ky * a.Kz;
    if (a.nx > TW_MAX || a.ny > TW_MAX || a.nz > TW_MAX) return cudaErrorInvalidValue;
    if (a.Kx <= 32 && a.nx <= DXR_NMAX) {
        const long long rows = (long long)a.ny * a.nz;
        const unsigned grid = (unsigned)((rows + DXR_R - 1) / DXR_R);
        const int nu = a.Kx / 2 + 1;
#define FLB_DXR(NUP) dft_x_rows_kernel<NUP><<<grid, DXR_R, dxr_smem<NUP>(a.nx), s>>>(a, rows)
        if (nu <= 2) FLB_DXR(2);
        else if (nu <= 4) FLB_DXR(4);
        else if (nu <= 6) FLB_DXR(6);
        else if (nu <= 10) FLB_DXR(10);
        else FLB_DXR(18);
#undef FLB_DXR
    } else {
        dft_x_kernel<<<(unsigned)((n1 + bs - 1) / bs), bs, sizeof(float2) * a.nx, s>>>(a);
    }
    const size_t ysm = sizeof(float2) * ((size_t)a.ny + (size_t)DYS_YC * a.Kx);
    if (a.Kx * a.Ky <= 1024 && ysm <= 48 * 1024) {
        const int nt = ((a.Kx * a.Ky + 31) / 32) * 32;
        dft_y_slab_kernel<<<(unsigned)a.nz, nt, ysm, s>>>(a);
    } else {
        dft_y_kernel<<<(unsigned)((n2 + bs - 1) / bs), bs, sizeof(float2) * a.ny, s>>>(a);
    }
    dft_z_acc_kernel<<<(unsigned)((n3 + DZ_WARPS - 1) / DZ_WARPS), 32 * DZ_WARPS, sizeof(float2) * a.nz, s>>>(a);
    return cudaGetLastError();
}

// Heights of the two psi = 0 surfaces of a slab normal to z: in every column the
// first sign change in z in [0, nz/2) and in [nz/2, nz) (the next node wrapping
// periodically), located by linear interpolation; a half-column without a sign
// change reports the centre of its half.
__global__ void heights_kernel(const Geom g, const float *__restrict__ psi, float *__restrict__ h)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long ncol = (long long)g.nx * g.ny;
    if (c >= ncol) return;
    const int x = (int)(c % g.nx), y = (int)(c / g.nx);
    const int half = g.nz / 2;
    for (int part = 0; part < 2; ++part) {
        const int lo = part == 0 ? 0 : half, hi = part == 0 ? half : g.nz;
        float hv = 0.5f * (float)(lo + hi);
        for (int z = lo; z < hi; ++z) {
            const float v0 = psi[g.pidx(x, y, z)], v1 = psi[g.pidx(x, y, z + 1 == g.nz ? 0 : z + 1)];
            if ((v0 < 0.f) != (v1 < 0.f)) {
                hv = (float)z + v0 / (v0 - v1);
                break;
            }
        }
        h[part * ncol + c] = hv;
    }
}

cudaError_t launch_heights(const Geom &g, const float *psi, float *h, cudaStream_t s)
{
    const long long ncol = (long long)g.nx * g.ny;
    heights_kernel<<<(unsigned)((ncol + 255) / 256), 256, 0, s>>>(g, psi, h);
    return cudaGetLastError();
}

}  // namespace flb

namespace flb {

__constant__ int8_t kWin19[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                     {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                     {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                     {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
__constant__ int8_t kWin15[15][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},
                                     {0, 0, 1},  {0, 0, -1}, {1, 1, 1},   {-1, -1, -1}, {1, 1, -1},
                                     {-1, -1, 1}, {1, -1, 1}, {-1, 1, -1}, {1, -1, -1}, {-1, 1, 1}};
__constant__ int8_t kWin9[9][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                                   {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};

// Gather the physical (streamed) population deviations and psi of a periodic window.
template <typename T>
__global__ void window_kernel(const Geom g, int q, const T *__restrict__ f, const float *__restrict__ psi, int x0,
                              int y0, int z0, int wx, int wy, int wz, float *__restrict__ out)
{
    const long long W = (long long)wx * wy * wz;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= W) return;
    const int x = (x0 + (int)(k % wx)) % g.nx;
    const int y = (y0 + (int)((k / wx) % wy)) % g.ny;
    const int z = (z0 + (int)(k / ((long long)wx * wy))) % g.nz;
    for (int i = 0; i < q; ++i) {
        const int8_t *c = q == 19 ? kWin19[i] : q == 15 ? kWin15[i] : kWin9[i];
        const long long src = g.sidx(wrapi(x - c[0], g.nx), wrapi(y - c[1], g.ny), g.dim == 3 ? wrapi(z - c[2], g.nz) : 0);
        out[(long long)i * W + k] = ldv(f, (long long)i * g.n + src);
    }
    out[(long long)q * W + k] = psi[g.pidx(x, y, z)];
}

cudaError_t launch_window(const Geom &g, int q, int storage, const void *f, const float *psi, int x0, int y0, int z0,
                          int wx, int wy, int wz, float *out, cudaStream_t s)
{
    const long long W = (long long)wx * wy * wz;
    const unsigned grid = (unsigned)((W + 255) / 256);
    if (storage == FLB_F16_DEV)
        window_kernel<__half><<<grid, 256, 0, s>>>(g, q, (const __half *)f, psi, x0, y0, z0, wx, wy, wz, out);
    else
        window_kernel<float><<<grid, 256, 0, s>>>(g, q, (const float *)f, psi, x0, y0, z0, wx, wy, wz, out);
    return cudaGetLastError();
}

}  // namespace flb

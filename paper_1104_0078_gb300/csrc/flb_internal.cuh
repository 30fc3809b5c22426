// flb_internal.cuh -- device-side building blocks shared by the library's
// kernels: the counter-based random numbers, lattice geometry of the padded
// psi/mu/u fields, and the argument blocks the host passes to each kernel.
#pragma once

#include <vector>

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/flb.h"
#include "flb_lane.cuh"

namespace flb {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).  Counter
// (site, step_lo, (stream << 16) | block, step_hi), key (seed_lo, seed_hi).
// ---------------------------------------------------------------------------
struct u32x4 {
    uint32_t x, y, z, w;
};

// Round keys of one seed: round r uses (seed_lo + r W0, seed_hi + r W1).  They
// are computed on the host and passed in the kernel parameters, so every round
// XORs a constant operand.
struct PhiloxKey {
    uint32_t k0[10], k1[10];
};

inline PhiloxKey philox_key(uint64_t seed)
{
    PhiloxKey K;
    uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        K.k0[r] = a;
        K.k1[r] = b;
        a += 0x9E3779B9u;
        b += 0xBB67AE85u;
    }
    return K;
}

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, const PhiloxKey &K)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = u32x4{(uint32_t)(p1 >> 32) ^ c.y ^ K.k0[r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ K.k1[r],
                  (uint32_t)p0};
    }
    return c;
}

// The same ten rounds with the round keys formed from round 0's (the seed
// words) by one add per key and round: for kernels whose arguments sit in
// shared memory, where reading the twenty stored keys costs a load each.
__device__ __forceinline__ u32x4 philox4x32_10_r0(u32x4 c, uint32_t a, uint32_t b)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = u32x4{(uint32_t)(p1 >> 32) ^ c.y ^ a, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ b, (uint32_t)p0};
        a += 0x9E3779B9u;
        b += 0xBB67AE85u;
    }
    return c;
}

// ---- Box-Muller by table lookup --------------------------------------------
// One Philox word w makes one Box-Muller pair: its top 20 bits give the radius
// uniform u = ((w >> 12) + 1/2) 2^-20 and its low 12 bits the angle uniform
// v = ((w & 0xFFF) + 1/2) 2^-12, both exact in binary32, so a block of four
// words yields eight normals.  The pair is (r cos 2 pi v, r sin 2 pi v) with
// r = sqrt(-2 ln u): its radius stops at sqrt(42 ln 2) = 5.40 (the pair falls
// beyond it with probability 4.8e-7) and the 4096 equally spaced angles make
// every moment of (cos, sin) of order below 4096 the continuous one.
// The two transcendental steps are specialised to these uniforms and
// evaluated from small tables, to single-precision accuracy with fewer
// instructions than the general logf and sincospif:
//  * ln u, u = (2k+1) 2^-21: the table-driven method of P. T. P. Tang (ACM
//    TOMS 16(4), 1990).  2k+1 = 2^e f with f in [sqrt(1/2), sqrt(2)); the bits
//    of f select one of 32 cells; ln f = -ln r_j + ln(1 + d) with d = f r_j - 1
//    formed by one FMA (|d| < 1/64) and ln(1 + d) by its series to d^5 (error
//    < 3e-12).  r_j is near 1/(cell centre) and exactly 1 in the cell holding 1,
//    where d = f - 1 is exact, so u near 1 keeps its relative accuracy.  The
//    radius needs -2 ln u: the series and the table carry the factor -2, which
//    is exact in binary arithmetic.
//  * sin, cos of 2 pi v, v = (m + 1/2) 2^-12: v = j/64 + t_lo, the table of
//    sin, cos(2 pi j/64) and the angle-addition formulas with sin b, cos b of
//    b = 2 pi t_lo < 2 pi/64 by their series (to b^5 and b^4; error < 2e-9).
// The tables are computed at compile time in double precision from the same
// series and rounded to float.
namespace bm {

struct alignas(16) SinCos {
    float s, c, ns, pad;  // sin, cos and -sin of 2 pi j/64
};
struct alignas(8) LogCell {
    float r, l2r;  // r_j and 2 ln r_j
};
struct Tables {
    SinCos sc[64];
    LogCell lg[32];
};

constexpr double kPi = 3.14159265358979323846;
constexpr uint32_t kSqrtHalfBits = 0x3F3504F3u;  // bits of sqrt(1/2) in binary32

// sin and cos of x in [0, pi/2] by their Taylor series (x^31 terms: < 1e-25)
constexpr double taylor_sin(double x)
{
    double term = x, sum = x;
    for (int n = 1; n < 16; ++n) {
        term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
        sum += term;
    }
    return sum;
}
constexpr double taylor_cos(double x)
{
    double term = 1.0, sum = 1.0;
    for (int n = 1; n < 16; ++n) {
        term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
        sum += term;
    }
    return sum;
}
// ln x for x in [0.5, 2] as 2 atanh((x - 1)/(x + 1)) (|s| <= 1/3; 40 terms)
constexpr double series_log(double x)
{
    const double s = (x - 1.0) / (x + 1.0);
    double p = s, sum = 0.0;
    for (int n = 0; n < 40; ++n) {
        sum += p / (2.0 * n + 1.0);
        p *= s * s;
    }
    return 2.0 * sum;
}
// the binary32 value with bits b, for b in [0x3F000000, 0x40000000)
constexpr double f32_of_bits(uint32_t b)
{
    return b < 0x3F800000u ? 0.5 * (1.0 + (double)(b - 0x3F000000u) / 8388608.0)
                           : 1.0 + (double)(b - 0x3F800000u) / 8388608.0;
}
constexpr Tables make_tables()
{
    Tables T{};
    for (int j = 0; j < 64; ++j) {
        const int q = j / 16;  // quadrant of 2 pi j/64
        const double x = 2.0 * kPi * (j % 16) / 64.0;
        const double s = taylor_sin(x), c = taylor_cos(x);
        const double sq[4] = {s, c, -s, -c}, cq[4] = {c, -s, -c, s};
        T.sc[j].s = (float)sq[q];
        T.sc[j].c = (float)cq[q];
        T.sc[j].ns = -(float)sq[q];
        T.sc[j].pad = 0.0f;
    }
    const int one = (int)((0x3F800000u - kSqrtHalfBits) >> 18);  // the cell holding 1
    for (int j = 0; j < 32; ++j) {
        if (j == one) {
            T.lg[j].r = 1.0f;
            T.lg[j].l2r = 0.0f;
            continue;
        }
        const double lo = f32_of_bits(kSqrtHalfBits + ((uint32_t)j << 18));
        const double hi = f32_of_bits(kSqrtHalfBits + ((uint32_t)(j + 1) << 18));
        const float r = (float)(2.0 / (lo + hi));
        T.lg[j].r = r;
        T.lg[j].l2r = -2.0f * (float)(-series_log((double)r));  // -2 x (the binary32 -ln r_j)
    }
    return T;
}

}  // namespace bm

// one copy per translation unit, read through the read-only cache
static __device__ const bm::Tables kBM = bm::make_tables();

// Box-Muller on V::L independent words at once, one per lane (F2: two words in
// Blackwell's packed FP32 registers): lane l turns word w[l] into
// g0 = r cos 2 pi v, g1 = r sin 2 pi v (u, v and r as above).
// SCALED: r is multiplied by sc first (lane-wise), so the outputs come scaled.
// The integer steps, table loads and the reciprocal square root run per lane;
// every FP32 step is one lane-generic operation, so a word gets the same bits
// in either lane type.
template <class V, bool SCALED = false>
__device__ __forceinline__ void bm_eval(const uint32_t *w, V sc, V &g0, V &g1)
{
    constexpr int L = V::L;
    float f[L], lr[L], l2r[L], eb[L], xm[L], sa[L], ca[L], nsa[L];
#pragma unroll
    for (int l = 0; l < L; ++l) {
        const float fn = __uint2float_rn((w[l] >> 11) | 1u);  // 2k+1 < 2^21, exact
        const int bits = __float_as_int(fn);
        const int t = bits - (int)bm::kSqrtHalfBits;
        const int e = t >> 23;                                // 2k+1 = 2^e f
        f[l] = __int_as_float(bits - (e << 23));              // f in [sqrt(1/2), sqrt(2))
        const float2 C = __ldg(reinterpret_cast<const float2 *>(&kBM.lg[(t >> 18) & 31]));  // (r_j, 2 ln r_j)
        lr[l] = C.x;
        l2r[l] = C.y;
        eb[l] = __int_as_float(0x4B400000 + e - 21);          // 1.5 2^23 + (e - 21), exact
        const uint32_t m = w[l] & 0xFFFu;
        const float4 A = __ldg(reinterpret_cast<const float4 *>(&kBM.sc[m >> 6]));  // (sin, cos, -sin)(2 pi j/64)
        sa[l] = A.x;
        ca[l] = A.y;
        nsa[l] = A.z;
        xm[l] = __int_as_float(0x4B000000u | (m & 63u));      // 2^23 + (m mod 64), exact
    }
    // -2 ln u = -2 (e - 21) ln 2 + 2 ln r_j - 2 ln(1 + d)
    const V d = vfma(vmake<V>(f), vmake<V>(lr), V::bc(-1.0f));
    V p = vfma(d, V::bc(-0.4f), V::bc(0.5f));  // -2 x the series of ln(1 + d)/d, Horner form
    p = vfma(d, p, V::bc(-2.0f / 3.0f));
    p = vfma(d, p, V::bc(1.0f));
    p = vfma(d, p, V::bc(-2.0f));
    const V em = vmake<V>(eb) - V::bc(12582912.0f);       // e - 21, exact
    const V e2 = vfma(d, p, vfma(em, V::bc(-2.0f * 0.693147180559945f), vmake<V>(l2r)));  // >= 9.5e-7
    float rs[L];
#pragma unroll
    for (int l = 0; l < L; ++l) rs[l] = rsqrtf(e2.lane(l));
    V rad = e2 * vmake<V>(rs);
    if (SCALED) rad = rad * sc;
    // sin, cos of 2 pi v by angle addition
    const V x = vfma(vmake<V>(xm) - V::bc(8388608.0f), V::bc((float)(2.0 * bm::kPi / 4096.0)),
                     V::bc((float)(bm::kPi / 4096.0)));
    const V x2 = x * x;
    const V cb = vfma(x2, vfma(x2, V::bc(1.0f / 24.0f), V::bc(-0.5f)), V::bc(1.0f));
    const V sb = x * vfma(x2, vfma(x2, V::bc(1.0f / 120.0f), V::bc(-1.0f / 6.0f)), V::bc(1.0f));
    const V s = vfma(vmake<V>(sa), cb, vmake<V>(ca) * sb);
    const V c = vfma(vmake<V>(ca), cb, vmake<V>(nsa) * sb);
    g0 = rad * c;
    g1 = rad * s;
}

__device__ __forceinline__ uint32_t word(const u32x4 &r, int k) { return k == 0 ? r.x : k == 1 ? r.y : k == 2 ? r.z : r.w; }

__device__ __forceinline__ u32x4 philox_ctr(int64_t step, uint32_t site, uint32_t stream, uint32_t block)
{
    return u32x4{site, (uint32_t)(uint64_t)step, (stream << 16) | block, (uint32_t)((uint64_t)step >> 32)};
}

// Normals 8 block .. 8 block + 2 NP - 1 of counter (site, step, stream): the
// Box-Muller pairs of the block's first NP words (normals 2k, 2k + 1 of a block
// come from its word k), two words evaluated together in one packed register.
// KEY_R0: form the round keys from K's round-0 keys (arguments in shared memory).
// SCALED: every normal multiplied by sc.
template <int NP, bool KEY_R0 = false, bool SCALED = false>
__device__ __forceinline__ void normals(const PhiloxKey &K, int64_t step, uint32_t site, uint32_t stream,
                                        uint32_t block, float *g, float sc = 1.0f)
{
    static_assert(NP >= 1 && NP <= 4, "a Philox block has four words");
    const u32x4 c = philox_ctr(step, site, stream, block);
    const u32x4 r = KEY_R0 ? philox4x32_10_r0(c, K.k0[0], K.k1[0]) : philox4x32_10(c, K);
#pragma unroll
    for (int k = 0; k + 1 < NP; k += 2) {
        const uint32_t w[2] = {word(r, k), word(r, k + 1)};
        F2 c0, s0;
        bm_eval<F2, SCALED>(w, F2::bc(sc), c0, s0);
        g[2 * k] = c0.v.x;
        g[2 * k + 1] = s0.v.x;
        g[2 * k + 2] = c0.v.y;
        g[2 * k + 3] = s0.v.y;
    }
    if constexpr ((NP & 1) != 0) {
        const uint32_t w = word(r, NP - 1);
        F1 c0, s0;
        bm_eval<F1, SCALED>(&w, F1{sc}, c0, s0);
        g[2 * NP - 2] = c0.v;
        g[2 * NP - 1] = s0.v;
    }
}

// Normals 8 b .. 8 b + NB - 1 (NB <= 8) of stream 0, block b, at the V::L sites
// site[l], scaled lane-wise by sc: n[k] holds normal 8 b + k of every lane's
// site (n has room for NB rounded up to even).  F2: the lanes are the two
// sites; F1: the site's words are evaluated in pairs in one packed register.
// A caller consumes one block's normals before drawing the next, so that at
// most eight are live.
template <int NB, bool KEY_R0, class V>
__device__ __forceinline__ void lane_block(const PhiloxKey &K, int64_t step, const uint32_t *site, uint32_t b, V sc,
                                           V *n)
{
    static_assert(NB >= 1 && NB <= 8, "a Philox block gives eight normals");
    constexpr int L = V::L, NPAIR = (NB + 1) / 2;
    u32x4 r[L];
#pragma unroll
    for (int l = 0; l < L; ++l) {
        const u32x4 c = philox_ctr(step, site[l], 0u, b);
        r[l] = KEY_R0 ? philox4x32_10_r0(c, K.k0[0], K.k1[0]) : philox4x32_10(c, K);
    }
    if constexpr (L == 2) {
#pragma unroll
        for (int k = 0; k < NPAIR; ++k) {
            const uint32_t w[2] = {word(r[0], k), word(r[1], k)};
            bm_eval<V, true>(w, sc, n[2 * k], n[2 * k + 1]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < NPAIR; k += 2) {
            const uint32_t w[2] = {word(r[0], k), word(r[0], k + 1)};
            F2 c0, s0;
            bm_eval<F2, true>(w, F2::bc(sc.lane(0)), c0, s0);
            n[2 * k] = V::bc(c0.v.x);
            n[2 * k + 1] = V::bc(s0.v.x);
            if (k + 1 < NPAIR) {
                n[2 * k + 2] = V::bc(c0.v.y);
                n[2 * k + 3] = V::bc(s0.v.y);
            }
        }
    }
}

// 4-byte asynchronous copy global -> shared (cp.async); src_bytes 0 writes a
// zero and reads nothing.  commit closes this thread's group of copies;
// wait1 waits until at most the newest group is still in flight.
__device__ __forceinline__ void cp_async4(float *dst, const float *src, int src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// ---------------------------------------------------------------------------
// Geometry.  Populations: SoA planes [q][N], N = nx*ny*nz, unpadded, periodic
// by index wrap.  psi, mu, u, J: padded planes with a ghost frame of GX (x)
// and GY, GZ cells that hold periodic images, so stencil reads never wrap.
// ---------------------------------------------------------------------------
constexpr int GX = 4;  // 16-byte aligned rows of FP32
constexpr int GY = 3;
constexpr int GZ3 = 3;

// launch geometry of the 3D kernels (shared with the host for the batched block lists)
constexpr int LB_BX = 32, LB_BY = 4, LB_BZ = 2;   // collide-stream and mu: one thread per site
constexpr int MU_BX = 32, MU_BY = 4, MU_ZC = 16;  // mu: column tile and planes of a block
// Ghost layers of the mu field written by the per-phase and batched mu kernels:
// 1 for the force's gradient, 2 for the FV psi stage 1, which reads mu on its
// flux region + 1.
constexpr int MU3_HALO = 2;
constexpr int PS_TX = 32, PS_TY = 16;  // psi stage: column tile of a block
constexpr int PS_ZC = 64;              // psi stage: default planes per block (the z chunk), tunable per replica
constexpr int PS_ZC_MIN = 1;           // smallest z chunk (sizes the batched block lists)

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
    __host__ __device__ __forceinline__ int pidx32(int x, int y, int z) const
    {
        return (x + GX) + px * ((y + GY) + py * (z + gz));
    }
    __host__ __device__ __forceinline__ long long sidx(int x, int y, int z) const
    {
        return (long long)x + (long long)nx * ((long long)y + (long long)ny * (long long)z);
    }
};

// Store v at interior site (x,y,z) of a padded plane and at every periodic image
// of it that lies in the ghost frame within `rad` cells of the interior.  When
// every edge is at least 2 rad long a site has at most one image per axis, and
// the images are the (at most 7) combinations of those offsets; shorter edges
// take the general path over all candidate images.  No local memory is used.
__device__ __forceinline__ void store_padded(float *a, const Geom &g, int x, int y, int z, float v, int rad)
{
    const int c = g.pidx32(x, y, z);
    a[c] = v;
    const bool ix = x >= rad && x < g.nx - rad, iy = y >= rad && y < g.ny - rad;
    const bool iz = g.dim == 2 || (z >= rad && z < g.nz - rad);
    if (ix && iy && iz) return;
    if (g.nx >= 2 * rad && g.ny >= 2 * rad && (g.dim == 2 || g.nz >= 2 * rad)) {
        const int ox = ix ? 0 : (x < rad ? g.nx : -g.nx);
        const int oy = iy ? 0 : (y < rad ? g.ny : -g.ny) * g.px;
        const int oz = iz ? 0 : (z < rad ? g.nz : -g.nz) * g.px * g.py;
        if (ox) a[c + ox] = v;
        if (oy) a[c + oy] = v;
        if (ox && oy) a[c + ox + oy] = v;
        if (oz) {
            a[c + oz] = v;
            if (ox) a[c + oz + ox] = v;
            if (oy) a[c + oz + oy] = v;
            if (ox && oy) a[c + oz + ox + oy] = v;
        }
        return;
    }
    const int xs[3] = {x, x + g.nx, x - g.nx};
    const bool vx[3] = {true, x < rad, x >= g.nx - rad};
    const int ys[3] = {y, y + g.ny, y - g.ny};
    const bool vy[3] = {true, y < rad, y >= g.ny - rad};
    const int zs[3] = {z, z + g.nz, z - g.nz};
    const bool vz[3] = {true, g.dim == 3 && z < rad, g.dim == 3 && z >= g.nz - rad};
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i)
                if ((i | j | k) && vz[k] && vy[j] && vx[i]) a[g.pidx(xs[i], ys[j], zs[k])] = v;
}

__host__ __device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// mu = A psi + B psi^3 - K lap_SO psi (Sec. II.A) from the partial sums of the SO
// stencil (Eq. solap): 22 lap_SO psi = 6 n1 + 3 n2 + n3 - 80 psi, with n1, n2, n3
// the sums over the faces, edges and corners.  Every operation is rounded
// explicitly, so the mu field and the FV stage's own mu get the same bits.
__device__ __forceinline__ float mu_so(float A, float B, float k22, float ps, float n1, float n2, float n3)
{
    const float l22 = __fmaf_rn(6.f, n1, __fmaf_rn(3.f, n2, __fmaf_rn(-80.f, ps, n3)));
    return __fmaf_rn(-k22, l22, __fmaf_rn(__fmul_rn(B, __fmul_rn(ps, ps)), ps, __fmul_rn(A, ps)));
}

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
    // D3Q19 collide-stream, in the units of its scaled stress Q = 4.5 B and scaled
    // ghosts: rq = 4.5 (1 - ws), 4.5 ws, 4.5 cs (cs = 1 - ws/2), 1.5 (wb - ws),
    // 3 (cb - cs); iso: wb != ws; k3T = kT / c_s^2; nq: the noise amplitudes
    // namp scaled to those units
    float rq[5];
    int iso;
    float k3T;
    float nq[15];
    int coupling;
    int force_kind;            // 0: -psi grad_CD mu, 1: -psi grad_FV mu (D3Q19), 2: -div sigma (stress
                               // form), 3: -psi grad_FV mu on the D3Q15 neighbourhood
    const float *sig;          // stress form: padded sigma planes xx, yy, zz, xy, xz, yz (2D: xx, yy, xy)
    PhiloxKey key;
    int64_t step;
};

// A Laplacian stencil of App. A by neighbour class: c0 at the centre, c1 on the
// faces, c2 on the edges, c3 on the corners (2D: c1 axes, c2 diagonals).
struct LapW {
    float c0, c1, c2, c3;
};

struct PsiArgs {
    Geom g;
    LapW lw;               // FD / naive: the Laplacian of mu and of M lap mu
    int q;                 // FV: the lattice of the gradient and divergence (9, 15 or 19)
    const float *psi;      // padded psi at the stage input
    const float *mu;       // padded mu of that psi, valid to halo 2
    const float *u;        // padded u, valid to halo 1
    const float *J;        // FV: padded deterministic node flux, valid to halo 1
    const float *eta;      // noise increment per site [N]
    const float *psi0;     // stage 2: Heun accumulator E [N]
    float *out;            // padded psi output (images to the full frame)
    float *acc;            // stage 1 of Heun: E = psi + D/2 + eta [N]; RK4: the running sum
    const float *base;     // RK4: padded psi^n
    float A, B, K, M;
    int coupling;
    int scheme;
    int stage;             // 1 or 2 (RK4: 1 to 4)
    int integrator;
};

struct NoiseArgs {
    Geom g;
    float *eta;            // [N]
    float kT, M;
    int scheme;
    int q;                 // FV: lattice of the noise divergence
    LapW lw;               // FD: link weights are the Laplacian's class coefficients
    PhiloxKey key;
    int64_t step;
};

// ---------------------------------------------------------------------------
// Batched mode: every replica of a handle advances in one launch per phase.
// Each launch walks a block list (replica, block coordinates); per-replica data
// sit in a device table of BatchRep records.  The step counter is a device
// value (dstep, steps since the table was written), so one captured graph of a
// step can be replayed: on even dstep the "A" buffers are current, on odd the
// "B" buffers.
// ---------------------------------------------------------------------------
struct alignas(128) BatchRep {
    CUtensorMap map_psi[2];  // tensor maps of psiA, psiB
    CUtensorMap map_psis;    // tensor map of psi* (Heun)
    CUtensorMap map_u;       // tensor map of u (3 components)
    CUtensorMap map_mu;      // tensor map of mu (FV stage 1 reads it when mu_in)
    LBArgs lb;               // fin = fA, fout = fB, psi = psiA; step = step0
    float *psi[2];           // psiA, psiB
    float *psis, *E;
    float A, B, K, M;
    int heun, advect, noise;
    int mu_in;               // the step forms mu of psi^n for the force (FV stage 1 may read it)
    int q15;                 // a D3Q15 replica
    int zc;                  // planes per psi block
    int pstep_tasks;         // persistent mode: tasks of this replica per step
};

struct BatchBlock {
    int rep, bx, by, bz;
};

// Site k (0 <= k < B) of a row-packed block of B sites (the persistent
// kernel's tasks: B = 2048, four per thread).  The block starts at (x0, y0, z0);
// a box with nx <= B packs B/nx whole x-rows into the block, a wider box takes
// a B-site chunk of one row.  Rows run y-fastest and are contiguous in the
// population planes, so a warp's loads stay coalesced.  False for an idle slot.
template <int B>
__device__ __forceinline__ bool packed_row(int nx, int ny, int nz, int x0, int y0, int z0, int k, int &x, int &y,
                                           int &z)
{
    int rl = 0;
    if (nx <= B) {
        rl = k / nx;
        if (rl >= B / nx) return false;
        x = k - rl * nx;
    } else {
        x = x0 + k;
        if (x >= nx) return false;
    }
    y = y0 + rl;
    z = z0;
    while (y >= ny) {
        y -= ny;
        ++z;
    }
    return z < nz;
}
template <int B>
__device__ __forceinline__ bool packed_site(const Geom &g, int x0, int y0, int z0, int k, int &x, int &y, int &z)
{
    return packed_row<B>(g.nx, g.ny, g.nz, x0, y0, z0, k, x, y, z);
}

// The batched collide-stream and velocity lists pack site pairs: the box's
// planes taken two at a time, (z, z+1) for even z, so that a thread works two
// sites in the lanes of packed FP32 as the plain kernels do.  Pair k of a block
// of B pairs: lanes at planes zl[0] and zl[1] (= zl[0] for the last plane of an
// odd nz, nl = 1).  The host builds the lists on pair_geom(g).
constexpr int LBB_NT = LB_BX * LB_BY;  // pairs (threads) of a batched collide-stream block
template <int B>
__device__ __forceinline__ bool packed_pair(const Geom &g, int x0, int y0, int z0, int k, int &x, int &y, int zl[2],
                                            int &nl)
{
    int zp;
    if (!packed_row<B>(g.nx, g.ny, (g.nz + 1) >> 1, x0, y0, z0, k, x, y, zp)) return false;
    const int z = 2 * zp;
    nl = z + 1 < g.nz ? 2 : 1;
    zl[0] = z;
    zl[1] = z + nl - 1;
    return true;
}
inline Geom pair_geom(const Geom &g)
{
    Geom h = g;
    h.nz = (g.nz + 1) / 2;
    return h;
}

// Entries of the row-packed list of one box for blocks of B sites (see packed_site).
inline int packed_blocks(const Geom &g, int B)
{
    if (g.nx <= B) {
        const int rpb = B / g.nx;
        return (int)(((long long)g.ny * g.nz + rpb - 1) / rpb);
    }
    return g.ny * g.nz * ((g.nx + B - 1) / B);
}

// The entries themselves, as (x0, y0, z0), in list order.
template <class F>
inline void for_packed_blocks(const Geom &g, int B, F &&emit)
{
    if (g.nx <= B) {
        const int rpb = B / g.nx;
        for (long long row = 0; row < (long long)g.ny * g.nz; row += rpb)
            emit(0, (int)(row % g.ny), (int)(row / g.ny));
    } else {
        for (int z = 0; z < g.nz; ++z)
            for (int y = 0; y < g.ny; ++y)
                for (int x0 = 0; x0 < g.nx; x0 += B) emit(x0, y, z);
    }
}

struct BatchLists {
    const BatchRep *reps;
    const BatchBlock *mu, *lb, *psi;
    int nmu, nlb, npsi;
    const long long *dstep;
    int *status;
};

cudaError_t encode_tensor_map_f32(CUtensorMap *map, const void *base, int rank, const uint64_t *dims,
                                  const uint64_t *strides_bytes, const uint32_t *box);
// mu_in: every replica's step forms mu of psi^n, so FV stage 1 reads it (map_mu)
// q15: D3Q15 replicas (collide-stream, velocity and the FV operators of D3Q15)
cudaError_t launch_batch_step(const BatchLists &L, int storage, bool ghost, bool force, int scheme_fv, bool heun,
                              bool noise, bool mu_in, bool q15, cudaStream_t st);
// the psi stage launches of a batched step alone (no state change: the autotuner times them)
cudaError_t launch_batch_psi(const BatchLists &L, bool heun, bool noise, bool mu_in, bool q15, cudaStream_t st);

// ---- persistent batched mode (flb_persist.cu) --------------------------------
enum { PH_MU = 0, PH_LB = 1, PH_VEL = 2, PH_S1 = 3, PH_S2 = 4, PH_COUNT = 5 };

struct PTask {
    int rep;       // replica
    int need;      // tasks of this replica listed before this one within a step
    short bx, by, bz;
    char phase, pad;
};

struct PersistArgs {
    BatchLists L;            // replica descriptors (pstep_tasks filled in)
    const PTask *tasks;      // one step's task list
    int ntask, nsteps;       // tasks per step, steps of this launch
    long long ds0;           // device step of the first step
    unsigned *ticket;        // dispatch counter, zero at launch
    unsigned *done;          // completed tasks per replica, zero at launch
    int *abort;              // raised by a block whose wait ran out, zero at launch
    int *status;             // handle status word (FLB_ETIMEOUT on a timeout)
    unsigned long long wait_ns;
};

size_t persist_smem_bytes();
void persist_tiles(const Geom &g, int zc, int coupling, int heun, int counts[PH_COUNT]);
void persist_tasks(std::vector<PTask> &v, int rep, int ph, const Geom &g, int zc, int need);
cudaError_t launch_persist(const PersistArgs &a, bool q15, cudaStream_t st);  // q15: D3Q15 replicas

// host launchers (flb_lb.cu, flb_psi.cu, flb_obs.cu)
cudaError_t launch_lb(const LBArgs &a, int q, int storage, cudaStream_t s);
// D3Q19 collide-stream that computes mu and the force itself from psi (flb_lb3d.cu)
cudaError_t launch_lb3d(const LBArgs &a, int storage, cudaStream_t s);
// order-parameter stress sigma on the interior + 1 ghost layer (flb_aux3d.cu, flb_psi.cu)
cudaError_t launch_sigma3(const Geom &g, const float *psi, float *sig, float A, float B, float K, cudaStream_t st);
cudaError_t launch_sigma2(const Geom &g, const float *psi, float *sig, float A, float B, float K, cudaStream_t st);
// velocity of the streamed state after a step, written to a.u (flb_aux3d.cu, flb_lb.cu)
cudaError_t launch_vel3(const LBArgs &a, int storage, cudaStream_t s);
cudaError_t launch_lb15(const LBArgs &a, int storage, cudaStream_t s);   // D3Q15 collide-stream
cudaError_t launch_vel15(const LBArgs &a, int storage, cudaStream_t s);  // D3Q15 velocity of the new state
// batched mu and velocity over the work lists (flb_aux3d.cu)
cudaError_t launch_mu3_batch(const BatchLists &L, cudaStream_t st);
cudaError_t launch_vel3_batch(const BatchLists &L, int storage, bool force, cudaStream_t st);
cudaError_t launch_vel2(const LBArgs &a, int storage, cudaStream_t s);
// one fused Runge-Kutta stage of psi on a 3D box (flb_psi3d.cu); q: the lattice
// of the FV operators (19 or 15); mu_in: the mu of the stage input on the
// interior and 2 ghost layers, or null (stage 1 then forms it)
cudaError_t launch_psi3(const Geom &g, int scheme, int q, int stage, bool noise, const float *psi, const float *u,
                        float *out, float *E, float A, float B, float K, float M, float kT, int advect, int heun,
                        const PhiloxKey &key, int64_t step, int zc, int rk4, const float *base, float *Dn,
                        const float *mu_in, int *status, cudaStream_t st, const LapW *lw = nullptr);
// mu on the interior and MU3_HALO = 2 ghost layers of a 3D box (flb_aux3d.cu)
// lw: the class weights of an App. A Laplacian (null: SO)
cudaError_t launch_mu3(const Geom &g, const float *psi, float *mu, float A, float B, float K, cudaStream_t st,
                       const LapW *lw = nullptr);
cudaError_t launch_init_eq(const Geom &g, int q, int storage, const float *rho, const float *u, float rho0, void *f,
                           cudaStream_t st);
cudaError_t launch_mu(const Geom &g, const float *psi, float *mu, float A, float B, float K, const LapW &lw,
                      cudaStream_t s);
// both Heun stages of the FV psi step in one launch by halo recompute (flb_heun1.cu)
cudaError_t launch_psi3_heun1(const Geom &g, int scheme, const float *psi, const float *u, float *out, float A, float B,
                              float K, float M, float kT, int advect, bool noise, const PhiloxKey &key, int64_t step,
                              int zc, cudaStream_t st);
// equilibrium start (flb_init.cu): populations into f (the current buffer), psi
// (padded) through an inverse DFT whose intermediates use `spare` (>= 16 bytes
// per site: the other population buffer)
cudaError_t launch_equilibrium_start(const Geom &g, int q, int storage, const LapW &lw, double rho0, double kT,
                                     double A, double K, uint64_t seed, void *f, void *spare, float *psi,
                                     cudaStream_t st);
cudaError_t launch_noise(const NoiseArgs &a, cudaStream_t s);
cudaError_t launch_flux(const Geom &g, int q, const float *psi, const float *mu, const float *u, float *J, float M,
                        int coupling, cudaStream_t s);
cudaError_t launch_psi_update(const PsiArgs &a, int q, cudaStream_t s);

}  // namespace flb

// flb_site3d.cuh -- the per-site work of the D3Q19 step kernels, shared by the
// per-phase kernels (flb_lb3d.cu, flb_aux3d.cu) and the persistent batched
// kernel (flb_persist.cu): population loads and stores (FP32 or FP16 storage),
// the 19-population pull, the force density of Sec. IV, the collide-stream of
// one site, the velocity of the new fluid state at one site, and the per-block
// arguments of a batched launch.  (The mu and sigma columns are in
// flb_mu3d.cuh.)
//
// D3Q19.  Plane order: 0 rest; pairs (1,2) +-x, (3,4) +-y, (5,6) +-z,
// (7,8) +-(1,1,0), (9,10) +-(1,-1,0), (11,12) +-(1,0,1), (13,14) +-(1,0,-1),
// (15,16) +-(0,1,1), (17,18) +-(0,1,-1).
#pragma once

#include "flb_internal.cuh"

namespace flb {

// Loads of fields written by earlier launches take the read-only path (COH
// false).  Inside the persistent batched kernel a field may have been written
// by another block of the same launch, so loads go to L2 (COH true): the
// read-only path and L1 are not coherent within a launch.
template <bool COH>
__device__ __forceinline__ float ldf(const float *p)
{
    if (COH) return __ldcg(p);
    return __ldg(p);
}
template <bool COH>
__device__ __forceinline__ float ld3(const float *p, int i)
{
    return ldf<COH>(p + i);
}
template <bool COH>
__device__ __forceinline__ float ld3(const __half *p, int i)
{
    return __half2float(COH ? __ldcg(p + i) : p[i]);
}

template <typename T>
__device__ __forceinline__ void st3(T *p, int i, float v);
template <>
__device__ __forceinline__ void st3<float>(float *p, int i, float v) { p[i] = v; }
template <>
__device__ __forceinline__ void st3<__half>(__half *p, int i, float v) { p[i] = __float2half_rn(v); }

// Addresses of the 19 population planes (plane i of N sites).  PlanesFromBase
// forms them from the buffers' bases, as the batched and persistent kernels must
// (their buffers swap with the device step); PlaneTable holds them, as a kernel
// parameter of the plain collide-stream, so a plane's address is one constant
// load instead of 64-bit arithmetic in every warp.
template <typename T>
struct PlanesFromBase {
    const T *fi;
    T *fo;
    long long N;
    __device__ __forceinline__ const T *in(int i) const { return fi + i * N; }
    __device__ __forceinline__ T *out(int i) const { return fo + i * N; }
};
template <typename T>
struct PlaneTable {
    const T *in_[19];
    T *out_[19];
    __device__ __forceinline__ const T *in(int i) const { return in_[i]; }
    __device__ __forceinline__ T *out(int i) const { return out_[i]; }
};

// The table of q planes of n sites from the buffers in and out (either may be
// null) (host).
template <typename T>
inline PlaneTable<T> plane_table(const void *in, void *out, long long n, int q)
{
    PlaneTable<T> P{};
    for (int i = 0; i < q; ++i) {
        P.in_[i] = in ? (const T *)in + i * n : nullptr;
        P.out_[i] = out ? (T *)out + i * n : nullptr;
    }
    return P;
}

// Pull of the 19 populations of the lanes' sites (x, y, zl[l]) from stored
// post-collision planes P.in(i): fbar_i(r) = stored_i(r - c_i).  Lane l of f[i]
// holds lane l's population i.
template <typename T, bool COH, class V, class PL>
__device__ __forceinline__ void pullv(const PL &P, const Geom &g, int x, int y, const int *zl, V f[19])
{
    constexpr int L = V::L;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const int row = nx, pl = nx * ny;
    const int sY0 = row * y, sYm = row * ym, sYp = row * yp;
    int sZ0[L], sZm[L], sZp[L];
#pragma unroll
    for (int l = 0; l < L; ++l) {
        const int z = zl[l];
        sZ0[l] = pl * z;
        sZm[l] = pl * (z == 0 ? nz - 1 : z - 1);
        sZp[l] = pl * (z == nz - 1 ? 0 : z + 1);
    }
    float t[L];
#define FLB_PULL(i, X, SY, SZ)                                                        \
    do {                                                                              \
        for (int l = 0; l < L; ++l) t[l] = ld3<COH>(P.in(i), X + SY + SZ[l]); \
        f[i] = vmake<V>(t);                                                           \
    } while (0)
    FLB_PULL(0, x, sY0, sZ0);
    FLB_PULL(1, xm, sY0, sZ0);
    FLB_PULL(2, xp, sY0, sZ0);
    FLB_PULL(3, x, sYm, sZ0);
    FLB_PULL(4, x, sYp, sZ0);
    FLB_PULL(5, x, sY0, sZm);
    FLB_PULL(6, x, sY0, sZp);
    FLB_PULL(7, xm, sYm, sZ0);
    FLB_PULL(8, xp, sYp, sZ0);
    FLB_PULL(9, xm, sYp, sZ0);
    FLB_PULL(10, xp, sYm, sZ0);
    FLB_PULL(11, xm, sY0, sZm);
    FLB_PULL(12, xp, sY0, sZp);
    FLB_PULL(13, xm, sY0, sZp);
    FLB_PULL(14, xp, sY0, sZm);
    FLB_PULL(15, x, sYm, sZm);
    FLB_PULL(16, x, sYp, sZp);
    FLB_PULL(17, x, sYm, sZp);
    FLB_PULL(18, x, sYp, sZm);
#undef FLB_PULL
}

// Force density of Sec. IV at the lanes' interior sites (x, y, zl[l]):
// F = -psi grad mu with the central difference or the FV gradient of mu, or
// F = -div sigma (stress form).
template <bool COH, class V>
__device__ __forceinline__ void force3v(const LBArgs &a, int x, int y, const int *zl, V &Fx, V &Fy, V &Fz)
{
    constexpr int L = V::L;
    const Geom &g = a.g;
    const int sy = g.px, sz = g.px * g.py;
    int pi[L];
#pragma unroll
    for (int l = 0; l < L; ++l) pi[l] = g.pidx32(x, y, zl[l]);
    auto LD = [&](const float *base, int off) {
        float t[L];
#pragma unroll
        for (int l = 0; l < L; ++l) t[l] = ldf<COH>(base + pi[l] + off);
        return vmake<V>(t);
    };
    if (a.force_kind == 2) {
        // F = -div sigma by central differences (stress form); sigma valid on the interior + 1
        const int pn = (int)g.pn;
        const float *xx = a.sig, *yy = xx + pn, *zz = yy + pn, *xy = zz + pn, *xz = xy + pn, *yz = xz + pn;
        Fx = (((LD(xx, 1) - LD(xx, -1)) + (LD(xy, sy) - LD(xy, -sy))) + (LD(xz, sz) - LD(xz, -sz))) * -0.5f;
        Fy = (((LD(xy, 1) - LD(xy, -1)) + (LD(yy, sy) - LD(yy, -sy))) + (LD(yz, sz) - LD(yz, -sz))) * -0.5f;
        Fz = (((LD(xz, 1) - LD(xz, -1)) + (LD(yz, sy) - LD(yz, -sy))) + (LD(zz, sz) - LD(zz, -sz))) * -0.5f;
        return;
    }
    // F = -psi grad mu, mu read from its field (valid on the interior + 1,
    // edges and corners included)
    const float *mu = a.mu;
    const V ps = LD(a.psi, 0);
    const V dx = LD(mu, 1) - LD(mu, -1);
    const V dy = LD(mu, sy) - LD(mu, -sy);
    const V dz = LD(mu, sz) - LD(mu, -sz);
    if (a.force_kind == 3) {
        // FV gradient on the D3Q15 neighbourhood: w = 1/9 (faces), 1/72 (corners),
        // so (1/c_s^2) sum_i w_i c_i mu(r + c_i) = (face difference)/3 + (sum of
        // the 8 corners signed by c_a)/24
        const V ppp = LD(mu, 1 + sy + sz), ppm = LD(mu, 1 + sy - sz);
        const V pmp = LD(mu, 1 - sy + sz), pmm = LD(mu, 1 - sy - sz);
        const V mpp = LD(mu, -1 + sy + sz), mpm = LD(mu, -1 + sy - sz);
        const V mmp = LD(mu, -1 - sy + sz), mmm = LD(mu, -1 - sy - sz);
        const V cx = ((ppp + ppm) + (pmp + pmm)) - ((mpp + mpm) + (mmp + mmm));
        const V cy = ((ppp + ppm) + (mpp + mpm)) - ((pmp + pmm) + (mmp + mmm));
        const V cz = ((ppp + pmp) + (mpp + mmp)) - ((ppm + pmm) + (mpm + mmm));
        const V nps = ps * -1.0f;
        Fx = nps * vfma(dx, 1.0f / 3.0f, cx * (1.0f / 24.0f));
        Fy = nps * vfma(dy, 1.0f / 3.0f, cy * (1.0f / 24.0f));
        Fz = nps * vfma(dz, 1.0f / 3.0f, cz * (1.0f / 24.0f));
    } else if (a.force_kind == 1) {
        // FV gradient (1/c_s^2) sum_i w_i c_i mu(r + c_i), Eq. (fvgrad): with
        // w = 1/18 (faces), 1/36 (edges) it is [2 (face difference) + sum of
        // the 8 edge neighbours signed by c_a] / 12
        const V xyp = LD(mu, 1 + sy), xym = LD(mu, 1 - sy);
        const V yxp = LD(mu, -1 + sy), yxm = LD(mu, -1 - sy);
        const V xzp = LD(mu, 1 + sz), xzm = LD(mu, 1 - sz);
        const V zxp = LD(mu, -1 + sz), zxm = LD(mu, -1 - sz);
        const V yzp = LD(mu, sy + sz), yzm = LD(mu, sy - sz);
        const V zyp = LD(mu, -sy + sz), zym = LD(mu, -sy - sz);
        // xyp = mu(+1,+1,0), xym = mu(+1,-1,0), yxp = mu(-1,+1,0), yxm = mu(-1,-1,0);
        // likewise in the (x,z) and (y,z) planes
        const V c = ps * (-1.0f / 12.0f);
        Fx = c * vfma(dx, 2.0f, ((xyp + xym) - (yxp + yxm)) + ((xzp + xzm) - (zxp + zxm)));
        Fy = c * vfma(dy, 2.0f, ((xyp - xym) + (yxp - yxm)) + ((yzp + yzm) - (zyp + zym)));
        Fz = c * vfma(dz, 2.0f, ((xzp - xzm) + (zxp - zxm)) + ((yzp - yzm) + (zyp - zym)));
    } else {
        const V c = ps * -0.5f;
        Fx = c * dx;
        Fy = c * dy;
        Fz = c * dz;
    }
}

// One site's force (the persistent kernel, one site per thread).
template <bool COH = false>
__device__ __forceinline__ void force3(const LBArgs &a, int x, int y, int z, float &Fx, float &Fy, float &Fz)
{
    F1 X, Y, Z;
    force3v<COH, F1>(a, x, y, &z, X, Y, Z);
    Fx = X.v;
    Fy = Y.v;
    Fz = Z.v;
}

// Per-block LBArgs of a batched launch, in shared memory: the replica's
// arguments with the population buffers swapped on odd device steps, the psi
// buffer of the step and the step's noise counter.
__device__ __forceinline__ void batch_lb_args(const BatchLists &L, const BatchRep &r, LBArgs &sa)
{
    // the batched kernels' blocks are one-dimensional, LBB_NT threads (a stride
    // fixed at compile time: a stride read from blockDim measured 2% slower)
    const int tid = threadIdx.x;
    {
        const int *src = reinterpret_cast<const int *>(&r.lb);
        int *dst = reinterpret_cast<int *>(&sa);
        for (int k = tid; k < (int)(sizeof(LBArgs) / sizeof(int)); k += LBB_NT) dst[k] = src[k];
    }
    __syncthreads();
    if (tid == 0) {
        const long long ds = *L.dstep;
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

// Collide-stream of the D3Q19 sites (x, y, zl[l]) of the lanes of V; the first
// nl lanes are stored (a lane past the box repeats lane 0's site and is
// dropped).  Pull, moments, relaxation with force and noise (Eq. bab, Sec. III),
// store.  The stress is carried as Q = 4.5 B (B: the relaxed second moment in
// the cartesian form of Eq. bab) and the ghost modes in the scaled forms
// G10..G12 = g/3, G13..G15 = g, G16 = g/3, G17, G18 = g/2, so that the
// back-transform f_i = w_i [drho + 3 c_i.(j + F) + 4.5 (c_i c_i - I/3):B +
// ghosts] needs no further scale factors; a.rq and a.nq carry the relaxation
// and noise coefficients in these units.
// KEY_R0: the arguments sit in shared memory (batched and persistent kernels).
// P: the planes it pulls from (P.in) and stores to (P.out).
template <class V, typename T, bool GHOST_RELAX, bool COH, bool KEY_R0, class PL>
__device__ __forceinline__ void lb_sites(const LBArgs &a, const PL &P, int x, int y, const int *zl, int nl, V Fx,
                                         V Fy, V Fz)
{
    constexpr int L = V::L;
    const Geom &g = a.g;
    int s[L];
#pragma unroll
    for (int l = 0; l < L; ++l) s[l] = x + g.nx * y + g.nx * g.ny * zl[l];

    V f[19];
    pullv<T, COH>(P, g, x, y, zl, f);

    V sp[10], dp[10];
#pragma unroll
    for (int p = 1; p <= 9; ++p) {
        sp[p] = f[2 * p - 1] + f[2 * p];
        dp[p] = f[2 * p - 1] - f[2 * p];
    }
    const V s45 = sp[4] + sp[5], s67 = sp[6] + sp[7], s89 = sp[8] + sp[9];
    const V drho = f[0] + ((sp[1] + sp[2] + sp[3]) + (s45 + s67 + s89));
    const V jx = dp[1] + (dp[4] + dp[5]) + (dp[6] + dp[7]);
    const V jy = dp[2] + (dp[4] - dp[5]) + (dp[8] + dp[9]);
    const V jz = dp[3] + (dp[6] - dp[7]) + (dp[8] - dp[9]);
    const V third = drho * (1.0f / 3.0f);
    const V Sxx = sp[1] + s45 + s67 - third;
    const V Syy = sp[2] + s45 + s89 - third;
    const V Szz = sp[3] + s67 + s89 - third;
    const V Sxy = sp[4] - sp[5], Sxz = sp[6] - sp[7], Syz = sp[8] - sp[9];

    const V rho = drho + a.rho0;
    float ir[L];
#pragma unroll
    for (int l = 0; l < L; ++l) ir[l] = __fdividef(1.0f, rho.lane(l));  // ~2 ulp
    const V irho = vmake<V>(ir);
    const V vx = vfma(Fx, 0.5f, jx) * irho, vy = vfma(Fy, 0.5f, jy) * irho, vz = vfma(Fz, 0.5f, jz) * irho;

    // Q = 4.5 [(1 - ws) S + ws rho v v + cs (v F + F v)] + the bulk correction,
    // with h = 4.5 (ws rho v + cs F) and c = 4.5 cs F
    const V cFx = Fx * a.rq[2], cFy = Fy * a.rq[2], cFz = Fz * a.rq[2];
    const V wr = rho * a.rq[1];
    const V hx = vfma(wr, vx, cFx), hy = vfma(wr, vy, cFy), hz = vfma(wr, vz, cFz);
    V Qxx = vfma(Sxx, a.rq[0], vx * (hx + cFx));
    V Qyy = vfma(Syy, a.rq[0], vy * (hy + cFy));
    V Qzz = vfma(Szz, a.rq[0], vz * (hz + cFz));
    if (a.iso) {  // bulk rate differs from the shear rate: the trace relaxes at its own rate
        const V P2 = vfma(vz, vz, vfma(vy, vy, vx * vx));
        const V vF = vfma(vz, Fz, vfma(vy, Fy, vx * Fx));
        const V trS = Sxx + Syy + Szz;
        const V isoq = vfma(vfma(rho, P2, trS * -1.0f), a.rq[3], vF * a.rq[4]);
        Qxx = Qxx + isoq;
        Qyy = Qyy + isoq;
        Qzz = Qzz + isoq;
    }
    V Qxy = vfma(Sxy, a.rq[0], vfma(vy, hx, vx * cFy));
    V Qxz = vfma(Sxz, a.rq[0], vfma(vz, hx, vx * cFz));
    V Qyz = vfma(Syz, a.rq[0], vfma(vz, hy, vy * cFz));

    V G10 = V::bc(0.f), G11 = V::bc(0.f), G12 = V::bc(0.f), G13 = V::bc(0.f), G14 = V::bc(0.f),
      G15 = V::bc(0.f), G16 = V::bc(0.f), G17 = V::bc(0.f), G18 = V::bc(0.f);
    if (GHOST_RELAX) {
        const V gg = V::bc(a.gamma_g);
        const V m10 = (dp[4] + dp[5] + dp[6] + dp[7]) * (1.f / 3.f) - dp[1] * (2.f / 3.f);
        const V m11 = (dp[4] - dp[5] + dp[8] + dp[9]) * (1.f / 3.f) - dp[2] * (2.f / 3.f);
        const V m12 = (dp[6] - dp[7] + dp[8] - dp[9]) * (1.f / 3.f) - dp[3] * (2.f / 3.f);
        const V m13 = dp[4] + dp[5] - dp[6] - dp[7];
        const V m14 = dp[5] - dp[4] + dp[8] + dp[9];
        const V m15 = dp[6] - dp[7] - dp[8] + dp[9];
        const V m16 = (f[0] + sp[4] + sp[5] + sp[6] + sp[7] + sp[8] + sp[9]) * (1.f / 3.f) -
                      (sp[1] + sp[2] + sp[3]) * (2.f / 3.f);
        const V m17 = (sp[2] + sp[3] + sp[4] + sp[5] + sp[6] + sp[7]) * 0.5f - sp[1] - (sp[8] + sp[9]);
        const V m18 = (sp[3] - sp[2] + sp[4] + sp[5] - sp[6] - sp[7]) * 0.5f;
        // gamma_g m_k / b_k in the scaled units above
        G10 = gg * m10 * 4.5f;
        G11 = gg * m11 * 4.5f;
        G12 = gg * m12 * 4.5f;
        G13 = gg * m13 * 4.5f;
        G14 = gg * m14 * 4.5f;
        G15 = gg * m15 * 4.5f;
        G16 = gg * m16 * 1.5f;
        G17 = gg * m17 * 1.5f;
        G18 = gg * m18 * 4.5f;
    }
    if (a.kT > 0.f) {
        // 15 normals (noise order: bulk, 3c_x^2-c^2, c_y^2-c_z^2, xy, yz, zx, then
        // the ghosts in basis order) scaled by sqrt(rho kT / c_s^2), lane-wise
        const V mun = rho * a.k3T;
        float sq[L];
#pragma unroll
        for (int l = 0; l < L; ++l) sq[l] = mun.lane(l) * rsqrtf(mun.lane(l));  // ~2 ulp
        uint32_t su[L];
#pragma unroll
        for (int l = 0; l < L; ++l) su[l] = (uint32_t)s[l];
        const V sc = vmake<V>(sq);
        V n[8];
        lane_block<8, KEY_R0>(a.key, a.step, su, 0u, sc, n);  // normals 0-7
        const V m0 = n[0] * a.nq[0], m1 = n[1] * a.nq[1], m2 = n[2] * a.nq[2];
        const V t01 = m0 - m1;
        Qxx = Qxx + vfma(m1, 2.0f, m0);
        Qyy = Qyy + (t01 + m2);
        Qzz = Qzz + (t01 - m2);
        Qxy = vfma(n[3], a.nq[3], Qxy);
        Qyz = vfma(n[4], a.nq[4], Qyz);
        Qxz = vfma(n[5], a.nq[5], Qxz);
        G10 = vfma(n[6], a.nq[6], G10);
        G11 = vfma(n[7], a.nq[7], G11);
        lane_block<7, KEY_R0>(a.key, a.step, su, 1u, sc, n);  // normals 8-14
        G12 = vfma(n[0], a.nq[8], G12);
        G13 = vfma(n[1], a.nq[9], G13);
        G14 = vfma(n[2], a.nq[10], G14);
        G15 = vfma(n[3], a.nq[11], G15);
        G16 = vfma(n[4], a.nq[12], G16);
        G17 = vfma(n[5], a.nq[13], G17);
        G18 = vfma(n[6], a.nq[14], G18);
    }

    // back-transform f_i = w_i (E_i +- O_i), E even and O odd in c_i
    auto store = [&](int i, V v) {
#pragma unroll
        for (int l = 0; l < L; ++l)
            if (l < nl) st3(P.out(i), s[l], v.lane(l));
    };
    const V d = vfma(Qxx + Qyy + Qzz, -1.0f / 3.0f, drho);  // drho - tr(Q)/3
    const V Dg = d + G16;
    store(0, Dg * (1.0f / 3.0f));
    const V a3x = (jx + Fx) * 3.0f, a3y = (jy + Fy) * 3.0f, a3z = (jz + Fz) * 3.0f;
    constexpr float w1 = 1.0f / 18.0f, w2 = 1.0f / 36.0f;
    {
        const V Dm = vfma(G16, -2.0f, d);
        const V t17 = Dm + G17;
        const V Ex = vfma(G17, -2.0f, Dm + Qxx), Ey = (t17 - G18) + Qyy, Ez = (t17 + G18) + Qzz;
        const V Ox = vfma(G10, -2.0f, a3x), Oy = vfma(G11, -2.0f, a3y), Oz = vfma(G12, -2.0f, a3z);
        store(1, (Ex + Ox) * w1);
        store(2, (Ex - Ox) * w1);
        store(3, (Ey + Oy) * w1);
        store(4, (Ey - Oy) * w1);
        store(5, (Ez + Oz) * w1);
        store(6, (Ez - Oz) * w1);
    }
    const V Ge = Dg + G17;
    {
        const V xyb = (Qxx + Qyy) + (Ge + G18);
        const V E7 = vfma(Qxy, 2.0f, xyb), E9 = vfma(Qxy, -2.0f, xyb);
        const V O7 = (a3x + a3y) + (G10 + G11) + (G13 - G14);
        const V O9 = (a3x - a3y) + (G10 - G11) + (G13 + G14);
        store(7, (E7 + O7) * w2);
        store(8, (E7 - O7) * w2);
        store(9, (E9 + O9) * w2);
        store(10, (E9 - O9) * w2);
    }
    {
        const V xzb = (Qxx + Qzz) + (Ge - G18);
        const V E11 = vfma(Qxz, 2.0f, xzb), E13 = vfma(Qxz, -2.0f, xzb);
        const V O11 = (a3x + a3z) + (G10 + G12) + (G15 - G13);
        const V O13 = (a3x - a3z) + (G10 - G12) - (G13 + G15);
        store(11, (E11 + O11) * w2);
        store(12, (E11 - O11) * w2);
        store(13, (E13 + O13) * w2);
        store(14, (E13 - O13) * w2);
    }
    {
        const V yzb = (Qyy + Qzz) + vfma(G17, -2.0f, Dg);
        const V E15 = vfma(Qyz, 2.0f, yzb), E17 = vfma(Qyz, -2.0f, yzb);
        const V O15 = (a3y + a3z) + (G11 + G12) + (G14 - G15);
        const V O17 = (a3y - a3z) + (G11 - G12) + (G14 + G15);
        store(15, (E15 + O15) * w2);
        store(16, (E15 - O15) * w2);
        store(17, (E17 + O17) * w2);
        store(18, (E17 - O17) * w2);
    }
}

// One site on the planes of a.fin and a.fout (the persistent kernel, one site per thread).
template <typename T, bool GHOST_RELAX, bool COH = false, bool KEY_R0 = false>
__device__ __forceinline__ void lb_site(const LBArgs &a, int x, int y, int z, float Fx, float Fy, float Fz)
{
    lb_sites<F1, T, GHOST_RELAX, COH, KEY_R0>(a, PlanesFromBase<T>{(const T *)a.fin, (T *)a.fout, a.g.n}, x, y, &z,
                                              1, F1{Fx}, F1{Fy}, F1{Fz});
}

// Velocity of the streamed state at the lanes' sites (x, y, zl[l]), the first
// nl stored: u = (sum fbar c + F/2)/rho with fbar the populations the next step
// pulls (a.fout) and F this step's force.  P.in: the planes of a.fout.
template <class V, typename T, bool FORCE, bool COH, class PL>
__device__ __forceinline__ void vel3_sites(const LBArgs &a, const PL &P, int x, int y, const int *zl, int nl)
{
    constexpr int L = V::L;
    const Geom &g = a.g;
    V f[19];
    pullv<T, COH>(P, g, x, y, zl, f);
    V sp[10], dp[10];
#pragma unroll
    for (int p = 1; p <= 9; ++p) {
        sp[p] = f[2 * p - 1] + f[2 * p];
        dp[p] = f[2 * p - 1] - f[2 * p];
    }
    const V s45 = sp[4] + sp[5], s67 = sp[6] + sp[7], s89 = sp[8] + sp[9];
    const V drho = f[0] + ((sp[1] + sp[2] + sp[3]) + (s45 + s67 + s89));
    const V jx = dp[1] + (dp[4] + dp[5]) + (dp[6] + dp[7]);
    const V jy = dp[2] + (dp[4] - dp[5]) + (dp[8] + dp[9]);
    const V jz = dp[3] + (dp[6] - dp[7]) + (dp[8] - dp[9]);
    V Fx = V::bc(0.f), Fy = V::bc(0.f), Fz = V::bc(0.f);
    if (FORCE && (a.coupling & FLB_COUPLE_FORCE)) force3v<COH>(a, x, y, zl, Fx, Fy, Fz);
    const V rho = drho + a.rho0;
    float ir[L];
#pragma unroll
    for (int l = 0; l < L; ++l) ir[l] = __fdividef(1.0f, rho.lane(l));
    const V irho = vmake<V>(ir);
    const V ux = vfma(Fx, 0.5f, jx) * irho, uy = vfma(Fy, 0.5f, jy) * irho, uz = vfma(Fz, 0.5f, jz) * irho;
#pragma unroll
    for (int l = 0; l < L; ++l) {
        if (l >= nl) break;
        store_padded(a.u, g, x, y, zl[l], ux.lane(l), 1);
        store_padded(a.u + g.pn, g, x, y, zl[l], uy.lane(l), 1);
        store_padded(a.u + 2 * g.pn, g, x, y, zl[l], uz.lane(l), 1);
    }
}

// The same at one site on the planes of a.fout.
template <typename T, bool FORCE, bool COH = false>
__device__ __forceinline__ void vel3_site(const LBArgs &a, int x, int y, int z)
{
    vel3_sites<F1, T, FORCE, COH>(a, PlanesFromBase<T>{(const T *)a.fout, nullptr, a.g.n}, x, y, &z, 1);
}

}  // namespace flb

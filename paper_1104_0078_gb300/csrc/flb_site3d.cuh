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

// Pull of the 19 populations of site (x, y, z) from stored post-collision
// planes P.in(i): fbar_i(r) = stored_i(r - c_i).
template <typename T, bool COH = false, class PL>
__device__ __forceinline__ void pull19(const PL &P, const Geom &g, int x, int y, int z, float f[19])
{
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    const int row = nx, pl = nx * ny;
    const int sY0 = row * y, sYm = row * ym, sYp = row * yp;
    const int sZ0 = pl * z, sZm = pl * zm, sZp = pl * zp;
    f[0] = ld3<COH>(P.in(0), x + sY0 + sZ0);
    f[1] = ld3<COH>(P.in(1), xm + sY0 + sZ0);
    f[2] = ld3<COH>(P.in(2), xp + sY0 + sZ0);
    f[3] = ld3<COH>(P.in(3), x + sYm + sZ0);
    f[4] = ld3<COH>(P.in(4), x + sYp + sZ0);
    f[5] = ld3<COH>(P.in(5), x + sY0 + sZm);
    f[6] = ld3<COH>(P.in(6), x + sY0 + sZp);
    f[7] = ld3<COH>(P.in(7), xm + sYm + sZ0);
    f[8] = ld3<COH>(P.in(8), xp + sYp + sZ0);
    f[9] = ld3<COH>(P.in(9), xm + sYp + sZ0);
    f[10] = ld3<COH>(P.in(10), xp + sYm + sZ0);
    f[11] = ld3<COH>(P.in(11), xm + sY0 + sZm);
    f[12] = ld3<COH>(P.in(12), xp + sY0 + sZp);
    f[13] = ld3<COH>(P.in(13), xm + sY0 + sZp);
    f[14] = ld3<COH>(P.in(14), xp + sY0 + sZm);
    f[15] = ld3<COH>(P.in(15), x + sYm + sZm);
    f[16] = ld3<COH>(P.in(16), x + sYp + sZp);
    f[17] = ld3<COH>(P.in(17), x + sYm + sZp);
    f[18] = ld3<COH>(P.in(18), x + sYp + sZm);
}

// Force density of Sec. IV at an interior site: F = -psi grad mu with the
// central difference or the FV gradient of mu, or F = -div sigma (stress form).
template <bool COH = false>
__device__ __forceinline__ void force3(const LBArgs &a, int x, int y, int z, float &Fx, float &Fy, float &Fz)
{
    const Geom &g = a.g;
    if (a.force_kind == 2) {
        // F = -div sigma by central differences (stress form); sigma valid on the interior + 1
        const int pi = g.pidx32(x, y, z);
        const int sy = g.px, sz = g.px * g.py, pn = (int)g.pn;
        const float *xx = a.sig, *yy = xx + pn, *zz = yy + pn, *xy = zz + pn, *xz = xy + pn, *yz = xz + pn;
        Fx = -0.5f * ((ldf<COH>(xx + pi + 1) - ldf<COH>(xx + pi - 1)) + (ldf<COH>(xy + pi + sy) - ldf<COH>(xy + pi - sy)) +
                      (ldf<COH>(xz + pi + sz) - ldf<COH>(xz + pi - sz)));
        Fy = -0.5f * ((ldf<COH>(xy + pi + 1) - ldf<COH>(xy + pi - 1)) + (ldf<COH>(yy + pi + sy) - ldf<COH>(yy + pi - sy)) +
                      (ldf<COH>(yz + pi + sz) - ldf<COH>(yz + pi - sz)));
        Fz = -0.5f * ((ldf<COH>(xz + pi + 1) - ldf<COH>(xz + pi - 1)) + (ldf<COH>(yz + pi + sy) - ldf<COH>(yz + pi - sy)) +
                      (ldf<COH>(zz + pi + sz) - ldf<COH>(zz + pi - sz)));
        return;
    }
    // F = -psi grad mu, mu read from its field (valid on the interior + 1,
    // edges and corners included)
    const int pi = g.pidx32(x, y, z);
    const int sy = g.px, sz = g.px * g.py;
    const float ps = ldf<COH>(a.psi + pi);
    const float *mu = a.mu;
    const float dx = ldf<COH>(mu + pi + 1) - ldf<COH>(mu + pi - 1);
    const float dy = ldf<COH>(mu + pi + sy) - ldf<COH>(mu + pi - sy);
    const float dz = ldf<COH>(mu + pi + sz) - ldf<COH>(mu + pi - sz);
    if (a.force_kind == 3) {
        // FV gradient on the D3Q15 neighbourhood: w = 1/9 (faces), 1/72 (corners),
        // so (1/c_s^2) sum_i w_i c_i mu(r + c_i) = (face difference)/3 + (sum of
        // the 8 corners signed by c_a)/24
        const float ppp = ldf<COH>(mu + pi + 1 + sy + sz), ppm = ldf<COH>(mu + pi + 1 + sy - sz);
        const float pmp = ldf<COH>(mu + pi + 1 - sy + sz), pmm = ldf<COH>(mu + pi + 1 - sy - sz);
        const float mpp = ldf<COH>(mu + pi - 1 + sy + sz), mpm = ldf<COH>(mu + pi - 1 + sy - sz);
        const float mmp = ldf<COH>(mu + pi - 1 - sy + sz), mmm = ldf<COH>(mu + pi - 1 - sy - sz);
        const float cx = ((ppp + ppm) + (pmp + pmm)) - ((mpp + mpm) + (mmp + mmm));
        const float cy = ((ppp + ppm) + (mpp + mpm)) - ((pmp + pmm) + (mmp + mmm));
        const float cz = ((ppp + pmp) + (mpp + mmp)) - ((ppm + pmm) + (mpm + mmm));
        Fx = -ps * (dx * (1.0f / 3.0f) + cx * (1.0f / 24.0f));
        Fy = -ps * (dy * (1.0f / 3.0f) + cy * (1.0f / 24.0f));
        Fz = -ps * (dz * (1.0f / 3.0f) + cz * (1.0f / 24.0f));
    } else if (a.force_kind == 1) {
        // FV gradient (1/c_s^2) sum_i w_i c_i mu(r + c_i), Eq. (fvgrad): with
        // w = 1/18 (faces), 1/36 (edges) it is [2 (face difference) + sum of
        // the 8 edge neighbours signed by c_a] / 12
        const float xyp = ldf<COH>(mu + pi + 1 + sy), xym = ldf<COH>(mu + pi + 1 - sy);
        const float yxp = ldf<COH>(mu + pi - 1 + sy), yxm = ldf<COH>(mu + pi - 1 - sy);
        const float xzp = ldf<COH>(mu + pi + 1 + sz), xzm = ldf<COH>(mu + pi + 1 - sz);
        const float zxp = ldf<COH>(mu + pi - 1 + sz), zxm = ldf<COH>(mu + pi - 1 - sz);
        const float yzp = ldf<COH>(mu + pi + sy + sz), yzm = ldf<COH>(mu + pi + sy - sz);
        const float zyp = ldf<COH>(mu + pi - sy + sz), zym = ldf<COH>(mu + pi - sy - sz);
        // xyp = mu(+1,+1,0), xym = mu(+1,-1,0), yxp = mu(-1,+1,0), yxm = mu(-1,-1,0);
        // likewise in the (x,z) and (y,z) planes
        const float c = -ps * (1.0f / 12.0f);
        Fx = c * (2.f * dx + ((xyp + xym) - (yxp + yxm)) + ((xzp + xzm) - (zxp + zxm)));
        Fy = c * (2.f * dy + ((xyp - xym) + (yxp - yxm)) + ((yzp + yzm) - (zyp + zym)));
        Fz = c * (2.f * dz + ((xzp - xzm) + (zxp - zxm)) + ((yzp - yzm) + (zyp - zym)));
    } else {
        Fx = -ps * 0.5f * dx;
        Fy = -ps * 0.5f * dy;
        Fz = -ps * 0.5f * dz;
    }
}

// Per-block LBArgs of a batched launch, in shared memory: the replica's
// arguments with the population buffers swapped on odd device steps, the psi
// buffer of the step and the step's noise counter.
__device__ __forceinline__ void batch_lb_args(const BatchLists &L, const BatchRep &r, LBArgs &sa)
{
    const int tid = threadIdx.x + LB_BX * (threadIdx.y + LB_BY * threadIdx.z);
    {
        const int *src = reinterpret_cast<const int *>(&r.lb);
        int *dst = reinterpret_cast<int *>(&sa);
        for (int k = tid; k < (int)(sizeof(LBArgs) / sizeof(int)); k += LB_BX * LB_BY * LB_BZ) dst[k] = src[k];
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

// One D3Q19 site: pull, moments, relaxation with force and noise, store.
// KEY_R0: the arguments sit in shared memory (batched and persistent kernels).
// P: the planes it pulls from (P.in) and stores to (P.out).
template <typename T, bool GHOST_RELAX, bool COH, bool KEY_R0, class PL>
__device__ __forceinline__ void lb_site_on(const LBArgs &a, const PL &P, int x, int y, int z, float Fx, float Fy,
                                           float Fz)
{
    const Geom &g = a.g;
    const int s = x + g.nx * y + g.nx * g.ny * z;

    float f[19];
    pull19<T, COH>(P, g, x, y, z, f);

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
        normals4<KEY_R0>(a.key, a.step, sid, 0u, 0u, G);
        normals4<KEY_R0>(a.key, a.step, sid, 0u, 1u, G + 4);
        normals4<KEY_R0>(a.key, a.step, sid, 0u, 2u, G + 8);
        normals4<KEY_R0>(a.key, a.step, sid, 0u, 3u, G + 12);
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
    st3(P.out(0), s, (1.f / 3.f) * (drho - e0 + h1 * g16));
    float E, O;
    E = drho + 4.5f * Bxx - e0 - h2 * g16 - g17;
    O = 3.f * Ax - h2 * g10;
    st3(P.out(1), s, w1 * (E + O));
    st3(P.out(2), s, w1 * (E - O));
    E = drho + 4.5f * Byy - e0 - h2 * g16 + 0.5f * g17 - 0.5f * g18;
    O = 3.f * Ay - h2 * g11;
    st3(P.out(3), s, w1 * (E + O));
    st3(P.out(4), s, w1 * (E - O));
    E = drho + 4.5f * Bzz - e0 - h2 * g16 + 0.5f * g17 + 0.5f * g18;
    O = 3.f * Az - h2 * g12;
    st3(P.out(5), s, w1 * (E + O));
    st3(P.out(6), s, w1 * (E - O));
    const float Gev = h1 * g16 + 0.5f * g17;
    E = drho + 4.5f * (Bxx + Byy + 2.f * Bxy) - e0 + Gev + 0.5f * g18;
    O = 3.f * (Ax + Ay) + h1 * (g10 + g11) + g13 - g14;
    st3(P.out(7), s, w2 * (E + O));
    st3(P.out(8), s, w2 * (E - O));
    E = drho + 4.5f * (Bxx + Byy - 2.f * Bxy) - e0 + Gev + 0.5f * g18;
    O = 3.f * (Ax - Ay) + h1 * (g10 - g11) + g13 + g14;
    st3(P.out(9), s, w2 * (E + O));
    st3(P.out(10), s, w2 * (E - O));
    E = drho + 4.5f * (Bxx + Bzz + 2.f * Bxz) - e0 + Gev - 0.5f * g18;
    O = 3.f * (Ax + Az) + h1 * (g10 + g12) - g13 + g15;
    st3(P.out(11), s, w2 * (E + O));
    st3(P.out(12), s, w2 * (E - O));
    E = drho + 4.5f * (Bxx + Bzz - 2.f * Bxz) - e0 + Gev - 0.5f * g18;
    O = 3.f * (Ax - Az) + h1 * (g10 - g12) - g13 - g15;
    st3(P.out(13), s, w2 * (E + O));
    st3(P.out(14), s, w2 * (E - O));
    E = drho + 4.5f * (Byy + Bzz + 2.f * Byz) - e0 + h1 * g16 - g17;
    O = 3.f * (Ay + Az) + h1 * (g11 + g12) + g14 - g15;
    st3(P.out(15), s, w2 * (E + O));
    st3(P.out(16), s, w2 * (E - O));
    E = drho + 4.5f * (Byy + Bzz - 2.f * Byz) - e0 + h1 * g16 - g17;
    O = 3.f * (Ay - Az) + h1 * (g11 - g12) + g14 + g15;
    st3(P.out(17), s, w2 * (E + O));
    st3(P.out(18), s, w2 * (E - O));
}

// The same site on the planes of a.fin and a.fout.
template <typename T, bool GHOST_RELAX, bool COH = false, bool KEY_R0 = false>
__device__ __forceinline__ void lb_site(const LBArgs &a, int x, int y, int z, float Fx, float Fy, float Fz)
{
    lb_site_on<T, GHOST_RELAX, COH, KEY_R0>(a, PlanesFromBase<T>{(const T *)a.fin, (T *)a.fout, a.g.n}, x, y, z,
                                             Fx, Fy, Fz);
}

// Velocity of the streamed state at (x, y, z): u = (sum fbar c + F/2)/rho with
// fbar the populations the next step pulls (a.fout) and F this step's force.
// P.in: the planes of a.fout.
template <typename T, bool FORCE, bool COH, class PL>
__device__ __forceinline__ void vel3_site_on(const LBArgs &a, const PL &P, int x, int y, int z)
{
    const Geom &g = a.g;
    float f[19];
    pull19<T, COH>(P, g, x, y, z, f);
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
    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
    if (FORCE && (a.coupling & FLB_COUPLE_FORCE)) force3<COH>(a, x, y, z, Fx, Fy, Fz);
    const float irho = __fdividef(1.0f, a.rho0 + drho);
    store_padded(a.u, g, x, y, z, (jx + 0.5f * Fx) * irho, 1);
    store_padded(a.u + g.pn, g, x, y, z, (jy + 0.5f * Fy) * irho, 1);
    store_padded(a.u + 2 * g.pn, g, x, y, z, (jz + 0.5f * Fz) * irho, 1);
}

// The same on the planes of a.fout.
template <typename T, bool FORCE, bool COH = false>
__device__ __forceinline__ void vel3_site(const LBArgs &a, int x, int y, int z)
{
    vel3_site_on<T, FORCE, COH>(a, PlanesFromBase<T>{(const T *)a.fout, nullptr, a.g.n}, x, y, z);
}

}  // namespace flb

// flb_site3d.cuh -- per-site pieces shared by the D3Q19 collide-stream and the
// velocity kernel: population loads and stores (FP32 or FP16 storage), the
// 19-population pull, the force density of Sec. IV and the per-block arguments
// of a batched launch.
//
// D3Q19.  Plane order: 0 rest; pairs (1,2) +-x, (3,4) +-y, (5,6) +-z,
// (7,8) +-(1,1,0), (9,10) +-(1,-1,0), (11,12) +-(1,0,1), (13,14) +-(1,0,-1),
// (15,16) +-(0,1,1), (17,18) +-(0,1,-1).
#pragma once

#include "flb_internal.cuh"

namespace flb {

template <typename T>
__device__ __forceinline__ float ld3(const T *p, int i);
template <>
__device__ __forceinline__ float ld3<float>(const float *p, int i) { return __ldg(p + i); }
template <>
__device__ __forceinline__ float ld3<__half>(const __half *p, int i) { return __half2float(p[i]); }

template <typename T>
__device__ __forceinline__ void st3(T *p, int i, float v);
template <>
__device__ __forceinline__ void st3<float>(float *p, int i, float v) { p[i] = v; }
template <>
__device__ __forceinline__ void st3<__half>(__half *p, int i, float v) { p[i] = __float2half_rn(v); }

// Pull of the 19 populations of site (x, y, z) from stored post-collision
// planes fi: fbar_i(r) = stored_i(r - c_i).
template <typename T>
__device__ __forceinline__ void pull19(const T *fi, const Geom &g, int x, int y, int z, float f[19])
{
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int N = (int)g.n;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    const int row = nx, pl = nx * ny;
    const int sY0 = row * y, sYm = row * ym, sYp = row * yp;
    const int sZ0 = pl * z, sZm = pl * zm, sZp = pl * zp;
    f[0] = ld3(fi, x + sY0 + sZ0);
    f[1] = ld3(fi + 1ll * N, xm + sY0 + sZ0);
    f[2] = ld3(fi + 2ll * N, xp + sY0 + sZ0);
    f[3] = ld3(fi + 3ll * N, x + sYm + sZ0);
    f[4] = ld3(fi + 4ll * N, x + sYp + sZ0);
    f[5] = ld3(fi + 5ll * N, x + sY0 + sZm);
    f[6] = ld3(fi + 6ll * N, x + sY0 + sZp);
    f[7] = ld3(fi + 7ll * N, xm + sYm + sZ0);
    f[8] = ld3(fi + 8ll * N, xp + sYp + sZ0);
    f[9] = ld3(fi + 9ll * N, xm + sYp + sZ0);
    f[10] = ld3(fi + 10ll * N, xp + sYm + sZ0);
    f[11] = ld3(fi + 11ll * N, xm + sY0 + sZm);
    f[12] = ld3(fi + 12ll * N, xp + sY0 + sZp);
    f[13] = ld3(fi + 13ll * N, xm + sY0 + sZp);
    f[14] = ld3(fi + 14ll * N, xp + sY0 + sZm);
    f[15] = ld3(fi + 15ll * N, x + sYm + sZm);
    f[16] = ld3(fi + 16ll * N, x + sYp + sZp);
    f[17] = ld3(fi + 17ll * N, x + sYm + sZp);
    f[18] = ld3(fi + 18ll * N, x + sYp + sZm);
}

// Force density F = -psi grad mu of Sec. IV at an interior site.
__device__ __forceinline__ void force3(const LBArgs &a, int x, int y, int z, float &Fx, float &Fy, float &Fz)
{
    const Geom &g = a.g;
    // F = -psi grad mu, mu read from its field (valid on the interior + 1,
    // edges and corners included)
    const int pi = g.pidx32(x, y, z);
    const int sy = g.px, sz = g.px * g.py;
    const float ps = __ldg(a.psi + pi);
    const float *mu = a.mu;
    const float dx = __ldg(mu + pi + 1) - __ldg(mu + pi - 1);
    const float dy = __ldg(mu + pi + sy) - __ldg(mu + pi - sy);
    const float dz = __ldg(mu + pi + sz) - __ldg(mu + pi - sz);
    if (a.fv_force) {
        // FV gradient (1/c_s^2) sum_i w_i c_i mu(r + c_i), Eq. (fvgrad): with
        // w = 1/18 (faces), 1/36 (edges) it is [2 (face difference) + sum of
        // the 8 edge neighbours signed by c_a] / 12
        const float xyp = __ldg(mu + pi + 1 + sy), xym = __ldg(mu + pi + 1 - sy);
        const float yxp = __ldg(mu + pi - 1 + sy), yxm = __ldg(mu + pi - 1 - sy);
        const float xzp = __ldg(mu + pi + 1 + sz), xzm = __ldg(mu + pi + 1 - sz);
        const float zxp = __ldg(mu + pi - 1 + sz), zxm = __ldg(mu + pi - 1 - sz);
        const float yzp = __ldg(mu + pi + sy + sz), yzm = __ldg(mu + pi + sy - sz);
        const float zyp = __ldg(mu + pi - sy + sz), zym = __ldg(mu + pi - sy - sz);
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

}  // namespace flb

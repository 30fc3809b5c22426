// flb_site15.cuh -- the per-site work of the D3Q15 step kernels (the lattice of
// the paper's own runs, Sec. VI), shared by the plain and batched kernels
// (flb_lb15.cu) and the persistent batched kernel (flb_persist.cu).
//
// Plane order: 0 rest; pairs (1,2) +-x, (3,4) +-y, (5,6) +-z, (7,8) +-(1,1,1),
// (9,10) +-(1,1,-1), (11,12) +-(1,-1,1), (13,14) +-(1,-1,-1).  Weights 2/9,
// 1/9, 1/72.
//
// The relaxation of the hydrodynamic moments (Eq. bab) is the same Cartesian
// algebra as on D3Q19: mass, momentum A = j + F and the second moment B, and
// the reconstruction w (rho + 3 A.c + 9/2 B:(cc - delta/3)).  The ghost space
// differs.  Gram-Schmidt under the weighted inner product gives the five
// D3Q15 ghosts and their norms
//   c_a (c^2 - 5/3)       b = 8/27   (a = x, y, z)
//   c_x c_y c_z           b = 1/9
//   c^4 - 3 c^2 + 4/3     b = 8/9
// each added back as w E_k g_k with g_k = (gamma_g m_k + noise_k)/b_k (the
// noise amplitude already carries 1/b_k).  Noise order: bulk, 3c_x^2-c^2,
// c_y^2-c_z^2, xy, yz, zx, the three c_a(c^2-5/3), c_xc_yc_z, c^4-3c^2+4/3:
// eleven normals from three Philox blocks of stream 0.
#pragma once

#include "flb_site3d.cuh"

namespace flb {

// fbar_i(r) = stored_i(r - c_i) for the 15 planes of site (x, y, z).
template <typename T, bool COH = false, class PL>
__device__ __forceinline__ void pull15(const PL &P, const Geom &g, int x, int y, int z, float f[15])
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
    f[7] = ld3<COH>(P.in(7), xm + sYm + sZm);    // (1,1,1)
    f[8] = ld3<COH>(P.in(8), xp + sYp + sZp);
    f[9] = ld3<COH>(P.in(9), xm + sYm + sZp);    // (1,1,-1)
    f[10] = ld3<COH>(P.in(10), xp + sYp + sZm);
    f[11] = ld3<COH>(P.in(11), xm + sYp + sZm);  // (1,-1,1)
    f[12] = ld3<COH>(P.in(12), xp + sYm + sZp);
    f[13] = ld3<COH>(P.in(13), xm + sYp + sZp);  // (1,-1,-1)
    f[14] = ld3<COH>(P.in(14), xp + sYm + sZm);
}

// Mass deviation and momentum of 15 populations; sp/dp the pair sums and differences.
__device__ __forceinline__ void moments15(const float f[15], float sp[8], float dp[8], float &drho, float &jx,
                                          float &jy, float &jz)
{
#pragma unroll
    for (int p = 1; p <= 7; ++p) {
        sp[p] = f[2 * p - 1] + f[2 * p];
        dp[p] = f[2 * p - 1] - f[2 * p];
    }
    drho = f[0] + ((sp[1] + sp[2] + sp[3]) + ((sp[4] + sp[5]) + (sp[6] + sp[7])));
    jx = dp[1] + ((dp[4] + dp[5]) + (dp[6] + dp[7]));
    jy = dp[2] + ((dp[4] + dp[5]) - (dp[6] + dp[7]));
    jz = dp[3] + ((dp[4] - dp[5]) + (dp[6] - dp[7]));
}

// The collide-stream of the D3Q15 sites (x, y, zl[l]) of the lanes of V (the
// first nl stored; a lane past the box repeats lane 0's site and is dropped).
// The second moment is carried as Q = 9/2 B, with the relaxation coefficients
// a.rq of the D3Q19 kernel (they do not depend on the lattice); the ghost
// amplitudes g_k stay in the units above.
// P: the planes it pulls from (P.in) and stores to (P.out).  COH: loads through
// L2 (fields written in the same launch); KEY_R0: round keys formed from round
// 0's (arguments in shared memory).
template <class V, typename T, bool GHOST_RELAX, bool COH = false, bool KEY_R0 = false, class PL>
__device__ __forceinline__ void lb15_sites(const LBArgs &a, const PL &P, int x, int y, const int *zl, int nl, V Fx,
                                           V Fy, V Fz)
{
    constexpr int L = V::L;
    const Geom &g = a.g;
    int s[L];
    V f[15];
    {
        float fl[L][15];
#pragma unroll
        for (int l = 0; l < L; ++l) {
            s[l] = x + g.nx * (y + g.ny * zl[l]);
            pull15<T, COH>(P, g, x, y, zl[l], fl[l]);
        }
#pragma unroll
        for (int i = 0; i < 15; ++i) {
            float t[L];
#pragma unroll
            for (int l = 0; l < L; ++l) t[l] = fl[l][i];
            f[i] = vmake<V>(t);
        }
    }
    V sp[8], dp[8];
#pragma unroll
    for (int p = 1; p <= 7; ++p) {
        sp[p] = f[2 * p - 1] + f[2 * p];
        dp[p] = f[2 * p - 1] - f[2 * p];
    }
    const V C = (sp[4] + sp[5]) + (sp[6] + sp[7]);
    const V drho = f[0] + ((sp[1] + sp[2] + sp[3]) + C);
    const V jx = dp[1] + ((dp[4] + dp[5]) + (dp[6] + dp[7]));
    const V jy = dp[2] + ((dp[4] + dp[5]) - (dp[6] + dp[7]));
    const V jz = dp[3] + ((dp[4] - dp[5]) + (dp[6] - dp[7]));
    const V third = drho * (1.0f / 3.0f);
    const V Sxx = sp[1] + C - third, Syy = sp[2] + C - third, Szz = sp[3] + C - third;
    const V Sxy = (sp[4] + sp[5]) - (sp[6] + sp[7]);
    const V Sxz = (sp[4] - sp[5]) + (sp[6] - sp[7]);
    const V Syz = (sp[4] - sp[5]) - (sp[6] - sp[7]);

    const V rho = drho + a.rho0;
    float ir[L];
#pragma unroll
    for (int l = 0; l < L; ++l) ir[l] = __fdividef(1.0f, rho.lane(l));
    const V irho = vmake<V>(ir);
    const V vx = vfma(Fx, 0.5f, jx) * irho, vy = vfma(Fy, 0.5f, jy) * irho, vz = vfma(Fz, 0.5f, jz) * irho;

    // Q = 4.5 [(1 - ws) S + ws rho v v + cs (v F + F v)] + the bulk correction
    const V cFx = Fx * a.rq[2], cFy = Fy * a.rq[2], cFz = Fz * a.rq[2];
    const V wr = rho * a.rq[1];
    const V hx = vfma(wr, vx, cFx), hy = vfma(wr, vy, cFy), hz = vfma(wr, vz, cFz);
    V Qxx = vfma(Sxx, a.rq[0], vx * (hx + cFx));
    V Qyy = vfma(Syy, a.rq[0], vy * (hy + cFy));
    V Qzz = vfma(Szz, a.rq[0], vz * (hz + cFz));
    if (a.iso) {
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

    // ghost amplitudes g_k (already divided by b_k)
    V gx = V::bc(0.f), gy = V::bc(0.f), gz = V::bc(0.f), gq = V::bc(0.f), g4 = V::bc(0.f);
    if (GHOST_RELAX) {
        const V gg = V::bc(a.gamma_g);
        const V mx = ((dp[4] + dp[5]) + (dp[6] + dp[7])) * (4.f / 3.f) - dp[1] * (2.f / 3.f);
        const V my = ((dp[4] + dp[5]) - (dp[6] + dp[7])) * (4.f / 3.f) - dp[2] * (2.f / 3.f);
        const V mz = ((dp[4] - dp[5]) + (dp[6] - dp[7])) * (4.f / 3.f) - dp[3] * (2.f / 3.f);
        const V mq = (dp[4] - dp[5]) - (dp[6] - dp[7]);
        const V m4 = (f[0] + C) * (4.f / 3.f) - (sp[1] + sp[2] + sp[3]) * (2.f / 3.f);
        gx = gg * mx * 3.375f;
        gy = gg * my * 3.375f;
        gz = gg * mz * 3.375f;
        gq = gg * mq * 9.0f;
        g4 = gg * m4 * 1.125f;
    }
    if (a.kT > 0.f) {
        // 11 normals from two Philox blocks, scaled by sqrt(rho kT / c_s^2) lane-wise
        const V mun = rho * a.k3T;
        float sq[L];
#pragma unroll
        for (int l = 0; l < L; ++l) sq[l] = mun.lane(l) * rsqrtf(mun.lane(l));
        uint32_t su[L];
#pragma unroll
        for (int l = 0; l < L; ++l) su[l] = (uint32_t)s[l];
        const V sc = vmake<V>(sq);
        V n[8];
        lane_block<8, KEY_R0>(a.key, a.step, su, 0u, sc, n);  // normals 0-7
        // the six stress modes enter Q as on D3Q19 (4.5 x 2/9 = 1, 4.5 x 1/9 = 1/2)
        const V m0 = n[0] * a.namp[0], m1 = n[1] * a.namp[1], m2 = n[2] * a.namp[2];
        const V t01 = m0 - m1;
        Qxx = Qxx + vfma(m1, 2.0f, m0);
        Qyy = Qyy + (t01 + m2);
        Qzz = Qzz + (t01 - m2);
        Qxy = vfma(n[3], 0.5f * a.namp[3], Qxy);
        Qyz = vfma(n[4], 0.5f * a.namp[4], Qyz);
        Qxz = vfma(n[5], 0.5f * a.namp[5], Qxz);
        gx = vfma(n[6], a.namp[6], gx);
        gy = vfma(n[7], a.namp[7], gy);
        lane_block<3, KEY_R0>(a.key, a.step, su, 1u, sc, n);  // normals 8-10
        gz = vfma(n[0], a.namp[8], gz);
        gq = vfma(n[1], a.namp[9], gq);
        g4 = vfma(n[2], a.namp[10], g4);
    }

    auto store = [&](int i, V v) {
#pragma unroll
        for (int l = 0; l < L; ++l)
            if (l < nl) st3(P.out(i), s[l], v.lane(l));
    };
    // B = Q / 4.5: e0 = 9/2 trB / 3 = trQ / 3, 9/2 B_aa = Q_aa, 9/2 trB - e0 = (2/3) trQ, 9 B_ab = 2 Q_ab
    const V trQ = Qxx + Qyy + Qzz;
    const V d = vfma(trQ, -1.0f / 3.0f, drho);  // drho - e0
    const float h2 = 2.f / 3.f, h4 = 4.f / 3.f;
    store(0, vfma(g4, h4, d) * (2.f / 9.f));
    const float w1 = 1.f / 9.f, w3 = 1.f / 72.f;
    const V Dm = vfma(g4, -h2, d);
    const V a3x = (jx + Fx) * 3.0f, a3y = (jy + Fy) * 3.0f, a3z = (jz + Fz) * 3.0f;
    {
        const V Ex = Dm + Qxx, Ey = Dm + Qyy, Ez = Dm + Qzz;
        const V Ox = vfma(gx, -h2, a3x), Oy = vfma(gy, -h2, a3y), Oz = vfma(gz, -h2, a3z);
        store(1, (Ex + Ox) * w1);
        store(2, (Ex - Ox) * w1);
        store(3, (Ey + Oy) * w1);
        store(4, (Ey - Oy) * w1);
        store(5, (Ez + Oz) * w1);
        store(6, (Ez - Oz) * w1);
    }
    // corners c = (1, a, b) and their opposites: B:cc = trB + 2(a Bxy + b Bxz + ab Byz)
    const V Ec = vfma(trQ, 2.0f / 3.0f, vfma(g4, h4, drho));
    const V gs = (gx + gy) * h4, gd = (gx - gy) * h4, gzh = gz * h4;
    const V sxy = a3x + a3y, dxy = a3x - a3y;
    {
        const V E = vfma(Qxy + Qxz + Qyz, 2.0f, Ec);
        const V O = ((sxy + a3z) + (gs + gzh)) + gq;
        store(7, (E + O) * w3);
        store(8, (E - O) * w3);
    }
    {
        const V E = vfma(Qxy - Qxz - Qyz, 2.0f, Ec);
        const V O = ((sxy - a3z) + (gs - gzh)) - gq;
        store(9, (E + O) * w3);
        store(10, (E - O) * w3);
    }
    {
        const V E = vfma(Qxz - Qxy - Qyz, 2.0f, Ec);
        const V O = ((dxy + a3z) + (gd + gzh)) - gq;
        store(11, (E + O) * w3);
        store(12, (E - O) * w3);
    }
    {
        const V E = vfma(Qyz - Qxy - Qxz, 2.0f, Ec);
        const V O = ((dxy - a3z) + (gd - gzh)) + gq;
        store(13, (E + O) * w3);
        store(14, (E - O) * w3);
    }
}

// u = (sum fbar c + F/2)/rho of the streamed state at (x, y, z), F this step's
// force; P.in: the planes of a.fout.
template <typename T, bool FORCE, bool COH = false, class PL>
__device__ __forceinline__ void vel15_site_on(const LBArgs &a, const PL &P, int x, int y, int z)
{
    const Geom &g = a.g;
    float f[15];
    pull15<T, COH>(P, g, x, y, z, f);
    float sp[8], dp[8], drho, jx, jy, jz;
    moments15(f, sp, dp, drho, jx, jy, jz);
    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
    if (FORCE && (a.coupling & FLB_COUPLE_FORCE)) force3<COH>(a, x, y, z, Fx, Fy, Fz);
    const float irho = __fdividef(1.0f, a.rho0 + drho);
    store_padded(a.u, g, x, y, z, (jx + 0.5f * Fx) * irho, 1);
    store_padded(a.u + g.pn, g, x, y, z, (jy + 0.5f * Fy) * irho, 1);
    store_padded(a.u + 2 * g.pn, g, x, y, z, (jz + 0.5f * Fz) * irho, 1);
}

// One site's collide-stream on the planes of a.fin and a.fout (the persistent
// kernel, one site per thread).
template <typename T, bool GHOST_RELAX, bool COH = false, bool KEY_R0 = false>
__device__ __forceinline__ void lb15_site(const LBArgs &a, int x, int y, int z, float Fx, float Fy, float Fz)
{
    lb15_sites<F1, T, GHOST_RELAX, COH, KEY_R0>(a, PlanesFromBase<T>{(const T *)a.fin, (T *)a.fout, a.g.n}, x, y,
                                                &z, 1, F1{Fx}, F1{Fy}, F1{Fz});
}

// The velocity at one site on the planes of a.fout.
template <typename T, bool FORCE, bool COH = false>
__device__ __forceinline__ void vel15_site(const LBArgs &a, int x, int y, int z)
{
    vel15_site_on<T, FORCE, COH>(a, PlanesFromBase<T>{(const T *)a.fout, nullptr, a.g.n}, x, y, z);
}

}  // namespace flb

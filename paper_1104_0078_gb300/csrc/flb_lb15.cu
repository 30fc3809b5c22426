// flb_lb15.cu -- D3Q15 fused collide-stream and the velocity of the new fluid
// state, one thread per site (the lattice of the paper's own runs, Sec. VI).
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
#include "flb_site3d.cuh"

namespace flb {

namespace {

// fbar_i(r) = stored_i(r - c_i) for the 15 planes of site (x, y, z).
template <typename T, class PL>
__device__ __forceinline__ void pull15(const PL &P, const Geom &g, int x, int y, int z, float f[15])
{
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    const int row = nx, pl = nx * ny;
    const int sY0 = row * y, sYm = row * ym, sYp = row * yp;
    const int sZ0 = pl * z, sZm = pl * zm, sZp = pl * zp;
    f[0] = ld3<false>(P.in(0), x + sY0 + sZ0);
    f[1] = ld3<false>(P.in(1), xm + sY0 + sZ0);
    f[2] = ld3<false>(P.in(2), xp + sY0 + sZ0);
    f[3] = ld3<false>(P.in(3), x + sYm + sZ0);
    f[4] = ld3<false>(P.in(4), x + sYp + sZ0);
    f[5] = ld3<false>(P.in(5), x + sY0 + sZm);
    f[6] = ld3<false>(P.in(6), x + sY0 + sZp);
    f[7] = ld3<false>(P.in(7), xm + sYm + sZm);    // (1,1,1)
    f[8] = ld3<false>(P.in(8), xp + sYp + sZp);
    f[9] = ld3<false>(P.in(9), xm + sYm + sZp);    // (1,1,-1)
    f[10] = ld3<false>(P.in(10), xp + sYp + sZm);
    f[11] = ld3<false>(P.in(11), xm + sYp + sZm);  // (1,-1,1)
    f[12] = ld3<false>(P.in(12), xp + sYm + sZp);
    f[13] = ld3<false>(P.in(13), xm + sYp + sZp);  // (1,-1,-1)
    f[14] = ld3<false>(P.in(14), xp + sYm + sZm);
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

// P: the planes it pulls from (P.in) and stores to (P.out).
template <typename T, bool GHOST_RELAX, class PL>
__device__ __forceinline__ void lb15_site(const LBArgs &a, const PL &P, int x, int y, int z, float Fx, float Fy,
                                          float Fz)
{
    const Geom &g = a.g;
    const int s = x + g.nx * (y + g.ny * z);

    float f[15];
    pull15<T>(P, g, x, y, z, f);
    float sp[8], dp[8], drho, jx, jy, jz;
    moments15(f, sp, dp, drho, jx, jy, jz);
    const float C = (sp[4] + sp[5]) + (sp[6] + sp[7]);
    const float third = drho * (1.0f / 3.0f);
    const float Sxx = sp[1] + C - third, Syy = sp[2] + C - third, Szz = sp[3] + C - third;
    const float Sxy = (sp[4] + sp[5]) - (sp[6] + sp[7]);
    const float Sxz = (sp[4] - sp[5]) + (sp[6] - sp[7]);
    const float Syz = (sp[4] - sp[5]) - (sp[6] - sp[7]);

    const float rho = a.rho0 + drho;
    const float irho = __fdividef(1.0f, rho);
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

    // ghost amplitudes g_k (already divided by b_k)
    float gx = 0.f, gy = 0.f, gz = 0.f, gq = 0.f, g4 = 0.f;
    if (GHOST_RELAX) {
        const float gg = a.gamma_g;
        const float mx = (4.f / 3.f) * ((dp[4] + dp[5]) + (dp[6] + dp[7])) - (2.f / 3.f) * dp[1];
        const float my = (4.f / 3.f) * ((dp[4] + dp[5]) - (dp[6] + dp[7])) - (2.f / 3.f) * dp[2];
        const float mz = (4.f / 3.f) * ((dp[4] - dp[5]) + (dp[6] - dp[7])) - (2.f / 3.f) * dp[3];
        const float mq = (dp[4] - dp[5]) - (dp[6] - dp[7]);
        const float m4 = (4.f / 3.f) * (f[0] + C) - (2.f / 3.f) * (sp[1] + sp[2] + sp[3]);
        gx = gg * mx * 3.375f;
        gy = gg * my * 3.375f;
        gz = gg * mz * 3.375f;
        gq = gg * mq * 9.0f;
        g4 = gg * m4 * 1.125f;
    }
    if (a.kT > 0.f) {
        float G[12];
        const uint32_t sid = (uint32_t)s;
        normals4(a.key, a.step, sid, 0u, 0u, G);
        normals4(a.key, a.step, sid, 0u, 1u, G + 4);
        normals4(a.key, a.step, sid, 0u, 2u, G + 8);
        const float mun = 3.0f * rho * a.kT;
        const float sq = mun * rsqrtf(mun);
        float n[11];
#pragma unroll
        for (int t = 0; t < 11; ++t) n[t] = sq * a.namp[t] * G[t];
        // the six stress modes enter B exactly as on D3Q19 (same polynomials)
        const float two9 = 2.0f / 9.0f, one9 = 1.0f / 9.0f;
        Bxx += two9 * (n[0] + 2.f * n[1]);
        Byy += two9 * (n[0] - n[1] + n[2]);
        Bzz += two9 * (n[0] - n[1] - n[2]);
        Bxy += one9 * n[3];
        Byz += one9 * n[4];
        Bxz += one9 * n[5];
        gx += n[6];
        gy += n[7];
        gz += n[8];
        gq += n[9];
        g4 += n[10];
    }

    const float trB = Bxx + Byy + Bzz;
    const float e0 = 1.5f * trB;  // 9/2 trB/3
    const float h2 = 2.f / 3.f, h4 = 4.f / 3.f;
    st3(P.out(0), s, (2.f / 9.f) * (drho - e0 + h4 * g4));
    const float w1 = 1.f / 9.f, w3 = 1.f / 72.f;
    float E, O;
    E = drho + 4.5f * Bxx - e0 - h2 * g4;
    O = 3.f * Ax - h2 * gx;
    st3(P.out(1), s, w1 * (E + O));
    st3(P.out(2), s, w1 * (E - O));
    E = drho + 4.5f * Byy - e0 - h2 * g4;
    O = 3.f * Ay - h2 * gy;
    st3(P.out(3), s, w1 * (E + O));
    st3(P.out(4), s, w1 * (E - O));
    E = drho + 4.5f * Bzz - e0 - h2 * g4;
    O = 3.f * Az - h2 * gz;
    st3(P.out(5), s, w1 * (E + O));
    st3(P.out(6), s, w1 * (E - O));
    // corners c = (1, a, b) and their opposites: B:cc = trB + 2(a Bxy + b Bxz + ab Byz)
    const float Ec = drho + 3.f * trB + h4 * g4;  // 9/2 trB - e0 = 3 trB
    E = Ec + 9.f * (Bxy + Bxz + Byz);
    O = 3.f * (Ax + Ay + Az) + h4 * (gx + gy + gz) + gq;
    st3(P.out(7), s, w3 * (E + O));
    st3(P.out(8), s, w3 * (E - O));
    E = Ec + 9.f * (Bxy - Bxz - Byz);
    O = 3.f * (Ax + Ay - Az) + h4 * (gx + gy - gz) - gq;
    st3(P.out(9), s, w3 * (E + O));
    st3(P.out(10), s, w3 * (E - O));
    E = Ec + 9.f * (-Bxy + Bxz - Byz);
    O = 3.f * (Ax - Ay + Az) + h4 * (gx - gy + gz) - gq;
    st3(P.out(11), s, w3 * (E + O));
    st3(P.out(12), s, w3 * (E - O));
    E = Ec + 9.f * (-Bxy - Bxz + Byz);
    O = 3.f * (Ax - Ay - Az) + h4 * (gx - gy - gz) + gq;
    st3(P.out(13), s, w3 * (E + O));
    st3(P.out(14), s, w3 * (E - O));
}

// P: the population planes (in: a.fin, out: a.fout), a table of addresses.
template <typename T, bool GHOST_RELAX, bool FORCE>
__global__ void __launch_bounds__(LB_BX *LB_BY *LB_BZ) lb15_kernel(const LBArgs a, const __grid_constant__ PlaneTable<T> P)
{
    const Geom &g = a.g;
    const int x = blockIdx.x * LB_BX + threadIdx.x;
    const int y = blockIdx.y * LB_BY + threadIdx.y;
    const int z = blockIdx.z * LB_BZ + threadIdx.z;
    if (x >= g.nx || y >= g.ny || z >= g.nz) return;
    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
    if (FORCE) force3<false>(a, x, y, z, Fx, Fy, Fz);
    lb15_site<T, GHOST_RELAX>(a, P, x, y, z, Fx, Fy, Fz);
}

// u = (sum fbar c + F/2)/rho of the streamed state, F this step's force (plane
// addresses formed from a.fout, as in the D3Q19 velocity gather).
template <typename T, bool FORCE>
__global__ void __launch_bounds__(LB_BX *LB_BY *LB_BZ) vel15_kernel(const LBArgs a)
{
    const Geom &g = a.g;
    const int x = blockIdx.x * LB_BX + threadIdx.x;
    const int y = blockIdx.y * LB_BY + threadIdx.y;
    const int z = blockIdx.z * LB_BZ + threadIdx.z;
    if (x >= g.nx || y >= g.ny || z >= g.nz) return;
    float f[15];
    pull15<T>(PlanesFromBase<T>{(const T *)a.fout, nullptr, g.n}, g, x, y, z, f);
    float sp[8], dp[8], drho, jx, jy, jz;
    moments15(f, sp, dp, drho, jx, jy, jz);
    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
    if (FORCE) force3<false>(a, x, y, z, Fx, Fy, Fz);
    const float irho = __fdividef(1.0f, a.rho0 + drho);
    store_padded(a.u, g, x, y, z, (jx + 0.5f * Fx) * irho, 1);
    store_padded(a.u + g.pn, g, x, y, z, (jy + 0.5f * Fy) * irho, 1);
    store_padded(a.u + 2 * g.pn, g, x, y, z, (jz + 0.5f * Fz) * irho, 1);
}

}  // namespace

cudaError_t launch_lb15(const LBArgs &a, int storage, cudaStream_t st)
{
    const dim3 block(LB_BX, LB_BY, LB_BZ);
    const dim3 grid((a.g.nx + LB_BX - 1) / LB_BX, (a.g.ny + LB_BY - 1) / LB_BY, (a.g.nz + LB_BZ - 1) / LB_BZ);
    const bool gr = a.gamma_g != 0.0f;
    const bool force = (a.coupling & FLB_COUPLE_FORCE) != 0;
#define FLB_LB15(T, G, F) lb15_kernel<T, G, F><<<grid, block, 0, st>>>(a, plane_table<T>(a.fin, a.fout, a.g.n, 15))
    if (storage == FLB_F16_DEV) {
        if (gr) { if (force) FLB_LB15(__half, true, true); else FLB_LB15(__half, true, false); }
        else { if (force) FLB_LB15(__half, false, true); else FLB_LB15(__half, false, false); }
    } else {
        if (gr) { if (force) FLB_LB15(float, true, true); else FLB_LB15(float, true, false); }
        else { if (force) FLB_LB15(float, false, true); else FLB_LB15(float, false, false); }
    }
#undef FLB_LB15
    return cudaGetLastError();
}

cudaError_t launch_vel15(const LBArgs &a, int storage, cudaStream_t st)
{
    const dim3 block(LB_BX, LB_BY, LB_BZ);
    const dim3 grid((a.g.nx + LB_BX - 1) / LB_BX, (a.g.ny + LB_BY - 1) / LB_BY, (a.g.nz + LB_BZ - 1) / LB_BZ);
    const bool force = (a.coupling & FLB_COUPLE_FORCE) != 0;
    if (storage == FLB_F16_DEV) {
        if (force) vel15_kernel<__half, true><<<grid, block, 0, st>>>(a);
        else vel15_kernel<__half, false><<<grid, block, 0, st>>>(a);
    } else {
        if (force) vel15_kernel<float, true><<<grid, block, 0, st>>>(a);
        else vel15_kernel<float, false><<<grid, block, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace flb

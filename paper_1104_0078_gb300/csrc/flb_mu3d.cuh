// flb_mu3d.cuh -- one column of the chemical potential mu = A psi + B psi^3
// - K lap_SO psi (Sec. II.A, Eq. solap) or of the order-parameter stress sigma
// (Sec. IV, Eq. muf) on the 3D padded grid, marching z with per-plane partial
// sums of the SO stencil; used by the per-phase, batched and persistent kernels.
#pragma once

#include "flb_site3d.cuh"

namespace flb {

// The column (x, y), output planes zb .. ze-1 of the mu field.  lw (may be
// null): the class weights of an App. A Laplacian instead of SO's,
// mu = A psi + B psi^3 - K [(c1 n1 + c2 n2) + (c3 n3 + c0 psi)] over the faces
// n1, edges n2 and corners n3 of the 3 x 3 x 3 neighbourhood.
template <bool COH = false>
__device__ __forceinline__ void mu3_column(const Geom &g, const float *__restrict__ psi, float *__restrict__ mu, float A,
                                           float B, float K, int x, int y, int zb, int ze, const LapW *lw = nullptr)
{
    const int Y = g.px, Z = g.px * g.py;
    const float k22 = K * (1.0f / 22.0f);
    int c = g.pidx32(x, y, zb - 1);
    float a0 = 0.f, b0 = 0.f, d0 = 0.f, a1 = 0.f, b1 = 0.f, d1 = 0.f;  // planes p-2, p-1
    for (int p = zb - 1; p <= ze; ++p, c += Z) {
        const float a2 = ldf<COH>(psi + c);
        const float b2 = (ldf<COH>(psi + c - 1) + ldf<COH>(psi + c + 1)) + (ldf<COH>(psi + c - Y) + ldf<COH>(psi + c + Y));
        const float d2 = (ldf<COH>(psi + c - 1 - Y) + ldf<COH>(psi + c + 1 - Y)) + (ldf<COH>(psi + c - 1 + Y) + ldf<COH>(psi + c + 1 + Y));
        if (p - 1 >= zb) {
            const float n1 = b1 + (a0 + a2), n2 = d1 + (b0 + b2), n3 = d0 + d2;
            mu[c - Z] = lw ? A * a1 + B * a1 * a1 * a1 - K * ((lw->c1 * n1 + lw->c2 * n2) + (lw->c3 * n3 + lw->c0 * a1))
                           : mu_so(A, B, k22, a1, n1, n2, n3);
        }
        a0 = a1; b0 = b1; d0 = d1;
        a1 = a2; b1 = b2; d1 = d2;
    }
}

// The column (x, y), planes zb .. ze-1, of the order-parameter stress (Sec. IV,
// Eq. muf): sigma_ab = K g_a g_b + delta_ab [A/2 psi^2 + 3B/4 psi^4
// - K psi lap_SO psi - K/2 |g|^2], g the central-difference gradient of psi.
// Per plane a thread keeps the centre, the faces and the diagonals of psi (the
// SO stencil, as in mu3_column) and the in-plane face differences.
template <bool COH = false>
__device__ __forceinline__ void sigma3_column(const Geom &g, const float *__restrict__ psi, float *__restrict__ sig,
                                              float A, float B, float K, int x, int y, int zb, int ze)
{
    const int Y = g.px, Z = g.px * g.py, pn = (int)g.pn;
    int c = g.pidx32(x, y, zb - 1);
    float a0 = 0.f, b0 = 0.f, d0 = 0.f, a1 = 0.f, b1 = 0.f, d1 = 0.f, gx1 = 0.f, gy1 = 0.f;
    for (int p = zb - 1; p <= ze; ++p, c += Z) {
        const float a2 = ldf<COH>(psi + c);
        const float xm = ldf<COH>(psi + c - 1), xp = ldf<COH>(psi + c + 1);
        const float ym = ldf<COH>(psi + c - Y), yp = ldf<COH>(psi + c + Y);
        const float b2 = (xm + xp) + (ym + yp);
        const float d2 = (ldf<COH>(psi + c - 1 - Y) + ldf<COH>(psi + c + 1 - Y)) + (ldf<COH>(psi + c - 1 + Y) + ldf<COH>(psi + c + 1 + Y));
        if (p - 1 >= zb) {  // plane p-1: centre a1, gradient (gx1, gy1, gz)
            const float n1 = b1 + (a0 + a2), n2 = d1 + (b0 + b2), n3 = d0 + d2;
            const float lap = (6.f * n1 + 3.f * n2 + n3 - 80.f * a1) * (1.0f / 22.0f);
            const float gz = 0.5f * (a2 - a0);
            const float ps2 = a1 * a1;
            const float iso = 0.5f * A * ps2 + 0.75f * B * ps2 * ps2 - K * a1 * lap -
                              0.5f * K * (gx1 * gx1 + gy1 * gy1 + gz * gz);
            const int o = c - Z;
            sig[o] = K * gx1 * gx1 + iso;
            sig[o + pn] = K * gy1 * gy1 + iso;
            sig[o + 2 * pn] = K * gz * gz + iso;
            sig[o + 3 * pn] = K * gx1 * gy1;
            sig[o + 4 * pn] = K * gx1 * gz;
            sig[o + 5 * pn] = K * gy1 * gz;
        }
        a0 = a1; b0 = b1; d0 = d1;
        a1 = a2; b1 = b2; d1 = d2;
        gx1 = 0.5f * (xp - xm);
        gy1 = 0.5f * (yp - ym);
    }
}

}  // namespace flb

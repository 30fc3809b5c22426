/*
 * flb_oracle.c -- plain FP64 CPU oracle for one coupled time step of the
 * hybrid model-H solver of Sumesh, Pagonabarraga & Adhikari (arXiv:1104.0078):
 * a fluctuating lattice Boltzmann step for the momentum (Sec. IV, App. B)
 * alternated with a stochastic method-of-lines step for the conserved order
 * parameter psi (Sec. V, finite-difference Sec. V.A and finite-volume Sec. V.B).
 *
 * TEST INFRASTRUCTURE. This file is the checker, not the product: only the
 * test-suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or constant with the CUDA library; the two
 * implement the same published definitions independently.
 *
 * Everything is written as plain loops over lattice sites in double precision,
 * in the order the paper states the algorithm.  Readings of passages that the
 * paper leaves open (force sign, tau convention, moment basis, ghost noise,
 * real-space finite-difference noise, time integrator, random-number mapping)
 * are named where they are used.
 *
 * Conventions
 *   lattice units dx = dt = 1 (Sec. VI), periodic boundaries, c_s^2 = 1/3.
 *   site index s = x + nx*(y + ny*z); population plane i at f[i*N + s].
 *   f holds the auxiliary distribution fbar(x,t) of Eq. (barreln) AFTER
 *   streaming, i.e. the pre-collision state at time t.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "flb_oracle.h"
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads the site loops use (OpenMP), for reporting the CPU baseline. */
int ora_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the site loops from now on (n >= 1). */
void ora_set_threads(int32_t n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11): ten rounds of a multiply-hi/lo bijection with a  */
/* Weyl-sequence key schedule.  The paper itself names no generator.          */
/* ------------------------------------------------------------------------- */
void ora_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint64_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = M0 * (uint64_t)x0;
        uint64_t p1 = M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One Box-Muller pair per 32-bit word w: the radius uniform from its top 20
 * bits, ((w >> 12) + 1/2) * 2^-20, and the angle uniform from its low 12 bits,
 * ((w & 0xFFF) + 1/2) * 2^-12.  Both values are exactly representable in
 * binary32 and binary64, so both sides of the parity check start every
 * Gaussian from the same real numbers. */
static double u_radius(uint32_t w) { return ((double)(w >> 12) + 0.5) * (1.0 / 1048576.0); }
static double u_angle(uint32_t w) { return ((double)(w & 0xFFFu) + 0.5) * (1.0 / 4096.0); }

/* Standard normals for (seed, step, site, stream): block b of the Philox
 * counter (site, step_lo, (stream << 16) | b, step_hi) under key (seed_lo,
 * seed_hi) yields four words x_0..x_3; word x_k gives normals 8b+2k and
 * 8b+2k+1 as r cos(2 pi v), r sin(2 pi v) with r = sqrt(-2 ln u), u and v the
 * radius and angle uniforms of x_k. */
void ora_gaussians(uint64_t seed, int64_t step, uint32_t site, uint32_t stream,
                   int32_t nblocks, double *g)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int b = 0; b < nblocks; ++b) {
        uint32_t ctr[4] = {site, (uint32_t)(uint64_t)step, (stream << 16) | (uint32_t)b,
                           (uint32_t)((uint64_t)step >> 32)};
        uint32_t x[4];
        ora_philox4x32_10(ctr, key, x);
        for (int k = 0; k < 4; ++k) {
            double r = sqrt(-2.0 * log(u_radius(x[k]))), t = u_angle(x[k]);
            g[8 * b + 2 * k] = r * cos(2.0 * M_PI * t);
            g[8 * b + 2 * k + 1] = r * sin(2.0 * M_PI * t);
        }
    }
}

/* The normals of ora_gaussians for nsites consecutive counter sites
 * site0 .. site0 + nsites - 1: g[s * 8 nblocks + k]. */
void ora_gaussians_sites(uint64_t seed, int64_t step, uint32_t site0, int64_t nsites, uint32_t stream,
                         int32_t nblocks, double *g)
{
    for (int64_t s = 0; s < nsites; ++s)
        ora_gaussians(seed, step, site0 + (uint32_t)s, stream, nblocks, g + (size_t)s * 8 * (size_t)nblocks);
}

/* ------------------------------------------------------------------------- */
/* Velocity sets and weights (Sec. IV; D3Q15 is the paper's own, Sec. VI).    */
/* Plane order: rest first, then opposite pairs (i, i+1).                     */
/* ------------------------------------------------------------------------- */
int ora_lattice(int32_t dim, int32_t q, int32_t *c, double *w)
{
    int n = 0;
    memset(c, 0, sizeof(int32_t) * 3 * (size_t)q);
    if (dim == 2 && q == 9) {
        static const int v[9][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1},
                                    {1, 1}, {-1, -1}, {1, -1}, {-1, 1}};
        for (n = 0; n < 9; ++n) {
            c[3 * n] = v[n][0]; c[3 * n + 1] = v[n][1];
            int len2 = v[n][0] * v[n][0] + v[n][1] * v[n][1];
            w[n] = len2 == 0 ? 4.0 / 9.0 : len2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0;
        }
        return 0;
    }
    if (dim == 3 && q == 19) {
        static const int v[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                     {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                     {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                     {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
        for (n = 0; n < 19; ++n) {
            int len2 = 0;
            for (int a = 0; a < 3; ++a) { c[3 * n + a] = v[n][a]; len2 += v[n][a] * v[n][a]; }
            w[n] = len2 == 0 ? 1.0 / 3.0 : len2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0;
        }
        return 0;
    }
    if (dim == 3 && q == 15) {
        static const int v[15][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0},   {0, 1, 0},  {0, -1, 0},
                                     {0, 0, 1},  {0, 0, -1},  {1, 1, 1},    {-1, -1, -1}, {1, 1, -1},
                                     {-1, -1, 1}, {1, -1, 1}, {-1, 1, -1}, {1, -1, -1}, {-1, 1, 1}};
        for (n = 0; n < 15; ++n) {
            int len2 = 0;
            for (int a = 0; a < 3; ++a) { c[3 * n + a] = v[n][a]; len2 += v[n][a] * v[n][a]; }
            w[n] = len2 == 0 ? 2.0 / 9.0 : len2 == 1 ? 1.0 / 9.0 : 1.0 / 72.0;
        }
        return 0;
    }
    return -1;
}

/* ------------------------------------------------------------------------- */
/* Moment basis (App. B asks for "the moment basis" without listing it).      */
/* Reading: Gram-Schmidt under <a,b> = sum_i w_i a_i b_i applied to the       */
/* ordered monomials below; b_k = <e_k, e_k>.  Classes: mass {0}, momentum    */
/* {1..d}, stress {d+1 .. d+d(d+1)/2}, ghosts = the rest.                     */
/* ------------------------------------------------------------------------- */
static double monomial(int dim, int q, int k, const int32_t *cv)
{
    double cx = cv[0], cy = cv[1], cz = cv[2];
    double c2 = cx * cx + cy * cy + cz * cz;
    if (dim == 3 && q == 15) {
        /* D3Q15: the stress and c^2 c_a rows as for D3Q19; the remaining
         * independent monomials on this set are c_x c_y c_z and c^4
         * (c_a(c_b^2 - c_g^2) vanishes and c^2(3c_x^2 - c^2) repeats 3c_x^2 - c^2) */
        if (k == 13) return cx * cy * cz;
        if (k == 14) return c2 * c2;
    }
    if (dim == 3) {
        switch (k) {
        case 0: return 1.0;
        case 1: return cx;
        case 2: return cy;
        case 3: return cz;
        case 4: return c2;
        case 5: return 3.0 * cx * cx - c2;
        case 6: return cy * cy - cz * cz;
        case 7: return cx * cy;
        case 8: return cy * cz;
        case 9: return cz * cx;
        case 10: return c2 * cx;
        case 11: return c2 * cy;
        case 12: return c2 * cz;
        case 13: return cx * (cy * cy - cz * cz);
        case 14: return cy * (cz * cz - cx * cx);
        case 15: return cz * (cx * cx - cy * cy);
        case 16: return c2 * c2;
        case 17: return c2 * (3.0 * cx * cx - c2);
        case 18: return c2 * (cy * cy - cz * cz);
        }
    } else {
        switch (k) {
        case 0: return 1.0;
        case 1: return cx;
        case 2: return cy;
        case 3: return c2;
        case 4: return cx * cx - cy * cy;
        case 5: return cx * cy;
        case 6: return c2 * cx;
        case 7: return c2 * cy;
        case 8: return c2 * c2;
        }
    }
    return 0.0;
}

int ora_moment_basis(int32_t dim, int32_t q, double *E, double *b)
{
    int32_t c[3 * 19];
    double w[19];
    if (!((dim == 3 && (q == 19 || q == 15)) || (dim == 2 && q == 9))) return -1;
    if (ora_lattice(dim, q, c, w)) return -1;
    for (int k = 0; k < q; ++k) {
        double *ek = E + (size_t)k * q;
        for (int i = 0; i < q; ++i) ek[i] = monomial(dim, q, k, c + 3 * i);
        for (int l = 0; l < k; ++l) {
            const double *el = E + (size_t)l * q;
            double dot = 0.0;
            for (int i = 0; i < q; ++i) dot += w[i] * ek[i] * el[i];
            for (int i = 0; i < q; ++i) ek[i] -= dot / b[l] * el[i];
        }
        double nrm = 0.0;
        for (int i = 0; i < q; ++i) nrm += w[i] * ek[i] * ek[i];
        if (nrm < 1e-12) return -2; /* monomials not independent on this lattice */
        b[k] = nrm;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Periodic lattice helpers                                                    */
/* ------------------------------------------------------------------------- */
typedef struct {
    int dim, nx, ny, nz;
    size_t n;
} box_t;

static box_t box_of(const ora_params *p)
{
    box_t g;
    g.dim = p->dim; g.nx = p->nx; g.ny = p->ny; g.nz = p->dim == 2 ? 1 : p->nz;
    g.n = (size_t)g.nx * g.ny * g.nz;
    return g;
}

static inline int wrap(int a, int n) { a %= n; return a < 0 ? a + n : a; }

static inline size_t site_at(const box_t *g, int x, int y, int z)
{
    return (size_t)wrap(x, g->nx) + (size_t)g->nx * ((size_t)wrap(y, g->ny) + (size_t)g->ny * (size_t)wrap(z, g->nz));
}

static inline void coords(const box_t *g, size_t s, int *x, int *y, int *z)
{
    *x = (int)(s % (size_t)g->nx);
    *y = (int)((s / (size_t)g->nx) % (size_t)g->ny);
    *z = (int)(s / ((size_t)g->nx * g->ny));
}

/* Counter id of a site: its index in the global lattice.  A box may be a
 * window (origin ox,oy,oz) of a larger periodic lattice gnx x gny x gnz so that
 * single sites of a big run can be recomputed from a small neighbourhood. */
static inline uint32_t rng_site(const ora_params *p, int x, int y, int z)
{
    int gx = p->gnx > 0 ? p->gnx : p->nx;
    int gy = p->gny > 0 ? p->gny : p->ny;
    int gz = p->gnz > 0 ? p->gnz : (p->dim == 2 ? 1 : p->nz);
    int X = wrap(p->ox + x, gx), Y = wrap(p->oy + y, gy), Z = wrap(p->oz + z, gz);
    return (uint32_t)((uint64_t)X + (uint64_t)gx * ((uint64_t)Y + (uint64_t)gy * (uint64_t)Z));
}

/* ------------------------------------------------------------------------- */
/* Laplacian stencils of App. A and the finite-volume operators of Sec. V.B   */
/* ------------------------------------------------------------------------- */

/* The Laplacian stencils of App. A on the 3D cubic neighbourhood, written by
 * neighbour class: a1 on the 6 nearest neighbours (N1), a2 on the 12 next
 * nearest (N2), a3 on the 8 corners (N3), and -(6 a1 + 12 a2 + 8 a3) at the
 * centre:
 *   kind 0 Shinozaki-Oono, Eq. (solap):  6/22, 3/22, 1/22 (centre -80/22)
 *   kind 1 central difference, Eq. (fdlap): 1, 0, 0 (centre -6)
 *   kind 2 Patra-Karttunen, Eq. (pklap): 14/30, 3/30, 1/30 (centre -128/30)
 *   kind 3 lattice Boltzmann, Eq. (lblap): 1/9 on all 26 (centre -26/9)
 * In 2D the paper gives no stencil; readings: SO 1/4 [2 sum N1 + sum N2 - 12 psi]
 * (the planar stencil with the same N1:N2 = 2:1 weighting) and CD the 5-point
 * stencil.  Returns -1 for a kind without a 2D form. */
static int lap_class_weights(int dim, int kind, double a[4])
{
    a[3] = 0.0;
    if (dim == 3) {
        switch (kind) {
        case 0: a[1] = 6.0 / 22.0; a[2] = 3.0 / 22.0; a[3] = 1.0 / 22.0; break;
        case 1: a[1] = 1.0; a[2] = 0.0; a[3] = 0.0; break;
        case 2: a[1] = 14.0 / 30.0; a[2] = 3.0 / 30.0; a[3] = 1.0 / 30.0; break;
        case 3: a[1] = 1.0 / 9.0; a[2] = 1.0 / 9.0; a[3] = 1.0 / 9.0; break;
        default: return -1;
        }
        a[0] = -(6.0 * a[1] + 12.0 * a[2] + 8.0 * a[3]);
        return 0;
    }
    switch (kind) {
    case 0: a[1] = 0.5; a[2] = 0.25; break;
    case 1: a[1] = 1.0; a[2] = 0.0; break;
    default: return -1;
    }
    a[0] = -(4.0 * a[1] + 4.0 * a[2]);
    return 0;
}

int ora_laplacian(int32_t dim, int32_t kind, int32_t nx, int32_t ny, int32_t nz, const double *in, double *out)
{
    double a[4];
    if (lap_class_weights(dim, kind, a)) return -1;
    box_t g; g.dim = dim; g.nx = nx; g.ny = ny; g.nz = dim == 2 ? 1 : nz;
    g.n = (size_t)g.nx * g.ny * g.nz;
    const int zr = dim == 3 ? 1 : 0;
#pragma omp parallel for schedule(static)
    for (long long s = 0; s < (long long)g.n; ++s) {
        int x, y, z;
        coords(&g, (size_t)s, &x, &y, &z);
        double acc = 0.0;
        for (int dz = -zr; dz <= zr; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int cls = abs(dx) + abs(dy) + abs(dz);
                    acc += a[cls] * in[site_at(&g, x + dx, y + dy, z + dz)];
                }
        out[s] = acc;
    }
    return 0;
}

void ora_laplacian_so(int32_t dim, int32_t nx, int32_t ny, int32_t nz, const double *in, double *out)
{
    ora_laplacian(dim, 0, nx, ny, nz, in, out);
}

/* Finite-volume gradient, Eq. (fvgrad): grad m(r) = (1/c_s^2) sum_i w_i c_i m(r + c_i).
 * (The paper's "c_s^2 delta = sum c c" drops the weights; sum_i w_i c_i c_i = c_s^2 delta is meant.) */
static void fv_gradient(const box_t *g, int q, const int32_t *c, const double *w, const double *m, double *grad)
{
    const double inv_cs2 = 3.0;
#pragma omp parallel for schedule(static)
    for (long long s = 0; s < (long long)g->n; ++s) {
        int x, y, z;
        coords(g, (size_t)s, &x, &y, &z);
        double gr[3] = {0, 0, 0};
        for (int i = 1; i < q; ++i) {
            double mv = m[site_at(g, x + c[3 * i], y + c[3 * i + 1], z + c[3 * i + 2])];
            for (int a = 0; a < g->dim; ++a) gr[a] += w[i] * c[3 * i + a] * mv;
        }
        for (int a = 0; a < g->dim; ++a) grad[(size_t)a * g->n + s] = inv_cs2 * gr[a];
    }
}

/* Finite-volume divergence of a node flux J through link-midpoint averages,
 * Eqs. (fvdiff), (fvflux), (noiseflux): div(r) = (2/c_s^2) sum_i w_i c_i . J^i,
 * J^i = (J(r) + J(r + c_i))/2.  Reading: the factor 2/c_s^2, garbled in the
 * paper, is the one that makes the operator tend to div as q -> 0 and that
 * reproduces Eq. (fvlapft) for D3Q15. */
static void fv_divergence(const box_t *g, int q, const int32_t *c, const double *w, const double *J, double *div)
{
    const double fac = 2.0 * 3.0;
#pragma omp parallel for schedule(static)
    for (long long s = 0; s < (long long)g->n; ++s) {
        int x, y, z;
        coords(g, (size_t)s, &x, &y, &z);
        double acc = 0.0;
        for (int i = 1; i < q; ++i) {
            size_t t = site_at(g, x + c[3 * i], y + c[3 * i + 1], z + c[3 * i + 2]);
            for (int a = 0; a < g->dim; ++a) {
                double link = 0.5 * (J[(size_t)a * g->n + (size_t)s] + J[(size_t)a * g->n + t]);
                acc += w[i] * c[3 * i + a] * link;
            }
        }
        div[s] = fac * acc;
    }
}

/* Laplacian that the finite-volume scheme applies to mu: div(grad m)
 * (App. A, Eq. (fvlapft) for D3Q15).  Exposed for the Fourier-symbol tests. */
int ora_fv_laplacian(int32_t dim, int32_t q, int32_t nx, int32_t ny, int32_t nz, const double *in, double *out)
{
    int32_t c[3 * 19];
    double w[19];
    if (ora_lattice(dim, q, c, w)) return -1;
    box_t g; g.dim = dim; g.nx = nx; g.ny = ny; g.nz = dim == 2 ? 1 : nz;
    g.n = (size_t)g.nx * g.ny * g.nz;
    double *grad = (double *)malloc(sizeof(double) * 3 * g.n);
    if (!grad) return -3;
    fv_gradient(&g, q, c, w, in, grad);
    fv_divergence(&g, q, c, w, grad, out);
    free(grad);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Chemical potential and force                                                */
/* ------------------------------------------------------------------------- */

/* mu = A psi + B psi^3 - K lap psi (Sec. II.A), lap the App. A stencil chosen
 * by p->laplacian (the paper's runs: SO). */
void ora_mu(const ora_params *p, const double *psi, double *mu)
{
    box_t g = box_of(p);
    double *lap = (double *)malloc(sizeof(double) * g.n);
    ora_laplacian(p->dim, p->laplacian, p->nx, p->ny, p->nz, psi, lap);
    for (size_t s = 0; s < g.n; ++s) {
        double ps = psi[s];
        mu[s] = p->A * ps + p->B * ps * ps * ps - p->K * lap[s];
    }
    free(lap);
}

/* Force density as the divergence of the order-parameter stress (Sec. IV,
 * Eq. muf), F = -div sigma with
 *   sigma_ab = K d_a psi d_b psi
 *            + delta_ab [A/2 psi^2 + 3B/4 psi^4 - K psi lap psi - K/2 |grad psi|^2]
 * (psi f' - f = A/2 psi^2 + 3B/4 psi^4 for f = A/2 psi^2 + B/4 psi^4), whose
 * continuum divergence is psi grad mu.  Reading: gradients by the symmetric
 * central difference, lap by the stencil of mu, and the divergence by
 * the central difference, so that sum_r F = 0 exactly (momentum is conserved
 * for B != 0 too) while F = -psi grad mu + O(h^2). */
static void stress_force(const ora_params *p, const box_t *g, const double *psi, double *F)
{
    const size_t N = g->n;
    const int d = g->dim;
    double *lap = (double *)malloc(sizeof(double) * N);
    double *sig = (double *)malloc(sizeof(double) * 9 * N);
    ora_laplacian(p->dim, p->laplacian, p->nx, p->ny, p->nz, psi, lap);
    for (size_t s = 0; s < N; ++s) {
        int x, y, z;
        coords(g, s, &x, &y, &z);
        double gr[3] = {0.5 * (psi[site_at(g, x + 1, y, z)] - psi[site_at(g, x - 1, y, z)]),
                        0.5 * (psi[site_at(g, x, y + 1, z)] - psi[site_at(g, x, y - 1, z)]),
                        d == 3 ? 0.5 * (psi[site_at(g, x, y, z + 1)] - psi[site_at(g, x, y, z - 1)]) : 0.0};
        const double ps = psi[s];
        const double g2 = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
        const double iso = 0.5 * p->A * ps * ps + 0.75 * p->B * ps * ps * ps * ps - p->K * ps * lap[s] - 0.5 * p->K * g2;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) sig[(size_t)(3 * a + b) * N + s] = p->K * gr[a] * gr[b] + (a == b ? iso : 0.0);
    }
    for (size_t s = 0; s < N; ++s) {
        int x, y, z;
        coords(g, s, &x, &y, &z);
        for (int a = 0; a < 3; ++a) {
            double div = 0.0;
            if (a < d)
                for (int b = 0; b < d; ++b) {
                    int e[3] = {0, 0, 0};
                    e[b] = 1;
                    const double *sab = sig + (size_t)(3 * a + b) * N;
                    div += 0.5 * (sab[site_at(g, x + e[0], y + e[1], z + e[2])] - sab[site_at(g, x - e[0], y - e[1], z - e[2])]);
                }
            F[(size_t)a * N + s] = -div;
        }
    }
    free(lap);
    free(sig);
}

/* Force density on the fluid from the order parameter (Sec. IV): F = -psi grad mu.
 * Reading of the sign: the paper prints +psi grad mu; only -psi grad mu makes
 * the advective work u.F cancel the advective change of the free energy, so
 * that free energy plus kinetic energy cannot grow without noise.
 * Gradient (force_grad): 1 -- the symmetric nearest-neighbour central difference
 * of Sec. IV; 2 -- the finite-volume lattice gradient of Eq. (fvgrad),
 * (1/c_s^2) sum_i w_i c_i mu(r + c_i); 0 -- the one matched to the psi scheme
 * (1 for FD, 2 for FV); 3 -- no gradient of mu: the divergence of the stress
 * (stress_force above).  Reading: the cancellation above holds on the lattice
 * only if the force uses the gradient whose negative adjoint is the divergence
 * that advects psi.  For the FD scheme (central-difference advection, Sec. V.A)
 * that is the central difference; for the FV scheme (advection through link
 * averages, Eq. fvflux) it is the FV gradient.  With the unmatched pair the
 * exchange leaves a residue that noise drives into growing short-wavelength
 * modes at an interface. */
void ora_force(const ora_params *p, const double *psi, const double *mu, double *F)
{
    box_t g = box_of(p);
    const int grad = p->force_grad == 0 ? (p->scheme == 1 ? 2 : 1) : p->force_grad;
    if (grad == 3) {
        stress_force(p, &g, psi, F);
        return;
    }
    if (grad == 2) {
        int32_t c[3 * 19];
        double w[19];
        ora_lattice(p->dim, p->q, c, w);
        double *grad = (double *)malloc(sizeof(double) * 3 * g.n);
        memset(grad, 0, sizeof(double) * 3 * g.n);
        fv_gradient(&g, p->q, c, w, mu, grad);
        for (size_t s = 0; s < g.n; ++s)
            for (int a = 0; a < 3; ++a) F[a * g.n + s] = a < g.dim ? -psi[s] * grad[a * g.n + s] : 0.0;
        free(grad);
        return;
    }
    for (size_t s = 0; s < g.n; ++s) {
        int x, y, z;
        coords(&g, s, &x, &y, &z);
        double gx = 0.5 * (mu[site_at(&g, x + 1, y, z)] - mu[site_at(&g, x - 1, y, z)]);
        double gy = 0.5 * (mu[site_at(&g, x, y + 1, z)] - mu[site_at(&g, x, y - 1, z)]);
        double gz = g.dim == 3 ? 0.5 * (mu[site_at(&g, x, y, z + 1)] - mu[site_at(&g, x, y, z - 1)]) : 0.0;
        F[s] = -psi[s] * gx;
        F[g.n + s] = -psi[s] * gy;
        F[2 * g.n + s] = -psi[s] * gz;
    }
}

/* ------------------------------------------------------------------------- */
/* Fluctuating lattice Boltzmann step (Sec. IV, App. B)                        */
/* ------------------------------------------------------------------------- */
/* stress and ghost modes: every mode but mass and momentum */
static int noisy_mode_count(int dim, int q) { return q - dim - 1; }

/* One collision at every site followed by streaming.  F is the force density
 * (3 x N; may be NULL).  u_out (d x N) receives the velocity of the streamed
 * populations, v = (sum fbar c + F/2)/rho with the F just applied: the fluid
 * velocity after this step, which advects psi (see ora_step).
 *
 *  Momentum relations (App. B, last paragraph): rho = sum fbar,
 *    rho v = sum fbar c + F dt/2.  Reading: the paper's "rho F" multiplies a
 *    force DENSITY by rho; F alone is meant.
 *  Post-collision moments, Eq. (bab): A = sum fbar c + F dt;
 *    B = S + omega(-S + rho v v + tau (v F + F v) + ...), omega = dt/(tau+dt/2)
 *    (so tau omega = 1 - omega/2).  Reading: tau is the paper's, with
 *    omega = 1/(tau + 1/2), viscosity c_s^2 tau.  A bulk rate different from
 *    the shear rate acts on the trace (isotropic) part only.
 *  Reconstruction: fbar* = w (rho + A.c/c_s^2 + B:Q/(2 c_s^4)), which projects
 *    the ghost modes out.
 *  Thermal noise (Sec. III, ref. adhikari2005: all non-conserved modes,
 *    ghosts included): each stress and ghost mode k receives
 *    sqrt(mu_n b_k (1 - gamma_k^2)) g_k with mu_n = rho kT / c_s^2, and a ghost
 *    mode keeps gamma_g of its pre-collision value (gamma_g = 0: projected).
 */
static void lb_collide_stream(const ora_params *p, const box_t *g, double *f, const double *F, double *u_out,
                              int64_t step)
{
    const int q = p->q, d = p->dim;
    int32_t c[3 * 19];
    double w[19], E[19 * 19], bk[19];
    ora_lattice(d, q, c, w);
    ora_moment_basis(d, q, E, bk);
    const double cs2 = 1.0 / 3.0;
    const double omega_s = 1.0 / (p->tau + 0.5);
    const double gamma_s = 1.0 - omega_s;
    const double gamma_b = isnan(p->gamma_bulk) ? gamma_s : p->gamma_bulk;
    const double omega_b = 1.0 - gamma_b;
    const double gamma_g = p->gamma_ghost;
    const int nstress = d * (d + 1) / 2;
    const int first_noisy = d + 1;
    const int nnoisy = noisy_mode_count(d, q);
    const size_t N = g->n;

    double *fnew = (double *)malloc(sizeof(double) * (size_t)q * N);

#pragma omp parallel for schedule(static)
    for (long long ss = 0; ss < (long long)N; ++ss) {
        size_t s = (size_t)ss;
        int x, y, z;
        coords(g, s, &x, &y, &z);
        double fs[19];
        for (int i = 0; i < q; ++i) fs[i] = f[(size_t)i * N + s];

        double Fv[3] = {p->gext[0], p->gext[1], p->gext[2]};
        if (F) for (int a = 0; a < 3; ++a) Fv[a] += F[(size_t)a * N + s];
        if (d == 2) Fv[2] = 0.0;

        double rho = 0.0, j[3] = {0, 0, 0};
        for (int i = 0; i < q; ++i) {
            rho += fs[i];
            for (int a = 0; a < d; ++a) j[a] += fs[i] * c[3 * i + a];
        }
        double v[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) v[a] = (j[a] + 0.5 * Fv[a]) / rho;

        /* stress of the auxiliary distribution, S = sum fbar Q, Q = c c - c_s^2 delta */
        double S[3][3] = {{0}};
        for (int i = 0; i < q; ++i)
            for (int a = 0; a < d; ++a)
                for (int bb = 0; bb < d; ++bb)
                    S[a][bb] += fs[i] * (c[3 * i + a] * c[3 * i + bb] - (a == bb ? cs2 : 0.0));

        /* Eq. (bab) with the trace relaxed at the bulk rate */
        double X[3][3], T[3][3], Bm[3][3];
        double trX = 0.0, trT = 0.0;
        for (int a = 0; a < d; ++a)
            for (int bb = 0; bb < d; ++bb) {
                X[a][bb] = -S[a][bb] + rho * v[a] * v[bb];
                T[a][bb] = v[a] * Fv[bb] + Fv[a] * v[bb];
            }
        for (int a = 0; a < d; ++a) { trX += X[a][a]; trT += T[a][a]; }
        for (int a = 0; a < d; ++a)
            for (int bb = 0; bb < d; ++bb) {
                double isoX = a == bb ? trX / d : 0.0, isoT = a == bb ? trT / d : 0.0;
                Bm[a][bb] = S[a][bb] + omega_s * (X[a][bb] - isoX) + omega_b * isoX +
                            (1.0 - 0.5 * omega_s) * (T[a][bb] - isoT) + (1.0 - 0.5 * omega_b) * isoT;
            }
        double Am[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) Am[a] = j[a] + Fv[a];

        double fpost[19];
        for (int i = 0; i < q; ++i) {
            double ac = 0.0, bq = 0.0;
            for (int a = 0; a < d; ++a) ac += Am[a] * c[3 * i + a];
            for (int a = 0; a < d; ++a)
                for (int bb = 0; bb < d; ++bb)
                    bq += Bm[a][bb] * (c[3 * i + a] * c[3 * i + bb] - (a == bb ? cs2 : 0.0));
            fpost[i] = w[i] * (rho + ac / cs2 + bq / (2.0 * cs2 * cs2));
        }

        /* ghost relaxation and thermal noise in the moment basis */
        double gs[16];
        int have_noise = p->kT > 0.0;
        if (have_noise) ora_gaussians(p->seed, step, rng_site(p, x, y, z), 0u, (nnoisy + 7) / 8, gs);
        const double mun = rho * p->kT / cs2;
        for (int t = 0; t < nnoisy; ++t) {
            int k = first_noisy + t;
            int is_ghost = t >= nstress;
            double gam = is_ghost ? gamma_g : (t == 0 ? gamma_b : gamma_s);
            double add = 0.0;
            if (is_ghost && gam != 0.0) {
                double mk = 0.0;
                for (int i = 0; i < q; ++i) mk += E[(size_t)k * q + i] * fs[i];
                add += gam * mk;
            }
            if (have_noise) add += sqrt(mun * bk[k] * (1.0 - gam * gam)) * gs[t];
            if (add != 0.0)
                for (int i = 0; i < q; ++i) fpost[i] += w[i] * E[(size_t)k * q + i] * add / bk[k];
        }

        /* streaming: fbar(x + c_i, t + 1) = fbar*(x, t) */
        for (int i = 0; i < q; ++i)
            fnew[(size_t)i * N + site_at(g, x + c[3 * i], y + c[3 * i + 1], z + c[3 * i + 2])] = fpost[i];
    }
    memcpy(f, fnew, sizeof(double) * (size_t)q * N);
    free(fnew);

    /* velocity of the new fluid state, with the force density applied in this step */
    if (u_out) {
#pragma omp parallel for schedule(static)
        for (long long ss = 0; ss < (long long)N; ++ss) {
            size_t s = (size_t)ss;
            double rho = 0.0, j[3] = {0, 0, 0};
            for (int i = 0; i < q; ++i) {
                rho += f[(size_t)i * N + s];
                for (int a = 0; a < d; ++a) j[a] += f[(size_t)i * N + s] * c[3 * i + a];
            }
            for (int a = 0; a < d; ++a) {
                double Fa = p->gext[a] + (F ? F[(size_t)a * N + s] : 0.0);
                u_out[(size_t)a * N + s] = (j[a] + 0.5 * Fa) / rho;
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Stochastic method of lines for psi (Sec. V)                                 */
/* ------------------------------------------------------------------------- */

/* Half-links of the finite-difference scheme: one of each +-c pair of the 3x3x3
 * neighbourhood, in the order x, y, z; (1,1,0), (1,-1,0), (1,0,1), (1,0,-1),
 * (0,1,1), (0,1,-1); (1,1,1), (1,1,-1), (1,-1,1), (1,-1,-1).  2D: (1,0), (0,1),
 * (1,1), (1,-1).  Their weights a_l are the class coefficients of the chosen
 * Laplacian (SO: 6/22, 3/22, 1/22; 2D 1/2, 1/4); a link of weight 0 carries no
 * noise. */
static const int FD_LINKS3[13][3] = {{1, 0, 0},  {0, 1, 0},  {0, 0, 1},  {1, 1, 0}, {1, -1, 0},
                                     {1, 0, 1},  {1, 0, -1}, {0, 1, 1},  {0, 1, -1}, {1, 1, 1},
                                     {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};
static const int FD_LINKS2[4][3] = {{1, 0, 0}, {0, 1, 0}, {1, 1, 0}, {1, -1, 0}};

static double fd_link_weight(const ora_params *p, const int *cl)
{
    double a[4];
    lap_class_weights(p->dim, p->laplacian, a);
    return a[abs(cl[0]) + abs(cl[1]) + abs(cl[2])];
}

/* Finite-difference noise eta(r) of Eq. (etafdt).  The paper builds eta in
 * Fourier space with <eta eta> = -2 kT M L_SO(q).  Reading: the same Gaussian
 * law is produced in real space by independent link noises
 * zeta_l ~ N(0, 2 kT M a_l / dt) on the half-links, eta(r) = sum_l
 * [zeta_l(r - c_l) - zeta_l(r)], whose spectrum is sum_l 2 var_l (1 - cos q.c_l)
 * = -2 kT M L(q) for the Laplacian L of class weights a_l (SO in the paper);
 * it is conservative by construction and needs no FFT. */
void ora_fd_noise(const ora_params *p, int64_t step, double *eta)
{
    box_t g = box_of(p);
    const int nl = p->dim == 3 ? 13 : 4;
    const int (*L)[3] = p->dim == 3 ? FD_LINKS3 : FD_LINKS2;
    double *zeta = (double *)malloc(sizeof(double) * (size_t)nl * g.n);
#pragma omp parallel for schedule(static)
    for (long long s = 0; s < (long long)g.n; ++s) {
        int x, y, z;
        coords(&g, (size_t)s, &x, &y, &z);
        double gs[16];
        ora_gaussians(p->seed, step, rng_site(p, x, y, z), 1u, (nl + 7) / 8, gs);
        for (int l = 0; l < nl; ++l)
            zeta[(size_t)l * g.n + (size_t)s] = sqrt(2.0 * p->kT * p->M * fd_link_weight(p, L[l])) * gs[l];
    }
    for (size_t s = 0; s < g.n; ++s) {
        int x, y, z;
        coords(&g, s, &x, &y, &z);
        double acc = 0.0;
        for (int l = 0; l < nl; ++l)
            acc += zeta[(size_t)l * g.n + site_at(&g, x - L[l][0], y - L[l][1], z - L[l][2])] - zeta[(size_t)l * g.n + s];
        eta[s] = acc;
    }
    free(zeta);
}

/* Finite-volume node noise xi_alpha(r) ~ N(0, 2 kT M / dt), Eq. (fdt_orderpara). */
static void fv_node_noise(const ora_params *p, const box_t *g, int64_t step, double *xi)
{
#pragma omp parallel for schedule(static)
    for (long long s = 0; s < (long long)g->n; ++s) {
        int x, y, z;
        coords(g, (size_t)s, &x, &y, &z);
        double gs[8];
        ora_gaussians(p->seed, step, rng_site(p, x, y, z), 1u, 1, gs);
        for (int a = 0; a < 3; ++a)
            xi[(size_t)a * g->n + (size_t)s] = a < g->dim ? sqrt(2.0 * p->kT * p->M) * gs[a] : 0.0;
    }
}

/* Right-hand side of the semi-discrete order-parameter equation (advdiff).
 * noise: eta (FD) or xi (FV, contrast) held fixed over the step; u: frozen velocity.
 *  FD: R = M lap(mu) - div_CD(u psi) + eta, with the conservative
 *      central-difference advection of Sec. V.A.
 *  FV: R = div_FV(J), J = M grad_FV(mu) - u psi + xi (Eqs. fvdiff-fvgrad).
 *  Contrast (Sec. III, the Petschek-Metiu discretisation): R = M lap(mu)
 *      - div_CD(u psi) + div_CD(xi), the node noise xi ~ N(0, 2 kT M) taken
 *      through the central-difference divergence [div xi](r) = (1/2) sum_a
 *      [xi_a(r + e_a) - xi_a(r - e_a)].  Reading: the paper names the method
 *      but not its stencils; we take the plain nearest-neighbour ones, the
 *      central difference for the divergence and the Laplacian chosen by
 *      p->laplacian (CD, Eq. fdlap, for the method as published).  Its noise
 *      spectrum 2 kT M sum_a sin^2 q_a differs from -2 kT M L(q), so the
 *      equilibrium ratio is sum_a sin^2 q_a / (-L(q)) instead of 1. */
static void psi_rhs(const ora_params *p, const box_t *g, const double *psi, const double *u, const double *noise,
                    double *R)
{
    const size_t N = g->n;
    const int advect = (p->coupling & 2) != 0;
    double *mu = (double *)malloc(sizeof(double) * N);
    ora_mu(p, psi, mu);
    if (p->scheme == 0 || p->scheme == 2) {
        double *lapmu = (double *)malloc(sizeof(double) * N);
        ora_laplacian(p->dim, p->laplacian, p->nx, p->ny, p->nz, mu, lapmu);
        for (size_t s = 0; s < N; ++s) {
            int x, y, z;
            coords(g, s, &x, &y, &z);
            double adv = 0.0, nz = 0.0;
            for (int a = 0; a < g->dim; ++a) {
                int e[3] = {0, 0, 0};
                e[a] = 1;
                size_t sp = site_at(g, x + e[0], y + e[1], z + e[2]);
                size_t sm = site_at(g, x - e[0], y - e[1], z - e[2]);
                if (advect) adv += 0.5 * (u[(size_t)a * N + sp] * psi[sp] - u[(size_t)a * N + sm] * psi[sm]);
                if (p->scheme == 2 && noise) nz += 0.5 * (noise[(size_t)a * N + sp] - noise[(size_t)a * N + sm]);
            }
            if (p->scheme == 0 && noise) nz = noise[s];
            R[s] = p->M * lapmu[s] - adv + nz;
        }
        free(lapmu);
    } else {
        int32_t c[3 * 19];
        double w[19];
        ora_lattice(p->dim, p->q, c, w);
        double *J = (double *)calloc(3 * N, sizeof(double));
        fv_gradient(g, p->q, c, w, mu, J);
        for (size_t s = 0; s < N; ++s)
            for (int a = 0; a < g->dim; ++a) {
                double val = p->M * J[(size_t)a * N + s];
                if (advect) val -= u[(size_t)a * N + s] * psi[s];
                if (noise) val += noise[(size_t)a * N + s];
                J[(size_t)a * N + s] = val;
            }
        fv_divergence(g, p->q, c, w, J, R);
        free(J);
    }
    free(mu);
}

/* One step of psi with u frozen.  Time integration (Sec. V, ref. wilkie2004:
 * Runge-Kutta with the noise held constant over the step).  Reading: the order
 * is not given; Euler (integrator 1), Heun/RK2 (integrator 2) and the classical
 * RK4 (integrator 4) are offered. */
static void psi_step(const ora_params *p, const box_t *g, double *psi, const double *u, int64_t step)
{
    const size_t N = g->n;
    double *noise = NULL;
    if (p->kT > 0.0) {
        if (p->scheme == 0) {
            noise = (double *)malloc(sizeof(double) * N);
            ora_fd_noise(p, step, noise);
        } else {
            noise = (double *)malloc(sizeof(double) * 3 * N);
            fv_node_noise(p, g, step, noise);
        }
    }
    double *R0 = (double *)malloc(sizeof(double) * N);
    psi_rhs(p, g, psi, u, noise, R0);
    if (p->integrator == 1) {
        for (size_t s = 0; s < N; ++s) psi[s] += R0[s];
    } else if (p->integrator == 4) {
        /* classical fourth-order Runge-Kutta with the noise held fixed over the
         * step (Wilkie): k1 = R(psi), k2 = R(psi + k1/2), k3 = R(psi + k2/2),
         * k4 = R(psi + k3), psi += (k1 + 2 k2 + 2 k3 + k4)/6 */
        double *ps = (double *)malloc(sizeof(double) * N);
        double *K = (double *)malloc(sizeof(double) * N);
        double *sum = (double *)malloc(sizeof(double) * N);
        for (size_t s = 0; s < N; ++s) {
            sum[s] = R0[s];
            ps[s] = psi[s] + 0.5 * R0[s];
        }
        psi_rhs(p, g, ps, u, noise, K);
        for (size_t s = 0; s < N; ++s) {
            sum[s] += 2.0 * K[s];
            ps[s] = psi[s] + 0.5 * K[s];
        }
        psi_rhs(p, g, ps, u, noise, K);
        for (size_t s = 0; s < N; ++s) {
            sum[s] += 2.0 * K[s];
            ps[s] = psi[s] + K[s];
        }
        psi_rhs(p, g, ps, u, noise, K);
        for (size_t s = 0; s < N; ++s) psi[s] += (sum[s] + K[s]) / 6.0;
        free(ps);
        free(K);
        free(sum);
    } else {
        double *pst = (double *)malloc(sizeof(double) * N);
        double *R1 = (double *)malloc(sizeof(double) * N);
        for (size_t s = 0; s < N; ++s) pst[s] = psi[s] + R0[s];
        psi_rhs(p, g, pst, u, noise, R1);
        for (size_t s = 0; s < N; ++s) psi[s] += 0.5 * (R0[s] + R1[s]);
        free(pst);
        free(R1);
    }
    free(R0);
    free(noise);
}

/* ------------------------------------------------------------------------- */
/* Coupled step (Sec. VI: FLBE and SMOL marched alternately every step).       */
/* Reading of the order (Gauss-Seidel): the LB step takes the force of psi^n   */
/* and advances the fluid to n+1; the psi step then advances psi^n with the    */
/* velocity of that new fluid state, (sum fbar^{n+1} c + F^n/2)/rho^{n+1}.     */
/* Advecting with the velocity of the fluid BEFORE it received F^n (both       */
/* halves reading time n) leaves the lattice's undamped staggered momentum     */
/* mode (k = pi, flipped by every streaming step) coupled to psi at an         */
/* interface through the force and the advection, and that loop grows.         */
/* ------------------------------------------------------------------------- */
int ora_step(const ora_params *p, double *f, double *psi, double *u, int64_t step0, int64_t nsteps)
{
    if (!((p->dim == 3 && (p->q == 19 || p->q == 15)) || (p->dim == 2 && p->q == 9))) return -1;
    if (p->nx <= 0 || p->ny <= 0 || (p->dim == 3 && p->nz <= 0)) return -1;
    if (!(p->tau > 0.0) || !(p->integrator == 1 || p->integrator == 2 || p->integrator == 4) || p->scheme < 0 ||
        p->scheme > 2)
        return -1;
    double lw[4];
    if (lap_class_weights(p->dim, p->laplacian, lw)) return -1;
    box_t g = box_of(p);
    const size_t N = g.n;
    double *mu = (double *)malloc(sizeof(double) * N);
    double *F = (double *)calloc(3 * N, sizeof(double));
    for (int64_t n = 0; n < nsteps; ++n) {
        int64_t step = step0 + n;
        if (p->lb_on) {
            int force = (p->coupling & 1) != 0;
            if (force) {
                ora_mu(p, psi, mu);
                ora_force(p, psi, mu, F);
            }
            lb_collide_stream(p, &g, f, force ? F : NULL, u, step);
        }
        psi_step(p, &g, psi, u, step);
    }
    free(mu);
    free(F);
    return 0;
}

/* Hydrodynamic moments of fbar at every site: rho, j = sum fbar c (no force
 * shift), and all q moments m_k = sum_i e_ki fbar_i of the basis above. */
int ora_moments(const ora_params *p, const double *f, double *rho, double *j, double *m)
{
    int32_t c[3 * 19];
    double w[19], E[19 * 19], bk[19];
    if (ora_lattice(p->dim, p->q, c, w) || ora_moment_basis(p->dim, p->q, E, bk)) return -1;
    box_t g = box_of(p);
    for (size_t s = 0; s < g.n; ++s) {
        double r = 0.0, jj[3] = {0, 0, 0};
        for (int i = 0; i < p->q; ++i) {
            double fi = f[(size_t)i * g.n + s];
            r += fi;
            for (int a = 0; a < 3; ++a) jj[a] += fi * c[3 * i + a];
        }
        if (rho) rho[s] = r;
        if (j) for (int a = 0; a < 3; ++a) j[(size_t)a * g.n + s] = jj[a];
        if (m)
            for (int k = 0; k < p->q; ++k) {
                double mk = 0.0;
                for (int i = 0; i < p->q; ++i) mk += E[(size_t)k * p->q + i] * f[(size_t)i * g.n + s];
                m[(size_t)k * g.n + s] = mk;
            }
    }
    return 0;
}

/* Exposed right-hand side of the psi equation for the operator tests. */
int ora_psi_rhs(const ora_params *p, const double *psi, const double *u, int64_t step, int32_t with_noise, double *R)
{
    box_t g = box_of(p);
    double *noise = NULL;
    if (with_noise && p->kT > 0.0) {
        if (p->scheme == 0) {
            noise = (double *)malloc(sizeof(double) * g.n);
            ora_fd_noise(p, step, noise);
        } else {
            noise = (double *)malloc(sizeof(double) * 3 * g.n);
            fv_node_noise(p, &g, step, noise);
        }
    }
    psi_rhs(p, &g, psi, u, noise, R);
    free(noise);
    return 0;
}

/* Equilibrium populations for given rho, u fields: w (rho + rho u.c/c_s^2 + rho u u:Q/(2 c_s^4)). */
int ora_equilibrium(const ora_params *p, const double *rho, const double *u, double *f)
{
    int32_t c[3 * 19];
    double w[19];
    if (ora_lattice(p->dim, p->q, c, w)) return -1;
    box_t g = box_of(p);
    const double cs2 = 1.0 / 3.0;
    for (size_t s = 0; s < g.n; ++s) {
        double v[3] = {0, 0, 0};
        for (int a = 0; a < p->dim; ++a) v[a] = u ? u[(size_t)a * g.n + s] : 0.0;
        double r = rho ? rho[s] : p->rho0;
        for (int i = 0; i < p->q; ++i) {
            double cu = 0.0, uuq = 0.0;
            for (int a = 0; a < p->dim; ++a) cu += c[3 * i + a] * v[a];
            for (int a = 0; a < p->dim; ++a)
                for (int b = 0; b < p->dim; ++b)
                    uuq += v[a] * v[b] * (c[3 * i + a] * c[3 * i + b] - (a == b ? cs2 : 0.0));
            f[(size_t)i * g.n + s] = w[i] * r * (1.0 + cu / cs2 + uuq / (2.0 * cs2 * cs2));
        }
    }
    return 0;
}

/*
 * flb_oracle.h -- interface of the plain FP64 CPU oracle (flb_oracle.c).
 *
 * TEST INFRASTRUCTURE: used only by the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg.  The CUDA library neither includes this header
 * nor links this code.
 *
 * All arrays are caller-owned, double precision, site-major planes:
 * value k of site s at a[k*N + s], s = x + nx*(y + ny*z), N = nx*ny*nz (nz = 1 in 2D).
 */
#ifndef FLB_ORACLE_H
#define FLB_ORACLE_H
#include <stdint.h>

typedef struct {
    int32_t dim, q;         /* 2/9 (D2Q9) or 3/19 (D3Q19) */
    int32_t nx, ny, nz;
    double rho0, tau;       /* omega = 1/(tau + 1/2), viscosity c_s^2 tau */
    double gamma_bulk;      /* NaN: same as shear (1 - omega) */
    double gamma_ghost;     /* 0: ghosts projected out before thermalisation */
    double kT, A, B, K, M;
    int32_t scheme;         /* 0 finite difference, 1 finite volume, 2 the naive contrast
                               scheme (node noise under a central-difference divergence) */
    int32_t integrator;     /* 1 Euler, 2 Heun */
    int32_t coupling;       /* bit 0: force -psi grad mu on the fluid; bit 1: advection of psi */
    int32_t lb_on;          /* 0: skip the lattice Boltzmann half (u stays as given) */
    uint64_t seed;
    double gext[3];         /* extra uniform body-force density (operator tests only) */
    int32_t gnx, gny, gnz;  /* global lattice for counter ids (0: this box) */
    int32_t ox, oy, oz;     /* origin of this box inside the global lattice */
    int32_t force_grad;     /* gradient of mu in the force: 1 central difference, 2 FV lattice
                               gradient, 0 the one matched to the psi scheme; 3 the
                               divergence of the order-parameter stress instead */
    int32_t laplacian;      /* App. A stencil of mu and of the FD/contrast psi equation:
                               0 SO, 1 CD, 2 PK, 3 LB (2D: SO or CD) */
} ora_params;

int ora_threads(void);
void ora_set_threads(int32_t n);
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void ora_gaussians(uint64_t seed, int64_t step, uint32_t site, uint32_t stream, int32_t nblocks, double *g);
void ora_gaussians_sites(uint64_t seed, int64_t step, uint32_t site0, int64_t nsites, uint32_t stream,
                         int32_t nblocks, double *g);
int ora_lattice(int32_t dim, int32_t q, int32_t *c, double *w);
int ora_moment_basis(int32_t dim, int32_t q, double *E, double *b);
void ora_laplacian_so(int32_t dim, int32_t nx, int32_t ny, int32_t nz, const double *in, double *out);
int ora_laplacian(int32_t dim, int32_t kind, int32_t nx, int32_t ny, int32_t nz, const double *in, double *out);
int ora_fv_laplacian(int32_t dim, int32_t q, int32_t nx, int32_t ny, int32_t nz, const double *in, double *out);
void ora_mu(const ora_params *p, const double *psi, double *mu);
void ora_force(const ora_params *p, const double *psi, const double *mu, double *F);
void ora_fd_noise(const ora_params *p, int64_t step, double *eta);
int ora_psi_rhs(const ora_params *p, const double *psi, const double *u, int64_t step, int32_t with_noise, double *R);
int ora_step(const ora_params *p, double *f, double *psi, double *u, int64_t step0, int64_t nsteps);
int ora_moments(const ora_params *p, const double *f, double *rho, double *j, double *m);
int ora_equilibrium(const ora_params *p, const double *rho, const double *u, double *f);

#endif

/*
 * flb.h -- C ABI of the GB300 library for the hybrid model-H solver of
 * Sumesh, Pagonabarraga & Adhikari, "Lattice Boltzmann - Langevin simulations
 * of binary mixtures" (arXiv:1104.0078), on D2Q9, D3Q19 and the paper's own
 * D3Q15 lattice.
 *
 * One time step advances, in this order (Sec. VI, "alternate marching"; the
 * psi step uses the velocity of the fluid state the LB step produced):
 *   1. the fluctuating lattice Boltzmann equation for the momentum (Sec. IV,
 *      App. B): pull-streaming of the auxiliary populations fbar, moments
 *      rho = sum fbar, rho v = sum fbar c + F/2, moment-space relaxation with
 *      the order-parameter force F = -psi grad mu and Landau-Lifshitz noise on
 *      every stress and ghost mode (Eq. bab, adhikari2005);
 *   2. the stochastic method-of-lines step of the order parameter psi
 *      (Sec. V): d psi/dt = -div(u psi) + M lap mu + div xi, with
 *      mu = A psi + B psi^3 - K lap psi (Sec. II.A, lap one of the App. A
 *      stencils, SO by default), in the finite-difference (Sec. V.A) or
 *      finite-volume (Sec. V.B) form, or the naive discretisation Sec. III
 *      contrasts with; noise held fixed over a Runge-Kutta step (Sec. V,
 *      wilkie2004).
 *
 * Units: lattice units, dx = dt = 1, c_s^2 = 1/3, periodic boundaries.
 * Threading: a handle is not thread-safe; calls on one handle must be
 * serialised by the caller.  All device work is issued on the stream given to
 * flb_init; functions documented as synchronising wait for that stream.
 * Memory: the library never allocates device memory.  The caller allocates one
 * device workspace of flb_workspace_bytes() bytes (e.g. a torch uint8 tensor)
 * and keeps it alive until flb_destroy().  Host buffers passed to any call are
 * caller-owned and are not retained after the call returns.
 * Errors: every int-returning call returns FLB_OK (0) or a negative FLB_E*
 * code; flb_strerror() names it.  Faults detected on the device (non-finite
 * values, a timed-out wait) are latched in a device status word and reported
 * by the next synchronising call.
 */
#ifndef FLB_H
#define FLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define FLB_OK 0
#define FLB_EINVAL (-1)        /* invalid argument or parameter combination */
#define FLB_ENOSPC (-2)        /* workspace or host buffer too small */
#define FLB_ECUDA (-3)         /* a CUDA runtime call failed */
#define FLB_ENONFINITE (-4)    /* a reduction met NaN or Inf in the fields */
#define FLB_ETIMEOUT (-5)      /* a bounded device-side wait gave up */
#define FLB_EUNSUPPORTED (-6)  /* valid request this build does not provide */

/* ---- enumerations ---- */
#define FLB_FD 0               /* finite-difference psi scheme, Sec. V.A */
#define FLB_FV 1               /* finite-volume psi scheme, Sec. V.B */
#define FLB_NAIVE 2            /* the naive contrast scheme of Sec. III (see psi_scheme) */
#define FLB_EULER 1            /* one-stage integrator */
#define FLB_HEUN 2             /* two-stage (RK2) integrator, noise held fixed */
#define FLB_RK4 4              /* classical fourth-order Runge-Kutta, noise held fixed */
#define FLB_F32_DEV 0          /* populations stored as FP32 deviations fbar_i - w_i rho0 */
#define FLB_F16_DEV 1          /* populations stored as FP16 deviations */
#define FLB_COUPLE_FORCE 1     /* psi exerts -psi grad mu on the fluid */
#define FLB_COUPLE_ADVECT 2    /* the fluid advects psi */
#define FLB_SQ_PSI 0           /* structure factor of psi */
#define FLB_SQ_HEIGHT 1        /* capillary spectrum of the two psi = 0 surfaces */
#define FLB_SQ_DYNAMIC 2       /* dynamic structure factor S(q, tau) of psi */
#define FLB_FORCE_MATCHED 0     /* force gradient matched to the psi scheme */
#define FLB_FORCE_CD 1          /* central difference of Sec. IV */
#define FLB_FORCE_FV 2          /* FV lattice gradient of Eq. (fvgrad) */
#define FLB_FORCE_STRESS 3      /* F = -div sigma, the order-parameter stress of Eq. (muf) */
#define FLB_LAP_SO 0           /* Shinozaki-Oono Laplacian, Eq. (solap) (the paper's runs) */
#define FLB_LAP_CD 1           /* central-difference Laplacian, Eq. (fdlap) */
#define FLB_LAP_PK 2           /* Patra-Karttunen Laplacian, Eq. (pklap) (3D only) */
#define FLB_LAP_LB 3           /* lattice-Boltzmann Laplacian, Eq. (lblap) (3D only) */
#define FLB_MODE_PLAIN 0       /* per-replica launch sequence */
#define FLB_MODE_BATCHED 1     /* all replicas in one launch per phase, CUDA-graph replay */
#define FLB_MODE_PERSISTENT 2  /* all replicas, n steps, one cooperative launch (FV, FP32 storage) */
#define FLB_INIT_REST 0        /* flb_init leaves every replica at rest */
#define FLB_INIT_EQUILIBRIUM 1 /* ... in the equilibrium of the Gaussian model (Sec. VI) */
#define FLB_INIT_USER 2        /* ... at rest, for the caller to set (flb_set_fields, flb_set_state) */
#define FLB_TUNE_FORCE 1       /* flb_autotune: time every candidate even if the cache has an entry */

/*
 * Parameters of one lattice (one replica).  Names follow the paper.
 *   dim, q      : 2 and 9 (D2Q9), 3 and 19 (D3Q19) or 3 and 15 (D3Q15, the
 *                 lattice of the paper's own runs, Sec. VI).
 *   nx, ny, nz  : lattice size, each in [4, 4096] (nz is ignored and taken as 1
 *                 in 2D); nx*ny*nz < 2^31.
 *   rho0        : reference density, > 0 (the populations are stored as
 *                 deviations from w_i rho0).
 *   tau         : the paper's relaxation time (App. B): omega = 1/(tau + 1/2),
 *                 shear viscosity c_s^2 tau; > 0.
 *   gamma_bulk  : relaxation factor of the trace of the stress, in (-1, 1);
 *                 NaN selects the shear factor 1 - omega (the paper's choice).
 *   gamma_ghost : relaxation factor of the ghost modes, in (-1, 1); 0 projects
 *                 them out before they are thermalised (Eq. bab, Sec. III).
 *   kT          : temperature, >= 0 (0 switches all noise off).
 *   A, B, K, M  : free energy f = A/2 psi^2 + B/4 psi^4 + K/2 |grad psi|^2
 *                 (Eqs. Feng, feng) and mobility M >= 0.
 *   psi_scheme  : FLB_FD, FLB_FV or FLB_NAIVE.  FLB_NAIVE is the Petschek-Metiu
 *                 discretisation Sec. III contrasts with: node noise
 *                 xi ~ N(0, 2 kT M) through the central-difference divergence,
 *                 dpsi/dt = M lap mu - div_CD(u psi) + div_CD xi.  Its noise
 *                 spectrum 2 kT M sum_a sin^2 q_a is not -2 kT M L(q), so it
 *                 breaks the fluctuation-dissipation theorem at high q (the
 *                 equilibrium ratio falls to sum_a sin^2 q_a / (-L(q))); it is
 *                 there to show that failure.
 *   integrator  : FLB_EULER, FLB_HEUN or FLB_RK4 (the noise is drawn once per
 *                 step and held fixed in every stage, Sec. V).  FLB_RK4 runs in
 *                 FLB_MODE_PLAIN only.
 *   storage     : FLB_F32_DEV or FLB_F16_DEV.
 *   coupling    : bit mask of FLB_COUPLE_FORCE | FLB_COUPLE_ADVECT (3 = model H;
 *                 0 = "diffusion alone" of Sec. VI.A).
 *   seed        : Philox key of this replica.
 *   sq_kmax     : structure-factor window: wavevector indices |k_a| <= sq_kmax
 *                 on every axis; <= 0 or >= n_a/2 keeps the whole axis.
 *   sq_lags     : lags kept for the dynamic structure factor S(q, tau) (0 = none,
 *                 at most 4096); lag l is l sampling intervals (flb_set_sampling).
 *   force_grad  : lattice gradient in the force F = -psi grad mu:
 *                 FLB_FORCE_MATCHED (default) takes the central difference
 *                 with FLB_FD and the FV gradient (1/c_s^2) sum_i w_i c_i
 *                 mu(r + c_i) of Eq. (fvgrad) with FLB_FV -- the gradient whose
 *                 negative adjoint is the divergence advecting psi, so that the
 *                 work u.F equals the free energy advection removes (Sec. II.B).
 *                 FLB_FORCE_CD or FLB_FORCE_FV force one choice.
 *                 FLB_FORCE_STRESS takes instead F = -div sigma with
 *                 sigma_ab = K d_a psi d_b psi + delta_ab [A/2 psi^2 + 3B/4 psi^4
 *                 - K psi lap_SO psi - K/2 |grad psi|^2] (Sec. IV, Eq. muf),
 *                 central differences for the gradient and the divergence: the
 *                 total momentum is then conserved exactly for B != 0 as well,
 *                 F = -psi grad mu + O(h^2), but the force is not the adjoint
 *                 of the psi advection (with FLB_FV, rough fields of amplitude
 *                 ~0.5 can go non-finite).  Needs laplacian FLB_LAP_SO.
 *   laplacian   : the App. A stencil of mu = A psi + B psi^3 - K lap psi and of
 *                 the diffusion M lap mu of FLB_FD and FLB_NAIVE (whose link
 *                 noise follows it, so FLB_FD keeps the fluctuation-dissipation
 *                 theorem with any of them): FLB_LAP_SO (default), FLB_LAP_CD,
 *                 FLB_LAP_PK or FLB_LAP_LB; 2D takes SO or CD.
 * D3Q19 and D3Q15 with FLB_LAP_SO and FLB_FD or FLB_FV run the tiled 3D
 * kernels; every other 3D combination (another Laplacian, FLB_NAIVE) runs
 * one-thread-per-site stencil kernels that keep mu, the noise increment and
 * the FV flux in HBM, in FLB_MODE_PLAIN only.
 */
typedef struct flb_params {
    int32_t dim, q;
    int32_t nx, ny, nz;
    double rho0, tau;
    double gamma_bulk, gamma_ghost;
    double kT, A, B, K, M;
    int32_t psi_scheme, integrator, storage, coupling;
    uint64_t seed;
    int32_t sq_kmax;
    int32_t force_grad;
    int32_t sq_lags;
    int32_t laplacian;
    int32_t init;
} flb_params;

typedef struct flb_handle flb_handle;

/* Fill *p with the defaults: D3Q19 32^3, rho0 1, tau 0.8, gamma_bulk NaN,
 * gamma_ghost 0, kT 0, A 0.05, B 0, K 0.04, M 0.1, FV, Heun, FP32, coupling 3,
 * seed 1, sq_kmax 0, force_grad FLB_FORCE_MATCHED, sq_lags 0, laplacian
 * FLB_LAP_SO, init FLB_INIT_REST. */
void flb_params_default(flb_params *p);

/* Device workspace needed for nrep replicas p[0..nrep-1]; 0 if any parameter
 * set is invalid.  Replicas may differ in size, seed and physical constants but
 * must share dim, q, psi_scheme, integrator and storage. */
size_t flb_workspace_bytes(const flb_params *p, int32_t nrep);

/* Create a handle.  dev_ws: device pointer, 256-byte aligned, ws_bytes >=
 * flb_workspace_bytes(p, nrep), caller-owned.  cuda_stream: a cudaStream_t
 * (NULL = legacy default stream).  Every replica starts at step 0 in the state
 * its flb_params.init names:
 *   FLB_INIT_REST, FLB_INIT_USER: at rest (fbar = w rho0, u = 0, psi = 0); USER
 *     marks that the caller sets the fields next (flb_set_fields, flb_set_state).
 *   FLB_INIT_EQUILIBRIUM: the equilibrium of the Gaussian model, as the paper's
 *     runs start (Sec. VI).  Population deviations independent N(0, rho0 kT w_i /
 *     c_s^2), the stationary law of the linearised fluctuating LB (Sec. III;
 *     Philox stream 3, step 0, counter = site); psi Gaussian with S(q) =
 *     kT/(A - K L(q)) on every q != 0 (Eq. test2; L the symbol of the chosen
 *     Laplacian; B is not part of it) and zero mean, drawn mode by mode (Philox
 *     stream 4, counter = the mode's FFT-order index) and summed on the device by
 *     an inverse DFT; u the velocity of those populations.  Needs A > 0, K >= 0.
 * Synchronising.  Errors: EINVAL, ENOSPC, ECUDA. */
int flb_init(const flb_params *p, int32_t nrep, void *dev_ws, size_t ws_bytes, void *cuda_stream,
             flb_handle **out);

/* Equilibrium initialisation of replica rep from host fields (FP64, site-major
 * s = x + nx*(y + ny*z)): rho[N] (NULL: rho0), u[dim][N] (NULL: 0), psi[N]
 * (NULL: 0).  fbar = w (rho + rho u.c/c_s^2 + rho uu:Q/(2 c_s^4)).  Also sets
 * the stored velocity to u.  The step counter is kept.  Synchronising.
 * Errors: EINVAL (no such replica), ECUDA. */
int flb_set_fields(flb_handle *h, int32_t rep, const double *rho, const double *u, const double *psi);

/* Physical populations fbar_i(x, t) after streaming, FP64 [q][N], the state the
 * paper's App. B evolves; set replaces the populations (psi and u are kept).
 * Synchronising.  Errors: EINVAL (no such replica, NULL f), ECUDA. */
int flb_get_populations(flb_handle *h, int32_t rep, double *f);
int flb_set_populations(flb_handle *h, int32_t rep, const double *f);

/* Order parameter psi(t) [N] and the velocity u [dim][N] that the last psi
 * step used (time t-1; the initial field before the first step).  Either pointer
 * may be NULL.  Synchronising.  Errors: EINVAL (no such replica), ECUDA. */
int flb_get_psi_u(flb_handle *h, int32_t rep, double *psi, double *u);

/* A periodic window of replica rep: origin (x0,y0,z0), size wx*wy*wz, populations
 * f[q][W] and psi[W] in window site order (either may be NULL).  Synchronising.
 * Errors: EINVAL (no such replica, sizes < 1), ENOSPC (W above 32768), ECUDA. */
int flb_get_window(flb_handle *h, int32_t rep, int32_t x0, int32_t y0, int32_t z0, int32_t wx, int32_t wy,
                   int32_t wz, double *f, double *psi);

/* Advance every replica by n >= 0 steps.  Asynchronous on the stream.
 * Errors: EINVAL (n < 0), EUNSUPPORTED (replicas outside the chosen mode),
 * ECUDA; device-side faults are reported by the next synchronising call. */
int flb_step(flb_handle *h, int64_t n);

/* Current step counter of replica rep.  Errors: EINVAL. */
int flb_get_step(flb_handle *h, int32_t rep, int64_t *step);

/* Conserved totals and velocity variance of replica rep, reduced on the device
 * in FP64: totals = {sum rho, sum j_x, sum j_y, [sum j_z,] sum psi} (2 + dim
 * values; j = sum fbar c), u2 = {<u_x^2>, <u_y^2>, [<u_z^2>]} of the stored
 * velocity.  Either pointer may be NULL.  Synchronising; returns ENONFINITE if
 * any population, psi or u value was NaN or Inf. */
int flb_moments(flb_handle *h, int32_t rep, double *totals, double *u2);

/* Per-mode mean squares of replica rep: msq[k] = (1/N) sum_r m_k(r)^2, k = 0..q-1,
 * with m_k(r) = sum_i E_ki (fbar_i(r) - w_i rho0) the projections of the
 * physical populations on the moment basis E (Gram-Schmidt under sum_i w_i a_i
 * b_i on the ordered monomials 1; c; c^2; 3c_x^2 - c^2; c_y^2 - c_z^2; c_x c_y;
 * c_y c_z; c_z c_x; c^2 c; c_x(c_y^2 - c_z^2), c_y(c_z^2 - c_x^2), c_z(c_x^2 - c_y^2);
 * c^4; c^2(3c_x^2 - c^2); c^2(c_y^2 - c_z^2) for D3Q19; D3Q15 ends c_x c_y c_z, c^4
 * after the c^2 c rows; D2Q9: 1; c; c^2; c_x^2 - c_y^2; c_x c_y; c^2 c; c^4).  In
 * equilibrium every non-conserved mode has <m_k^2> = (rho kT / c_s^2) b_k, b_k =
 * sum_i w_i E_ki^2 (Sec. III).  msq: host FP64 [q].  Reduced in FP64 on the device;
 * synchronising; returns ENONFINITE if any population was NaN or Inf. */
int flb_mode_variances(flb_handle *h, int32_t rep, double *msq);

/* Sampling of the structure factors during flb_step: every every_m steps
 * (0 = never) the psi spectrum (mask bit 1), the interface-height spectrum
 * (mask bit 2) and/or the dynamic structure factor (mask bit 4: the psi
 * spectrum's Fourier components are kept for the last sq_lags samples and
 * correlated with every new one) of every replica are accumulated in FP64. */
int flb_set_sampling(flb_handle *h, int32_t every_m, int32_t mask);

/* Take one sample now (same mask bits).  Asynchronous. */
int flb_sample(flb_handle *h, int32_t mask);

/* Accumulated mean spectrum of replica rep.  which = FLB_SQ_PSI: out has
 * Kz*Ky*Kx values <|psi~(q)|^2> with psi~(q) = N^-1/2 sum psi e^{-iq.r}
 * (Eqs. test1, test2); each axis lists indices k = 0..kmax then n-kmax..n-1
 * (all n indices when the whole axis is kept), x fastest.  which =
 * FLB_SQ_HEIGHT: out has ny*nx values <|h~(q)|^2> (Eq. flucinterf) averaged over
 * the two interfaces of a slab normal to z.  which = FLB_SQ_DYNAMIC: out has
 * sq_lags blocks of Kz*Ky*Kx values (lag slowest), block l holding
 * S(q, l m) = < Re psi~(q, t) psi~(q, t - l m)^* > over the samples t that
 * have a sample l intervals before them (the paper's S(q, tau), Sec. VI.A,
 * Eq. strf; the same window and normalisation as FLB_SQ_PSI).  *nsamples
 * receives the sample count (of lag 0 for FLB_SQ_DYNAMIC).  Synchronising. */
int flb_structure_factor(flb_handle *h, int32_t rep, int32_t which, double *out, int64_t *nsamples);

/* Number of values flb_structure_factor writes for `which`. */
int64_t flb_structure_factor_size(flb_handle *h, int32_t rep, int32_t which);

/* Zero the accumulated spectra of replica rep (-1: all). */
int flb_sq_reset(flb_handle *h, int32_t rep);

/*
 * Launch mode for flb_step:
 *   FLB_MODE_PLAIN       every replica's kernels launched one replica after another;
 *   FLB_MODE_BATCHED     all replicas in one launch per phase (mu, collide-stream,
 *                        velocity, psi stages), replayed as a CUDA graph (D3Q19
 *                        or D3Q15, FV, FLB_LAP_SO, Euler or Heun);
 *   FLB_MODE_PERSISTENT  all replicas advanced the n steps of one flb_step call
 *                        by one cooperative launch per stretch between sampling
 *                        steps (as FLB_MODE_BATCHED, with FP32 storage).  Its blocks take tile tasks
 *                        from a list in order and wait, per replica, for the
 *                        previous phase of that replica only (a per-replica phase
 *                        barrier), each wait bounded by flb_set_wait_limit.
 * All three give bitwise identical results.  flb_step returns EUNSUPPORTED when
 * the replicas do not fit the chosen mode.
 */
int flb_set_mode(flb_handle *h, int32_t mode);

/* Limit of one inter-block wait of FLB_MODE_PERSISTENT, in seconds (default 1,
 * at most 60).  A wait that runs out latches FLB_ETIMEOUT in the handle's status
 * word and ends the launch (every block stops taking tasks), leaving the step in
 * progress incomplete; the next synchronising call returns FLB_ETIMEOUT.  The
 * state must then be set again (flb_set_fields / flb_set_state) before stepping. */
int flb_set_wait_limit(flb_handle *h, double seconds);

/*
 * Tiling of the 3D psi stage.  A psi block owns a 32 x 16 column of sites and
 * marches psi_zchunk planes of it in z (default 64).  Smaller chunks give more
 * blocks (small boxes fill the GPU) at the cost of recomputing the stencil halo
 * of 6 planes per chunk.  The choice changes no result bit: every site's
 * arithmetic is the same.  (A performance knob of this implementation; the
 * paper has no counterpart.)
 *
 * flb_get_tuning / flb_set_tuning read / set psi_zchunk of replica rep (-1 sets
 * every replica), 1 <= psi_zchunk <= 4096; EINVAL otherwise.  Setting it drops
 * the batched mode's captured graph, which the next batched flb_step rebuilds.
 *
 * flb_autotune times the candidates 4, 8, ... (up to the first value that
 * covers the box depth) on the handle's own buffers and keeps the fastest: in
 * FLB_MODE_PLAIN per distinct replica configuration (box, lattice, scheme,
 * integrator, noise, advection) on that replica's psi stages; in
 * FLB_MODE_BATCHED and FLB_MODE_PERSISTENT one value for all replicas on the
 * batched psi launches, then, deepest boxes first, one value per distinct box
 * depth nz over the even splits ceil(nz / k), k = 1..16, the other depths held
 * (kept when at least 1% faster).  The
 * timed launches write only step scratch and the spare psi buffer, so the state
 * (populations, psi, step counters, spectra) is unchanged.  cache_path (may be
 * NULL) names a text file of "key<TAB>planes" lines, keyed by the device name,
 * its SM count and the configuration (batched: one line for the shared value
 * and one per box depth): entries found there are applied without
 * timing (unless flags has FLB_TUNE_FORCE), new results are appended.  An
 * unreadable or unwritable file only disables the cache.  Synchronising; call
 * with the handle's device current and outside stream capture.  2D replicas and
 * the 3D combinations on one-thread-per-site kernels (see laplacian) are left as
 * they are.
 */
int flb_get_tuning(flb_handle *h, int32_t rep, int32_t *psi_zchunk);
int flb_set_tuning(flb_handle *h, int32_t rep, int32_t psi_zchunk);

/* Single-pass Heun (tuning flag, default off): with on != 0 every replica's psi
 * step runs both Runge-Kutta stages of Sec. V in one launch by halo recompute:
 * stage 1 on a halo of the tile (tile + 3 for the FV scheme, tile + 2 for FD),
 * so that stage 2's stencils find psi* in the block; psi* and the Heun
 * accumulator stay in shared memory and only psi^n and u are read.  The noise is
 * the two-stage form's (same counters), so both forms give the same step up to
 * FP32 rounding.  Applies to Heun with the SO Laplacian in plain mode: the FV
 * scheme on D3Q19, the FD scheme on either lattice; the z chunk is
 * flb_set_tuning's value.  Errors: EINVAL
 * (NULL handle), EUNSUPPORTED (on != 0 and some replica is not of that kind, or
 * the handle is not in plain mode).  Mode changes (flb_set_mode) turn it off. */
int flb_set_psi_fused(flb_handle *h, int32_t on);
int flb_autotune(flb_handle *h, const char *cache_path, int32_t flags);

/* Bitwise checkpoint of replica rep: flb_state_bytes() bytes holding the step
 * counter, the stored populations (in the storage precision), psi and u exactly
 * as kept on the device.  Restoring gives a bitwise-identical continuation (the
 * noise is counter-based).  Synchronising.  Errors: EINVAL (no such replica,
 * NULL buffer), ENOSPC (bytes too small), ECUDA. */
size_t flb_state_bytes(flb_handle *h, int32_t rep);
int flb_get_state(flb_handle *h, int32_t rep, void *host, size_t bytes);
int flb_set_state(flb_handle *h, int32_t rep, const void *host, size_t bytes);

/* Wait for the stream and return any latched device error. */
int flb_synchronize(flb_handle *h);

/* Kernel launches issued by this handle since creation (for accounting). */
int64_t flb_launch_count(flb_handle *h);

/* Per-phase device timing.  While on, flb_step records CUDA events around the
 * lattice Boltzmann collide-stream kernel and around the other kernels of every
 * replica step.  flb_kernel_times() synchronises and returns the summed
 * milliseconds and launch counts of {collide-stream kernel, the other step
 * kernels (mu, velocity of the new fluid state, psi stages), sampling} since the
 * last flb_set_profiling(h, 1), which clears them.  ms and counts: 3 entries.
 * In batched mode the whole graph-launched step counts as the first entry. */
int flb_set_profiling(flb_handle *h, int32_t on);
int flb_kernel_times(flb_handle *h, double *ms, int64_t *counts);

/*
 * Structure factor of one device field without any device allocation.
 * No counterpart in the paper: this serves callers that cannot obtain device
 * memory where they want a spectrum (a memory pool that forbids cudaMalloc, a
 * plug-in given only pointers and a stream, a loop that must not allocate).
 *   psi_dev : device pointer, FP32, nz*ny*nx values, x fastest (caller-owned).
 *   kmax    : wavevector window per axis as flb_params.sq_kmax.
 *   S_dev   : device pointer, FP64, Kz*Ky*Kx values (the layout of
 *             flb_structure_factor), WRITTEN (not accumulated) with
 *             |psi~(q)|^2 = |sum psi e^{-iq.r}|^2 / N.
 *   cuda_stream : cudaStream_t (NULL: legacy default stream); asynchronous.
 * Scratch: the two DFT intermediates use a fixed array in device memory that the
 * library declares at file scope (2 x FLB_NOALLOC_MAX_VALUES complex FP32 values,
 * 8 MiB), held by every GPU that loads the library until the process exits.
 * Limit: Kx*ny*nz and Kx*Ky*nz must each be <= FLB_NOALLOC_MAX_VALUES, else the
 * call returns FLB_ENOSPC without launching anything (e.g. 64^3 whole grid fits;
 * 128^3 needs kmax <= 15).  Other errors: EINVAL (null pointer, size < 1, kmax < 0,
 * N >= 2^31), ECUDA (also, before any launch, when an earlier CUDA error is
 * still pending on the calling thread; that error is left for its owner).  The
 * call allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress); the first call on a device may load the library's
 * device code there, so make it before any stream capture.  All calls on a device share the array,
 * which keeps the last call's contents; calls that overlap on the GPU (on
 * different streams, or from several threads) race on it and must be ordered by
 * the caller.
 */
#define FLB_NOALLOC_MAX_VALUES (1 << 19)
int flb_structure_factor_noalloc(const float *psi_dev, int32_t nx, int32_t ny, int32_t nz, int32_t kmax,
                                 double *S_dev, void *cuda_stream);

/* The standard normals the kernels draw (reading of the paper's noise: Philox
 * counter-based normals, held fixed over each step's Runge-Kutta stages), for
 * tests and for users who reproduce a run's noise elsewhere.  For sites
 * site0 .. site0+nsites-1 and Philox blocks 0 .. nblocks-1 of (seed, step,
 * stream) it writes dev_out[s*8*nblocks + 8*b + j], j = 0..7: normals 2k
 * and 2k+1 of block b are Box-Muller on its word x_k (k = 0..3), with the
 * radius uniform u = ((x_k >> 12) + 1/2) 2^-20 from the top 20 bits and the
 * angle uniform v = ((x_k & 0xFFF) + 1/2) 2^-12 from the low 12 bits,
 * g = sqrt(-2 ln u) (cos, sin)(2 pi v).  Stream 0 feeds the collide-stream
 * (mode noise), stream 1 the psi equation, streams 3 and 4 the equilibrium
 * start; the site id of a lattice point is x + nx*(y + ny*z).
 *   dev_out     : device pointer, FP32, nsites*8*nblocks values (caller-owned).
 *   cuda_stream : cudaStream_t (NULL: legacy default stream); asynchronous.
 * Errors: EINVAL (null dev_out, nsites < 0, nblocks outside [1, 16], stream >
 * 0xFFFF, site0 + nsites > 2^32), ECUDA. */
int flb_gaussians(uint64_t seed, int64_t step, uint32_t stream, uint32_t site0, int64_t nsites, int32_t nblocks,
                  float *dev_out, void *cuda_stream);

const char *flb_strerror(int code);

/* Release the handle (not the caller's workspace or stream). */
void flb_destroy(flb_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* FLB_H */

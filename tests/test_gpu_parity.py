"""GPU parity: the CUDA path against the FP64 oracle, element by element, from the
same seeded binary32-exact inputs, through the C ABI (flb_* via the binding).

Tolerance: per-step field error <= 1e-5 (max |gpu - oracle| over the RMS
deviation of the oracle field) -- the FP32 path rounds every quantity at
~6e-8 relative and the dynamics is contractive, so after tens to a hundred
steps the accumulated error stays two orders below that bound."""
import numpy as np
import pytest

import oracle as O
import paper_1104_0078_gb300 as F
from paper_1104_0078_gb300 import inputs as I

from gpu_helpers import field_error, flb_params, oracle_params, weights_column

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _run_pair(d, nsteps, amp_f=2e-3, amp_psi=0.05, seed=7):
    """Advance the same random start nsteps on the GPU and in the oracle."""
    fp = flb_params(d)
    op = oracle_params(d)
    N = op.n
    w = weights_column(op.q)
    f0 = w * op.rho0 + I.random_deviations(op.q, N, amp_f, seed)
    psi0 = I.random_field(N, amp_psi, seed + 1)
    s = F.Solver(fp)
    s.set_fields(psi=psi0)
    s.set_populations(f0)
    s.step(nsteps)
    s.synchronize()
    fg = s.get_populations()
    pg, ug = s.get_psi_u()
    st = O.State(op, f0.copy(), psi0.copy(), np.zeros((3, N)), 0)
    st.advance(nsteps)
    return s, (fg, pg, ug), st, w * op.rho0


CASES = []
for dim, q, shape in ((2, 9, (13, 10, 1)), (3, 19, (11, 7, 9)), (3, 19, (37, 23, 19)), (3, 15, (11, 7, 9)),
                      (3, 15, (37, 23, 19))):
    for scheme in ((0,) if q == 15 else (0, 1)):    # D3Q15: the FD psi scheme on the device
        for integ in (1, 2, 4):
            if shape == (37, 23, 19) and integ == 1:
                continue
            CASES.append((dim, q, shape, scheme, integ))


@pytest.mark.parametrize("dim,q,shape,scheme,integ", CASES)
def test_coupled_step_matches_oracle(dim, q, shape, scheme, integ):
    d = dict(dim=dim, q=q, nx=shape[0], ny=shape[1], nz=shape[2], tau=0.8, kT=1e-4, A=0.05, B=0.3, K=0.04, M=0.1,
             scheme=scheme, integrator=integ, coupling=3, seed=3)
    s, (fg, pg, ug), st, feq = _run_pair(d, 25)
    assert field_error(fg, st.f, feq) < TOL
    assert field_error(pg, st.psi) < TOL
    assert field_error(ug[:dim], st.u[:dim]) < TOL
    assert s.get_step() == 25


@pytest.mark.parametrize("integ", [1, 2, 4])
def test_noise_free_coupled_fv_matches_oracle(integ):
    # kT = 0 with the force coupled: FV stage 1 without noise, taking mu of psi^n
    # from the force's mu field, on a box of several ragged tiles.  A > 0: a large
    # psi relaxes and drives the fluid (in a quench the FP32 trajectory separates
    # from the FP64 one exponentially, and without noise the deviations the error
    # is measured against stay small)
    d = dict(dim=3, q=19, nx=37, ny=23, nz=19, tau=0.8, kT=0.0, A=0.05, B=0.3, K=0.04, M=0.1, scheme=1,
             integrator=integ, coupling=3, seed=21)
    s, (fg, pg, ug), st, feq = _run_pair(d, 20, amp_psi=0.3)
    assert field_error(fg, st.f, feq) < TOL
    assert field_error(pg, st.psi) < TOL
    assert field_error(ug, st.u) < TOL


FORCE_CASES = [(dim, q, scheme, fg) for dim, q in ((2, 9), (3, 19)) for scheme in (0, 1) for fg in (1, 2, 3)]
FORCE_CASES += [(3, 15, 0, 1), (3, 15, 0, 3)]


@pytest.mark.parametrize("dim,q,scheme,force_grad", FORCE_CASES)
def test_force_gradient_choices_match_oracle(dim, q, scheme, force_grad):
    # both lattice gradients in the force with both psi schemes (the matched pair
    # is the default of the cases above); a deep quench so the force is large
    shape = (10, 9, 7)
    d = dict(dim=dim, q=q, nx=shape[0], ny=shape[1], nz=shape[2], tau=0.8, kT=1e-4, A=-0.05, B=0.3, K=0.04, M=0.1,
             scheme=scheme, integrator=2, coupling=3, seed=13, force_grad=force_grad)
    s, (fg, pg, ug), st, feq = _run_pair(d, 20, amp_psi=0.3)
    assert field_error(fg, st.f, feq) < TOL
    assert field_error(pg, st.psi) < TOL
    assert field_error(ug[:dim], st.u[:dim]) < TOL


@pytest.mark.parametrize("dim,q", [(2, 9), (3, 19), (3, 15)])
def test_relaxation_variants_match_oracle(dim, q):
    # bulk rate different from shear, partially relaxed ghosts, only advection coupling
    shape = (9, 8, 6)
    for extra in (dict(gamma_bulk=-0.4, gamma_ghost=0.35), dict(coupling=2, gamma_ghost=-0.2),
                  dict(coupling=0, kT=0.0), dict(M=0.0, coupling=1)):
        d = dict(dim=dim, q=q, nx=shape[0], ny=shape[1], nz=shape[2], tau=0.6, kT=2e-4, A=-0.02, B=0.1, K=0.03,
                 M=0.2, scheme=0 if q == 15 else 1, integrator=2, coupling=3, seed=11)
        d.update(extra)
        s, (fg, pg, ug), st, feq = _run_pair(d, 15)
        assert field_error(fg, st.f, feq) < TOL, extra
        assert field_error(pg, st.psi) < TOL, extra


def test_bulk_3d_100_steps_from_rest():
    # D3Q19 64^3, tau 0.8, kT 1e-5, A 0.05, B 0, K 0.04, M 0.1, FV, Heun, from rest:
    # field error after 100 steps <= 1e-5 for populations, psi and u
    d = dict(I.WORKLOADS["bulk_3d"], integrator=2)
    fp = flb_params(d)
    op = oracle_params(d)
    s = F.Solver(fp)
    s.step(100)
    s.synchronize()
    fg = s.get_populations()
    pg, ug = s.get_psi_u()
    st = O.State.rest(op)
    st.advance(100)
    feq = weights_column(19) * op.rho0
    assert field_error(fg, st.f, feq) < TOL
    assert field_error(pg, st.psi) < TOL
    assert field_error(ug, st.u) < TOL


@pytest.mark.parametrize("q", [19, 15])
def test_conserved_totals_drift(q):
    # mass, momentum (B = 0) and psi drift over 400 steps on the GPU, reduced in FP64
    d = dict(I.WORKLOADS["bulk_3d"], nx=32, ny=32, nz=32, kT=1e-4, q=q, scheme=0 if q == 15 else 1)
    s = F.Solver(flb_params(d))
    N = 32 ** 3
    s.set_fields(psi=I.random_field(N, 0.1, 5))
    t0, _, rc0 = s.moments()
    s.step(400)
    t1, u2, rc1 = s.moments()
    assert rc0 == rc1 == F.FLB_OK
    f = s.get_populations()
    c, _ = O.lattice(3, q)
    jabs = np.abs(np.einsum("ia,in->an", c.astype(float), f)).sum()
    psi, _ = s.get_psi_u()
    assert abs(t1[0] - t0[0]) / (N * 1.0) < 1e-6
    assert np.abs(t1[1:4] - t0[1:4]).max() / jabs < 1e-6
    assert abs(t1[4] - t0[4]) / np.abs(psi).sum() < 1e-6


@pytest.mark.parametrize("scheme", [0, 1])
def test_stress_force_conserves_momentum(scheme):
    # force_grad 3 (F = -div sigma): with B != 0 and noise the total momentum,
    # reduced in FP64 on the device, stays at zero to FP32 round-off over 300
    # steps (the stored populations' rounding walks it to ~1e-6), while
    # -psi grad mu drives a net momentum thousands of times larger
    d = dict(dim=3, q=19, nx=24, ny=20, nz=18, tau=0.8, kT=1e-4, A=-0.05, B=0.3, K=0.04, M=0.1, scheme=scheme,
             integrator=2, coupling=3, seed=9)
    N = 24 * 20 * 18
    out = {}
    for fg in (3, 0):
        s = F.Solver(flb_params(d, force_grad=fg))
        s.set_fields(psi=I.random_field(N, 0.05, 21))
        s.step(300)
        t1, _, rc = s.moments()
        assert rc == F.FLB_OK
        out[fg] = np.abs(t1[1:4]).max()
    assert out[3] < 1e-2 * out[0] and out[3] < 1e-9 * N


def test_structure_factor_matches_oracle():
    # same seed: accumulated S(q) on the GPU (separable DFT, FP64 sums) against the
    # oracle's FFT of its own trajectory, every 5 steps over 100 steps
    d = dict(dim=3, q=19, nx=16, ny=12, nz=10, tau=0.8, kT=1e-4, A=0.1, B=0.0, K=0.04, M=0.2, scheme=1,
             integrator=2, seed=2)
    s = F.Solver(flb_params(d))
    s.set_sampling(5, 1)
    s.step(100)
    S_gpu, ns = s.structure_factor()
    op = oracle_params(d)
    st = O.State.rest(op)
    acc = np.zeros(op.shape)
    for _ in range(20):
        st.advance(5)
        acc += O.structure_factor(op, st.psi)
    acc /= 20
    assert ns == 20
    S_gpu = S_gpu.reshape(op.shape)
    big = acc > 1e-3 * acc.max()
    assert np.max(np.abs(S_gpu[big] - acc[big]) / acc[big]) < 1e-4


@pytest.mark.parametrize("kmax", [0, 3])
def test_dynamic_structure_factor_matches_oracle(kmax):
    # same seed: S(q, l) accumulated on the GPU (Fourier snapshots kept on the
    # device, FP64 lag sums) against the oracle's estimator on its own trajectory,
    # sampled every 4 steps over 80 steps, 6 lags; full grid and a window
    d = dict(dim=3, q=19, nx=16, ny=12, nz=10, tau=0.8, kT=1e-4, A=0.1, B=0.0, K=0.04, M=0.2, scheme=1,
             integrator=2, seed=4)
    fp = flb_params(d, sq_kmax=kmax)
    fp.sq_lags = 6
    s = F.Solver(fp)
    s.set_sampling(4, 1 | 4)
    s.step(80)
    S_gpu, ns = s.structure_factor(which=F.FLB_SQ_DYNAMIC)
    S_static, _ = s.structure_factor()
    assert ns == 20
    op = oracle_params(d)
    st = O.State.rest(op)
    psis = []
    for _ in range(20):
        st.advance(4)
        psis.append(st.psi.copy())
    ref = O.dynamic_structure_factor(op, psis, 6)
    if kmax:
        sel = [np.r_[0:kmax + 1, n - kmax:n] for n in op.shape]
        ref = ref[:, sel[0]][:, :, sel[1]][:, :, :, sel[2]]
    S_gpu = S_gpu.reshape(ref.shape)
    assert np.allclose(S_gpu[0].ravel(), S_static, rtol=1e-6, atol=0)   # lag 0 is the static S(q)
    scale = np.abs(ref[0]).max()
    assert np.max(np.abs(S_gpu - ref)) < 2e-4 * scale


def test_structure_factor_window():
    # sq_kmax keeps |k_a| <= kmax on every axis, in FFT order; sampled at step 0
    # from a seeded field, against the oracle's FFT of the same field
    d = dict(dim=3, q=19, nx=16, ny=16, nz=12, tau=0.8, kT=1e-4, A=0.1, B=0.0, K=0.04, M=0.2, scheme=0,
             integrator=1, seed=4, sq_kmax=3)
    s = F.Solver(flb_params(d))
    psi0 = I.random_field(16 * 16 * 12, 0.2, 12)
    s.set_fields(psi=psi0)
    s.sample(1)
    s.sample(1)
    S_gpu, ns = s.structure_factor()
    op = oracle_params(d)
    full = O.structure_factor(op, psi0)
    ks = lambda n: list(range(0, 4)) + list(range(n - 3, n))
    sel = full[np.ix_(ks(12), ks(16), ks(16))]
    assert S_gpu.size == 7 * 7 * 7 and ns == 2
    assert np.allclose(S_gpu.reshape(7, 7, 7), sel, rtol=1e-4, atol=1e-6 * sel.max())
    s.sq_reset()
    S0, n0 = s.structure_factor()
    assert n0 == 0 and not S0.any()


def test_interface_heights_match_oracle():
    # slab with two tanh interfaces, a few noisy steps, heights spectrum GPU vs oracle
    d = dict(dim=3, q=19, nx=16, ny=12, nz=32, tau=0.8, kT=2e-5, A=-0.0625, B=0.0625, K=0.04, M=0.1, scheme=1,
             integrator=2, seed=9)
    op = oracle_params(d)
    psi0 = I.slab_profile(16, 12, 32, d["A"], d["B"], d["K"], 8.0, 24.0)
    s = F.Solver(flb_params(d))
    s.set_fields(psi=psi0)
    s.step(20)
    s.sample(2)
    H_gpu, ns = s.structure_factor(which=F.FLB_SQ_HEIGHT)
    st = O.State.rest(op, psi=psi0)
    st.advance(20)
    h1, h2 = O.interface_heights(op, st.psi)
    assert not np.isnan(h1).any() and not np.isnan(h2).any()
    H = 0.5 * (O.height_spectrum(h1) + O.height_spectrum(h2))
    H[0, 0] = 0.0
    assert ns == 1
    H_gpu = H_gpu.reshape(12, 16)
    # heights located from FP32 psi carry an absolute error dh <~ 2e-5 lattice units
    # (psi error <~ 1e-5 over an interface slope >~ 0.5); |h~|^2 then moves by at
    # most 2 |h~| dh + dh^2 per mode
    dh = 2e-5
    assert np.all(np.abs(H_gpu - H) <= 2 * np.sqrt(H) * dh + dh * dh)
    assert H.max() > 1e-4
    # the same surfaces located by the oracle in the device's own FP32 psi: the
    # crossing cells are decided on the same values, so what remains is the FP32
    # arithmetic of the device's heights and of its DFT, which transforms the raw
    # heights (|h| < 32, mean included) with FP32 products and lane sums: ~1e-5
    # per mode, the same bound as above, now without the trajectories' divergence
    pg, _ = s.get_psi_u()
    g1, g2 = O.interface_heights(op, pg.astype(np.float64))
    assert not np.isnan(g1).any() and not np.isnan(g2).any()
    Hs = 0.5 * (O.height_spectrum(g1) + O.height_spectrum(g2))
    Hs[0, 0] = 0.0
    assert np.all(np.abs(H_gpu - Hs) <= 2 * np.sqrt(Hs) * dh + dh * dh)


def test_checkpoint_resume_bitwise():
    d = dict(dim=3, q=19, nx=12, ny=10, nz=8, tau=0.8, kT=1e-4, A=0.05, B=0.2, K=0.04, M=0.1, scheme=1,
             integrator=2, seed=5)
    a = F.Solver(flb_params(d))
    a.set_fields(psi=I.random_field(960, 0.1, 1))
    a.step(50)
    blob = a.get_state()
    a.step(50)
    fa = a.get_populations()
    pa, ua = a.get_psi_u()
    b = F.Solver(flb_params(d))
    b.set_state(blob)
    assert b.get_step() == 50
    b.step(50)
    fb = b.get_populations()
    pb, ub = b.get_psi_u()
    assert np.array_equal(fa, fb) and np.array_equal(pa, pb) and np.array_equal(ua, ub)


def test_determinism_two_runs():
    d = dict(dim=2, q=9, nx=20, ny=16, tau=1.0, kT=1e-4, A=0.05, B=0.1, K=0.04, M=0.1, scheme=0, integrator=2,
             seed=8)
    out = []
    for _ in range(2):
        s = F.Solver(flb_params(d))
        s.step(30)
        out.append((s.get_populations(), s.get_psi_u()[0]))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_minimum_box_and_errors():
    # the smallest admitted box (4^3) still matches, on both 3D lattices; invalid
    # calls return codes
    for q in (15, 19):
        d = dict(dim=3, q=q, nx=4, ny=4, nz=4, tau=0.8, kT=1e-4, A=0.05, B=0.3, K=0.04, M=0.1, scheme=0,
                 integrator=2, seed=3)
        s, (fg, pg, ug), st, feq = _run_pair(d, 10)
        assert field_error(fg, st.f, feq) < TOL and field_error(pg, st.psi) < TOL, q
    lib = F.load_library()
    assert lib.flb_step(s.h, -1) == F.FLB_EINVAL
    assert lib.flb_get_window(s.h, 0, 0, 0, 0, 64, 64, 64, None, None) == F.FLB_ENOSPC
    assert lib.flb_set_mode(s.h, 7) == F.FLB_EINVAL


# The one-thread-per-site path: another App. A Laplacian, the naive scheme of
# Sec. III, FV on D3Q15; and the tiled D3Q15 FD path with the explicit FV force
STENCIL_CASES = [
    (3, 19, 0, 2, dict(laplacian=1)), (3, 19, 0, 2, dict(laplacian=2)), (3, 19, 0, 4, dict(laplacian=3)),
    (3, 19, 1, 2, dict(laplacian=1)), (3, 19, 2, 2, dict(laplacian=1)), (3, 19, 2, 1, dict(laplacian=0)),
    (3, 15, 1, 2, {}), (3, 15, 1, 4, {}), (3, 15, 1, 1, dict(laplacian=2)), (3, 15, 2, 2, dict(laplacian=1)),
    (3, 15, 0, 2, dict(force_grad=2)), (3, 15, 0, 2, dict(laplacian=3)),
    (2, 9, 0, 2, dict(laplacian=1)), (2, 9, 2, 2, dict(laplacian=1)), (2, 9, 2, 4, {}),
]


@pytest.mark.parametrize("dim,q,scheme,integ,extra", STENCIL_CASES)
def test_stencil_options_match_oracle(dim, q, scheme, integ, extra):
    shape = (13, 10, 1) if dim == 2 else (11, 9, 7)
    d = dict(dim=dim, q=q, nx=shape[0], ny=shape[1], nz=shape[2], tau=0.8, kT=1e-4, A=-0.05, B=0.3, K=0.04, M=0.1,
             scheme=scheme, integrator=integ, coupling=3, seed=17, **extra)
    s, (fg, pg, ug), st, feq = _run_pair(d, 20, amp_psi=0.2)
    assert field_error(fg, st.f, feq) < TOL
    assert field_error(pg, st.psi) < TOL
    assert field_error(ug[:dim], st.u[:dim]) < TOL


def test_d3q15_fp16_storage_tracks_fp32():
    # FP16 deviations on D3Q15: the same seeded start advanced 40 steps stays within
    # the half-precision rounding of the FP32 path (unit roundoff 2^-11 on
    # deviations of ~2e-3, re-rounded every step)
    d = dict(dim=3, q=15, nx=20, ny=18, nz=16, tau=0.8, kT=1e-4, A=0.05, B=0.3, K=0.04, M=0.1, scheme=0,
             integrator=2, coupling=3, seed=6)
    N = 20 * 18 * 16
    out = {}
    for stg in (F.FLB_F32_DEV, F.FLB_F16_DEV):
        s = F.Solver(flb_params(d, storage=stg))
        s.set_fields(psi=I.random_field(N, 0.05, 2))
        s.set_populations(weights_column(15) + I.random_deviations(15, N, 2e-3, 3))
        s.step(40)
        out[stg] = (s.get_populations(), s.get_psi_u()[0])
    feq = weights_column(15)
    assert field_error(out[F.FLB_F16_DEV][0], out[F.FLB_F32_DEV][0], feq) < 5e-2
    assert field_error(out[F.FLB_F16_DEV][1], out[F.FLB_F32_DEV][1]) < 1e-3


@pytest.mark.parametrize("dim,q,shape", [(3, 19, (13, 9, 7)), (3, 15, (8, 11, 6)), (2, 9, (17, 6, 1))])
def test_set_fields_equilibrium_and_fields(dim, q, shape):
    # flb_set_fields with rho, u and psi: the populations are the second-order
    # equilibrium of (rho, u) (Sec. IV) element by element, psi and u come back
    # as given (FP32), and a coupled step from there still matches the oracle
    d = dict(dim=dim, q=q, nx=shape[0], ny=shape[1], nz=shape[2], tau=0.8, kT=1e-4, A=0.05, B=0.3, K=0.04, M=0.1,
             scheme=0, integrator=2, coupling=3, seed=23)
    op = oracle_params(d)
    N = op.n
    rho = I.f32(1.0 + I.random_field(N, 0.01, 31))       # binary32-exact inputs on both sides
    u = np.zeros((3, N))
    u[:dim] = I.random_field(dim * N, 0.02, 32).reshape(dim, N)
    psi = I.random_field(N, 0.1, 33)
    s = F.Solver(flb_params(d))
    s.set_fields(rho=rho, u=u[:dim], psi=psi)
    feq = O.equilibrium(op, rho=rho, u=u)
    w = weights_column(q) * op.rho0
    # the device evaluates the equilibrium deviations in FP32 (a few ulp)
    assert field_error(s.get_populations(), feq, w) < 2e-6
    pg, ug = s.get_psi_u()
    assert np.array_equal(pg, I.f32(psi)) and np.array_equal(ug[:dim], I.f32(u[:dim]))
    s.step(5)
    st = O.State(op, feq.copy(), psi.copy(), u.copy(), 0)
    st.advance(5)
    assert field_error(s.get_populations(), st.f, w) < TOL
    assert field_error(s.get_psi_u()[0], st.psi) < TOL


@pytest.mark.parametrize("dim,q,shape", [(3, 19, (11, 9, 7)), (3, 15, (10, 8, 9)), (2, 9, (17, 12, 1))])
def test_mode_variances_match_oracle(dim, q, shape):
    # flb_mode_variances against the oracle's projection of its own trajectory:
    # the mean over sites of m_k^2, m = E (fbar - w rho0), for every mode k
    d = dict(dim=dim, q=q, nx=shape[0], ny=shape[1], nz=shape[2], tau=0.8, kT=1e-4, A=0.05, B=0.3, K=0.04, M=0.1,
             scheme=0, integrator=2, coupling=3, seed=19, gamma_ghost=0.2)
    s, (fg, pg, ug), st, feq = _run_pair(d, 12)
    E, b = O.moment_basis(dim, q)
    m = E @ (st.f - feq)
    ref = np.mean(m ** 2, axis=1)
    got = s.mode_variances()
    assert np.allclose(got, ref, rtol=1e-4, atol=0), (got, ref)


def test_nonfinite_is_reported():
    d = dict(dim=2, q=9, nx=8, ny=8, tau=1.0, kT=0.0, A=0.05, B=0.0, K=0.04, M=0.1, scheme=0, integrator=1)
    s = F.Solver(flb_params(d))
    psi = np.zeros(64)
    psi[5] = np.nan
    s.set_fields(psi=psi)
    _, _, rc = s.moments()
    assert rc == F.FLB_ENONFINITE


def test_structure_factor_long_rows():
    # the x pass of the windowed DFT sums blocks of 128 rows against staged
    # twiddles (only k >= 0, the rest as conjugates) for windows of K_x <= 32 and
    # rows up to 1024, the y pass a plane per block: rows of 512 as in the 512^3
    # workload (16 chunks of 32 columns), kmax = 8 as the bench samples, a seeded
    # field at step 0, every value of the window against the oracle's FFT of the
    # same field
    d = dict(dim=3, q=19, nx=512, ny=48, nz=40, tau=0.8, kT=1e-4, A=0.1, B=0.0, K=0.04, M=0.2, scheme=1,
             integrator=2, seed=4, sq_kmax=8)
    s = F.Solver(flb_params(d))
    N = 512 * 48 * 40
    psi0 = I.uniform_field(N, -0.01, 0.01, 31)
    s.set_fields(psi=psi0)
    s.sample(1)
    S_gpu, ns = s.structure_factor()
    assert ns == 1 and S_gpu.size == 17 ** 3
    full = O.structure_factor(oracle_params(d), psi0)
    ks = lambda n: list(range(0, 9)) + list(range(n - 8, n))
    ref = full[np.ix_(ks(40), ks(48), ks(512))]
    assert np.allclose(S_gpu.reshape(17, 17, 17), ref, rtol=1e-4, atol=1e-6 * ref.max())


@pytest.mark.parametrize("shape,kmax", [((15, 13, 9), 0), ((33, 10, 7), 4), ((21, 17, 1), 0), ((40, 9, 1), 5)])
def test_structure_factor_odd_and_planar_boxes(shape, kmax):
    # the row-block x pass sums k >= 0 and writes the partners as conjugates:
    # odd extents (no self-conjugate k = n/2), a window on a wider row, a
    # ragged last block of rows, and planar boxes (one plane: the y pass alone
    # in its block, the z pass over one plane); every value against the
    # oracle's FFT of the same seeded field at step 0
    nx, ny, nz = shape
    dim = 2 if nz == 1 else 3
    d = dict(dim=dim, q=9 if dim == 2 else 19, nx=nx, ny=ny, nz=nz, tau=0.8, kT=1e-4, A=0.1, B=0.0, K=0.04,
             M=0.2, scheme=1, integrator=2, seed=4, sq_kmax=kmax)
    s = F.Solver(flb_params(d))
    N = nx * ny * nz
    psi0 = I.uniform_field(N, -0.01, 0.01, 37)
    s.set_fields(psi=psi0)
    s.sample(1)
    S_gpu, ns = s.structure_factor()
    full = O.structure_factor(oracle_params(d), psi0)
    keep = lambda n: list(range(n)) if kmax <= 0 or 2 * kmax + 1 >= n else list(range(kmax + 1)) + list(range(n - kmax, n))
    kz, ky, kx = keep(nz), keep(ny), keep(nx)
    assert ns == 1 and S_gpu.size == len(kx) * len(ky) * len(kz)
    ref = full.reshape(nz, ny, nx)[np.ix_(kz, ky, kx)]
    assert np.allclose(S_gpu.reshape(len(kz), len(ky), len(kx)), ref, rtol=1e-4, atol=1e-6 * ref.max())

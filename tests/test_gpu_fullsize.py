"""Parity at the full 512^3 quench size, in the launch configuration bench.py
times (D3Q19, FV, Heun) and in that of its D3Q15/FD variant: after two steps
from the seeded start (rest populations, psi0 uniform in [-0.01, 0.01]) sampled
sites are compared with the FP64 oracle run on a 32^3 window around each
(periodic window, counter ids of the global lattice).  Two steps of either
path depend on psi0 within 12 cells and on the populations within 11, so the
central 8^3 of each window is exact; plus conservation of mass and psi over the
run."""
import numpy as np
import pytest

import oracle as O
import paper_1104_0078_gb300 as F
from paper_1104_0078_gb300 import inputs as I

from gpu_helpers import field_error

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.mark.parametrize("q,scheme", [(19, 1), (15, 0)])
def test_quench_512_windows_match_oracle(q, scheme):
    d = dict(I.WORKLOADS["quench"])
    n = 512
    N = n ** 3
    p = F.flb_params_default(q=q, nx=n, ny=n, nz=n, tau=d["tau"], kT=d["kT"], A=d["A"], B=d["B"], K=d["K"],
                             M=d["M"], psi_scheme=scheme, integrator=F.FLB_HEUN, seed=d["seed"], sq_kmax=8)
    psi0 = I.uniform_field(N, -0.01, 0.01, 11)
    s = F.Solver(p)
    s.set_fields(psi=psi0)
    t0, _, _ = s.moments()
    s.step(2)
    t1, _, rc = s.moments()
    assert rc == F.FLB_OK
    assert abs(t1[0] - t0[0]) / N < 1e-6
    psi_cube = psi0.reshape(n, n, n)
    rng = np.random.default_rng(5)
    W = 32
    _, w = O.lattice(3, q)
    for origin in [(0, 0, 0), (n - 16, 100, 250), (240, 496, 8)] + [tuple(rng.integers(0, n, 3)) for _ in range(3)]:
        x0, y0, z0 = (int(v) for v in origin)
        fg, pg = s.get_window((x0, y0, z0), (W, W, W))
        idx = [(np.arange(W) + o) % n for o in (z0, y0, x0)]
        win_psi = psi_cube[np.ix_(*idx)].reshape(-1)
        op = O.Params(dim=3, q=q, nx=W, ny=W, nz=W, tau=d["tau"], kT=d["kT"], A=d["A"], B=d["B"], K=d["K"],
                      M=d["M"], scheme=scheme, integrator=2, coupling=3, seed=d["seed"], gdims=(n, n, n),
                      origin=(x0, y0, z0))
        st = O.State.rest(op, psi=win_psi)
        st.advance(2)
        c = slice(12, 20)
        f_o = st.f.reshape(q, W, W, W)[:, c, c, c].reshape(q, -1)
        f_g = fg.reshape(q, W, W, W)[:, c, c, c].reshape(q, -1)
        p_o = st.psi.reshape(W, W, W)[c, c, c].reshape(-1)
        p_g = pg.reshape(W, W, W)[c, c, c].reshape(-1)
        assert field_error(f_g, f_o, w[:, None]) < TOL
        assert field_error(p_g, p_o, p_o.mean()) < TOL


def test_structure_factor_512_sampled_wavevectors():
    # the S(q) window the bench samples on the 512^3 quench (|k_a| <= 8, FFT
    # order), on the seeded initial field: sampled wavevectors of the window,
    # negative and zero components included, against the oracle's direct sum
    # of the definition over all 512^3 sites
    d = dict(I.WORKLOADS["quench"])
    n, kmax = 512, 8
    p = F.flb_params_default(nx=n, ny=n, nz=n, tau=d["tau"], kT=d["kT"], A=d["A"], B=d["B"], K=d["K"], M=d["M"],
                             psi_scheme=F.FLB_FV, integrator=F.FLB_HEUN, seed=d["seed"], sq_kmax=kmax)
    psi0 = I.uniform_field(n ** 3, -0.01, 0.01, 11)
    s = F.Solver(p)
    s.set_fields(psi=psi0)
    s.sample(1)
    S_gpu, ns = s.structure_factor()
    del s
    K = 2 * kmax + 1
    S_gpu = S_gpu.reshape(K, K, K)
    slot = lambda k: k if k >= 0 else K + k   # window index of k in FFT order
    ks = [(1, 0, 0), (0, 0, 1), (8, 8, 8), (-8, 3, -5), (2, -7, 0), (-1, -1, -1), (5, 1, 8), (0, 6, -3)]
    op = O.Params(dim=3, q=19, nx=n, ny=n, nz=n, tau=d["tau"], kT=d["kT"], A=d["A"], B=d["B"], K=d["K"], M=d["M"])
    ref = O.structure_factor_at(op, psi0, ks)
    got = np.array([S_gpu[slot(kz), slot(ky), slot(kx)] for kx, ky, kz in ks])
    assert np.allclose(got, ref, rtol=1e-4, atol=1e-6 * ref.max()), (got, ref)


def test_fp16_storage_on_the_512_quench():
    # the FP16-deviation storage form on the 512^3 spinodal quench (A -0.0625,
    # B 0.0625, K 0.04, M 0.1, kT 1e-5, psi0 uniform in [-0.01, 0.01]), 2000 steps
    # beside FP32 from the same seed and start.  The run is out of equilibrium,
    # so equipartition is checked where it must hold: every ghost mode of the
    # stored populations keeps <m_g^2> = (rho0 kT / c_s^2) b_g within 1% (the
    # ghosts are projected and re-drawn each step, Sec. III); mass and psi are
    # conserved within 1e-6; and <u_a^2> of FP16 matches FP32 within 1%
    d = dict(I.WORKLOADS["quench"])
    n = 512
    N = n ** 3
    psi0 = I.uniform_field(N, -0.01, 0.01, 11)
    _, b = O.moment_basis(3, 19)
    u2 = {}
    for st in (F.FLB_F32_DEV, F.FLB_F16_DEV):
        p = F.flb_params_default(nx=n, ny=n, nz=n, tau=d["tau"], kT=d["kT"], A=d["A"], B=d["B"], K=d["K"],
                                 M=d["M"], psi_scheme=F.FLB_FV, integrator=F.FLB_HEUN, storage=st, seed=d["seed"])
        s = F.Solver(p)
        s.set_fields(psi=psi0)
        t0, _, _ = s.moments()
        s.step(2000)
        t1, uu, rc = s.moments()
        assert rc == F.FLB_OK
        assert abs(t1[0] - t0[0]) / (N * p.rho0) < 1e-6
        assert abs(t1[4] - t0[4]) / np.abs(psi0).sum() < 1e-6
        ratio = s.mode_variances() / (p.rho0 * d["kT"] * 3.0 * b)
        assert np.all(np.abs(ratio[10:] - 1) < 0.01), (st, ratio)
        u2[st] = uu
        del s
    assert np.all(np.abs(u2[F.FLB_F16_DEV] / u2[F.FLB_F32_DEV] - 1) < 0.01), u2

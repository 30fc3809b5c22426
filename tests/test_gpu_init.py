"""The equilibrium start (flb_params.init = FLB_INIT_EQUILIBRIUM; the paper's runs
start from equilibrium, Sec. VI) against the oracle's State.equilibrium: element
by element on ragged boxes, and statistically against the closed forms --
S(q) = kT/(A - K L(q)) at t = 0 (Eq. test2) and <u_a^2> = kT/rho0 from the first
step on, without the transient a start from rest has."""
import numpy as np
import pytest

import oracle as O
import paper_1104_0078_gb300 as F
from oracle import theory as T
from paper_1104_0078_gb300 import inputs as I

from gpu_helpers import field_error, flb_params, oracle_params, weights_column

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.mark.parametrize("dim,q,shape,lap,storage", [(3, 19, (13, 10, 7), 0, 0), (3, 15, (9, 11, 6), 0, 0),
                                                     (3, 19, (8, 6, 5), 2, 0), (2, 9, (13, 10, 1), 0, 0),
                                                     (2, 9, (7, 12, 1), 1, 0)])
def test_equilibrium_start_matches_oracle(dim, q, shape, lap, storage):
    nx, ny, nz = shape
    d = dict(dim=dim, q=q, nx=nx, ny=ny, nz=nz, tau=0.8, kT=2e-4, A=0.05, B=0.0, K=0.04, M=0.1, scheme=0,
             integrator=2, laplacian=lap, seed=9)
    s = F.Solver(flb_params(d, init=F.FLB_INIT_EQUILIBRIUM, storage=storage))
    st = O.State.equilibrium(oracle_params(d))
    f = s.get_populations()
    psi, u = s.get_psi_u()
    assert field_error(f, st.f, weights_column(q)) < TOL
    assert field_error(psi, st.psi) < TOL
    assert field_error(u, st.u[:dim]) < TOL


def test_equilibrium_start_rejects_unstable_free_energy():
    p = F.flb_params_default(nx=8, ny=8, nz=8, A=-0.0625, B=0.0625, init=F.FLB_INIT_EQUILIBRIUM)
    with pytest.raises(F.FlbError):
        F.Solver(p)


def test_equilibrium_start_statistics():
    # the bulk 3D workload (64^3, FV, Heun) from its equilibrium: two seeds; S(q)
    # at t = 0 per |q| shell within 2% of kT/(A - K L_SO) (>= 4e4 modes per shell:
    # s.d. <= 0.5%), <u_a^2> within 1% of kT/rho0 at t = 0 and over the next 2000
    # steps, and S(q) over those steps within 2% of the stationary theory of the
    # discrete scheme (no transient factor)
    d = dict(I.WORKLOADS["bulk_3d"], integrator=2)
    op = oracle_params(d)
    qg = T.q_grid(op.shape)
    c, w = O.lattice(3, 19)
    th0 = d["kT"] / (d["A"] - d["K"] * T.L_so(qg))
    Lm = T.L_fv(qg, c, w)
    th = T.static_structure_factor(qg, op, Lm)
    qm = np.sqrt((qg ** 2).sum(-1))
    edges = np.linspace(1e-9, qm.max() + 1e-9, 13)
    S0 = np.zeros(op.shape)
    S1 = np.zeros(op.shape)
    u20 = np.zeros(3)
    u21 = np.zeros(3)
    for seed in (1, 2):
        s = F.Solver(flb_params(d, init=F.FLB_INIT_EQUILIBRIUM, seed=seed))
        _, uu, _ = s.moments()
        u20 += uu / 2
        s.sample(1)
        S, ns = s.structure_factor()
        S0 += S.reshape(op.shape) / 2
        s.sq_reset()
        acc = np.zeros(3)
        for _ in range(200):
            s.step(10)
            s.sample(1)
            _, uu, rc = s.moments()
            assert rc == F.FLB_OK
            acc += uu
        u21 += acc / 200 / 2
        S, ns = s.structure_factor()
        S1 += S.reshape(op.shape) / 2
    checked = 0
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (qm >= lo) & (qm < hi)
        if sel.sum() >= 2e4:
            assert abs((S0[sel] / th0[sel]).mean() - 1) < 0.02, (lo, hi)
            assert abs((S1[sel] / th[sel]).mean() - 1) < 0.02, (lo, hi)
            checked += 1
    assert checked >= 6
    assert np.all(np.abs(u20 / d["kT"] - 1) < 0.01), u20 / d["kT"]
    assert np.all(np.abs(u21 / d["kT"] - 1) < 0.01), u21 / d["kT"]

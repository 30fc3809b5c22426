"""The single-pass Heun psi step (flb_set_psi_fused; Sec. V's Runge-Kutta step
with the noise held fixed, both stages in one launch by halo recompute) against
the FP64 oracle element by element, against the two-launch form, and for the
bitwise independence of its z chunk."""
import numpy as np
import pytest

import oracle as O
import paper_1104_0078_gb300 as F
from paper_1104_0078_gb300 import inputs as I

from gpu_helpers import field_error, flb_params, oracle_params, weights_column

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _start(d, fused, zc=None, amp_f=2e-3, amp_psi=0.05, seed=7):
    op = oracle_params(d)
    N = op.n
    w = weights_column(op.q)
    f0 = w * op.rho0 + I.random_deviations(op.q, N, amp_f, seed)
    psi0 = I.random_field(N, amp_psi, seed + 1)
    s = F.Solver(flb_params(d))
    s.set_fields(psi=psi0)
    s.set_populations(f0)
    if zc is not None:
        s.set_tuning(zc)
    if fused:
        s.set_psi_fused(True)
    return s, op, f0, psi0, w * op.rho0


CASES = [((13, 10, 9), 1e-4, 0.05, 0.3), ((37, 23, 19), 1e-4, 0.05, 0.3), ((8, 6, 5), 1e-4, -0.05, 0.3),
         ((37, 23, 19), 0.0, 0.05, 0.3)]


@pytest.mark.parametrize("scheme,q", [(1, 19), (0, 19), (0, 15)])
@pytest.mark.parametrize("shape,kT,A,B", CASES)
def test_fused_heun_matches_oracle(shape, kT, A, B, scheme, q):
    # ragged tiles, a box smaller than the tile + halo region (its periodic
    # images wrap several times), a quench, and the noise-free stage; the FV
    # scheme (D3Q19) and the FD scheme on both lattices
    d = dict(dim=3, q=q, nx=shape[0], ny=shape[1], nz=shape[2], tau=0.8, kT=kT, A=A, B=B, K=0.04, M=0.1,
             scheme=scheme, integrator=2, coupling=3, seed=3)
    s, op, f0, psi0, feq = _start(d, True, amp_psi=0.3 if kT == 0 else 0.05)
    s.step(20)
    fg = s.get_populations()
    pg, ug = s.get_psi_u()
    st = O.State(op, f0.copy(), psi0.copy(), np.zeros((3, op.n)), 0)
    st.advance(20)
    assert field_error(fg, st.f, feq) < TOL
    assert field_error(pg, st.psi) < TOL
    assert field_error(ug, st.u) < TOL


@pytest.mark.parametrize("scheme", [1, 0])
def test_fused_heun_matches_two_launch_form(scheme):
    # the bulk 3D workload from a random start: 50 coupled steps with each form
    d = dict(I.WORKLOADS["bulk_3d"], integrator=2, scheme=scheme)
    out = {}
    for fused in (False, True):
        s, op, f0, psi0, feq = _start(d, fused)
        s.step(50)
        out[fused] = (s.get_populations(), s.get_psi_u()[0])
    assert field_error(out[True][0], out[False][0], feq) < TOL
    assert field_error(out[True][1], out[False][1]) < TOL


@pytest.mark.parametrize("scheme", [1, 0])
def test_fused_heun_z_chunk_changes_no_bit(scheme):
    d = dict(dim=3, q=19, nx=40, ny=20, nz=33, tau=0.8, kT=1e-4, A=0.05, B=0.3, K=0.04, M=0.1, scheme=scheme,
             integrator=2, coupling=3, seed=5)
    ref = None
    for zc in (1, 4, 7, 64):
        s, *_ = _start(d, True, zc=zc)
        s.step(5)
        psi, _ = s.get_psi_u()
        if ref is None:
            ref = psi
        assert np.array_equal(psi, ref), zc


def test_fused_heun_scope():
    base = dict(dim=3, q=19, nx=8, ny=8, nz=8, tau=0.8, kT=1e-4, A=0.05, B=0.0, K=0.04, M=0.1, scheme=1,
                integrator=2, coupling=3, seed=1)
    # the Euler integrator, FV on D3Q15, FD with an App. A Laplacian (the per-site path)
    for kw in (dict(integrator=1), dict(q=15), dict(laplacian=2, scheme=0), dict(integrator=1, scheme=0)):
        s = F.Solver(flb_params(base, **kw))
        assert s.lib.flb_set_psi_fused(s.h, 1) == F.FLB_EUNSUPPORTED
    for kw in (dict(scheme=0), dict(scheme=0, q=15)):  # FD with the SO Laplacian, either lattice
        s = F.Solver(flb_params(base, **kw))
        assert s.lib.flb_set_psi_fused(s.h, 1) == F.FLB_OK
    s = F.Solver(flb_params(base))
    s.set_mode(F.FLB_MODE_BATCHED)
    assert s.lib.flb_set_psi_fused(s.h, 1) == F.FLB_EUNSUPPORTED
    s.set_mode(F.FLB_MODE_PLAIN)
    assert s.lib.flb_set_psi_fused(s.h, 1) == F.FLB_OK
    assert s.lib.flb_set_psi_fused(s.h, 0) == F.FLB_OK

"""Batched mode (all replicas in one launch per phase, replayed as a CUDA graph)
against the plain per-replica launch sequence on the same uneven replica set:
the per-site arithmetic is shared, so every field must agree bitwise."""
import numpy as np
import pytest

import paper_1104_0078_gb300 as F
from paper_1104_0078_gb300 import inputs as I

from gpu_helpers import flb_params

pytestmark = pytest.mark.gpu

SHAPES = [(16, 16, 16), (12, 10, 20), (40, 18, 9), (33, 7, 70)]


def _replicas(**kw):
    ps = []
    for r, (nx, ny, nz) in enumerate(SHAPES):
        d = dict(dim=3, q=19, nx=nx, ny=ny, nz=nz, tau=0.8, kT=1e-5 * (1 + r), A=0.05, B=0.2, K=0.04, M=0.1,
                 scheme=1, integrator=2, seed=100 + r)
        d.update(kw)
        ps.append(flb_params(d))
    return ps


def _run(mode, ps, nsteps, sample=0):
    s = F.Solver(ps)
    for r, p in enumerate(ps):
        s.set_fields(rep=r, psi=I.random_field(p.nx * p.ny * p.nz, 0.05, 10 + r))
    s.set_mode(mode)
    if sample:
        s.set_sampling(sample, 1)
    s.step(nsteps)
    s.synchronize()
    out = [(s.get_populations(r), s.get_psi_u(r)[0], s.get_step(r)) for r in range(len(ps))]
    sq = [s.structure_factor(r)[0] for r in range(len(ps))] if sample else None
    return out, sq, s


@pytest.mark.parametrize("integrator", [1, 2])
def test_batched_equals_plain(integrator):
    ps = _replicas(integrator=integrator)
    plain, _, _ = _run(F.FLB_MODE_PLAIN, ps, 7)
    batched, _, s = _run(F.FLB_MODE_BATCHED, ps, 7)
    for (fa, pa, sa), (fb, pb, sb) in zip(plain, batched):
        assert sa == sb == 7
        assert np.array_equal(fa, fb)
        assert np.array_equal(pa, pb)
    # a second call continues from the device-side step counter and buffer parity
    s.step(3)
    plain10, _, _ = _run(F.FLB_MODE_PLAIN, ps, 10)
    for r, (fa, pa, _) in enumerate(plain10):
        assert np.array_equal(fa, s.get_populations(r))
        assert np.array_equal(pa, s.get_psi_u(r)[0])


def test_batched_row_packing_of_wide_and_narrow_boxes_equals_plain():
    # the batched collide-stream and velocity work site pairs (z, z+1) and pack
    # 128/nx whole rows of plane pairs per block (nx <= 128, here 4, 5 and 100:
    # rows wrap into the next plane pair inside a block; an odd nz leaves the
    # last pair with one plane) or take 128-pair chunks of a row (nx = 300: two
    # full chunks and a partial one; nx = 129: a full chunk and a 1-pair one);
    # every field must still agree bitwise with the plain launches
    shapes = [(4, 4, 5), (5, 7, 4), (100, 6, 5), (300, 4, 4), (129, 4, 5)]
    ps = [flb_params(dict(dim=3, q=19, nx=nx, ny=ny, nz=nz, tau=0.8, kT=2e-5, A=0.05, B=0.2, K=0.04, M=0.1,
                          scheme=1, integrator=2, seed=300 + r)) for r, (nx, ny, nz) in enumerate(shapes)]
    plain, _, _ = _run(F.FLB_MODE_PLAIN, ps, 5)
    batched, _, _ = _run(F.FLB_MODE_BATCHED, ps, 5)
    for (fa, pa, _), (fb, pb, _) in zip(plain, batched):
        assert np.array_equal(fa, fb)
        assert np.array_equal(pa, pb)


def test_batched_stress_force_equals_plain():
    ps = _replicas(A=-0.05, B=0.3, force_grad=3)
    plain, _, _ = _run(F.FLB_MODE_PLAIN, ps, 6)
    batched, _, _ = _run(F.FLB_MODE_BATCHED, ps, 6)
    for (fa, pa, _), (fb, pb, _) in zip(plain, batched):
        assert np.array_equal(fa, fb)
        assert np.array_equal(pa, pb)


def test_batched_sampling_and_launch_count():
    ps = _replicas(kT=2e-4)
    _, sq_plain, sp = _run(F.FLB_MODE_PLAIN, ps, 12, sample=4)
    _, sq_batch, sb = _run(F.FLB_MODE_BATCHED, ps, 12, sample=4)
    for a, b in zip(sq_plain, sq_batch):
        assert np.array_equal(a, b)
    # the batched step issues 5 kernels for all replicas instead of 4 per replica
    assert sb.launch_count() < sp.launch_count()


def test_batched_rejects_fd():
    ps = _replicas(scheme=0)
    s = F.Solver(ps)
    s.set_mode(F.FLB_MODE_BATCHED)
    with pytest.raises(F.FlbError) as e:
        s.step(1)
    assert e.value.code == F.FLB_EUNSUPPORTED


@pytest.mark.parametrize("integrator,kT", [(1, 1e-4), (2, 1e-4), (2, 0.0)])
def test_batched_d3q15_equals_plain(integrator, kT):
    # D3Q15 replicas (the paper's lattice, Sec. VI), uneven sizes, FV: the batched
    # launches (one site per thread on row-packed lists, the D3Q15 stage
    # operators) against the plain two-sites-per-thread path, bitwise; and again
    # after the step counter and buffer parity have advanced on the device
    ps = _replicas(q=15, integrator=integrator, kT=kT)
    plain, _, _ = _run(F.FLB_MODE_PLAIN, ps, 6)
    batched, _, s = _run(F.FLB_MODE_BATCHED, ps, 6)
    for (fa, pa, sa), (fb, pb, sb) in zip(plain, batched):
        assert sa == sb == 6
        assert np.array_equal(fa, fb)
        assert np.array_equal(pa, pb)
    s.step(3)
    plain9, _, _ = _run(F.FLB_MODE_PLAIN, ps, 9)
    for r, (fa, pa, _) in enumerate(plain9):
        assert np.array_equal(fa, s.get_populations(r))
        assert np.array_equal(pa, s.get_psi_u(r)[0])

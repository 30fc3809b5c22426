"""Persistent batched mode: every replica advanced by one cooperative launch with
per-replica phase barriers.  The per-site arithmetic is that of the plain path,
so every field and spectrum must agree bitwise; a wait that runs out must end
the launch with FLB_ETIMEOUT and leave the context usable."""
import numpy as np
import pytest

import paper_1104_0078_gb300 as F
from paper_1104_0078_gb300 import inputs as I

from gpu_helpers import flb_params

pytestmark = pytest.mark.gpu

SHAPES = [(16, 16, 16), (12, 10, 20), (40, 18, 9), (33, 7, 70), (24, 24, 24)]


def _replicas(**kw):
    ps = []
    for r, (nx, ny, nz) in enumerate(SHAPES):
        d = dict(dim=3, q=19, nx=nx, ny=ny, nz=nz, tau=0.8, kT=1e-5 * (1 + r), A=-0.05, B=0.2, K=0.04, M=0.1,
                 scheme=1, integrator=2, seed=200 + r)
        d.update(kw)
        ps.append(flb_params(d))
    return ps


def _solver(mode, ps, sample=0, chunks=None):
    s = F.Solver(ps)
    for r, p in enumerate(ps):
        s.set_fields(rep=r, psi=I.random_field(p.nx * p.ny * p.nz, 0.1, 30 + r))
        if chunks:
            s.set_tuning(chunks[r], rep=r)
    s.set_mode(mode)
    if sample:
        s.set_sampling(sample, 1)
    return s


def _fields(s, nrep):
    return [(s.get_populations(r), *s.get_psi_u(r), s.get_step(r)) for r in range(nrep)]


def _same(a, b):
    for ra, rb in zip(a, b):
        for x, y in zip(ra, rb):
            assert np.array_equal(x, y)


def test_persistent_row_packing_equals_plain():
    # collide-stream and velocity tasks are row-packed blocks of 2048 sites:
    # narrow boxes pack 2048/nx rows that wrap into the next planes (nx = 4, 5,
    # 100), a box wider than 2048 takes chunks of a row (nx = 2100: a full and a
    # partial chunk)
    shapes = [(4, 4, 5), (5, 7, 4), (100, 6, 5), (2100, 4, 4)]
    ps = [flb_params(dict(dim=3, q=19, nx=nx, ny=ny, nz=nz, tau=0.8, kT=2e-5, A=0.05, B=0.2, K=0.04, M=0.1,
                          scheme=1, integrator=2, seed=400 + r)) for r, (nx, ny, nz) in enumerate(shapes)]
    out = {}
    for mode in (F.FLB_MODE_PLAIN, F.FLB_MODE_PERSISTENT):
        s = _solver(mode, ps)
        s.step(5)
        s.synchronize()
        out[mode] = _fields(s, len(ps))
    _same(out[F.FLB_MODE_PLAIN], out[F.FLB_MODE_PERSISTENT])


@pytest.mark.parametrize("integrator", [1, 2])
def test_persistent_equals_plain(integrator):
    ps = _replicas(integrator=integrator)
    plain = _solver(F.FLB_MODE_PLAIN, ps, sample=4)
    pers = _solver(F.FLB_MODE_PERSISTENT, ps, sample=4)
    for n in (7, 3, 1):
        plain.step(n)
        pers.step(n)
        pers.synchronize()
        _same(_fields(plain, len(ps)), _fields(pers, len(ps)))
    for r in range(len(ps)):
        sa, na = plain.structure_factor(r)
        sb, nb = pers.structure_factor(r)
        assert na == nb == 2 and np.array_equal(sa, sb)
    tp, u2p, _ = plain.moments(0)
    tq, u2q, rc = pers.moments(0)
    assert rc == F.FLB_OK and np.array_equal(tp, tq) and np.array_equal(u2p, u2q)


def test_persistent_mixed_zchunks_and_coupling():
    ps = _replicas()
    ps[1].coupling = F.FLB_COUPLE_ADVECT     # a replica without force: no mu tasks
    ps[2].gamma_ghost = 0.3                  # ghost relaxation path
    ps[3].force_grad = F.FLB_FORCE_STRESS    # stress-form force: sigma instead of mu
    chunks = [4, 7, 64, 16, 3]
    plain = _solver(F.FLB_MODE_PLAIN, ps)
    pers = _solver(F.FLB_MODE_PERSISTENT, ps, chunks=chunks)
    plain.step(9)
    pers.step(9)
    _same(_fields(plain, len(ps)), _fields(pers, len(ps)))


def test_persistent_wait_that_runs_out():
    ps = _replicas()
    s = _solver(F.FLB_MODE_PERSISTENT, ps)
    s.set_wait_limit(0.0)                    # every wait not met at the first poll gives up
    s.step(20)
    with pytest.raises(F.FlbError) as e:
        s.synchronize()
    assert e.value.code == F.FLB_ETIMEOUT
    # the context stays usable: restarted from a checkpoint it steps on as the plain path does
    s.set_wait_limit(1.0)
    ref = _solver(F.FLB_MODE_PLAIN, ps)
    for r in range(len(ps)):
        s.set_state(ref.get_state(r), rep=r)
    s.step(5)
    ref.step(5)
    s.synchronize()
    a, b = _fields(s, len(ps)), _fields(ref, len(ps))
    _same(a, b)


def test_persistent_unsupported_configurations():
    for kw in (dict(storage=F.FLB_F16_DEV), dict(scheme=0), dict(integrator=4)):
        s = _solver(F.FLB_MODE_PERSISTENT, _replicas(**kw))
        with pytest.raises(F.FlbError) as e:
            s.step(1)
        assert e.value.code == F.FLB_EUNSUPPORTED


@pytest.mark.parametrize("kT", [0.0, 1e-4])
def test_persistent_d3q15_equals_plain(kT):
    # D3Q15 replicas (the paper's lattice, Sec. VI): the persistent launch runs
    # their collide-stream and velocity one site per thread and the FV stage with
    # the D3Q15 operators; the plain path runs two sites per thread in packed
    # FP32.  The per-site arithmetic is the same lane-generic code, so every
    # field, spectrum and total agrees bitwise
    ps = _replicas(q=15, kT=kT)
    plain = _solver(F.FLB_MODE_PLAIN, ps, sample=4)
    pers = _solver(F.FLB_MODE_PERSISTENT, ps, sample=4)
    for n in (5, 4):
        plain.step(n)
        pers.step(n)
        pers.synchronize()
        _same(_fields(plain, len(ps)), _fields(pers, len(ps)))
    for r in range(len(ps)):
        sa, na = plain.structure_factor(r)
        sb, nb = pers.structure_factor(r)
        assert na == nb == 2 and np.array_equal(sa, sb)

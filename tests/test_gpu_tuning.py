"""The psi z chunk (planes per psi block) and its autotuner.  The chunk is a tiling
knob: every site's arithmetic is the same whatever its value, so every field
must agree bitwise; the autotuner must leave the state untouched and honour its
cache file."""
import numpy as np
import pytest

import paper_1104_0078_gb300 as F
from paper_1104_0078_gb300 import inputs as I

from gpu_helpers import flb_params, weights_column

pytestmark = pytest.mark.gpu

RAGGED = dict(dim=3, q=19, nx=37, ny=23, nz=19, tau=0.8, kT=1e-4, A=-0.05, B=0.3, K=0.04, M=0.1, integrator=2,
              coupling=3, seed=3)


def _start(s, d, rep=0):
    N = d["nx"] * d["ny"] * d["nz"]
    s.set_fields(rep=rep, psi=I.random_field(N, 0.05, 8 + rep))
    s.set_populations(weights_column(d["q"]) + I.random_deviations(d["q"], N, 2e-3, 7 + rep), rep=rep)


def _fields(s, rep=0):
    psi, u = s.get_psi_u(rep)
    return s.get_populations(rep), psi, u


@pytest.mark.parametrize("q,scheme", [(19, 0), (19, 1), (15, 1)])
def test_zchunk_changes_no_bit(q, scheme):
    d = dict(RAGGED, q=q, scheme=scheme)
    ref = None
    for zc in (64, 1, 3, 8, 19):
        s = F.Solver(flb_params(d))
        _start(s, d)
        s.set_tuning(zc)
        assert s.get_tuning(0) == zc
        s.step(12)
        out = _fields(s)
        if ref is None:
            ref = out
        else:
            for a, b in zip(ref, out):
                assert np.array_equal(a, b), zc


def test_batched_with_mixed_zchunks_equals_plain():
    shapes = [(16, 16, 16), (12, 10, 20), (40, 18, 9), (33, 7, 70)]
    ds = [dict(RAGGED, nx=nx, ny=ny, nz=nz, scheme=1, kT=1e-5 * (1 + r), seed=100 + r)
          for r, (nx, ny, nz) in enumerate(shapes)]
    ps = [flb_params(d) for d in ds]
    runs = []
    for mode, chunks in ((F.FLB_MODE_PLAIN, (64, 64, 64, 64)), (F.FLB_MODE_BATCHED, (4, 7, 64, 16))):
        s = F.Solver(ps)
        for r, d in enumerate(ds):
            _start(s, d, r)
            s.set_tuning(chunks[r], rep=r)
        s.set_mode(mode)
        s.step(6)
        s.set_tuning(5, rep=3)              # a change between calls rebuilds the batched graph
        s.step(3)
        runs.append([_fields(s, r) for r in range(len(ps))])
    for ra, rb in zip(*runs):
        for a, b in zip(ra, rb):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("mode", [0, 1])
def test_autotune_keeps_state_and_uses_cache(tmp_path, mode):
    cache = str(tmp_path / "tune.txt")
    d = dict(RAGGED, scheme=1)
    ps = [flb_params(d), flb_params(dict(d, nx=20, ny=20, nz=40, seed=9))]
    s = F.Solver(ps)
    for r in range(2):
        _start(s, dict(d, nx=ps[r].nx, ny=ps[r].ny, nz=ps[r].nz), r)
    s.set_mode(mode)
    s.step(2)
    before = [_fields(s, r) for r in range(2)] + [s.get_step(0)]
    chosen = s.autotune(cache=cache)
    after = [_fields(s, r) for r in range(2)] + [s.get_step(0)]
    for a, b in zip(before[:2], after[:2]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    assert before[2] == after[2] == 2
    lines = open(cache).read().splitlines()
    if mode == F.FLB_MODE_BATCHED:
        # one shared value, then one per box depth: a listed value or an even split ceil(nz / k)
        for c, p in zip(chosen, ps):
            assert c in (4, 8, 16, 32, 64) or any(c == -(-p.nz // k) for k in range(1, 17))
        assert len(lines) == 1 + len({p.nz for p in ps})
    else:
        assert all(c in (4, 8, 16, 32, 64) for c in chosen)
        assert len(lines) == 2
    # a second handle of the same configuration takes the cached values without timing
    s2 = F.Solver(ps)
    s2.set_mode(mode)
    assert s2.autotune(cache=cache) == chosen
    assert open(cache).read().splitlines() == lines
    # forcing re-times and appends; the state still steps on identically
    s2.autotune(cache=cache, force=True)
    assert len(open(cache).read().splitlines()) == 2 * len(lines)
    s.step(3)
    ref = F.Solver(ps)
    for r in range(2):
        _start(ref, dict(d, nx=ps[r].nx, ny=ps[r].ny, nz=ps[r].nz), r)
    ref.step(5)
    for r in range(2):
        for x, y in zip(_fields(s, r), _fields(ref, r)):
            assert np.array_equal(x, y)


def test_tuning_argument_checks():
    s = F.Solver(flb_params(dict(RAGGED, scheme=1)))
    for bad in (0, -3, 5000):
        with pytest.raises(F.FlbError):
            s.set_tuning(bad)
    with pytest.raises(F.FlbError):
        s.set_tuning(8, rep=3)

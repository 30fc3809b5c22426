"""The allocation-free structure factor, flb_structure_factor_noalloc().

It exists for callers that cannot allocate device memory where they want a
spectrum; its DFT intermediates live in a fixed device array of the library.
This file is collected last on purpose: it runs after every other test in the
same process (the shared array then already holds earlier contents) and also
passes alone in a fresh process.  Each case compares two calls in a row with the
handle-based path (flb_sample + flb_structure_factor) on the same field."""
import ctypes

import numpy as np
import pytest

import paper_1104_0078_gb300 as F
from paper_1104_0078_gb300 import inputs as I

pytestmark = pytest.mark.gpu

RTOL = 1e-4   # the structure-factor tolerance of the other GPU tests


def _noalloc(psi_t, shape, kmax, S_t, stream):
    nz, ny, nx = shape
    return F.load_library().flb_structure_factor_noalloc(
        ctypes.c_void_p(psi_t.data_ptr()), nx, ny, nz, kmax, ctypes.c_void_p(S_t.data_ptr()),
        ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("shape,kmax", [((16, 20, 24), 0), ((12, 16, 16), 3), ((1, 30, 40), 0)])
def test_noalloc_matches_handle_path_twice(shape, kmax):
    import torch
    nz, ny, nx = shape
    dim = 2 if nz == 1 else 3
    p = F.flb_params_default(dim=dim, q=9 if dim == 2 else 19, nx=nx, ny=ny, nz=nz, sq_kmax=kmax)
    psi0 = I.random_field(nx * ny * nz, 0.3, 17)
    s = F.Solver(p)
    s.set_fields(psi=psi0)
    s.sample(1)
    ref, ns = s.structure_factor()
    assert ns == 1
    psi_t = torch.tensor(psi0, dtype=torch.float32, device="cuda:0")
    S_t = torch.full((ref.size,), -1.0, dtype=torch.float64, device="cuda:0")
    st = torch.cuda.Stream()
    for _ in range(2):
        assert _noalloc(psi_t, shape, kmax, S_t, st) == F.FLB_OK
        st.synchronize()
        got = S_t.cpu().numpy()
        assert np.allclose(got, ref, rtol=RTOL, atol=1e-12 * ref.max())
        S_t.fill_(-1.0)


def test_noalloc_rejects_oversize_and_bad_arguments():
    import torch
    st = torch.cuda.Stream()
    big = torch.zeros(128 ** 3, dtype=torch.float32, device="cuda:0")
    out = torch.zeros(128 ** 3, dtype=torch.float64, device="cuda:0")
    assert _noalloc(big, (128, 128, 128), 0, out, st) == F.FLB_ENOSPC
    st.synchronize()
    lib = F.load_library()
    assert lib.flb_structure_factor_noalloc(None, 4, 4, 4, 0, ctypes.c_void_p(out.data_ptr()), None) == F.FLB_EINVAL
    assert _noalloc(big, (128, 128, 128), -1, out, st) == F.FLB_EINVAL


def test_noalloc_near_limit_window_matches_handle_path():
    """The largest accepted layout: 128^3 with kmax = 15 fills Kx*ny*nz =
    507,904 of the 524,288 scratch values; its values are compared twice with
    the handle path on the same field."""
    import torch
    n, kmax = 128, 15
    p = F.flb_params_default(nx=n, ny=n, nz=n, sq_kmax=kmax)
    psi0 = I.random_field(n ** 3, 0.3, 23)
    s = F.Solver(p)
    s.set_fields(psi=psi0)
    s.sample(1)
    ref, ns = s.structure_factor()
    assert ns == 1 and ref.size == (2 * kmax + 1) ** 3
    del s
    psi_t = torch.tensor(psi0, dtype=torch.float32, device="cuda:0")
    S_t = torch.full((ref.size,), -1.0, dtype=torch.float64, device="cuda:0")
    st = torch.cuda.Stream()
    for _ in range(2):
        assert _noalloc(psi_t, (n, n, n), kmax, S_t, st) == F.FLB_OK
        st.synchronize()
        got = S_t.cpu().numpy()
        assert np.allclose(got, ref, rtol=RTOL, atol=1e-12 * ref.max())
        S_t.fill_(-1.0)

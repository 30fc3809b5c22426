"""The device normals against the oracle's generator, value by value: the same
Philox4x32-10 words (bit-exact integer work) and Box-Muller in FP32 on the
device (radius by table-driven ln u, angle by table and angle addition) against
FP64 in the oracle."""
import numpy as np
import pytest

import oracle as O
import paper_1104_0078_gb300 as F

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,step,stream,site0", [(1, 0, 0, 0), (0x1234ABCD5678EF01, 987654321012, 1, 4000000000),
                                                    (7, -3, 0xFFFF, 123456789)])
def test_device_normals_match_oracle(seed, step, stream, site0):
    n, nb = 40000, 4
    g = F.gaussians(seed, step, stream, site0, n, nb).cpu().numpy().astype(np.float64)
    ref = np.stack([O.gaussians(seed, step, (site0 + i) & 0xFFFFFFFF, stream, nb) for i in range(n)])
    err = np.abs(g - ref)
    # FP32 evaluation: a few units in the last place of the radius and the angle
    assert np.all(err <= 1e-6 * np.maximum(1.0, np.abs(ref))), err.max()
    assert err.mean() < 1e-7
    # the sample is a standard normal sample
    assert abs(ref.mean()) < 5 / np.sqrt(ref.size) and abs(ref.var() - 1) < 0.01


def test_device_normals_argument_checks():
    import torch
    lib = F.load_library()
    buf = torch.empty(64, device="cuda")
    assert lib.flb_gaussians(1, 0, 0, 0, 4, 0, buf.data_ptr(), None) == F.FLB_EINVAL
    assert lib.flb_gaussians(1, 0, 0x10000, 0, 4, 1, buf.data_ptr(), None) == F.FLB_EINVAL
    assert lib.flb_gaussians(1, 0, 0, 0xFFFFFFFF, 4, 1, buf.data_ptr(), None) == F.FLB_EINVAL
    assert lib.flb_gaussians(1, 0, 0, 0, 4, 1, None, None) == F.FLB_EINVAL
    assert lib.flb_gaussians(1, 0, 0, 0, 0, 1, buf.data_ptr(), None) == F.FLB_OK


def test_device_normals_moments_and_tails_1e8():
    """10^8 device normals (6.25e6 sites x 16, one LB stream): mean 0, variance 1,
    skewness 0 and kurtosis 3 within 5 sigma of their sampling errors, and the
    frequencies of |z| > 3, 4, 5 within 5 sigma of the normal law's.  The tails
    come from the smallest radius uniforms (u down to 2^-21, |z| <= 5.40), where
    the table-driven ln u works on the lowest cells."""
    import math
    import torch
    nsites, nb = 6_250_000, 2
    g = F.gaussians(20240601, 12345, 0, 7, nsites, nb).double().flatten()
    n = g.numel()
    assert n == 100_000_000 and bool(torch.isfinite(g).all())
    m1 = g.mean().item()
    c = g - m1
    m2 = (c * c).mean().item()
    m3 = (c * c * c).mean().item() / m2**1.5
    m4 = ((c * c) ** 2).mean().item() / m2**2
    assert abs(m1) < 5 * math.sqrt(1 / n), m1
    assert abs(m2 - 1) < 5 * math.sqrt(2 / n), m2
    assert abs(m3) < 5 * math.sqrt(6 / n), m3
    assert abs(m4 - 3) < 5 * math.sqrt(24 / n), m4
    a = g.abs()
    for t in (3.0, 4.0, 5.0):
        p = math.erfc(t / math.sqrt(2))  # P(|z| > t)
        k = int((a > t).sum().item())
        assert abs(k - n * p) < 5 * math.sqrt(n * p * (1 - p)) + 1, (t, k, n * p)
    # 20-bit radius uniforms, u >= 2^-21, bound the draws by sqrt(42 ln 2) = 5.396
    assert a.max().item() <= math.sqrt(42 * math.log(2)) + 1e-5

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

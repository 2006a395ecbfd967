"""The allocation-free matvec entry point (mb_mobility_matvec_noalloc).

It serves callers that cannot allocate device memory: applications whose
framework owns the whole device-memory budget, and latency-critical code
that cannot take cudaMalloc's implicit synchronisation.  Its scratch is a
fixed device array inside the library.  These tests call it through the C
ABI and check it against the regular entry point, mb_mobility_matvec with
MB_FP32_KAHAN, within the FP32 matvec tolerance the other tests use (1e-5).
The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest
import torch

import paper_1602_02170_gb300 as mb
from paper_1602_02170_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _rel(got, ref):
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def test_noalloc_matches_regular_entry_point_twice():
    """Two calls in a row (different sizes, with and without the wall) agree
    with the regular entry point, and the second call leaves the device's
    free memory unchanged."""
    r1, f1, a = I.config_matvec_cloud(21, n=mb.NOALLOC_MAX_BLOBS)
    r2, f2 = I.blob_cloud(22, 5000, 0.5, 60.0, 0.5, 1.5)
    cases = [(r1, f1, a, True), (r2, f2, 0.5, False)]
    dev = [(torch.from_numpy(r).cuda(), torch.from_numpy(f).cuda(), a, w) for r, f, a, w in cases]
    with mb.Context(0) as ctx:
        refs = [ctx.mobility_matvec(r, f, a, 1.0, w, "fp32").cpu().numpy() for r, f, a, w in dev]
    outs = [torch.empty_like(r) for r, _, _, _ in dev]
    torch.cuda.synchronize()
    got = []
    for k, ((r, f, a, w), out) in enumerate(zip(dev, outs)):
        free_before = torch.cuda.mem_get_info()[0]
        mb.mobility_matvec_noalloc(r, f, a, 1.0, w, out=out)
        torch.cuda.synchronize()
        if k > 0:  # the first call on a device may load the library's module
            assert torch.cuda.mem_get_info()[0] == free_before
        got.append(out.cpu().numpy())
    for g, ref in zip(got, refs):
        assert np.isfinite(g).all()
        assert _rel(g, ref) <= TOL
        assert np.abs(g - ref).max() <= TOL * np.abs(ref).max()


def test_noalloc_rejects_sizes_above_its_maximum():
    n = mb.NOALLOC_MAX_BLOBS + 1
    r = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(mb.MBError) as ei:
        mb.mobility_matvec_noalloc(r, r, 0.5, out=torch.empty_like(r))
    assert ei.value.name == "MB_EINVAL"
    assert "MB_NOALLOC_MAX_BLOBS" in str(ei.value)

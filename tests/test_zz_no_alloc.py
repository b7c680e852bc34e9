"""The allocation-free orthonormalisation, for callers that cannot allocate
device memory when they need the step.  Its result must equal that of
lrs_orthonormalize, which allocates its scratch per call, on two calls in a
row (the second call reuses the shared scratch the first one left behind).

Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

from tests.gpu_helpers import gpu_available

pytestmark = pytest.mark.gpu


def test_noalloc_orthonormalize_matches_allocating_call_twice():
    if not gpu_available():
        pytest.skip("no CUDA device")
    import torch
    from paper_2311_03824_gb300 import build
    build.build()
    from paper_2311_03824_gb300 import lrs as L
    rng = np.random.default_rng(2024)
    for n, r in [(1000, 5), (4096, 10)]:           # two calls in a row
        Z = torch.from_numpy(rng.standard_normal((n, r)).astype(np.float32)).cuda()
        Q_ref = torch.empty_like(Z)
        Q_na = torch.full_like(Z, float("nan"))
        L.lrs_orthonormalize(Z, Q_ref)
        L.lrs_orthonormalize_noalloc(Z, Q_na)
        torch.cuda.synchronize()
        diff = (Q_na - Q_ref).abs().max().item()
        assert diff <= 2e-5, (n, r, diff)
        QtQ = (Q_na.double().T @ Q_na.double()).cpu().numpy()
        assert np.abs(QtQ - np.eye(r)).max() < 1e-5


def test_noalloc_rejects_sizes_beyond_its_scratch():
    if not gpu_available():
        pytest.skip("no CUDA device")
    import torch
    from paper_2311_03824_gb300 import lrs as L
    Z = torch.zeros((65537, 2), device="cuda")
    with pytest.raises(L.LrsError) as e:
        L.lrs_orthonormalize_noalloc(Z, Z)
    assert e.value.status == L.LRS_ERR_ARG
    assert "65536" in str(e.value)

"""lrs_orthonormalize (the QR step of Algorithm 1) against numpy's Householder
QR with the signs of diag(R) made positive."""
import numpy as np
import pytest

import oracle.altgdmin_lrs as O
from tests.gpu_helpers import gpu_available

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,r", [(1000, 5), (4096, 10), (17, 16), (300, 1)])
def test_orthonormalize_matches_positive_qr(n, r):
    if not gpu_available():
        pytest.skip("no CUDA device")
    import torch
    from paper_2311_03824_gb300 import lrs as L
    Z = np.random.default_rng(n + r).standard_normal((n, r)).astype(np.float32)
    Zd = torch.from_numpy(Z).cuda()
    Qd = torch.empty_like(Zd)
    L.lrs_orthonormalize(Zd, Qd)
    Q = Qd.cpu().numpy().astype(np.float64)
    Qo, _ = O.qr_positive(Z.astype(np.float64))
    assert np.abs(Q - Qo).max() < 2e-5
    assert np.abs(Q.T @ Q - np.eye(r)).max() < 1e-5

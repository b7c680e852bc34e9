"""The numerics the task engine's small steps rely on, checked on the CPU in
numpy (no GPU): an FP32 Cholesky inverse of the r x r Gram W^T W refined by
one FP64 Newton-Schulz step X <- X (2I - G X) reaches the FP64 inverse to
about (cond(G) * 1e-7)^2, far below the float32 resolution the solver
works at, for the Gram matrices of W = A_k U with m >= r; and the residual
update A s_new = A s - mu A g_G on a support that HardThreshold keeps."""
import numpy as np
import pytest


def chol_inverse_fp32(G):
    """G^{-1} from a float32 Cholesky (row by row, as the kernel does)."""
    r = G.shape[0]
    Gf = G.astype(np.float32)
    L = np.zeros((r, r), np.float32)
    for j in range(r):
        s = Gf[j, j] - np.float32(np.dot(L[j, :j], L[j, :j]))
        assert s > 1e-5 * Gf[j, j]
        ij = np.float32(1.0) / np.sqrt(s, dtype=np.float32)
        L[j, j] = s * ij
        for i in range(j + 1, r):
            L[i, j] = (Gf[i, j] - np.float32(np.dot(L[i, :j], L[j, :j]))) * ij
    Li = np.linalg.inv(L.astype(np.float64)).astype(np.float32)   # the triangular inverse
    return (Li.T @ Li).astype(np.float32)


def newton_schulz(G, X0):
    X0 = X0.astype(np.float64)
    return 2.0 * X0 - X0 @ (G @ X0)


@pytest.mark.parametrize("m,r,seed", [(150, 5, 0), (512, 10, 1), (48, 16, 2), (24, 1, 3),
                                      (40, 8, 4), (80, 3, 5)])
def test_one_newton_schulz_step_squares_the_fp32_error(m, r, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, 3 * r + 7)).astype(np.float32)
    U, _ = np.linalg.qr(rng.standard_normal((A.shape[1], r)))
    W = (A.astype(np.float64) @ U).astype(np.float32)
    G = (W.T.astype(np.float32) @ W.astype(np.float32)).astype(np.float64)   # the FP32 Gram
    exact = np.linalg.inv(G)
    cond = np.linalg.cond(G)
    X0 = chol_inverse_fp32(G)
    e0 = np.linalg.norm(X0 - exact) / np.linalg.norm(exact)
    X1 = newton_schulz(G, X0)
    e1 = np.linalg.norm(X1 - exact) / np.linalg.norm(exact)
    assert e0 < 50 * cond * 6e-8                     # the FP32 inverse: ~cond * eps32
    assert e1 < max(10 * e0 * e0 * cond, 1e-13)      # one step squares it (up to cond)
    assert e1 < 1e-9                                 # far below float32 resolution


def test_residual_update_on_a_kept_support_matches_the_gather():
    """The task engine's residual shortcut: when HardThreshold keeps the
    support G, the new values are s - mu g on G, so A s_new = A s - mu A g_G.
    Checked on a noiseless instance through the oracle's own IHT sweeps
    (HardThreshold of s - mu g with the support-restricted mu of Algorithm 2):
    wherever a sweep keeps the support, the update equals the direct product."""
    import oracle.altgdmin_lrs as O
    rng = np.random.default_rng(7)
    m, n, rho = 60, 120, 4
    A = rng.standard_normal((m, n))
    x = np.zeros(n)
    x[rng.choice(n, rho, replace=False)] = rng.uniform(1, 10, rho) * rng.choice([-1, 1], rho)
    y = A @ x
    s = np.zeros(n)
    idx = O.hard_threshold((A.T @ -y)[None], rho)[0][0]        # zero start, as Algorithm 2
    kept = 0
    for _ in range(12):
        g = A.T @ (A @ s - y)
        gG = np.zeros(n)
        gG[idx] = g[idx]
        mu = np.dot(gG, gG) / np.dot(A @ gG, A @ gG)
        idx_new, vals, _ = O.hard_threshold((s - mu * g)[None], rho)
        s_new = O.densify(idx_new, vals, n)[0]
        if set(idx_new[0]) == set(idx) and np.any(s):
            kept += 1
            np.testing.assert_allclose(A @ s - mu * (A @ gG), A @ s_new, rtol=1e-12, atol=1e-12)
        s, idx = s_new, idx_new[0]
    assert kept >= 5

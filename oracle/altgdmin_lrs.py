"""FP64 CPU oracle for AltGDmin-LR+S (Babu & Vaswani, "A Fast Algorithm for Low
Rank + Sparse column-wise Compressive Sensing", arXiv 2311.03824).

TEST INFRASTRUCTURE.  This module exists to check the CUDA solver.  Only the
tests, the smoke check and the benchmark's CPU-baseline leg may import or run
it; the solver library never does, and the two share no code.

It follows Algorithm 1 (AltGDmin-L+S) and Algorithm 2 (IHT) step by step, in
the paper's order and notation, with every linear-algebra step done the plain,
definitional way in float64 (numpy library primitives: matmul, SVD-based
pseudo-inverse, Householder QR, SVD, FFT).  Work that is independent across
columns k (the "for k in [q]" steps of Algorithm 1) is written as one
batched numpy expression over k; nothing is reordered beyond that.

Readings taken where the paper is silent or garbled (each is listed with its
reason in the design notes of this repository):
  * IHT step size (Algorithm 2, normalised IHT of Blumensath & Davies):
    mu = ||g_G||^2 / ||M g_G||^2, with g = M^T (M s - z) and g_G its
    restriction to the current support G (the support kept by the previous
    HardThreshold; for the all-zero start, the rho largest |g_i|).  The printed
    ratio of unsquared full-gradient norms is not invariant to scaling
    (A, y) -> (cA, cy) and diverges on the paper's Gaussian setting; the
    squared full-gradient ratio (`mu_rule="full"`) stalls far from the
    solution; the support-restricted step converges to the float32 floor on
    the Fig. 1 setting, as the paper reports.  `mu_rule="printed"` and
    `mu_rule="full"` keep the other two forms for the record.
  * A column whose ||M g|| is exactly 0 stops its IHT loop (s unchanged).
  * HardThreshold keeps exactly rho entries; ties in magnitude go to the lower
    index; the kept indices are reported ascending.
  * Gradient: the paper's grad_U f = sum_k A_k^T (A_k(U b_k + s_k) - y_k) b_k^T
    (Section II-A), i.e. half the derivative of f; eta = c_eta / ||grad||_2
    (spectral norm, Section I-A notation) from the t = 1 gradient, then frozen.
  * QR: Q factor of the Householder QR with the signs fixed so diag(R) > 0.
  * Output iterate after iteration t: X_t = U_t B_t + S_t with U_t taken after
    that iteration's QR (Algorithm 1, Output).
  * Complex (Fourier) data: transpose becomes conjugate transpose, |.| is the
    modulus, the 2D DFT is unitary (norm="ortho") in natural index order.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


# ------------------------------------------------------------ operators --

class GaussianOperator:
    """A_k dense m x n (float64 copies of the stored float32 values).

    dtype: the arithmetic of every step that uses this operator (float64 for
    the oracle; float32 only for studies of what float32 arithmetic can
    resolve, never for a parity reference)."""

    def __init__(self, A, dtype=np.float64):
        self.dtype = np.dtype(dtype)
        self.M = np.asarray(A, dtype=self.dtype)          # (q, m, n)
        self.q, self.m, self.n = self.M.shape
        self.complex = False

    def subset(self, ks):
        return GaussianOperator(self.M[ks], self.dtype)

    def A(self, X):                 # X: (q, n) -> (q, m): A_k x_k
        return (self.M @ X[:, :, None])[:, :, 0]

    def AH(self, V):                # V: (q, m) -> (q, n): A_k^T v_k
        return (V[:, None, :] @ self.M)[:, 0, :]

    def AU(self, U):                # U: (n, r) -> (q, m, r): A_k U
        return self.M @ U

    def explicit(self):
        return self.M


class FourierOperator:
    """A_k x = (F2 x)[Omega_k], F2 the unitary 2D DFT of an nx x ny frame.

    Section I-A: A_k is a random subset of rows of the (2D) DFT matrix.
    The adjoint is A_k^H v = F2^H(zero-fill_k v).  Rows are indexed
    kx*ny + ky in natural (unshifted) order.
    """

    def __init__(self, masks, nx, ny, dtype=np.complex128):
        self.masks = np.asarray(masks, dtype=np.int64)   # (q, m)
        self.nx, self.ny = nx, ny
        self.q, self.m = self.masks.shape
        self.n = nx * ny
        self.complex = True
        self.dtype = np.dtype(dtype)    # complex128; complex64 only for float32 studies

    def subset(self, ks):
        return FourierOperator(self.masks[ks], self.nx, self.ny, self.dtype)

    def _fft(self, X):              # (..., n) -> (..., n)
        sh = X.shape[:-1]
        F = np.fft.fft2(X.reshape(sh + (self.nx, self.ny)), norm="ortho")
        return F.reshape(sh + (self.n,))

    def _ifft(self, X):
        sh = X.shape[:-1]
        F = np.fft.ifft2(X.reshape(sh + (self.nx, self.ny)), norm="ortho")
        return F.reshape(sh + (self.n,))

    def A(self, X):
        return np.take_along_axis(self._fft(X.astype(self.dtype)), self.masks, axis=1)

    def AH(self, V):
        Z = np.zeros((V.shape[0], self.n), dtype=self.dtype)
        np.put_along_axis(Z, self.masks, V, axis=1)
        return self._ifft(Z)

    def AU(self, U):
        FU = self._fft(U.T.astype(self.dtype))             # (r, n): F2 u_j
        return np.stack([FU[:, mk].T for mk in self.masks])  # (q, m, r)

    def explicit(self):
        """Dense A_k (small frames only): rows of the unitary 2D DFT matrix."""
        E = self._fft(np.eye(self.n, dtype=np.complex128))   # row i = F2 e_i
        F2 = E.T                                              # F2[:, i] = F2 e_i
        return np.stack([F2[mk, :] for mk in self.masks])


# ----------------------------------------------------------- primitives --

def hard_threshold(V, rho):
    """HardThreshold(v, rho) (Algorithm 2): keep the rho largest |v_i|.

    Ties in |v| go to the lower index (stable sort on -|v|).  Returns
    (idx ascending (K, rho), values (K, rho), margin (K,)), where
    margin = (|v|_(rho) - |v|_(rho+1)) / max|v| is the gap that decides the
    support (inf when rho = n, nan when v = 0).
    """
    V = np.atleast_2d(V)
    K, n = V.shape
    a = np.abs(V)
    order = np.argsort(-a, axis=1, kind="stable")
    keep = np.sort(order[:, :rho], axis=1)
    vals = np.take_along_axis(V, keep, axis=1)
    margin = np.full(K, np.inf)
    if 0 < rho < n:
        amax = a.max(axis=1)
        r_in = np.take_along_axis(a, order[:, rho - 1:rho], axis=1)[:, 0]
        r_out = np.take_along_axis(a, order[:, rho:rho + 1], axis=1)[:, 0]
        with np.errstate(invalid="ignore", divide="ignore"):
            margin = (r_in - r_out) / amax
    return keep, vals, margin


def densify(idx, vals, n):
    K = idx.shape[0]
    S = np.zeros((K, n), dtype=vals.dtype if vals.size else np.float64)
    if idx.size:
        np.put_along_axis(S, idx, vals, axis=1)
    return S


def iht(z, M, MH, rho, tau, s0, mu_rule="support", idx0=None, perturb=None):
    """Algorithm 2 (IHT), batched over columns.

    z: (K, m); M(s) -> (K, m) and MH(u) -> (K, n) apply M_k and M_k^H;
    s0: (K, n) dense start whose support is idx0 (K, rho) (None: s0 = 0).
    For t = 1..tau: g = M^H(M s - z) (the gradient of ||M s - z||^2 up to the
    factor 2, which cancels in mu g); mu = ||g_G||^2 / ||M g_G||^2 on the
    current support G; s <- HardThreshold(s - mu g, rho).
    Returns (s (K, n), support (K, rho) ascending, margin (K,)) where margin is
    the smallest HardThreshold margin of the column over the sweeps (the gap
    that any arithmetic must resolve to reproduce the supports).
    perturb: None, or a function applied to v = s - mu g before each
    HardThreshold.  It is a test aid only (a relative perturbation of
    rounding size shows whether a column's sweeps amplify rounding); every
    plain run leaves it None.
    """
    s = np.array(s0, copy=True)
    K, n = s.shape
    margin = np.full(K, np.inf)
    idx_cur = None if idx0 is None else np.array(idx0, copy=True)
    for _ in range(tau):
        g = MH(M(s) - z)
        if mu_rule == "support":
            G = idx_cur if idx_cur is not None else hard_threshold(g, rho)[0]
            gG = np.zeros_like(g)
            np.put_along_axis(gG, G, np.take_along_axis(g, G, axis=1), axis=1)
        else:
            gG = g
        num = np.sum(np.abs(gG) ** 2, axis=1)
        den = np.sum(np.abs(M(gG)) ** 2, axis=1)
        active = den > 0
        if idx_cur is None:
            idx_cur = np.tile(np.arange(rho, dtype=np.int64), (K, 1))
        if not np.any(active):
            break
        mu = np.zeros(K, dtype=num.dtype)
        if mu_rule == "printed":        # literal ||g|| / ||M g||
            mu[active] = np.sqrt(num[active]) / np.sqrt(den[active])
        else:
            mu[active] = num[active] / den[active]
        v = s - mu[:, None] * g
        if perturb is not None:
            v = perturb(v)
        idx, vals, mg = hard_threshold(v, rho)
        s_new = densify(idx, vals, n)
        s[active] = s_new[active]
        idx_cur[active] = idx[active]
        margin[active] = np.minimum(margin[active], mg[active])
    if idx_cur is None:
        idx_cur = np.tile(np.arange(rho, dtype=np.int64), (K, 1))
    return s, idx_cur, margin


def pinv_apply(W, V):
    """(A_k U)^dagger v_k via the SVD pseudo-inverse (Eq. bk_LS)."""
    return np.einsum("krm,km->kr", np.linalg.pinv(W), V)


def projector_perp(W):
    """P_perp_k = I - W_k W_k^dagger (explicit m x m, Section II-B)."""
    K, m, _ = W.shape
    P = np.einsum("kmr,krj->kmj", W, np.linalg.pinv(W))
    return np.eye(m)[None] - P


def gradient_U(op, U, B, S, Y):
    """grad_U f = sum_k A_k^H (A_k(U b_k + s_k) - y_k) b_k^H (Section II-A)."""
    X = (U @ B).T + S                       # (q, n): x_k = U b_k + s_k
    R = op.A(X) - Y                         # (q, m)
    H = op.AH(R)                            # (q, n)
    return H.T @ B.conj().T                 # (n, r)


def qr_positive(Z):
    """Q factor of the Householder QR of Z with diag(R) made real positive."""
    Q, R = np.linalg.qr(Z)
    d = np.diag(R)
    ph = np.where(np.abs(d) > 0, d / np.abs(d), 1.0)
    return Q * ph.conj()[None, :], R * ph.conj()[:, None]


def top_r_left(L0, r):
    """Top-r left singular vectors of L0 (n x q), by the full SVD."""
    Uf, sv, _ = np.linalg.svd(L0, full_matrices=False)
    return Uf[:, :r], sv


def rank_count(n, q, m):
    """How many leading singular values of L0 the automatic rank looks at
    (Section II-F, parameter setting): the first min(n/10, q/10, m/10), taken
    as floor(min(n, q, m) / 10) and at least one."""
    return max(1, min(n, q, m) // 10)


def rank_from_singular_values(sv, N, energy=0.65):
    """The b% energy threshold (Section II-F) on the first N singular values
    sv (descending): the smallest r in 1..N whose leading r values hold at
    least the fraction `energy` of the energy sum_{i<=N} sigma_i^2."""
    e = np.asarray(sv, dtype=np.float64)[:N] ** 2
    total = e.sum()
    if not total > 0:
        return 1
    acc = 0.0
    for j in range(len(e)):
        acc += e[j]
        if acc >= energy * total:
            return j + 1
    return len(e)


def auto_rank(L0, m, energy=0.65):
    """Automatic rank of Section II-F from L0 (n x q): the energy threshold
    on the first rank_count(n, q, m) singular values of the full SVD.
    Returns (r, the singular values used)."""
    n, q = L0.shape
    N = rank_count(n, q, m)
    sv = np.linalg.svd(L0, compute_uv=False)[:N]
    return rank_from_singular_values(sv, N, energy), sv


def init_L0(op, Y, rho, tau0=10, mu_rule="support"):
    """L0 of Algorithm 1, Initialization: s_k = IHT(y_k, A_k, rho, tau0, 0)
    and column k = A_k^H (y_k - A_k s_k) (n x q).  It does not depend on r."""
    dt = op.dtype
    Y = np.asarray(Y, dtype=dt)
    S, _, _ = iht(Y, op.A, op.AH, rho, tau0, np.zeros((op.q, op.n), dtype=dt), mu_rule)
    return op.AH(Y - op.A(S)).T


def spectral_norm(G):
    return float(np.linalg.norm(G, 2)) if G.size else 0.0


# ------------------------------------------------------------ algorithm --

@dataclass
class OracleState:
    U: np.ndarray
    B: np.ndarray          # (r, q)
    S: np.ndarray          # (q, n) dense
    S_idx: np.ndarray      # (q, rho) support kept by the last HardThreshold
    eta: float = None
    t: int = 0


@dataclass
class OracleLog:
    t: list = field(default_factory=list)
    err: list = field(default_factory=list)
    X: list = field(default_factory=list)          # X_t (n, q) when kept
    U: list = field(default_factory=list)
    B: list = field(default_factory=list)
    S_idx: list = field(default_factory=list)
    S_val: list = field(default_factory=list)
    margin: list = field(default_factory=list)
    eta: float = None
    init_sv: np.ndarray = None


def init_alg1(op, Y, r, rho, tau0=10, mu_rule="support", perturb=None):
    """Algorithm 1, Initialization: IHT(y_k, A_k, rho, tau0, 0); L0; U0; b_k.
    perturb: see `iht` (test aid, None in plain runs)."""
    q, n = op.q, op.n
    dt = op.dtype
    Y = np.asarray(Y, dtype=dt)
    S, S_idx, margin = iht(Y, op.A, op.AH, rho, tau0, np.zeros((q, n), dtype=dt), mu_rule,
                           perturb=perturb)
    L0 = op.AH(Y - op.A(S)).T               # n x q, column k = A_k^H (y_k - A_k s_k)
    U0, sv = top_r_left(L0, r)
    W = op.AU(U0)
    B = pinv_apply(W, Y - op.A(S)).T        # r x q
    return OracleState(U=U0, B=B, S=S, S_idx=S_idx), L0, sv, margin


def iterate_alg1(op, Y, st, rho, tau=3, c_eta=0.14, mu_rule="support", chunk=None,
                 perturb=None):
    """One GDmin iteration of Algorithm 1 (t = st.t + 1), in place on `st`.

    z_k = P_perp y_k, M_k = P_perp A_k (explicit matrices for the Gaussian
    operator, the same definition as an operator for the Fourier one);
    s_k = IHT(z_k, M_k, rho, tau, s_k); b_k = (A_k U)^dagger (y_k - A_k s_k);
    grad = sum_k A_k^H (A_k(U b_k + s_k) - y_k) b_k^H; eta at t = 1;
    U <- QR(U - eta grad).  Returns the per-column margins of the last HT.
    perturb: see `iht` (test aid, None in plain runs).
    """
    q, n = op.q, op.n
    dt = op.dtype
    Y = np.asarray(Y, dtype=dt)
    chunk = chunk or q
    margins = np.empty(q)
    grad = np.zeros((n, st.U.shape[1]), dtype=dt)
    for k0 in range(0, q, chunk):
        ks = np.arange(k0, min(q, k0 + chunk))
        opc = op.subset(ks)
        Yc = Y[ks]
        W = opc.AU(st.U)                                    # A_k U
        Wp = np.linalg.pinv(W)                              # (A_k U)^dagger
        z = Yc - np.einsum("kmr,kr->km", W, np.einsum("krm,km->kr", Wp, Yc))
        if not op.complex:
            Am = opc.explicit()
            Mm = Am - W @ (Wp @ Am)                     # M_k = A_k - A_k U (A_k U)^dagger A_k
            M = lambda s, Mm=Mm: (Mm @ s[:, :, None])[:, :, 0]
            MH = lambda u, Mm=Mm: (u[:, None, :] @ Mm)[:, 0, :]
        else:
            def M(s, opc=opc, W=W, Wp=Wp):
                As = opc.A(s)
                return As - np.einsum("kmr,kr->km", W, np.einsum("krm,km->kr", Wp, As))

            def MH(u, opc=opc, W=W, Wp=Wp):
                Pu = u - np.einsum("kmr,kr->km", W, np.einsum("krm,km->kr", Wp, u))
                return opc.AH(Pu)
        S_c, I_c, mg = iht(z, M, MH, rho, tau, st.S[ks], mu_rule, st.S_idx[ks], perturb)
        st.S[ks] = S_c
        st.S_idx[ks] = I_c
        margins[ks] = mg
        Bc = np.einsum("krm,km->kr", Wp, Yc - opc.A(S_c)).T   # r x |ks|
        st.B[:, ks] = Bc
        grad += gradient_U(opc, st.U, Bc, S_c, Yc)
    st.t += 1
    if st.t == 1:
        gn = spectral_norm(grad)
        st.eta = c_eta / gn if gn > 0 else 0.0
    st.U, _ = qr_positive(st.U - st.eta * grad)
    return margins, grad


def relative_error(X, Xstar):
    return float(np.linalg.norm(X - Xstar) / np.linalg.norm(Xstar))


def run_alg1(op, Y, r, rho, T, tau0=10, tau=3, c_eta=0.14, Xstar=None,
             keep=(), mu_rule="support", chunk=None, init=None):
    """Algorithm 1 end to end.  Logs err_t for every t (when Xstar is given)
    and keeps (X_t, U_t, B_t, supports, margins) for t in `keep` (t = 0 is the
    initial state)."""
    log = OracleLog()
    if init is None:
        st, L0, sv, m0 = init_alg1(op, Y, r, rho, tau0, mu_rule)
    else:
        st, m0 = init, np.full(op.q, np.inf)
        sv = None
    log.init_sv = sv

    def record(t, margin):
        X = st.U @ st.B + st.S.T
        if Xstar is not None:
            log.t.append(t)
            log.err.append(relative_error(X, Xstar))
        if t in keep:
            log.X.append(X.copy())
            log.U.append(st.U.copy())
            log.B.append(st.B.copy())
            log.S_idx.append(st.S_idx.copy())
            log.S_val.append(np.take_along_axis(st.S, st.S_idx, axis=1) if st.S_idx.size
                             else np.zeros((op.q, 0)))
            log.margin.append(margin.copy())

    record(0, m0)
    for _ in range(T):
        mg, _ = iterate_alg1(op, Y, st, rho, tau, c_eta, mu_rule, chunk)
        record(st.t, mg)
    log.eta = st.eta
    return st, log

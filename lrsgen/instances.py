"""Seeded synthetic LR+S column-wise compressive-sensing instances.

Data model (Section I-A): X* = L* + S*, L* = U* B* with U* (n x r)
orthonormal, S* with rho nonzeros per column, y_k = A_k x*_k.  Value laws
follow the paper's simulations (Section III): U* = orthonormalised N(0,1)
n x r matrix, B* i.i.d. N(0,1), A_k i.i.d. N(0,1), supports uniform without
replacement; sparse magnitudes are +-U[1,10] * RMS(L*) unless another law is
named.  The stored instance is the float32 A_k and y_k (complex64 for the
Fourier operator); everything the solvers see is those stored values.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .philox import ln_pos, normals, uniforms

TAG_U, TAG_B, TAG_SUPP, TAG_SVAL, TAG_A, TAG_NOISE, TAG_MASK, TAG_PHASE = range(1, 9)


def sample_without_replacement(u, n, k):
    """Partial Fisher-Yates: first k entries of a shuffle of range(n) driven by u."""
    perm = {}
    out = np.empty(k, dtype=np.int64)
    for i in range(k):
        j = i + min(int(u[i] * (n - i)), n - i - 1)
        vi = perm.get(i, i)
        vj = perm.get(j, j)
        perm[i], perm[j] = vj, vi
        out[i] = vj
    return out


def _orth(Z):
    Q, R = np.linalg.qr(Z)
    d = np.diag(R)
    ph = np.where(np.abs(d) > 0, d / np.abs(d), 1.0)
    return Q * ph.conj()


def gaussian_A(seed, k, m, n):
    """A_k: i.i.d. N(0,1), row-major m x n, stored as float32."""
    return normals(seed, TAG_A, k, m * n).reshape(m, n).astype(np.float32)


@dataclass
class GaussianInstance:
    n: int
    q: int
    r: int
    m: int
    rho: int
    seed: int
    s_law: str = "pm_u1_10"
    alpha: float = 6.0
    y_float64: bool = False    # keep y_k in float64 (exact-recovery checks)
    identity_A: bool = False   # A_k = I (robust-PCA special case, m = n)
    noise: float = 0.0         # y_k = A_k x*_k + noise * ||x*_k|| * N(0, I_m)
    Ustar: np.ndarray = field(repr=False, default=None)
    Bstar: np.ndarray = field(repr=False, default=None)
    S_idx: np.ndarray = field(repr=False, default=None)   # (q, rho) ascending
    S_val: np.ndarray = field(repr=False, default=None)   # (q, rho)
    _A: np.ndarray = field(repr=False, default=None)
    _Y: np.ndarray = field(repr=False, default=None)

    def __post_init__(self):
        n, q, r, rho, seed = self.n, self.q, self.r, self.rho, self.seed
        self.Ustar = _orth(normals(seed, TAG_U, 0, n * r).reshape(n, r))
        self.Bstar = normals(seed, TAG_B, 0, r * q).reshape(r, q)
        L = self.Ustar @ self.Bstar
        rms = float(np.sqrt(np.mean(L * L))) if L.size else 1.0
        self.rms_L = rms
        self.S_idx = np.zeros((q, rho), dtype=np.int64)
        self.S_val = np.zeros((q, rho))
        for k in range(q):
            idx = sample_without_replacement(uniforms(seed, TAG_SUPP, k, rho), n, rho)
            u = uniforms(seed, TAG_SVAL, k, 2 * rho)
            if self.s_law == "pm_u1_10":        # +-U[1,10] RMS(L*)
                val = np.where(u[rho:] < 0.5, -1.0, 1.0) * (1.0 + 9.0 * u[:rho]) * rms
            elif self.s_law == "S1":            # U[-alpha, alpha] (Fig. 1)
                val = (2.0 * u[:rho] - 1.0) * self.alpha
            elif self.s_law == "S2":            # {+-1, +-10, +-100} (Fig. 2)
                mag = 10.0 ** np.floor(3.0 * u[:rho])
                val = np.where(u[rho:] < 0.5, -1.0, 1.0) * mag
            else:
                raise ValueError(self.s_law)
            o = np.argsort(idx)
            self.S_idx[k] = idx[o]
            self.S_val[k] = val[o]

    @property
    def Sstar(self):
        S = np.zeros((self.n, self.q))
        for k in range(self.q):
            S[self.S_idx[k], k] = self.S_val[k]
        return S

    @property
    def Xstar(self):
        return self.Ustar @ self.Bstar + self.Sstar

    def x_col(self, k):
        x = self.Ustar @ self.Bstar[:, k]
        x[self.S_idx[k]] += self.S_val[k]
        return x

    def A_col(self, k):
        if self.identity_A:
            return np.eye(self.n, dtype=np.float32)
        return gaussian_A(self.seed, k, self.m, self.n)

    def y_col(self, k, A_k=None):
        A_k = self.A_col(k) if A_k is None else A_k
        x = self.x_col(k)
        y = A_k.astype(np.float64) @ x
        if self.noise:
            # relative to ||x*_k||, the RMS of y_k's entries for Gaussian A_k
            y = y + self.noise * np.linalg.norm(x) * normals(self.seed, TAG_NOISE, k, len(y))
        return y if self.y_float64 else y.astype(np.float32)

    @property
    def A(self):
        """(q, m, n) float32; column k's A_k is A[k] (row-major m x n)."""
        if self._A is None:
            self._A = np.stack([self.A_col(k) for k in range(self.q)])
        return self._A

    @property
    def Y(self):
        """(q, m) float32; row k is y_k (so memory is m x q column-major)."""
        if self._Y is None:
            self._Y = np.stack([self.y_col(k, self.A[k]) for k in range(self.q)])
        return self._Y

    def columns(self, ks):
        """A_k and y_k for a subset of columns without building the whole A."""
        As = np.stack([self.A_col(k) for k in ks])
        Ys = np.stack([self.y_col(k, As[i]) for i, k in enumerate(ks)])
        return As, Ys


# ---------------------------------------------------------------- Fourier --

def vd_mask(seed, k, nx, ny, m, center):
    """Variable-density row mask of the 2D DFT, natural (unshifted) order.

    The centre `center` x `center` block of fftshift-ed k-space is always
    sampled; the other m - center^2 points are drawn without replacement with
    weight (1 + k_r/8)^-2 (k_r: distance to the k-space centre in index units),
    by the exponential-key method (Efraimidis-Spirakis).  Returns sorted int64
    row indices kx*ny + ky of the n = nx*ny DFT rows.
    """
    cx, cy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    dx, dy = cx - nx // 2, cy - ny // 2
    kr = np.sqrt(dx * dx + dy * dy)
    central = (dx >= -(center // 2)) & (dx < center - center // 2) & \
              (dy >= -(center // 2)) & (dy < center - center // 2)
    w = (1.0 + kr / 8.0) ** -2
    u = uniforms(seed, TAG_MASK, k, nx * ny).reshape(nx, ny)
    key = ln_pos(np.maximum(u, 2.0 ** -60)) / w          # larger is better
    key[central] = np.inf
    flat = np.argsort(-key.ravel(), kind="stable")[:m]
    sx, sy = np.unravel_index(flat, (nx, ny))
    kx = (sx - nx // 2) % nx
    ky = (sy - ny // 2) % ny
    return np.sort(kx * ny + ky)


@dataclass
class FourierInstance:
    nx: int
    ny: int
    q: int
    r: int
    m: int
    rho: int
    seed: int
    center: int = 16
    s_law: str = "blobs"
    mask_law: str = "vd"       # "vd": variable density; "uniform": uniform rows
    b_law: str = "dct"         # "dct": smooth temporal basis; "gauss": i.i.d. N(0,1)
    Ustar: np.ndarray = field(repr=False, default=None)
    Bstar: np.ndarray = field(repr=False, default=None)

    def __post_init__(self):
        nx, ny, q, r, rho, seed = self.nx, self.ny, self.q, self.r, self.rho, self.seed
        n = self.n = nx * ny
        z = normals(seed, TAG_U, 0, 2 * n * r).reshape(n, r, 2)
        self.Ustar = _orth((z[..., 0] + 1j * z[..., 1]) / np.sqrt(2.0))
        if self.b_law == "dct":
            j = np.arange(r)[:, None]
            kk = np.arange(q)[None, :]
            B = (2.0 ** (-j / 2.0)) * np.cos(np.pi * j * (kk + 0.5) / q)
            L = self.Ustar @ B
            B = B / np.sqrt(np.mean(np.abs(L) ** 2))
        else:
            B = normals(seed, TAG_B, 0, r * q).reshape(r, q)
        self.Bstar = B
        self.rms_L = float(np.sqrt(np.mean(np.abs(self.Ustar @ B) ** 2)))
        self.S_idx = np.zeros((q, rho), dtype=np.int64)
        self.S_val = np.zeros((q, rho), dtype=np.complex128)
        for k in range(q):
            idx = self._blobs(k) if self.s_law == "blobs" else \
                np.sort(sample_without_replacement(uniforms(seed, TAG_SUPP, k, rho), n, rho))
            u = uniforms(seed, TAG_SVAL, k, 2 * rho)
            if self.s_law == "S1":              # real U[-6, 6] (Fig. 1 law)
                val = (2.0 * u[:rho] - 1.0) * 6.0 + 0j
            else:                               # U[1,10] RMS(L*), uniform phase
                val = (1.0 + 9.0 * u[:rho]) * self.rms_L * np.exp(2j * np.pi * u[rho:])
            self.S_idx[k] = idx
            self.S_val[k] = val
        if self.mask_law == "vd":
            self.masks = np.stack([vd_mask(seed, k, nx, ny, self.m, self.center)
                                   for k in range(q)])
        else:
            self.masks = np.stack([np.sort(sample_without_replacement(
                uniforms(seed, TAG_MASK, k, self.m), n, self.m)) for k in range(q)])
        self._Y = None

    def _blobs(self, k):
        """3x3 blobs at uniform centres (clipped at the frame edge) until rho pixels."""
        nx, ny, rho = self.nx, self.ny, self.rho
        got = []
        seen = set()
        u = uniforms(self.seed, TAG_SUPP, k, 4 * rho + 64)
        t = 0
        while len(got) < rho:
            c = min(int(u[t] * nx * ny), nx * ny - 1)
            t += 1
            px, py = divmod(c, ny)
            for ddx in (-1, 0, 1):
                for ddy in (-1, 0, 1):
                    x, y = px + ddx, py + ddy
                    if 0 <= x < nx and 0 <= y < ny and len(got) < rho:
                        p = x * ny + y
                        if p not in seen:
                            seen.add(p)
                            got.append(p)
        return np.sort(np.array(got, dtype=np.int64))

    @property
    def Sstar(self):
        S = np.zeros((self.n, self.q), dtype=np.complex128)
        for k in range(self.q):
            S[self.S_idx[k], k] = self.S_val[k]
        return S

    @property
    def Xstar(self):
        return self.Ustar @ self.Bstar + self.Sstar

    @property
    def Y(self):
        """(q, m) complex64: y_k = (unitary 2D DFT of frame k)[mask_k]."""
        if self._Y is None:
            X = self.Xstar.T.reshape(self.q, self.nx, self.ny)
            F = np.fft.fft2(X, norm="ortho").reshape(self.q, self.n)
            self._Y = np.take_along_axis(F, self.masks, axis=1).astype(np.complex64)
        return self._Y

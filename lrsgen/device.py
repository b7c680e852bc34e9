"""Device-resident Gaussian instances for the large workloads, where drawing
every A_k on the host would take longer than the measurement itself.

Same data model and laws as `GaussianInstance` (U*, B*, supports and sparse
values come from it, so they equal the host instance's), except that the
i.i.d. N(0,1) entries of A_k are drawn by torch's seeded device generator
instead of the counter-based host stream: the instance is synthetic data
of the same law, not the host instance's values.  y_k = A_k x*_k is formed
in float64 and stored as float32, like the host instance.
"""
from __future__ import annotations

import numpy as np

from .instances import GaussianInstance


class DeviceGaussianInstance:
    def __init__(self, n, q, r, m, rho, seed, device="cuda", chunk=64):
        import torch
        self.n, self.q, self.r, self.m, self.rho, self.seed = n, q, r, m, rho, seed
        host = GaussianInstance(n=n, q=q, r=r, m=m, rho=rho, seed=seed)
        self.Xstar = host.Xstar                       # n x q float64 (host)
        g = torch.Generator(device=device)
        g.manual_seed(int(seed) * 1000003 + 12345)
        self.A = torch.empty((q, m, n), dtype=torch.float32, device=device)
        self.Y = torch.empty((q, m), dtype=torch.float32, device=device)
        X = torch.from_numpy(np.ascontiguousarray(self.Xstar.T)).to(device)   # q x n float64
        for k0 in range(0, q, chunk):
            k1 = min(q, k0 + chunk)
            self.A[k0:k1] = torch.randn((k1 - k0, m, n), generator=g, device=device,
                                        dtype=torch.float32)
            y = torch.bmm(self.A[k0:k1].double(), X[k0:k1, :, None])[:, :, 0]
            self.Y[k0:k1] = y.float()
        torch.cuda.current_stream().synchronize()  # this stream only: others keep running

    def free(self):
        self.A = None
        self.Y = None

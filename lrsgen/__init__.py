"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

Holds only input generation (counter-based random numbers and the instance
recipes); none of the solver's arithmetic lives here.
"""
from .philox import normals, uniforms, philox4x32_10, ln_pos, sincos_turns  # noqa: F401
from .instances import (GaussianInstance, FourierInstance, gaussian_A,  # noqa: F401
                        vd_mask, sample_without_replacement)

# The five workloads, by what they are.
C0 = dict(n=200, q=200, r=3, m=80, rho=4, seed=1, T=300)          # small Gaussian
C1 = dict(n=1000, q=1000, r=5, m=150, rho=10, seed=2, T=200)      # FP32 Gaussian
C2 = dict(n=4096, q=2048, r=10, m=512, rho=40, seed=3, T=100)     # precision forms
C3 = dict(nx=128, ny=128, q=256, r=6, m=2048, rho=82, seed=4, T=150)  # Fourier/MRI

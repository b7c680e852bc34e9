"""The paper's simulations (Section III) run through the CUDA solver.

    python tests/paper_experiments.py [--runs R] [--out FILE]

* Fig. 1: Gaussian A_k, n = q = 600, m = 80, r = 4, rho in {2, 5, 6, 7},
  rho_max = 7, sparse values by law S1 (U[-6, 6]), T = 200 (tau0 = 10,
  tau = 3): the error ||X* - X_t||_F / ||X*||_F against t.
* Fig. 2 (this solver's curves only; the comparison method's code is not
  part of this project): the same setting with rho = 2, rho_max = 5, laws S1
  and S2 ({+-1, +-10, +-100}).
* Table 1: random DFT rows (uniform masks), 20 x 20 frames (n = 400), q = 400,
  r = 4, rho = 2, rho_max = 5, T = 10, law S1: the error after T iterations
  for m = 40 ... 300, for AltGDmin-L+S and for AltGDmin (the rho = 0 solver
  on the same measurements), beside the paper's printed values
  (tests/golden/table1_fourier_altgdmin_lps.txt).

The paper averages 100 Monte Carlo runs; R seeded runs per setting here
(default 10).  Errors are measured by the library against X* stored in
float32, so they stop near 1e-7.  Writes a markdown report (default
profiles/paper_experiments_fig1_fig2_table1.md)."""
import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from lrsgen import FourierInstance, GaussianInstance  # noqa: E402

FIG_T = (0, 10, 25, 50, 100, 150, 200)


def rel_err(solver, Xstar):
    X = solver.X()                      # U B + S, assembled by the library
    return float(np.linalg.norm(X - Xstar) / np.linalg.norm(Xstar))


def error_curve(solver, Xstar, T):
    """Errors after the initialisation and after each of T iterations (the
    library's error log against X* in float32)."""
    from paper_2311_03824_gb300 import lrs as L
    L.lrs_set_reference(solver.h, np.ascontiguousarray(Xstar.T, np.float32))
    solver.init()
    e0 = rel_err(solver, Xstar)
    log = np.zeros(T)
    if T:
        solver.iterate(T, log)
    return np.concatenate([[e0], log])


def gaussian_run(n, q, r, m, rho, rho_max, law, seed, T):
    from paper_2311_03824_gb300 import Solver
    inst = GaussianInstance(n=n, q=q, r=r, m=m, rho=rho, seed=seed, s_law=law)
    s = Solver(n, m, q, r, rho, rho_max=rho_max)
    try:
        s.set_measurements(np.ascontiguousarray(inst.Y, np.float32),
                           np.ascontiguousarray(inst.A, np.float32))
        return error_curve(s, inst.Xstar, T)
    finally:
        s.close()


def fourier_run(m, rho_solver, rho_max, seed, T, nx=20, ny=20, q=400, r=4, rho=2):
    from paper_2311_03824_gb300 import LRS_OP_DFT2D_MASK, Solver
    inst = FourierInstance(nx=nx, ny=ny, q=q, r=r, m=m, rho=rho, seed=seed, s_law="S1",
                           mask_law="uniform", b_law="gauss")
    s = Solver(inst.n, m, q, r, rho_solver, kind=LRS_OP_DFT2D_MASK, nx=nx, ny=ny,
               rho_max=rho_max)
    try:
        s.set_measurements(np.ascontiguousarray(inst.Y, np.complex64),
                           np.ascontiguousarray(inst.masks, np.int32))
        s.init()
        s.iterate(T)
        return rel_err(s, inst.Xstar)
    finally:
        s.close()


def table1_paper():
    rows = {}
    p = os.path.join(ROOT, "tests", "golden", "table1_fourier_altgdmin_lps.txt")
    for line in open(p):
        if line.strip() and not line.startswith("#"):
            m, e = line.split()
            rows[int(m)] = float(e)
    return rows


def curve_rows(title, curves):
    out = [f"| {title} | " + " | ".join(f"t={t}" for t in FIG_T) + " | runs < 1e-5 at t=200 |",
           "|---|" + "---|" * (len(FIG_T) + 1)]
    for label, C in curves:
        C = np.asarray(C)
        med = np.median(C, axis=0)
        ok = int(np.sum(C[:, -1] < 1e-5))
        out.append(f"| {label} | " + " | ".join(f"{med[t]:.2e}" for t in FIG_T) +
                   f" | {ok}/{len(C)} |")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--runs", type=int, default=10)
    ap.add_argument("--out", default=os.path.join(ROOT, "profiles",
                                                  "paper_experiments_fig1_fig2_table1.md"))
    args = ap.parse_args()
    from paper_2311_03824_gb300 import build
    build.build()
    R = args.runs
    t0 = time.time()
    lines = ["# Section III simulations through the CUDA solver", "",
             f"Command: `python tests/paper_experiments.py --runs {R}` (one GB300).  Median "
             f"of {R} seeded runs per setting (the paper: 100).  Error "
             "||X* - X_t||_F / ||X*||_F, measured by the library against X* in float32.", ""]
    fig1 = []
    for rho in (2, 5, 6, 7):
        C = [gaussian_run(600, 600, 4, 80, rho, 7, "S1", 1000 * rho + i, 200) for i in range(R)]
        fig1.append((f"rho={rho}, rho_max=7", C))
    lines += ["## Fig. 1 (n = q = 600, m = 80, r = 4, S1, rho_max = 7)", ""]
    lines += curve_rows("setting", fig1) + [""]
    fig2 = []
    for law in ("S1", "S2"):
        C = [gaussian_run(600, 600, 4, 80, 2, 5, law, 5000 + 100 * (law == "S2") + i, 200)
             for i in range(R)]
        fig2.append((f"{law}, rho=2, rho_max=5", C))
    lines += ["## Fig. 2, this solver's curves (n = q = 600, m = 80, r = 4, rho = 2, "
              "rho_max = 5)", ""]
    lines += curve_rows("law", fig2) + [""]
    paper = table1_paper()
    lines += ["## Table 1 (DFT rows, 20 x 20 frames, q = 400, r = 4, rho = 2, rho_max = 5, "
              "T = 10, S1)", "",
              "| m | AltGDmin (rho = 0), mean | AltGDmin-L+S, mean | AltGDmin-L+S, median | "
              "paper AltGDmin-L+S |", "|---|---|---|---|---|"]
    for m in sorted(paper):
        lps = [fourier_run(m, 2, 5, 9000 + m * 10 + i, 10) for i in range(R)]
        lr = [fourier_run(m, 0, 0, 9000 + m * 10 + i, 10) for i in range(R)]
        lines.append(f"| {m} | {np.mean(lr):.4f} | {np.mean(lps):.4f} | {np.median(lps):.4f} | "
                     f"{paper[m]:.4f} |")
    lines += ["", f"Wall time {time.time() - t0:.0f} s (instance generation on the host "
              "included)."]
    text = "\n".join(lines) + "\n"
    with open(args.out, "w") as f:
        f.write(text)
    print(text)


if __name__ == "__main__":
    main()

"""Writes large_hf_1024_R32_100steps.txt: the FP64 oracle's solutions of the large
high-fidelity configuration (1024 x 1024, delta = 32h, 3209-point disc, smoothed-noise IC,
eps = 0.02 U[0.8, 1.2], tau = 1e-3) after 100 steps, samples 0..3 of its seeds: per sample the
OoI f, the mean of u, and u at 512 fixed lattice points (the points come from numpy's
default_rng(1024)).  Only the oracle computes these values; run it from the repository root:

    python tests/golden/make_large_hf_fixture.py

It takes several minutes of CPU time per sample.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle as O  # noqa: E402

N, R, STEPS, SAMPLES, POINTS = 1024, 32, 100, 4, 512
SEED0 = 20231016 + 1000003 * 4
KW = dict(n=N, delta=R / N, eps=0.02, eps_lo=0.016, eps_hi=0.024, tau=1e-3, nsteps=STEPS, ic=1, ic_amp=0.05)


def points():
    rng = np.random.default_rng(1024)
    return rng.integers(0, N, size=(POINTS, 2))


def main():
    o = O.OracleModel(**KW)
    pts = points()
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "large_hf_1024_R32_100steps.txt")
    lines = ["# FP64 oracle (oracle/nlch_oracle.c), 1024 x 1024, delta = 32h, 100 steps, smoothed-noise IC,",
             "# eps = 0.02 U[0.8, 1.2], tau = 1e-3; written by tests/golden/make_large_hf_fixture.py.",
             "# columns: sample seed f mean, then u at the 512 points of numpy default_rng(1024)",
             "# (pairs (y, x) from integers(0, 1024, size=(512, 2)))"]
    for s in range(SAMPLES):
        seed = SEED0 + s
        f, mean, uT, _ = o.solve_sample(seed)
        vals = " ".join(repr(float(uT[y, x])) for y, x in pts)
        lines.append(f"{s} {seed} {f!r} {mean!r} {vals}")
        print(f"sample {s}: f = {f:.15g}", flush=True)
    with open(out, "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()

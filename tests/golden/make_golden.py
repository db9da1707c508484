"""Writes the stored expected values under tests/golden/ from the FP64 oracle alone.

The inputs are closed-form (no random generator), so the files are reproducible on
any machine. Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import tracker as O  # noqa: E402


def tiny_inputs():
    """Nx = 8, Ny = 6, R = 2, four frames: factors, frames and masks from closed forms."""
    Nx, Ny, R, T = 8, 6, 2, 4
    i, j, r = np.arange(Nx)[:, None], np.arange(Ny)[:, None], np.arange(R)[None, :]
    A = np.cos(0.7 * i + 1.3 * r) + 1j * np.sin(0.4 * i - 0.9 * r)
    B = np.cos(0.5 * j - 0.6 * r) + 1j * np.sin(1.1 * j + 0.2 * r)
    frames, masks = [], []
    for t in range(T):
        u, v = np.arange(Nx)[:, None], np.arange(Ny)[None, :]
        L = np.exp(-((u - 3.5 - 0.3 * t) ** 2) / 6.0 - ((v - 2.5) ** 2) / 4.0) * (1 + 0.1 * t)
        frames.append(O.fft2(L))
        m = np.zeros(Nx, np.uint8)
        m[[0, 1, 7, (2 + 3 * t) % Nx, (4 + t) % Nx]] = 1
        masks.append(m)
    return dict(Nx=Nx, Ny=Ny, R=R, T=T, A=A, B=B, frames=frames, masks=masks)


def c2list(z):
    z = np.asarray(z).reshape(-1)
    return [[float(v.real), float(v.imag)] for v in z]


def main():
    d = tiny_inputs()
    out = {"source": "oracle/tracker.py (FP64), inputs of tests/golden/make_golden.py:tiny_inputs",
           "passage": "Alg. 3 with one coil, Gauss-Seidel MM iterations, forgetting (readings in oracle header)",
           "lambda_forget": 0.9, "mu": 0.05, "mm_iters": 3, "images": []}
    tr = O.Tracker(d["Nx"], d["Ny"], d["R"], 0.9, 0.05, 3, A=d["A"], B=d["B"])
    for t in range(d["T"]):
        rows = np.flatnonzero(d["masks"][t])
        x = tr.push_frame(d["frames"][t][rows], d["masks"][t])
        out["images"].append(c2list(x))
    out["abar_A"], out["abar_B"], out["w"] = tr.abar_A, tr.abar_B, tr.w
    with open(os.path.join(HERE, "tiny_track.json"), "w") as f:
        json.dump(out, f, indent=0)

    # line draws (Alg. 4 with integer CDF + Philox) for closed-form probabilities
    Nx = 64
    p = 1.0 / (1.0 + np.minimum(np.arange(Nx), Nx - np.arange(Nx)))
    p = p / p.sum()
    draws = {"source": "oracle/tracker.py:sample_lines_from_probs", "passage": "Alg. 4, §VI-C",
             "p": "1/(1+min(i,Nx-i)) normalised, Nx=64", "cases": []}
    for seed, ctr, k, wr in ((0, 0, 16, False), (7, 123, 16, False), (2 ** 40 + 5, 2 ** 41 + 3, 32, False),
                             (11, 5, 20, True)):
        m = O.sample_lines_from_probs(p, k, 8, seed, ctr, wr)
        draws["cases"].append({"seed": seed, "ctr": ctr, "k_lines": k, "with_replacement": wr,
                               "lines": [int(v) for v in np.flatnonzero(m)]})
    with open(os.path.join(HERE, "line_draws.json"), "w") as f:
        json.dump(draws, f, indent=1)


if __name__ == "__main__":
    main()

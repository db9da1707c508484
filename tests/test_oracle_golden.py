"""The oracle reproduces the stored values written by tests/golden/make_golden.py
(which calls only the oracle): guards the oracle against unintended changes."""
import json
import os

import numpy as np

from oracle import tracker as O
from tests.golden.make_golden import tiny_inputs

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_tiny_track_golden():
    g = json.load(open(os.path.join(HERE, "tiny_track.json")))
    d = tiny_inputs()
    tr = O.Tracker(d["Nx"], d["Ny"], d["R"], g["lambda_forget"], g["mu"], g["mm_iters"],
                   A=d["A"], B=d["B"])
    for t in range(d["T"]):
        rows = np.flatnonzero(d["masks"][t])
        x = tr.push_frame(d["frames"][t][rows], d["masks"][t])
        ref = np.array([complex(a, b) for a, b in g["images"][t]]).reshape(x.shape)
        np.testing.assert_allclose(x, ref, rtol=1e-10, atol=1e-12)
    assert abs(tr.abar_A - g["abar_A"]) <= 1e-10 * g["abar_A"]


def test_line_draws_golden():
    g = json.load(open(os.path.join(HERE, "line_draws.json")))
    Nx = 64
    p = 1.0 / (1.0 + np.minimum(np.arange(Nx), Nx - np.arange(Nx)))
    p = p / p.sum()
    for c in g["cases"]:
        m = O.sample_lines_from_probs(p, c["k_lines"], 8, c["seed"], c["ctr"], c["with_replacement"])
        assert [int(v) for v in np.flatnonzero(m)] == c["lines"]

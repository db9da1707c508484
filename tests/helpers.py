"""Shared test drivers: run the FP64 oracle and the CUDA tracker on the same inputs."""
from __future__ import annotations

import numpy as np

from oracle import tracker as O
from paper_1609_04104_gb300 import inputs

# Image parity bound: per-frame NRMSE of the FP32 CUDA path against the FP64 oracle.
NRMSE_TOL = 1e-4


def workload_inputs(w: inputs.Workload, T: int):
    L = inputs.phantom(w, T)
    Y = inputs.kspace(w, L)
    A0, B0 = inputs.init_factors(w.Nx, w.Ny, w.R, w.seed)
    return L, Y, A0, B0


def run_oracle(w: inputs.Workload, T: int, Y, A0, B0, masks=None, update="gauss_seidel", seed=None):
    """Oracle trajectory. With masks None the lines come from the oracle's own
    informative draws (after the fully-sampled warm-up frames). Returns (images,
    masks, states)."""
    tr = O.Tracker(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, w.mm_iters, update=update, A=A0, B=B0)
    imgs, used, states = [], [], []
    for t in range(T):
        if masks is not None:
            m = masks[t]
        elif t < w.warmup_frames:
            m = np.ones(w.Nx, np.uint8)
        else:
            m = tr.next_mask(w.k_lines, w.central_lines, seed=w.seed if seed is None else seed)
        states.append(tr.state())
        imgs.append(tr.push_frame(inputs.observed_rows(Y[t], m), m))
        used.append(np.asarray(m, np.uint8))
    states.append(tr.state())
    return np.array(imgs), np.array(used), states


def run_gpu(tts, w: inputs.Workload, T: int, Y, A0, B0, masks, **cfg):
    trk = tts.Tracker(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, mm_iters=w.mm_iters,
                      central_lines=w.central_lines, **cfg)
    trk.set_factors(A0, B0)
    imgs = []
    for t in range(T):
        trk.push_frame(inputs.observed_rows(Y[t], masks[t]), masks[t])
        imgs.append(trk.image(t))
    return trk, np.array(imgs)


def nrmse_per_frame(x, ref):
    return np.array([O.nrmse(x[t], ref[t]) for t in range(len(ref))])

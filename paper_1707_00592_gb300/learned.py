"""Training pipeline of the learned smooth-face gate, on the GPU, through the
library's own kernels (ws_face_samples, ws_mlp_grad, ws_mlp_adam,
ws_mlp_forward).

1. Sample labelled faces from plain (ungated) mixed-precision runs of the
   gas-water tube (1D), the shock-bubble (2D) and the water drop (3D).
2. Train the 24 -> 32 -> 32 -> 1 MLP with Adam on the weighted binary
   cross-entropy.
3. Choose the logit threshold on held-out faces so that at least `recall` of
   the faces that need WENO-IS stay above it.
"""
from __future__ import annotations

import math

import numpy as np

from . import workloads as wl
from . import (MLP_NIN, MLP_NPARAM, Solver, ws_face_samples, ws_mlp_adam, ws_mlp_forward, ws_mlp_grad)


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal initial weights, zero biases (layout W1, b1, W2, b2, W3, b3)."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0.0, math.sqrt(2.0 / 24), 32 * 24), np.zeros(32),
             rng.normal(0.0, math.sqrt(2.0 / 32), 32 * 32), np.zeros(32),
             rng.normal(0.0, math.sqrt(1.0 / 32), 32), np.zeros(1)]
    p = np.concatenate(parts)
    assert p.size == MLP_NPARAM
    return p


def _collect(solver, U, stride, budget, feats_out, labels_out):
    import torch
    n = ws_face_samples(solver.ctx, U, stride, budget, feats_out, labels_out)
    torch.cuda.synchronize()
    return n


def sample_faces(total: int = 10_000_000, seed: int = 0, sizes=(200, 1024, 96), steps=(255, 2000, 100),
                 snapshots: int = 8, share=(0.02, 0.68, 0.3)):
    """Labelled faces from plain mixed-precision runs of the three workloads
    (the gas-water tube, the shock-bubble and the water drop at the given
    sizes, each over its run of `steps` steps, sampled at `snapshots` evenly
    spaced states).  Returns (feats [n, 24] FP32 CUDA tensor, labels [n] uint8
    CUDA tensor)."""
    import torch
    cases = [wl.gas_water_tube(sizes[0]), wl.shock_bubble_2d(sizes[1]), wl.drop_3d(sizes[2], seed=seed)]
    feats = torch.empty((total, MLP_NIN), dtype=torch.float32, device="cuda")
    labels = torch.empty(total, dtype=torch.uint8, device="cuda")
    out = 0
    for case, nsteps, frac in zip(cases, steps, share):
        s = Solver(case.ndim, case.n, case.dx, case.bc, precision="mixed")
        U = s.prim_to_cons(s.tensor(case.Q))
        nf = sum((case.n[d] + 1) * case.cells // case.n[d] for d in range(case.ndim))
        budget_case = int(total * frac)
        per_snap = max(1, budget_case // snapshots)
        stride = max(1, nf // per_snap)
        every = max(1, nsteps // snapshots)
        got = 0
        for k in range(nsteps):
            if k % every == 0 and got < budget_case and out < total:
                room = min(per_snap, budget_case - got, total - out)
                n = _collect(s, U, stride, room, feats[out:], labels[out:])
                out += n
                got += n
            s.step(U)
        s.close()
    return feats[:out], labels[:out]


def train(feats, labels, epochs: int = 4, batch: int = 65536, lr: float = 3e-3, seed: int = 0,
          pos_weight: float | None = None, log=None):
    """Adam on the weighted BCE with the library's gradient kernel.  Returns the
    FP32 parameters as a CUDA tensor."""
    import torch
    n = feats.shape[0]
    if pos_weight is None:
        pos = float(labels.float().mean().item())
        pos_weight = max(1.0, (1.0 - pos) / max(pos, 1e-6))
    P = torch.tensor(init_params(seed), dtype=torch.float32, device="cuda")
    M = torch.zeros_like(P)
    V = torch.zeros_like(P)
    G = torch.empty_like(P)
    L = torch.empty(1, dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=gen)
        Xs, Ys = feats[perm].contiguous(), labels[perm].contiguous()
        for b0 in range(0, n - batch + 1, batch):
            step += 1
            ws_mlp_grad(P, Xs[b0:b0 + batch], Ys[b0:b0 + batch], pos_weight, G, L)
            ws_mlp_adam(P, M, V, G, step, lr * (0.5 ** ep))
        if log:
            log(f"epoch {ep}: loss {L.item():.5f}")
    torch.cuda.synchronize()
    return P


def logits(P, feats):
    import torch
    z = torch.empty(feats.shape[0], dtype=torch.float32, device="cuda")
    ws_mlp_forward(P, feats, z)
    torch.cuda.synchronize()
    return z


def choose_threshold(P, feats, labels, recall: float = 0.999) -> float:
    """Largest logit threshold keeping >= recall of the label-1 faces at or
    above it (those faces keep WENO-IS)."""
    import torch
    z = logits(P, feats)
    pos = z[labels > 0]
    if pos.numel() == 0:
        return float(z.max().item()) + 1.0
    k = max(1, int(math.floor((1.0 - recall) * pos.numel())))
    thr = torch.kthvalue(pos.cpu(), k).values.item()
    return float(thr)


def train_gate(total: int = 10_000_000, epochs: int = 4, recall: float = 0.999, seed: int = 0, log=None):
    """Sample, train, and pick the threshold.  Returns (params CUDA tensor,
    threshold, report dict)."""
    import torch
    feats, labels = sample_faces(total=total, seed=seed)
    n = feats.shape[0]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed + 1)
    perm = torch.randperm(n, device="cuda", generator=gen)
    cut = int(0.9 * n)
    tr, te = perm[:cut], perm[cut:]
    P = train(feats[tr].contiguous(), labels[tr].contiguous(), epochs=epochs, seed=seed, log=log)
    Xte, Yte = feats[te].contiguous(), labels[te].contiguous()
    thr = choose_threshold(P, Xte, Yte, recall)
    z = logits(P, Xte)
    smooth = z < thr
    pos = Yte > 0
    rep = {"samples": int(n), "positives": float(pos.float().mean().item()),
           "recall": float(((~smooth) & pos).sum().item() / max(1, int(pos.sum().item()))),
           "smooth_fraction": float(smooth.float().mean().item()), "threshold": thr}
    return P, thr, rep

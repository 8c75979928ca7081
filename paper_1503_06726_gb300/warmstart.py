"""Learned warm start of the steady morphogen solve.

Pipeline (every numerical step runs in the library's CUDA kernels; torch
only holds device memory):
  * ``tissue_tensors``: cell labels and source maps of a list of tissues,
    computed on the device by ``lbib_label_cells``;
  * ``make_dataset``: cold steady solves (``lbib_steady_solve``, residual
    1e-6) of many tissues, batched by similar decay so that a batch ends
    together -- the training pairs the LB solver itself generates;
  * ``train``: minibatch Adam on the neural operator
    (``lbib_nop_train_step``);
  * ``evaluate``: per tissue, steps and wall time to the residual from a cold
    start and from the network's prediction (inference time included), and
    whether the solve abandoned the prediction for the cold start.
"""
from __future__ import annotations

import time
from typing import List, Sequence

import numpy as np

from . import lbib


class _AllSources:
    """A tissue view whose every cell is flagged: its source map is the cell mask."""

    def __init__(self, T):
        self.cell_off, self.xy = T.cell_off, T.xy
        self.src_flag = np.full(T.n_cells, 0xF, np.uint8)
        self.n_cells = T.n_cells


def tissue_tensors(tissues: Sequence, H: int, W: int, device="cuda"):
    """(mask, src) uint8 CUDA tensors (n, H, W) of periodic tissues: the
    cell mask and the source map, both written by the labelling kernel."""
    import torch
    n = len(tissues)
    mask = torch.empty((n, H, W), dtype=torch.uint8, device=device)
    src = torch.empty((n, H, W), dtype=torch.uint8, device=device)
    for i, T in enumerate(tissues):
        _, srt = lbib.label_cells(W, H, 0, T, device=device)
        _, inside = lbib.label_cells(W, H, 0, _AllSources(T), device=device)
        src[i].copy_(srt)
        mask[i].copy_(inside)
    return mask, src


def _tensor_params(params):
    D = np.array([p.D[0] for p in params], np.float64)
    k = np.array([p.decay[0] for p in params], np.float64)
    s = np.array([p.src_rate[0] for p in params], np.float64)
    return D, k, s


class Dataset:
    def __init__(self, mask, src, D, k, s, phi, steps):
        self.mask, self.src, self.D, self.k, self.s = mask, src, D, k, s
        self.phi, self.steps = phi, steps

    def __len__(self):
        return self.mask.shape[0]


def make_dataset(items, H: int = 256, W: int = 256, batch: int = 256, tol: float = 1e-6,
                 max_steps: int = 400000, device="cuda") -> Dataset:
    """items: list of (params, tissue).  Cold-solves every tissue to `tol`."""
    import torch
    params = [p for p, _ in items]
    tissues = [t for _, t in items]
    D, k, s = _tensor_params(params)
    # similar decay -> similar convergence time within a batch; the dataset is
    # kept in this order
    order = np.argsort(k, kind="stable")
    D, k, s = D[order], k[order], s[order]
    tissues = [tissues[i] for i in order]
    n = len(items)
    mask = torch.empty((n, H, W), dtype=torch.uint8, device=device)
    src = torch.empty((n, H, W), dtype=torch.uint8, device=device)
    phi = torch.empty((n, H, W), dtype=torch.float32, device=device)
    steps = np.zeros(n, np.int64)
    for b0 in range(0, n, batch):
        b1 = min(n, b0 + batch)
        m, sr = tissue_tensors(tissues[b0:b1], H, W, device)
        out, st, res = lbib.steady_solve(sr, D[b0:b1], k[b0:b1], s[b0:b1], tol=tol,
                                         max_steps=max_steps)
        mask[b0:b1].copy_(m)
        src[b0:b1].copy_(sr)
        phi[b0:b1].copy_(out)
        steps[b0:b1] = st
    return Dataset(mask, src, D, k, s, phi, steps)


def train(net: "lbib.NeuralOperator", data: Dataset, epochs: int, batch: int,
          lr: float = 1e-3, lr_end: float = 1e-4, seed: int = 0, log=None) -> List[float]:
    """Minibatch Adam with a geometric learning-rate decay; returns the
    mean loss of every epoch."""
    import torch
    rng = np.random.default_rng(seed)
    n = len(data)
    steps_total = max(1, epochs * (n // batch))
    losses = []
    step = 0
    for ep in range(epochs):
        perm = rng.permutation(n)
        tot = 0.0
        nb = 0
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            ii = torch.as_tensor(idx, device=data.mask.device)
            cur = lr * (lr_end / lr) ** (step / steps_total)
            tot += net.train_step(data.mask[ii].contiguous(), data.src[ii].contiguous(),
                                  data.D[idx], data.k[idx], data.s[idx],
                                  data.phi[ii].contiguous(), lr=cur)
            nb += 1
            step += 1
        losses.append(tot / max(nb, 1))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.4e}")
    return losses


def evaluate(net: "lbib.NeuralOperator", items, H: int = 256, W: int = 256, tol: float = 1e-6,
             max_steps: int = 400000, device="cuda"):
    """Per tissue (one at a time, as a user would run it): steps and wall
    seconds to `tol` from a cold start and from the network's prediction
    (inference included), and the relative L-inf gap of the two solutions."""
    import torch
    params = [p for p, _ in items]
    D, k, s = _tensor_params(params)
    mask, src = tissue_tensors([t for _, t in items], H, W, device)
    rows = []
    for i in range(len(items)):
        m, sr = mask[i:i + 1], src[i:i + 1]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pc, sc, rc = lbib.steady_solve(sr, D[i:i + 1], k[i:i + 1], s[i:i + 1], tol=tol,
                                       max_steps=max_steps)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        p0 = net.forward(m, sr, D[i:i + 1], k[i:i + 1], s[i:i + 1])
        pw, sw, rw, fb = lbib.steady_solve(sr, D[i:i + 1], k[i:i + 1], s[i:i + 1], phi0=p0,
                                           tol=tol, max_steps=max_steps, with_fallback=True)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        a = pc.cpu().numpy()
        b = pw.cpu().numpy()
        rows.append({"cold_steps": int(sc[0]), "warm_steps": int(sw[0]),
                     "cold_s": t1 - t0, "warm_s": t2 - t1,
                     "fallback": int(fb[0]),
                     "gap": float(np.abs(a - b).max() / max(np.abs(a).max(), 1e-30)),
                     "pred_err": float(np.abs(p0.cpu().numpy() - a).max() /
                                       max(np.abs(a).max(), 1e-30))})
    return rows


def summarize(rows):
    cs = np.array([r["cold_steps"] for r in rows], float)
    ws = np.array([r["warm_steps"] for r in rows], float)
    ct = np.array([r["cold_s"] for r in rows])
    wt = np.array([r["warm_s"] for r in rows])
    pe = np.array([r["pred_err"] for r in rows])
    return {
        "n": len(rows),
        "cold_steps_mean": float(cs.mean()), "warm_steps_mean": float(ws.mean()),
        "cold_steps_median": float(np.median(cs)), "warm_steps_median": float(np.median(ws)),
        "cold_steps_p95": float(np.percentile(cs, 95)), "warm_steps_p95": float(np.percentile(ws, 95)),
        "cold_ms_mean": float(ct.mean() * 1e3), "warm_ms_mean": float(wt.mean() * 1e3),
        "step_ratio_mean": float((cs / np.maximum(ws, 1)).mean()),
        "pred_rel_linf_median": float(np.median(pe)),
        "warm_faster_fraction": float((wt < ct).mean()),
        "fallbacks": int(sum(r["fallback"] for r in rows)),
    }

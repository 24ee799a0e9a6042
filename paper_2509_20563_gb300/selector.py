"""Training and storage of the per-block predictor selector network.

The training loop is driven from Python, but every step runs in the
library's kernels: labels and features come from fz_block_report (the
exhaustive trial over the four predictors), gradients from fz_mlp_grad
and updates from fz_mlp_adam.  torch only holds the device buffers and
draws the minibatch order.

A weights blob is the FZ_SELECTOR_WEIGHTS bfloat16 values followed by
their float32 master copy; ``save``/``load`` write and check it together
with a SHA-256 digest.
"""
from __future__ import annotations

import hashlib
import json
import math
import os

import numpy as np
import torch

from . import SELECTOR_FEATURES, SELECTOR_WEIGHTS, block_report, mlp_adam, mlp_grad

N_FEAT, N_HID, N_PRED = SELECTOR_FEATURES, 64, 4


def init_weights(seed: int = 0, device="cuda") -> torch.Tensor:
    """He-style initialisation of the float32 master weights (layout W1, b1,
    W2, b2); features are log2-scaled statistics of order 10."""
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    w1 = torch.randn(N_HID * N_FEAT, generator=g) * math.sqrt(2.0 / N_FEAT) / 10.0
    b1 = torch.zeros(N_HID)
    w2 = torch.randn(N_PRED * N_HID, generator=g) * math.sqrt(1.0 / N_HID)
    b2 = torch.zeros(N_PRED)
    return torch.cat([w1, b1, w2, b2]).to(device=device, dtype=torch.float32).contiguous()


def to_bf16_bits(w: torch.Tensor) -> torch.Tensor:
    return w.to(torch.bfloat16).view(torch.int16).contiguous()


def collect(fields, eb: float, mode: str = "rel"):
    """Features and exhaustive labels of all blocks of the given 3D fields."""
    feats, labs = [], []
    for x in fields:
        lab, _, fea = block_report(x, eb, mode, costs=False)
        feats.append(fea)
        labs.append(lab)
    return torch.cat(feats).contiguous(), torch.cat(labs).contiguous()


def train(feat: torch.Tensor, labels: torch.Tensor, epochs: int = 8, batch: int = 4096, lr: float = 3e-3,
          seed: int = 0, w0: torch.Tensor | None = None, log=None):
    """Adam on minibatches; returns (master weights, bf16 bits, loss history)."""
    dev = feat.device
    w = init_weights(seed, dev) if w0 is None else w0.clone()
    m = torch.zeros_like(w)
    v = torch.zeros_like(w)
    wb = torch.empty(SELECTOR_WEIGHTS, dtype=torch.int16, device=dev)
    grad = torch.empty_like(w)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    n = labels.numel()
    step = 0
    hist = []
    for ep in range(epochs):
        order = torch.randperm(n, generator=g, device=dev)
        tot, cnt = 0.0, 0
        for s in range(0, n - batch + 1, batch):
            idx = order[s:s + batch]
            fb = feat[idx].contiguous()
            lb = labels[idx].contiguous()
            step += 1
            want = (s // batch) % 64 == 0
            _, loss = mlp_grad(w, fb, lb, grad, want_loss=want)
            lr_t = lr * (0.5 * (1 + math.cos(math.pi * ep / max(1, epochs))))
            mlp_adam(w, grad, m, v, step, lr_t, w_bf16=wb)
            if want:
                tot += loss
                cnt += 1
        hist.append(tot / max(1, cnt))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4f}")
    return w, wb, hist


def accuracy(wb: torch.Tensor, feat: torch.Tensor, labels: torch.Tensor) -> float:
    """Share of blocks where the network's choice equals the exhaustive
    label (evaluated with torch in float32, for reporting only)."""
    w = wb.view(torch.bfloat16).float()
    o1 = N_HID * N_FEAT
    W1 = w[:o1].view(N_HID, N_FEAT)
    b1 = w[o1:o1 + N_HID]
    W2 = w[o1 + N_HID:o1 + N_HID + N_PRED * N_HID].view(N_PRED, N_HID)
    b2 = w[-N_PRED:]
    f = feat.view(torch.bfloat16).float()
    h = torch.relu(f @ W1.T + b1)
    pred = (h @ W2.T + b2).argmax(1)
    return float((pred == labels.long()).float().mean())


def save(path: str, wb: torch.Tensor, w: torch.Tensor, meta: dict | None = None) -> str:
    blob = wb.cpu().numpy().astype(np.int16).tobytes() + w.cpu().numpy().astype(np.float32).tobytes()
    digest = hashlib.sha256(blob).hexdigest()
    with open(path, "wb") as f:
        f.write(blob)
    with open(path + ".json", "w") as f:
        json.dump({"sha256": digest, "n_weights": SELECTOR_WEIGHTS, **(meta or {})}, f, indent=1)
    return digest


def load(path: str, device="cuda"):
    blob = open(path, "rb").read()
    meta = json.load(open(path + ".json"))
    if hashlib.sha256(blob).hexdigest() != meta["sha256"]:
        raise ValueError(f"{path}: checksum mismatch")
    nb = 2 * SELECTOR_WEIGHTS
    wb = torch.from_numpy(np.frombuffer(blob[:nb], np.int16).copy()).to(device)
    w = torch.from_numpy(np.frombuffer(blob[nb:], np.float32).copy()).to(device)
    return wb, w, meta

"""Learned ACA rank model: data from the method itself, training on the GPU.

Training pairs come from H-matrices built without the model: for every
admissible block the library reports its 8 geometric features and the rank ACA
reached (hm_block_features). The MLP 8 -> 64 -> 64 -> 1 is trained with the
library's own forward/backward kernels (hm_mlp_loss_grad) and Adam
(hm_mlp_adam); this module only drives the loop. The trained weights are passed
to hm_build_ex (rank_model_theta), which reserves ceil(1.25 (2^yhat - 1) + 2)
columns per block and re-runs the blocks whose prediction was too small.
"""
from __future__ import annotations

import json
import time

import numpy as np

from . import hm, inputs

NPARAM = hm.MLP_NPARAM

# Training workloads: the families of the benchmark workloads at smaller sizes
# and other seeds than the ones the model is evaluated on.
TRAIN_SETS = (
    dict(points="uniform", n=4096, d=2, kernel=0, ell=0.1, leaf=32, eta=1.0, eps=1e-8,
         adm_max=True, seed=1101),
    dict(points="mixture", n=1 << 18, d=2, kernel=0, ell=0.1, leaf=64, eta=1.0, eps=1e-6,
         adm_max=False, seed=1103),
    dict(points="uniform", n=1 << 17, d=3, kernel=1, ell=0.2, leaf=64, eta=1.0, eps=1e-6,
         adm_max=False, seed=1102),
)


def init_theta(seed: int = 77) -> np.ndarray:
    """He-uniform weights, zero biases, flattened in the library's order."""
    w1 = inputs.he_uniform(8, 64, seed)
    w2 = inputs.he_uniform(64, 64, seed + 1)
    w3 = inputs.he_uniform(64, 1, seed + 2)
    th = np.concatenate([w1.ravel(), np.zeros(64), w2.ravel(), np.zeros(64), w3.ravel(),
                         [1.5]])
    assert th.size == NPARAM
    return th.astype(np.float32)


def block_data(points, kernel, ell, leaf, eta, eps, adm_max=False, precision=hm.PREC_MIXED):
    """(features, targets) of all admissible blocks of one build without the model."""
    H = hm.HMatrix(points, kernel, ell, leaf, eta, eps, adm_max=adm_max, precision=precision)
    F, T = H.features()
    H.free()
    return F, T


def training_data(sets=TRAIN_SETS, precision=hm.PREC_MIXED):
    Fs, Ts = [], []
    for s in sets:
        if s["points"] == "uniform":
            pts = inputs.uniform_points(s["n"], s["d"], s["seed"])
        else:
            pts = inputs.mixture_points(s["n"], s["d"], s["seed"])
        F, T = block_data(pts, s["kernel"], s["ell"], s["leaf"], s["eta"], s["eps"],
                          s.get("adm_max", False), precision)
        Fs.append(F)
        Ts.append(T)
    return np.concatenate(Fs), np.concatenate(Ts)


def train(F, T, epochs: int = 20, batch: int = 16384, lr: float = 2e-3, seed: int = 5,
          theta0=None, verbose: bool = False):
    """Adam on the GPU with the library kernels; returns (theta, history)."""
    import torch
    dev = "cuda"
    Fd = torch.from_numpy(np.ascontiguousarray(F, np.float32)).to(dev)
    Td = torch.from_numpy(np.ascontiguousarray(T, np.float32)).to(dev)
    th = torch.from_numpy(init_theta() if theta0 is None else np.asarray(theta0, np.float32)).to(dev)
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    g = torch.zeros_like(th)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    n = F.shape[0]
    rng = np.random.default_rng(seed)
    step = 0
    hist = []
    t0 = time.time()
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(n)).to(dev)
        Fe = Fd[perm].contiguous()
        Te = Td[perm].contiguous()
        tot = 0.0
        nb = 0
        for b0 in range(0, n, batch):
            Fb = Fe[b0:b0 + batch]
            Tb = Te[b0:b0 + batch]
            hm.mlp_loss_grad(th, Fb, Tb, g, loss)
            step += 1
            hm.mlp_adam(th, g, m, v, step, lr=lr)
            tot += float(loss.item()) if (nb % 16 == 0) else 0.0
            nb += 1
        # full-data loss at the end of the epoch
        hm.mlp_loss_grad(th, Fd, Td, g, loss)
        hist.append(float(loss.item()))
        if verbose:
            print("epoch %d loss %.4f (%.1fs)" % (ep, hist[-1], time.time() - t0))
    torch.cuda.synchronize()
    return th.cpu().numpy(), hist


def predict(theta, F):
    """yhat = MLP(F) with the library's forward kernel."""
    import torch
    th = torch.from_numpy(np.asarray(theta, np.float32)).cuda()
    Fd = torch.from_numpy(np.ascontiguousarray(F, np.float32)).cuda()
    out = torch.empty(F.shape[0], dtype=torch.float32, device="cuda")
    hm.mlp_forward(th, Fd, out)
    return out.cpu().numpy()


def reserved_rank(yhat):
    """Columns the build reserves for a prediction (before clamping)."""
    return np.maximum(np.ceil(1.25 * (np.exp2(np.minimum(yhat, 8.0)) - 1.0) + 2.0), 1.0)


LAYOUT = "W1 (64 x 8), b1 (64), W2 (64 x 64), b2 (64), W3 (1 x 64), b3 (1); row-major, float32"


def save(path, theta, meta=None) -> None:
    """Write trained weights (the library's flat order, NPARAM float32 values)
    and a JSON description (features, training sets, losses, ...) to an .npz
    file, so that later builds reuse a model without training it again."""
    theta = np.asarray(theta, np.float32).ravel()
    if theta.size != NPARAM:
        raise ValueError("theta has %d values, the model has %d" % (theta.size, NPARAM))
    m = dict(meta or {})
    m["nparam"] = NPARAM
    m["layout"] = LAYOUT
    np.savez(path, theta=theta, meta=np.frombuffer(json.dumps(m).encode(), np.uint8))


def load(path):
    """(theta, meta) written by save(); raises ValueError for another layout."""
    with np.load(path) as z:
        theta = np.array(z["theta"], np.float32)
        meta = json.loads(bytes(z["meta"]).decode())
    if theta.size != NPARAM or meta.get("nparam") != NPARAM or meta.get("layout") != LAYOUT:
        raise ValueError("not a weight file of this model")
    return theta, meta

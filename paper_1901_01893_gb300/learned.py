"""Learned warm start: data, training and evaluation on the GPU (host logic only).

Every computation runs in the library's kernels through the C ABI (smsm.py):
the synthetic acquisitions are imaged by ``smsm_forward``, the training targets
are plain-method reconstructions by ``smsm_reconstruct``, the network is trained
by ``smsm_cnn_train_step`` and applied by ``smsm_learned_start``.  This module
only draws the seeded inputs (``synth``), moves tensors and keeps the books.

The paper has no learned component; the network seeds the iteration of Eq. 10
(its first k-space, Gram and annihilating filters, Eq. 9).  The plain iteration
remains the arbiter: a learned solve whose data residual ||A x - y|| / ||y|| is
above the plain method's residuals on the training set (their largest value,
with a 5 % margin) is thrown away and the group is solved again by the plain
method from A^H y (the fallback), and its cost is counted.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import smsm, synth


@dataclass
class Workload:
    L: int
    Ns: int
    Nc: int
    N: int
    r: int
    K: int = 20
    J: int = 15
    lam: float = 1e-2
    snr: float = 30.0
    field: bool = True
    caipi_div: int = 0

    @property
    def B(self) -> int:
        return self.L * self.Ns


def synthesize(w: Workload, seeds, one: smsm.Plan, dev) -> dict:
    """y (RMS 1), the truth x_true = F(rho phi) (same scale) for the seeded groups, on the GPU.
    Every group shares the coil maps of `one` (the generator's maps depend only on the geometry)."""
    c64 = lambda a: torch.from_numpy(np.ascontiguousarray(a).astype(np.complex64)).to(dev)  # noqa: E731
    ys, xts = [], []
    for s in seeds:
        g = synth.make_group(w.L, w.Ns, w.Nc, w.N, int(s), field=w.field)
        xt = one.fft2c(c64(g["rho"][:, None] * g["phase"]))  # x_true = F(rho phi), Eq. 4
        yc = one.forward(xt)
        nz = c64(g["noise"])
        yd = yc + nz * (torch.linalg.vector_norm(yc) / (w.snr * torch.linalg.vector_norm(nz)))
        sc = torch.sqrt(torch.mean(torch.abs(yd) ** 2))
        ys.append(yd / sc)
        xts.append(xt / sc)
    return {"y": torch.stack(ys), "xt": torch.stack(xts)}


def sens_of(w: Workload) -> np.ndarray:
    return synth.make_group(w.L, w.Ns, w.Nc, w.N, 0, field=False)["sens"]


def plain_params(w: Workload, K: int | None = None, **kw) -> smsm.Params:
    return smsm.default_params(lam=w.lam, outer_iters=w.K if K is None else K, cg_iters=w.J, **kw)


def solve_batches(w: Workload, plan: smsm.Plan, y: torch.Tensor, prm: smsm.Params, x0: torch.Tensor | None = None):
    """Reconstruct every group of y [n][...] with the batched plan (D per call); x0 = warm starts."""
    D = plan.D
    out = torch.empty((y.shape[0],) + tuple(plan.x_shape[1:]), dtype=torch.complex64, device=y.device)
    for i in range(0, y.shape[0], D):
        n = min(D, y.shape[0] - i)
        yb = y[i:i + D]
        if n < D:  # pad the last batch by repeating its first group
            yb = torch.cat([yb, yb[:1].expand(D - n, *yb.shape[1:])])
        xb = torch.empty(plan.x_shape, dtype=torch.complex64, device=y.device)
        if x0 is not None:
            xs = x0[i:i + D]
            xb.copy_(torch.cat([xs, xs[:1].expand(D - n, *xs.shape[1:])]) if n < D else xs)
        xb, rep = plan.reconstruct(yb.contiguous(), x=xb, params=prm)
        out[i:i + n] = xb[:n]
    return out


def images(plan_one: smsm.Plan, x: torch.Tensor) -> torch.Tensor:
    """F^-1 of k-space [n][L][Ns][N][N] -> [n][L*Ns][N][N] images."""
    n = x.shape[0]
    return plan_one.fft2c(x.reshape(n, -1, x.shape[-2], x.shape[-1]).contiguous(), inverse=True)


def residual(plan_one: smsm.Plan, x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """||A x - y|| / ||y|| per group."""
    out = []
    for k in range(x.shape[0]):
        r = plan_one.forward(x[k].contiguous()) - y[k]
        out.append(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(y[k]))
    return torch.stack(out)


def nrmse(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """||a - b|| / ||b|| per group (first axis)."""
    n = a.shape[0]
    return torch.linalg.vector_norm((a - b).reshape(n, -1), dim=1) / torch.linalg.vector_norm(b.reshape(n, -1), dim=1)


def init_params(w: Workload, width: int, layers: int, seed: int, dev, last_scale: float = 0.1) -> torch.Tensor:
    """He-style complex initialisation (zero bias); the last layer scaled so the network
    starts close to x0 = a."""
    rng = np.random.default_rng(seed)
    ch = [w.B] + [width] * (layers - 1) + [w.B]
    parts = []
    for k in range(layers):
        ci, co = ch[k], ch[k + 1]
        std = math.sqrt(2.0 / (9 * ci)) / math.sqrt(2.0)
        W = std * (rng.standard_normal((co, ci, 3, 3)) + 1j * rng.standard_normal((co, ci, 3, 3)))
        if k + 1 == layers:
            W *= last_scale
        parts += [W.ravel(), np.zeros(co)]
    return torch.from_numpy(np.concatenate(parts).astype(np.complex64)).to(dev)


@dataclass
class TrainReport:
    losses: list = field(default_factory=list)
    seconds: float = 0.0
    steps: int = 0


def train(net: smsm.CNN, a: torch.Tensor, t: torch.Tensor, epochs: int, batch: int, lr: float,
          seed: int = 0) -> TrainReport:
    """Adam on mini-batches of (a, t) [n][B][N][N]; a seeded shuffle per epoch; cosine-decayed lr."""
    rep = TrainReport()
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = a.shape[0]
    nsteps = epochs * (n // batch)
    step = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(a.device)
        tot = 0.0
        for i in range(0, n - batch + 1, batch):
            idx = perm[i:i + batch]
            lr_k = lr * 0.5 * (1 + math.cos(math.pi * step / max(nsteps, 1)))
            tot += net.train_step(a[idx].contiguous(), t[idx].contiguous(), max(lr_k, 1e-3 * lr))
            step += 1
        rep.losses.append(tot / max(1, n // batch))
    torch.cuda.synchronize()
    rep.seconds = time.perf_counter() - t0
    rep.steps = step
    return rep

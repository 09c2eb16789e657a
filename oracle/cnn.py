"""FP64 CPU oracle of the learned warm start's complex CNN -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this module; it shares no code with the CUDA path.

The paper has no learned component: this network is the warm start that seeds
the k-space and the annihilating filters (Eq. 9) of the IRLS solve of Eq. 10.
It maps the aliased, zero-filled image of every (slice, shot),
a = F^-1(A^H y), to a starting image x0 = a + f(a), the residual f computed by
six complex 3x3 convolutions (channels B -> 64 -> 64 -> 64 -> 64 -> 64 -> B,
B = L * Ns) with CReLU between them (ReLU on the real and on the imaginary part).

Complex convolution (cross-correlation, zero padding, one pixel of halo):
    z[o, p] = b[o] + sum_c sum_{k in {0,1,2}^2} W[o, c, k] h[c, p + k - 1].
Gradients of a real loss L are carried as G = dL/dRe + i dL/dIm; for z = W h
that gives dL/dh = conj(W) G and dL/dW = conj(h) G, so
    dW[o, c, k] = sum_p G[o, p] conj(h[c, p + k - 1]),   db[o] = sum_p G[o, p],
    Gh[c, q]    = sum_o sum_k conj(W[o, c, k]) G[o, q - k + 1],
and CReLU passes each component of G where that component of its input is > 0.
Loss of one sample: ||x0 - t||^2 / ||t||^2 (the squared NRMSE of the start
against the target image t).

Written as plain loops over the 3x3 taps with NumPy array products, in FP64.
"""
from __future__ import annotations

import numpy as np

WIDTH = 64
LAYERS = 6


def layer_shapes(B: int, width: int = WIDTH, layers: int = LAYERS) -> list[tuple[int, int]]:
    """(out, in) channels of every convolution."""
    ch = [B] + [width] * (layers - 1) + [B]
    return [(ch[k + 1], ch[k]) for k in range(layers)]


def conv3x3(h: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """z[o] = b[o] + sum_c sum_k W[o, c, k] h[c, p + k - 1]; h [Cin][H][W'], W [Cout][Cin][3][3]."""
    C, H, Wd = h.shape
    hp = np.zeros((C, H + 2, Wd + 2), dtype=np.complex128)
    hp[:, 1:H + 1, 1:Wd + 1] = h
    z = np.zeros((W.shape[0], H, Wd), dtype=np.complex128) + b[:, None, None]
    for ky in range(3):
        for kx in range(3):
            win = hp[:, ky:ky + H, kx:kx + Wd].reshape(C, H * Wd)
            z += (W[:, :, ky, kx] @ win).reshape(-1, H, Wd)
    return z


def conv3x3_grads(h: np.ndarray, W: np.ndarray, G: np.ndarray):
    """Gradients through one convolution: (dW, db, Gh) for the output gradient G."""
    C, H, Wd = h.shape
    hp = np.zeros((C, H + 2, Wd + 2), dtype=np.complex128)
    hp[:, 1:H + 1, 1:Wd + 1] = h
    Gf = G.reshape(G.shape[0], H * Wd)
    dW = np.zeros_like(W, dtype=np.complex128)
    Ghp = np.zeros((C, H + 2, Wd + 2), dtype=np.complex128)
    for ky in range(3):
        for kx in range(3):
            win = hp[:, ky:ky + H, kx:kx + Wd].reshape(C, H * Wd)
            dW[:, :, ky, kx] = Gf @ np.conj(win).T
            Ghp[:, ky:ky + H, kx:kx + Wd] += (np.conj(W[:, :, ky, kx]).T @ Gf).reshape(C, H, Wd)
    return dW, Gf.sum(axis=1), Ghp[:, 1:H + 1, 1:Wd + 1]


def crelu(z: np.ndarray) -> np.ndarray:
    return np.maximum(z.real, 0.0) + 1j * np.maximum(z.imag, 0.0)


def crelu_grad(z: np.ndarray, G: np.ndarray) -> np.ndarray:
    return G.real * (z.real > 0) + 1j * (G.imag * (z.imag > 0))


def forward(a: np.ndarray, params: list, keep: bool = False):
    """x0 = a + f(a) for one sample a [B][H][W]; params = [(W, b)] per layer.
    With ``keep`` also returns the layer inputs and pre-activations."""
    h, hs, zs = a, [], []
    for k, (W, b) in enumerate(params):
        hs.append(h)
        z = conv3x3(h, W, b)
        zs.append(z)
        h = crelu(z) if k + 1 < len(params) else z
    out = a + h
    return (out, hs, zs) if keep else out


def loss(out: np.ndarray, t: np.ndarray) -> float:
    return float(np.sum(np.abs(out - t) ** 2) / np.sum(np.abs(t) ** 2))


def backward(a: np.ndarray, t: np.ndarray, params: list):
    """Loss of one sample and its gradients [(dW, db)] per layer (manual backward)."""
    out, hs, zs = forward(a, params, keep=True)
    G = 2.0 * (out - t) / np.sum(np.abs(t) ** 2)
    grads = [None] * len(params)
    for k in reversed(range(len(params))):
        if k + 1 < len(params):
            G = crelu_grad(zs[k], G)
        dW, db, G = conv3x3_grads(hs[k], params[k][0], G)
        grads[k] = (dW, db)
    return loss(out, t), grads


def init_params(rng: np.random.Generator, B: int, width: int = WIDTH, layers: int = LAYERS,
                last_scale: float = 0.1) -> list:
    """He-style initialisation of complex weights (variance 2 / (9 Cin) split between
    the real and imaginary parts), zero bias; the last layer scaled down so the
    network starts near the identity map x0 = a."""
    params = []
    shapes = layer_shapes(B, width, layers)
    for k, (co, ci) in enumerate(shapes):
        std = np.sqrt(2.0 / (9 * ci)) / np.sqrt(2.0)
        W = std * (rng.standard_normal((co, ci, 3, 3)) + 1j * rng.standard_normal((co, ci, 3, 3)))
        if k + 1 == len(shapes):
            W *= last_scale
        params.append((W, np.zeros(co, dtype=np.complex128)))
    return params

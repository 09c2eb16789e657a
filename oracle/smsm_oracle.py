"""FP64 CPU oracle for the SMS-MUSSELS reconstruction (Mani et al., 1901.01893).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may call it.  It shares no code with the CUDA path.

Plain NumPy complex128, written to be checked against the paper by eye: the
Hankel matrix is formed explicitly, the Gram is ``H^H H``, the eigensolver is
``numpy.linalg.eigh`` and CG is the textbook recurrence.

Conventions (readings of the paper, where it is silent or garbled):

* Centred unitary DFT ``F_c = fftshift . fft2(norm='ortho') . ifftshift``;
  k-space index n has DC at n = N/2 (the Hankel patches of Eq. 8 must
  surround DC, which needs centred k-space).
* Shot i (0-based) keeps the phase-encode lines n = m*Ns + i (Eq. 2, with the
  1-based line count of the paper shifted to 0-based indices).
* CAIPI phase of slice l (0-based) on line n: exp(-j 2 pi l (n - N/2) / Ldiv)
  (Eq. 1 and Eq. 3; the garbled Delta k_y factor is read as the centred line
  index, which differs from the paper's 1-based n only by a constant phase
  per slice).  Ldiv defaults to L (an FOV/L shift).
* Hankel lifting (Eq. 8): rows are the VALID patch origins k in [0, N-r]^2
  (row-major), columns (i, py, px) -> i*r*r + py*r + px, entry x_i[k + p].
  The PERIODIC variant (``periodic=True``) takes every origin k in [0, N)^2
  with the entry x_i[(k + p) mod N] (k-space treated as periodic).
* Solver: the paper minimises Eq. 10 with an augmented-Lagrangian scheme
  whose pseudo-code lives in another paper; here the same cost is minimised
  by iteratively reweighted least squares (IRLS): the nuclear norm is
  majorised with W = (G + eps I)^(-1/2), G = H^H H, and each outer iteration
  solves (A^H A + lam P_W) x = A^H y by J steps of CG, with
  P_W(x) = H^*(H(x) W) per slice.  ``lam`` here is the weight in these normal
  equations (it equals the lambda of Eq. 10 up to the factor 1/2 of the
  majoriser).
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft as _sfft

# the library FFT (pocketfft) run on every host core: the same transform as
# numpy.fft, threaded over the leading axes
_WORKERS = os.cpu_count() or 1

# ---------------------------------------------------------------------------
# Centred unitary DFT (Fig. 1, steps (i) and (iii))
# ---------------------------------------------------------------------------


def fft2c(img: np.ndarray) -> np.ndarray:
    """Centred unitary 2D DFT over the last two axes."""
    ax = (-2, -1)
    return np.fft.fftshift(_sfft.fft2(np.fft.ifftshift(img, axes=ax), norm="ortho", workers=_WORKERS), axes=ax)


def ifft2c(ksp: np.ndarray) -> np.ndarray:
    """Inverse of :func:`fft2c` (its adjoint: it is unitary)."""
    ax = (-2, -1)
    return np.fft.fftshift(_sfft.ifft2(np.fft.ifftshift(ksp, axes=ax), norm="ortho", workers=_WORKERS), axes=ax)


# ---------------------------------------------------------------------------
# Blipped-CAIPI phase and the multi-shot sampling (Eqs. 1-3)
# ---------------------------------------------------------------------------


def caipi_ramp(L: int, N: int, Ldiv: int | None = None) -> np.ndarray:
    """theta[l][n] = exp(-j 2 pi l (n - N/2) / Ldiv): slice l shifted by l*FOV/Ldiv (Eq. 1)."""
    Ldiv = L if Ldiv is None else Ldiv
    l = np.arange(L)[:, None]
    n = np.arange(N)[None, :]
    return np.exp(-2j * np.pi * l * (n - N / 2) / Ldiv)


def shot_lines(Ns: int, N: int, i: int, offsets=None) -> np.ndarray:
    """Phase-encode lines kept by shot i: n = m*Ns + i, m = 0..N/Ns-1 (Eq. 2).

    ``offsets`` (a permutation of 0..Ns-1, default the identity) lets shot i
    acquire the interleave n = m*Ns + offsets[i] instead: the same sampling
    with the shots relabelled, which the shot-permutation pin uses."""
    o = i if offsets is None else int(offsets[i])
    return np.arange(N // Ns) * Ns + o


# ---------------------------------------------------------------------------
# Forward operator A and its adjoint (Fig. 1; the data term of Eq. 10)
# ---------------------------------------------------------------------------


def forward(x: np.ndarray, sens: np.ndarray, Ns: int | None = None, Ldiv: int | None = None,
            phase: np.ndarray | None = None, full: bool = False, offsets=None) -> np.ndarray:
    """y = A(x), Fig. 1 steps (i)-(v).

    x     : [L][Ns][N][N] per-shot centred k-space (the unknown of Eq. 10), or
            [L][1][N][N] shared k-space when ``phase`` is given (Eq. 4 model).
    sens  : [L][Nc][N][N] coil sensitivities (image domain).
    phase : optional [L][Ns][N][N] image-domain shot phase phi_{l,i} (Eq. 4).
    full  : keep every line for every shot (used only by the exact-recovery pin).
    offsets : line interleave of each shot (see :func:`shot_lines`).
    returns y : [Ns][Nc][N/Ns][N] (or [Ns][Nc][N][N] when ``full``).
    """
    L, S1, N, _ = x.shape
    Nc = sens.shape[1]
    if phase is not None:
        Ns = phase.shape[1]
    elif Ns is None:
        Ns = S1
    theta = caipi_ramp(L, N, Ldiv)
    rows = N if full else N // Ns
    y = np.zeros((Ns, Nc, rows, N), dtype=np.complex128)
    img_all = ifft2c(x)                                  # (i) F^-1 per slice/shot
    for i in range(Ns):
        img = img_all[:, 0 if phase is not None else i]  # [L][N][N]
        if phase is not None:
            img = img * phase[:, i]                      # Eq. 4: rho_l * phi_{l,i}
        coil = sens * img[:, None]                       # (ii) [L][Nc][N][N]
        K = fft2c(coil)                                  # (iii)
        Ksum = np.sum(theta[:, None, :, None] * K, axis=0)  # (iv) CAIPI phase + slice sum
        lines = np.arange(N) if full else shot_lines(Ns, N, i, offsets)
        y[i] = Ksum[:, lines, :]                         # (v) shot mask
    return y


def adjoint(y: np.ndarray, sens: np.ndarray, L: int, Ldiv: int | None = None,
            phase: np.ndarray | None = None, full: bool = False, offsets=None) -> np.ndarray:
    """x = A^H(y): the transpose of each step of :func:`forward`, in reverse order."""
    Ns, Nc, rows, N = y.shape
    theta = caipi_ramp(L, N, Ldiv)
    out = np.zeros((L, 1 if phase is not None else Ns, N, N), dtype=np.complex128)
    for i in range(Ns):
        Kfull = np.zeros((Nc, N, N), dtype=np.complex128)
        lines = np.arange(N) if full else shot_lines(Ns, N, i, offsets)
        Kfull[:, lines, :] = y[i]                                 # (v)^H
        K = np.conj(theta)[:, None, :, None] * Kfull[None]        # (iv)^H [L][Nc][N][N]
        coil = ifft2c(K)                                          # (iii)^H
        img = np.sum(np.conj(sens) * coil, axis=1)                # (ii)^H [L][N][N]
        if phase is not None:
            out[:, 0] += np.conj(phase[:, i]) * img
        else:
            out[:, i] = img
    return fft2c(out)                                             # (i)^H


def normal(x: np.ndarray, sens: np.ndarray, Ldiv: int | None = None, offsets=None) -> np.ndarray:
    """A^H A x for the per-shot unknown."""
    L, Ns = x.shape[:2]
    return adjoint(forward(x, sens, Ns=Ns, Ldiv=Ldiv, offsets=offsets), sens, L, Ldiv=Ldiv, offsets=offsets)


# ---------------------------------------------------------------------------
# Hankel lifting, Gram, weights (Eqs. 8-9; nuclear norm of Eq. 10)
# ---------------------------------------------------------------------------


def hankel(xl: np.ndarray, r: int, periodic: bool = False) -> np.ndarray:
    """Block Hankel matrix H_l = [H(x_{l,1}) ... H(x_{l,Ns})] of Eq. 9.

    xl : [Ns][N][N]; returns [(N-r+1)^2][Ns*r*r] with entry x_i[k + p]
    (periodic: [N^2][Ns*r*r] with entry x_i[(k + p) mod N]).
    """
    Ns, N, _ = xl.shape
    if periodic:
        # wrap the first r-1 rows and columns around, then the VALID windows of
        # the extended image are exactly the N^2 periodic patches
        xl = np.concatenate([xl, xl[:, : r - 1, :]], axis=1)
        xl = np.concatenate([xl, xl[:, :, : r - 1]], axis=2)
    win = np.lib.stride_tricks.sliding_window_view(xl, (r, r), axis=(1, 2))
    # win[i, ky, kx, py, px] = xl[i, ky+py, kx+px]
    V = N if periodic else N - r + 1
    return np.ascontiguousarray(win.transpose(1, 2, 0, 3, 4)).reshape(V * V, Ns * r * r)


def hankel_adjoint(Y: np.ndarray, Ns: int, N: int, r: int, periodic: bool = False) -> np.ndarray:
    """H^*(Y): every entry Y[k, (i,p)] goes back to pixel k + p (mod N when
    periodic) of shot i."""
    V = N if periodic else N - r + 1
    Yr = Y.reshape(V, V, Ns, r, r)
    out = np.zeros((Ns, N, N), dtype=np.complex128)
    for py in range(r):
        for px in range(r):
            blk = Yr[:, :, :, py, px].transpose(2, 0, 1)
            if periodic:
                out += np.roll(blk, (py, px), axis=(1, 2))
            else:
                out[:, py:py + V, px:px + V] += blk
    return out


def gram(x: np.ndarray, r: int, periodic: bool = False) -> np.ndarray:
    """G_l = H_l^H H_l for every slice: [L][C][C], C = Ns*r*r."""
    out = []
    for l in range(x.shape[0]):
        H = hankel(x[l], r, periodic)
        out.append(H.conj().T @ H)
    return np.stack(out)


def irls_weight(G: np.ndarray, eps: float) -> tuple[np.ndarray, np.ndarray]:
    """W = V diag((s + eps)^(-1/2)) V^H per slice (majoriser of the nuclear norm, Eq. 10).

    Eigenvalues are clamped at 0 first (G is PSD; rounding can leave tiny
    negatives).  Returns (W [L][C][C], eigenvalues [L][C] ascending).
    """
    Ws, ss = [], []
    for Gl in G:
        s, V = np.linalg.eigh(Gl)
        f = 1.0 / np.sqrt(np.maximum(s, 0.0) + eps)
        Ws.append((V * f[None, :]) @ V.conj().T)
        ss.append(s)
    return np.stack(Ws), np.stack(ss)


def nullspace_weight(G: np.ndarray, rank: int) -> tuple[np.ndarray, np.ndarray]:
    """W = V_n V_n^H onto the C - rank smallest eigenvectors (one rank for every
    slice, the Methods' choice of a common rank)."""
    Ws, ss = [], []
    for Gl in G:
        s, V = np.linalg.eigh(Gl)
        Vn = V[:, : Gl.shape[0] - rank]
        Ws.append(Vn @ Vn.conj().T)
        ss.append(s)
    return np.stack(Ws), np.stack(ss)


def penalty(x: np.ndarray, W: np.ndarray, r: int, periodic: bool = False) -> np.ndarray:
    """P_W(x)_l = H_l^*(H_l(x_l) W_l): the gradient (up to 2) of ||H_l(x) W^(1/2)||_F^2."""
    L, Ns, N, _ = x.shape
    out = np.empty_like(x, dtype=np.complex128)
    for l in range(L):
        H = hankel(x[l], r, periodic)
        out[l] = hankel_adjoint(H @ W[l], Ns, N, r, periodic)
    return out


# ---------------------------------------------------------------------------
# Textbook conjugate gradients
# ---------------------------------------------------------------------------


def vdot(a: np.ndarray, b: np.ndarray) -> complex:
    """<a, b> = sum conj(a) b."""
    return np.vdot(a.ravel(), b.ravel())


def cg(apply_N, b: np.ndarray, x: np.ndarray, J: int) -> tuple[np.ndarray, list[float]]:
    """J steps of CG on the Hermitian positive definite system N x = b, from x."""
    r = b - apply_N(x)
    p = r.copy()
    rr = vdot(r, r).real
    hist = [rr]
    for _ in range(J):
        q = apply_N(p)
        alpha = rr / vdot(p, q).real
        x = x + alpha * p
        r = r - alpha * q
        rr_new = vdot(r, r).real
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        hist.append(rr)
    return x, hist


# ---------------------------------------------------------------------------
# The reconstruction (Eq. 10 by IRLS + CG)
# ---------------------------------------------------------------------------

DEFAULT_PARAMS = dict(lam=1e-2, eps0_rel=1e-2, eta=1.5, eps_min_rel=1e-2, K=10, J=10,
                      mode="irls", rank=0, periodic=False)


def reconstruct(y: np.ndarray, sens: np.ndarray, r: int, params: dict | None = None,
                x0: np.ndarray | None = None, Ldiv: int | None = None,
                report: dict | None = None, offsets=None) -> np.ndarray:
    """SMS-MUSSELS joint recovery of the slice-unfolded per-shot k-space.

    Outer iteration k = 1..K: G_l = H_l^H H_l of the current x; eigen-
    decomposition; weight W_l; then J CG steps on
    (A^H A + lam P_W) x = A^H y from the current x.
    eps_1 = eps0_rel * max_l s_max(G_l) at k = 1, eps_k = max(eps_{k-1}/eta,
    eps_min_rel * eps_1).

    ``report`` (a dict, optional) receives ``hist``: per outer iteration its
    eps and the CG residual norms; with ``report["keep_iterates"]`` true also
    the weight W used and the iterate x after that iteration's CG steps.
    ``offsets``: line interleave of each shot (see :func:`shot_lines`).
    """
    p = dict(DEFAULT_PARAMS)
    if params:
        p.update(params)
    Ns = y.shape[0]
    L = sens.shape[0]
    b = adjoint(y, sens, L, Ldiv=Ldiv, offsets=offsets)
    x = b.copy() if x0 is None else np.array(x0, dtype=np.complex128)
    eps = eps_min = None
    hist = []
    keep = bool(report is not None and report.get("keep_iterates"))
    per = bool(p["periodic"])
    for k in range(p["K"]):
        G = gram(x, r, per)
        if p["mode"] == "nullspace":
            W, s = nullspace_weight(G, p["rank"])
        else:
            if k == 0:
                s0 = np.max([np.linalg.eigvalsh(Gl)[-1] for Gl in G])
                eps = p["eps0_rel"] * s0
                eps_min = p["eps_min_rel"] * eps
            else:
                eps = max(eps / p["eta"], eps_min)
            W, s = irls_weight(G, eps)
        lam = p["lam"]

        def apply_N(v, W=W):
            return normal(v, sens, Ldiv, offsets) + lam * penalty(v, W, r, per)

        x, h = cg(apply_N, b, x, p["J"])
        hist.append(dict(eps=eps, rr=h, W=W, x=x.copy()) if keep else dict(eps=eps, rr=h))
    if report is not None:
        report["hist"] = hist
    return x


def sense(y: np.ndarray, sens: np.ndarray, L: int, J: int, phase: np.ndarray | None = None,
          Ldiv: int | None = None) -> np.ndarray:
    """SMS-SENSE, the comparison reconstruction of the paper's figures: the k-space
    data of all shots combined into one k-space per slice (the shot-shared model of
    Eq. 4, with the image-domain phase ``phase`` or, when it is None, without any
    phase correction) and the slices unfolded by least squares, J CG steps on
    A^H A x = A^H y from x = 0.  Returns x [L][1][N][N]."""
    Ns, _, _, N = y.shape
    ph = np.ones((L, Ns, N, N), dtype=np.complex128) if phase is None else phase
    b = adjoint(y, sens, L, Ldiv=Ldiv, phase=ph)

    def apply_N(v):
        return adjoint(forward(v, sens, Ldiv=Ldiv, phase=ph), sens, L, Ldiv=Ldiv, phase=ph)

    x, _ = cg(apply_N, b, np.zeros_like(b), J)
    return x


# ---------------------------------------------------------------------------
# Outputs and error measures
# ---------------------------------------------------------------------------


def magnitude(x: np.ndarray) -> np.ndarray:
    """rho_hat_l = sqrt(sum_i |F^-1 x_{l,i}|^2 / Ns): the shot phase is dropped
    (the paper ignores the phase once the shots are recovered, Eqs. 4-5)."""
    return np.sqrt(np.mean(np.abs(ifft2c(x)) ** 2, axis=1))


def nrmse(a: np.ndarray, b: np.ndarray, axis=None) -> np.ndarray:
    """||a - b|| / ||b|| (per slice when ``axis`` names the non-slice axes)."""
    if axis is None:
        return np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.asarray(b).ravel())
    return np.sqrt(np.sum(np.abs(a - b) ** 2, axis=axis) / np.sum(np.abs(b) ** 2, axis=axis))


def make_data(group: dict, snr: float | None, Ldiv: int | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Ground truth x_true = F_c(rho_l phi_{l,i}) (Eq. 4) and y = A x_true + noise.

    The noise draws of ``group`` are scaled so ||noise|| / ||A x_true|| = 1/snr
    (SNR read as a linear amplitude ratio); ``snr=None`` gives noiseless data.
    """
    rho, phase, sens = group["rho"], group["phase"], group["sens"]
    x_true = fft2c(rho[:, None] * phase)
    y = forward(x_true, sens, Ldiv=Ldiv)
    if snr is not None:
        n = group["noise"]
        y = y + n * (np.linalg.norm(y) / (snr * np.linalg.norm(n)))
    return x_true, y

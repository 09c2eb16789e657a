"""Seeded synthetic acquisitions shaped like the paper's SMS multi-shot DWI data.

This module only draws random numbers and rasterises simple shapes; it holds
none of the reconstruction's arithmetic (no Fourier transform, no CAIPI phase,
no Hankel lifting).  It is the one module that both the CUDA path (through
``bench.py``) and the FP64 oracle (through the tests) read their inputs from.

What is drawn, per slice group (the paper's own data -- in-vivo 128x128,
32-channel, MB 2-3, 2/4-shot acquisitions, Methods section -- is not
available, so these stand in for it):

* ``rho[L][N][N]``: the magnitude DWI of each slice (the rho_l of Eq. 4):
  10 random ellipses with additive intensities U(0.1, 1).
* ``phase[L][Ns][N][N]``: the per-shot, per-slice phase phi_{l,i} of Eq. 4:
  exp(j * (cubic polynomial with U(-pi, pi) coefficients in FOV units [-1/2, 1/2)^2
  [+ a real field band-limited to k-radius 3, scaled to +-pi])).
* ``sens[L][Nc][N][N]``: Gaussian coil maps centred on a ring (two rows of
  coils; each slice at its own height), constant phase 2*pi*c/Nc, normalised
  to root-sum-of-squares 1.
* ``noise[Ns][Nc][N/Ns][N]``: unit complex Gaussian draws; the caller scales
  them to the requested SNR against its own noiseless data.

Coordinates: pixel index n in [0, N) maps to u = (n - N/2) / (N/2) in [-1, 1).
Arrays are C-ordered with the x (readout, kx) index fastest.
"""
from __future__ import annotations

import functools

import numpy as np

__all__ = ["CONFIGS", "make_group", "coords", "bandlimited_phase", "draw_phase_coeffs", "phase_from_coeffs"]

# Workloads: the acquisitions the paper reconstructs (Methods: 128x128, 32
# channels, MB 2-3, 2- and 4-shot, filter 4x4 / 6x6), at the sizes the tests
# and the benchmark use.  ``K`` outer (weight) iterations x ``J`` CG iterations.
CONFIGS = {
    "tiny": dict(L=2, Ns=4, Nc=8, N=64, r=5, K=10, J=10, seed=1, field=False,
                 snr=30.0),
    "plain": dict(L=2, Ns=4, Nc=32, N=128, r=6, K=20, J=15, seed=2, field=True,
                  snr=30.0),
    "precision": dict(L=3, Ns=4, Nc=32, N=256, r=6, K=20, J=15, seed=3,
                      field=True, snr=30.0),
}


def coords(N: int) -> np.ndarray:
    """Normalised coordinate u = (n - N/2)/(N/2) of pixel index n."""
    return (np.arange(N, dtype=np.float64) - N / 2) / (N / 2)


def _ellipses(rng: np.random.Generator, N: int, count: int = 10) -> np.ndarray:
    u = coords(N)
    X, Y = np.meshgrid(u, u, indexing="xy")  # X varies along the last axis
    img = np.zeros((N, N), dtype=np.float64)
    for _ in range(count):
        cx, cy = rng.uniform(-0.3, 0.3, size=2)
        a, b = rng.uniform(0.1, 0.4, size=2)
        th = rng.uniform(0.0, np.pi)
        amp = rng.uniform(0.1, 1.0)
        dx, dy = X - cx, Y - cy
        xr = dx * np.cos(th) + dy * np.sin(th)
        yr = -dx * np.sin(th) + dy * np.cos(th)
        img += amp * (((xr / a) ** 2 + (yr / b) ** 2) <= 1.0)
    return img


def _poly_phase(rng: np.random.Generator, N: int) -> np.ndarray:
    # "scaled to the FOV": the polynomial's variables are positions in FOV
    # units, x/FOV in [-1/2, 1/2)
    u = coords(N) / 2
    X, Y = np.meshgrid(u, u, indexing="xy")
    ph = np.zeros((N, N), dtype=np.float64)
    for a in range(4):
        for b in range(4 - a):
            ph += rng.uniform(-np.pi, np.pi) * X ** a * Y ** b
    return ph


def _field(rng: np.random.Generator, N: int, kmax: int = 3) -> np.ndarray:
    """Real field with spatial frequencies |k| <= kmax cycles per FOV, max |f| = pi."""
    u = coords(N)
    k = np.arange(-kmax, kmax + 1)
    # one FOV is 2 units of u, so k cycles per FOV is exp(j*pi*k*u); the 2-D waves are
    # products of 1-D ones, so the sum is E_y^T C E_x with the coefficients C on |k| <= kmax
    E = np.exp(1j * np.pi * np.outer(k, u))  # [k][n]
    Cf = np.zeros((2 * kmax + 1, 2 * kmax + 1), dtype=np.complex128)
    for ky in range(-kmax, kmax + 1):
        for kx in range(-kmax, kmax + 1):
            if kx * kx + ky * ky > kmax * kmax:
                continue
            Cf[ky + kmax, kx + kmax] = rng.standard_normal() + 1j * rng.standard_normal()
    f = np.real(E.T @ Cf @ E)  # f[y][x] = Re sum_{ky,kx} C exp(j pi (ky u_y + kx u_x))
    return f * (np.pi / np.max(np.abs(f)))


@functools.lru_cache(maxsize=8)
def _coils_cached(L: int, Nc: int, N: int) -> np.ndarray:
    S = _coils(L, Nc, N)
    S.setflags(write=False)
    return S


def _coils(L: int, Nc: int, N: int, ring: float = 1.2, sigma: float = 0.6,
           dz_coil: float = 0.4, dz_slice: float = 0.6) -> np.ndarray:
    """Gaussian receive maps of Nc coils on a ring of radius ``ring``.

    Coils alternate between two rows at heights +-dz_coil; slice l sits at
    height (l - (L-1)/2) * dz_slice, so simultaneously excited slices see
    different maps (what SENSE slice unfolding relies on).  Coil c carries the
    constant phase 2*pi*c/Nc.  Each slice's maps are normalised to
    root-sum-of-squares 1 per pixel.
    """
    u = coords(N)
    X, Y = np.meshgrid(u, u, indexing="xy")
    S = np.zeros((L, Nc, N, N), dtype=np.complex128)
    for l in range(L):
        z = (l - (L - 1) / 2) * dz_slice
        for c in range(Nc):
            ang = 2 * np.pi * c / Nc
            zc = dz_coil if c % 2 == 0 else -dz_coil
            d2 = (X - ring * np.cos(ang)) ** 2 + (Y - ring * np.sin(ang)) ** 2 + (z - zc) ** 2
            S[l, c] = np.exp(-d2 / (2 * sigma ** 2)) * np.exp(2j * np.pi * c / Nc)
        S[l] /= np.sqrt(np.sum(np.abs(S[l]) ** 2, axis=0))[None]
    return S


def make_group(L: int, Ns: int, Nc: int, N: int, seed: int, field: bool = False,
               **_unused) -> dict:
    """Draw one slice group.  Same seed -> same arrays on any machine (PCG64)."""
    if N % Ns:
        raise ValueError("N must be a multiple of the shot count")
    rng = np.random.default_rng(seed)
    rho = np.stack([_ellipses(rng, N) for _ in range(L)])
    phase = np.empty((L, Ns, N, N), dtype=np.complex128)
    for l in range(L):
        for i in range(Ns):
            ph = _poly_phase(rng, N)
            if field:
                ph = ph + _field(rng, N)
            phase[l, i] = np.exp(1j * ph)
    sens = _coils_cached(L, Nc, N).copy()  # the maps depend on the geometry only
    noise = (rng.standard_normal((Ns, Nc, N // Ns, N))
             + 1j * rng.standard_normal((Ns, Nc, N // Ns, N))) / np.sqrt(2.0)
    return dict(rho=rho, phase=phase, sens=sens, noise=noise)


def bandlimited_phase(rng: np.random.Generator, L: int, Ns: int, N: int, s: int) -> np.ndarray:
    """Complex 'phase' images whose centred spectrum is supported on s x s samples.

    Used for the rank pins of the annihilation relation (Eqs. 6-9): with such
    phi, the per-slice block Hankel matrix has rank <= (r + s - 1)^2.  Returned
    as the s x s centred k-space coefficient blocks; the caller places them at
    DC and transforms with its own centred DFT.
    """
    return (rng.standard_normal((L, Ns, s, s)) + 1j * rng.standard_normal((L, Ns, s, s)))


def draw_phase_coeffs(rng: np.random.Generator, L: int, Ns: int, field: bool, kmax: int = 3) -> dict:
    """The random coefficients of one direction's shot phases (the draws of _poly_phase and
    _field for every slice and shot), without rasterising them: poly [L][Ns][10] (the a + b <= 3
    monomials in the order of _poly_phase) and, with ``field``, band [L][Ns][2k+1][2k+1]
    complex (zero outside |k| <= kmax).  For workloads with many directions, whose phases are
    then rasterised on the device by phase_from_coeffs."""
    poly = np.zeros((L, Ns, 10))
    band = np.zeros((L, Ns, 2 * kmax + 1, 2 * kmax + 1), dtype=np.complex128) if field else None
    for l in range(L):
        for i in range(Ns):
            poly[l, i] = rng.uniform(-np.pi, np.pi, size=10)
            if field:
                for ky in range(-kmax, kmax + 1):
                    for kx in range(-kmax, kmax + 1):
                        if kx * kx + ky * ky <= kmax * kmax:
                            band[l, i, ky + kmax, kx + kmax] = rng.standard_normal() + 1j * rng.standard_normal()
    return {"poly": poly, "band": band}


def phase_from_coeffs(coefs: dict, N: int, xp=np, device=None):
    """exp(j (polynomial [+ field])) for coefficients from draw_phase_coeffs, with the array
    namespace ``xp`` (numpy, or torch for a device tensor): the same formulas as
    _poly_phase and _field."""
    def arr(a):
        return xp.asarray(a) if xp is np else xp.as_tensor(a, device=device)
    u = coords(N)
    U = arr(u / 2)
    poly = arr(coefs["poly"])  # [L][Ns][10]
    X = U[None, :]
    Y = U[:, None]
    ph = 0
    t = 0
    for a in range(4):
        for b in range(4 - a):
            ph = ph + poly[..., t, None, None] * (X ** a) * (Y ** b)
            t += 1
    if coefs["band"] is not None:
        kmax = (coefs["band"].shape[-1] - 1) // 2
        k = np.arange(-kmax, kmax + 1)
        E = arr(np.exp(1j * np.pi * np.outer(k, u)))   # [k][n]
        C = arr(coefs["band"])                         # [L][Ns][ky][kx]
        f = (E.T @ C @ E).real                         # [L][Ns][y][x]
        m = f.abs().amax(dim=(-2, -1), keepdim=True) if xp is not np else np.abs(f).max(axis=(-2, -1), keepdims=True)
        ph = ph + f * (np.pi / m)
    return xp.exp(1j * ph)

"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each test checks one oracle function against the mathematics the paper fixes:
explicit DFT sums, closed forms, the Fourier shift theorem behind the
blipped-CAIPI phase (Eq. 1), the annihilation/low-rank relation (Eqs. 6-9),
brute-force sums and textbook properties of CG.  All run on the CPU.
"""
import numpy as np
import pytest

import oracle as O
from paper_1901_01893_gb300 import synth

RNG = np.random.default_rng(1234)


def crandn(*shape, rng=RNG):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def dft_matrix(N):
    """Centred unitary DFT written out: F[n, y] = exp(-j 2 pi (n-N/2)(y-N/2)/N)/sqrt(N)."""
    n = np.arange(N)[:, None] - N / 2
    y = np.arange(N)[None, :] - N / 2
    return np.exp(-2j * np.pi * n * y / N) / np.sqrt(N)


# --- centred DFT -------------------------------------------------------------

@pytest.mark.parametrize("N", [6, 8, 10])
def test_fft2c_is_the_centred_dft_sum(N):
    F = dft_matrix(N)
    x = crandn(3, N, N)
    ref = np.einsum("ay,lyx,bx->lab", F, x, F)
    assert np.allclose(O.fft2c(x), ref, atol=1e-12 * np.abs(ref).max())
    assert np.allclose(O.ifft2c(ref), x, atol=1e-12 * np.abs(x).max())


@pytest.mark.parametrize("N", [4, 6, 8])
def test_fft2c_checkerboard_identity(N):
    # For even N, F_c(x) = D F(D x) with D = (-1)^(x+y) and F the plain unitary DFT.
    D = (-1.0) ** np.add.outer(np.arange(N), np.arange(N))
    x = crandn(N, N)
    assert np.allclose(O.fft2c(x), D * np.fft.fft2(D * x, norm="ortho"), atol=1e-12)


# --- acquisition model (Fig. 1, Eqs. 1-3) ------------------------------------

def test_forward_is_identity_in_the_trivial_case():
    # One slice, one shot, one coil of unit sensitivity, all lines: A = I.
    N = 8
    x = crandn(1, 1, N, N)
    S = np.ones((1, 1, N, N), dtype=complex)
    y = O.forward(x, S)
    assert y.shape == (1, 1, N, N)
    assert np.allclose(y[0, 0], x[0, 0], atol=1e-13)
    assert np.allclose(O.adjoint(y, S, 1), x, atol=1e-13)


@pytest.mark.parametrize("L,N", [(2, 8), (4, 8), (3, 12)])
def test_caipi_integer_shift_is_a_circular_roll(L, N):
    # Fourier shift theorem: the phase exp(-j 2 pi l (n - N/2)/L) on line n moves
    # slice l by +l*N/L pixels along y (the FOV/L shift of blipped CAIPI).
    S = np.ones((L, 1, N, N), dtype=complex)
    for l in range(1, L):
        img = crandn(N, N)
        x = np.zeros((L, 1, N, N), dtype=complex)
        x[l, 0] = O.fft2c(img)
        alias = O.ifft2c(O.forward(x, S)[0, 0])
        assert np.allclose(alias, np.roll(img, l * N // L, axis=0), atol=1e-12)


def test_shot_lines_interleave():
    Ns, N = 4, 16
    got = np.sort(np.concatenate([O.shot_lines(Ns, N, i) for i in range(Ns)]))
    assert np.array_equal(got, np.arange(N))
    assert np.all(O.shot_lines(Ns, N, 3) % Ns == 3)


def test_forward_matches_dense_brute_force():
    # Every step written as a dense sum from the definitions (no FFT).
    L, Ns, Nc, N = 2, 2, 3, 8
    F = dft_matrix(N)
    x = crandn(L, Ns, N, N)
    S = crandn(L, Nc, N, N)
    img = np.einsum("ya,lsab,xb->lsyx", F.conj(), x, F.conj())    # F^-1 along both axes
    coil = S[:, None] * img[:, :, None]                              # [L][Ns][Nc][N][N]
    K = np.einsum("ny,lscyx,kx->lscnk", F, coil, F)
    ref = np.zeros((Ns, Nc, N // Ns, N), dtype=complex)
    for i in range(Ns):
        for m in range(N // Ns):
            n = m * Ns + i
            for l in range(L):
                ref[i, :, m, :] += np.exp(-2j * np.pi * l * (n - N / 2) / L) * K[l, i, :, n, :]
    assert np.allclose(O.forward(x, S), ref, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("phase", [False, True])
def test_adjoint_dot_product(phase):
    # <A x, y> = <x, A^H y>; L=3 with N=16 makes the CAIPI shift sub-pixel.
    L, Ns, Nc, N = 3, 4, 5, 16
    S = crandn(L, Nc, N, N)
    ph = np.exp(1j * RNG.uniform(-np.pi, np.pi, (L, Ns, N, N))) if phase else None
    x = crandn(L, 1 if phase else Ns, N, N)
    y = crandn(Ns, Nc, N // Ns, N)
    lhs = O.vdot(O.forward(x, S, Ns=Ns, phase=ph), y)
    rhs = O.vdot(x, O.adjoint(y, S, L, phase=ph))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# --- Hankel lifting and Gram (Eqs. 8-9) ---------------------------------------

def test_hankel_entries_and_adjoint():
    Ns, N, r = 3, 9, 4
    x = crandn(Ns, N, N)
    H = O.hankel(x, r)
    V = N - r + 1
    assert H.shape == (V * V, Ns * r * r)
    for _ in range(50):
        ky, kx = RNG.integers(0, V, 2)
        i, py, px = RNG.integers(0, Ns), *RNG.integers(0, r, 2)
        assert H[ky * V + kx, i * r * r + py * r + px] == x[i, ky + py, kx + px]
    Y = crandn(*H.shape)
    lhs = O.vdot(H, Y)
    rhs = O.vdot(x, O.hankel_adjoint(Y, Ns, N, r))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_gram_trace_hermitian_psd():
    L, Ns, N, r = 2, 3, 10, 3
    x = crandn(L, Ns, N, N)
    G = O.gram(x, r)
    V = N - r + 1
    for l in range(L):
        tr = sum(np.sum(np.abs(x[l, i, py:py + V, px:px + V]) ** 2)
                 for i in range(Ns) for py in range(r) for px in range(r))
        assert np.isclose(np.trace(G[l]).real, tr, rtol=1e-12)
        assert np.allclose(G[l], G[l].conj().T, atol=1e-12 * tr)
        s = np.linalg.eigvalsh(G[l])
        assert s.min() >= -1e-12 * s.max()


def _rank(A, tol=1e-9):
    s = np.linalg.svd(A, compute_uv=False)
    return int(np.sum(s > tol * s[0]))


def test_rank_bound_zero_shot_phase():
    # Identical shots: H_l = [H H ... H], rank <= r^2 (Eq. 9 with phi = 1).
    N, r, Ns = 20, 4, 3
    rho = RNG.uniform(0.1, 1.0, (N, N))
    xl = np.repeat(O.fft2c(rho)[None], Ns, axis=0)
    assert _rank(O.hankel(xl, r)) == r * r


def test_rank_bound_bandlimited_shot_phase():
    # m_i = rho * phi_i with phi_i's spectrum on s x s samples: every Hankel row is a
    # combination of (r+s-1)^2 shifted samples of rho_hat, so rank(H_l) <= (r+s-1)^2
    # (the annihilation relation of Eqs. 6-9); generic data attains the bound.
    N, r, Ns, s = 24, 5, 4, 3
    rng = np.random.default_rng(7)
    rho = rng.uniform(0.1, 1.0, (N, N))
    coef = synth.bandlimited_phase(rng, 1, Ns, N, s)[0]
    xl = np.empty((Ns, N, N), dtype=complex)
    for i in range(Ns):
        ph_hat = np.zeros((N, N), dtype=complex)
        c0 = N // 2 - s // 2
        ph_hat[c0:c0 + s, c0:c0 + s] = coef[i]
        xl[i] = O.fft2c(rho * O.ifft2c(ph_hat))
    assert _rank(O.hankel(xl, r)) == (r + s - 1) ** 2 == 49


# --- weights (nuclear-norm majoriser / fixed-rank nullspace) ------------------

def test_irls_weight_is_inverse_square_root():
    C, eps = 12, 1e-3
    H = crandn(40, C)
    G = (H.conj().T @ H)[None]
    W, s = O.irls_weight(G, eps)
    assert np.allclose(W[0] @ W[0] @ (G[0] + eps * np.eye(C)), np.eye(C), atol=1e-9)
    assert np.allclose(W[0], W[0].conj().T, atol=1e-12)
    assert np.allclose(s[0], np.sort(np.linalg.eigvalsh(G[0])), atol=1e-9)


def test_nullspace_weight_projects_and_annihilates():
    N, r, Ns = 16, 3, 3
    rho = RNG.uniform(0.1, 1.0, (N, N))
    xl = np.repeat(O.fft2c(rho)[None], Ns, axis=0)[None]     # rank(H) = r^2
    G = O.gram(xl, r)
    W, _ = O.nullspace_weight(G, r * r)
    C = Ns * r * r
    assert np.allclose(W[0] @ W[0], W[0], atol=1e-10)
    assert np.isclose(np.trace(W[0]).real, C - r * r)
    H = O.hankel(xl[0], r)
    assert np.linalg.norm(H @ W[0]) <= 1e-9 * np.linalg.norm(H)


# --- annihilating-filter penalty ----------------------------------------------

def _penalty_brute(x, W, r):
    """P_W(x)_i[n] = sum_p [n-p in V] sum_{i',q} W[(i',q),(i,p)] x_i'[n-p+q] (loops)."""
    L, Ns, N, _ = x.shape
    V = N - r + 1
    out = np.zeros_like(x)
    for l in range(L):
        for i in range(Ns):
            for ny in range(N):
                for nx in range(N):
                    acc = 0j
                    for py in range(r):
                        for px in range(r):
                            ky, kx = ny - py, nx - px
                            if not (0 <= ky < V and 0 <= kx < V):
                                continue
                            for j in range(Ns):
                                for qy in range(r):
                                    for qx in range(r):
                                        acc += (W[l, j * r * r + qy * r + qx, i * r * r + py * r + px]
                                                * x[l, j, ky + qy, kx + qx])
                    out[l, i, ny, nx] = acc
    return out


def _random_hermitian(L, C, rng=RNG):
    A = crandn(L, C, C, rng=rng)
    return A + np.conj(np.swapaxes(A, 1, 2))


def test_penalty_matches_brute_force():
    L, Ns, N, r = 1, 2, 7, 3
    x = crandn(L, Ns, N, N)
    W = _random_hermitian(L, Ns * r * r)
    assert np.allclose(O.penalty(x, W, r), _penalty_brute(x, W, r), atol=1e-11)


def test_penalty_with_identity_weight():
    # W = I: pixel n is counted once per patch covering it, c(n) = prod_d min(n+1, r, N-n, N-r+1).
    L, Ns, N, r = 2, 3, 11, 4
    x = crandn(L, Ns, N, N)
    W = np.broadcast_to(np.eye(Ns * r * r), (L, Ns * r * r, Ns * r * r))
    n = np.arange(N)
    c1 = np.minimum.reduce([n + 1, np.full(N, r), N - n, np.full(N, N - r + 1)])
    assert np.allclose(O.penalty(x, W, r), np.outer(c1, c1) * x, atol=1e-12)


@pytest.mark.parametrize("periodic", [False, True])
def test_penalty_is_self_adjoint_for_hermitian_weight(periodic):
    # P_W = H^* (H(.) W) with W Hermitian: <P_W x, y> = tr((Hy)^H (Hx) W) = <x, P_W y>.
    # The image-domain shot coupling m_ii' of the periodic part is then Hermitian in
    # (i, i'), which is what lets the GPU store only its upper triangle.
    L, Ns, N, r = 2, 3, 12, 3
    x, y = crandn(L, Ns, N, N), crandn(L, Ns, N, N)
    W = _random_hermitian(L, Ns * r * r)
    lhs = np.vdot(O.penalty(x, W, r, periodic=periodic), y)
    rhs = np.vdot(x, O.penalty(y, W, r, periodic=periodic))
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    # and a non-Hermitian weight breaks it (the test can fail)
    A = crandn(L, Ns * r * r, Ns * r * r)
    lhs = np.vdot(O.penalty(x, A, r, periodic=periodic), y)
    rhs = np.vdot(x, O.penalty(y, A, r, periodic=periodic))
    assert abs(lhs - rhs) > 1e-3 * abs(lhs)


def test_penalty_interior_equals_periodic_fft_convolution():
    # Away from the border (n in [r-1, N-r]^2) every patch is valid and the
    # penalty is the multichannel correlation with wt_{ii'}[d] = sum_{q-p=d} W[(i',q),(i,p)],
    # computed here with FFTs (periodic).  Two independent routes must agree.
    L, Ns, N, r = 2, 3, 16, 4
    x = crandn(L, Ns, N, N)
    W = _random_hermitian(L, Ns * r * r)
    ref = np.zeros_like(x)
    for l in range(L):
        for i in range(Ns):
            for j in range(Ns):
                K = np.zeros((N, N), dtype=complex)       # K[-d mod N] = wt[d]
                for py in range(r):
                    for px in range(r):
                        for qy in range(r):
                            for qx in range(r):
                                dy, dx = qy - py, qx - px
                                K[(-dy) % N, (-dx) % N] += W[l, j * r * r + qy * r + qx,
                                                             i * r * r + py * r + px]
                ref[l, i] += np.fft.ifft2(np.fft.fft2(K) * np.fft.fft2(x[l, j]))
    got = O.penalty(x, W, r)
    sl = slice(r - 1, N - r + 1)
    assert np.allclose(got[..., sl, sl], ref[..., sl, sl], atol=1e-10)


# --- PERIODIC boundary (every origin k in [0, N)^2, indices mod N) -------------

def test_periodic_hankel_entries_and_adjoint():
    Ns, N, r = 2, 7, 3
    x = crandn(Ns, N, N)
    H = O.hankel(x, r, periodic=True)
    assert H.shape == (N * N, Ns * r * r)
    for _ in range(60):
        ky, kx = RNG.integers(0, N, 2)
        i, py, px = RNG.integers(0, Ns), *RNG.integers(0, r, 2)
        assert H[ky * N + kx, i * r * r + py * r + px] == x[i, (ky + py) % N, (kx + px) % N]
    Y = crandn(*H.shape)
    lhs = O.vdot(H, Y)
    rhs = O.vdot(x, O.hankel_adjoint(Y, Ns, N, r, periodic=True))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_periodic_gram_is_circular_cross_correlation():
    # Every origin is used, so G[(i,p),(j,q)] = sum_k conj(x_i[k]) x_j[k + q - p]: the
    # circular cross-correlation of shots i and j at lag q - p, here by the correlation
    # theorem (FFTs) -- a route that never forms H.
    L, Ns, N, r = 1, 2, 8, 3
    x = crandn(L, Ns, N, N)
    G = O.gram(x, r, periodic=True)[0]
    F = [np.fft.fft2(x[0, i]) for i in range(Ns)]
    for i in range(Ns):
        for j in range(Ns):
            c = np.fft.ifft2(np.conj(F[i]) * F[j])  # c[d] = sum_k conj(x_i[k]) x_j[k + d]
            for py in range(r):
                for px in range(r):
                    for qy in range(r):
                        for qx in range(r):
                            ref = c[(qy - py) % N, (qx - px) % N]
                            got = G[i * r * r + py * r + px, j * r * r + qy * r + qx]
                            assert abs(got - ref) <= 1e-10 * np.abs(c).max()


def test_periodic_penalty_identity_weight_and_fft_convolution():
    L, Ns, N, r = 1, 2, 9, 3
    x = crandn(L, Ns, N, N)
    C = Ns * r * r
    # W = I: every pixel lies in exactly r*r periodic patches
    assert np.allclose(O.penalty(x, np.eye(C)[None], r, periodic=True), r * r * x, atol=1e-12)
    # general W: the multichannel correlation holds at every pixel (no border band)
    W = _random_hermitian(L, C)
    ref = np.zeros_like(x)
    for i in range(Ns):
        for j in range(Ns):
            K = np.zeros((N, N), dtype=complex)
            for py in range(r):
                for px in range(r):
                    for qy in range(r):
                        for qx in range(r):
                            K[(-(qy - py)) % N, (-(qx - px)) % N] += W[0, j * r * r + qy * r + qx,
                                                                      i * r * r + py * r + px]
            ref[0, i] += np.fft.ifft2(np.fft.fft2(K) * np.fft.fft2(x[0, j]))
    assert np.allclose(O.penalty(x, W, r, periodic=True), ref, atol=1e-10)


# --- SMS-SENSE comparison reconstruction --------------------------------------

def test_sense_is_the_least_squares_solution():
    # Dense route: the matrix of the shot-shared forward model (columns = images of the
    # unit vectors), solved by numpy's least squares; CG to convergence must agree.
    L, Ns, Nc, N = 2, 2, 3, 8
    sens = crandn(L, Nc, N, N)
    phase = np.exp(1j * RNG.uniform(-np.pi, np.pi, (L, Ns, N, N)))
    n = L * N * N
    A = np.zeros((Ns * Nc * (N // Ns) * N, n), dtype=complex)
    for k in range(n):
        e = np.zeros(n, dtype=complex)
        e[k] = 1.0
        A[:, k] = O.forward(e.reshape(L, 1, N, N), sens, phase=phase).ravel()
    y = crandn(Ns, Nc, N // Ns, N)
    x_ls = np.linalg.lstsq(A, y.ravel(), rcond=None)[0].reshape(L, 1, N, N)
    x_cg = O.sense(y, sens, L, J=3 * n, phase=phase)
    assert O.nrmse(x_cg, x_ls) < 1e-8
    # no phase given = unit phase (no phase correction)
    x0 = O.sense(y, sens, L, J=40)
    x1 = O.sense(y, sens, L, J=40, phase=np.ones((L, Ns, N, N), dtype=complex))
    assert np.allclose(x0, x1, atol=1e-12)


# --- CG ------------------------------------------------------------------------

def test_cg_solves_small_hpd_system_exactly():
    n = 12
    B = crandn(n, n)
    A = B.conj().T @ B + n * np.eye(n)
    b = crandn(n)
    x, hist = O.cg(lambda v: A @ v, b, np.zeros(n, dtype=complex), n)
    assert np.allclose(x, np.linalg.solve(A, b), atol=1e-10)
    assert hist[-1] < 1e-20 * hist[0]


# --- whole solver ----------------------------------------------------------------

def test_exact_recovery_with_full_sampling():
    # Every shot keeps every line, no shot phase, no noise, lam = 0, Nc >= L:
    # CG on A^H A x = A^H y recovers the slice-unfolded k-space exactly.
    L, Ns, Nc, N = 2, 2, 4, 16
    rng = np.random.default_rng(5)
    S = crandn(L, Nc, N, N, rng=rng)
    rho = rng.uniform(0.1, 1.0, (L, N, N))
    xt = np.repeat(O.fft2c(rho)[:, None], Ns, axis=1)
    y = O.forward(xt, S, full=True)

    def AhA(v):
        return O.adjoint(O.forward(v, S, full=True), S, L, full=True)

    b = O.adjoint(y, S, L, full=True)
    x, _ = O.cg(AhA, b, np.zeros_like(b), 300)
    assert O.nrmse(x, xt) <= 1e-10


def _small_problem(seed=3, L=2, Ns=2, Nc=6, N=16):
    g = synth.make_group(L, Ns, Nc, N, seed)
    xt, y = O.make_data(g, 30.0)
    return g, xt, y


def test_epsilon_schedule():
    g, xt, y = _small_problem()
    rep = {}
    p = dict(K=6, J=2, eps0_rel=1e-2, eta=2.0, eps_min_rel=0.1)
    O.reconstruct(y, g["sens"], 3, p, report=rep)
    eps = [h["eps"] for h in rep["hist"]]
    x0 = O.adjoint(y, g["sens"], 2)
    smax = max(np.linalg.eigvalsh(G)[-1] for G in O.gram(x0, 3))
    assert np.isclose(eps[0], 1e-2 * smax, rtol=1e-10)
    assert np.allclose(eps, [eps[0] * max(0.5 ** k, 0.1) for k in range(6)], rtol=1e-12)


def test_slice_phase_equivariance():
    # Multiplying slice l's coil maps by exp(-j c_l) multiplies the recovered
    # slice l by exp(+j c_l): data term unchanged, ||H_l||_* unchanged, and every
    # CG iterate transforms the same way.
    g, xt, y = _small_problem()
    c = np.array([0.7, -2.1])
    p = dict(K=3, J=4)
    x1 = O.reconstruct(y, g["sens"], 3, p)
    x2 = O.reconstruct(y, g["sens"] * np.exp(-1j * c)[:, None, None, None], 3, p)
    assert np.allclose(x2, x1 * np.exp(1j * c)[:, None, None, None], atol=1e-10 * np.abs(x1).max())


def test_global_phase_equivariance():
    g, xt, y = _small_problem()
    p = dict(K=3, J=4)
    x1 = O.reconstruct(y, g["sens"], 3, p)
    x2 = O.reconstruct(np.exp(0.9j) * y, g["sens"], 3, p)
    assert np.allclose(x2, np.exp(0.9j) * x1, atol=1e-10 * np.abs(x1).max())


def test_magnitude_recovers_rho_from_unit_phase_shots():
    # Eqs. 4-5: shot i of slice l is rho_l * phi_{l,i} with |phi| = 1, so the root mean
    # square over the shots of |F^-1 x| is rho_l exactly, whatever the phases; and a
    # magnitude that differs between shots averages in the square (not in the modulus).
    rng = np.random.default_rng(5)
    L, Ns, N = 2, 4, 16
    rho = rng.uniform(0.1, 1.0, (L, N, N))
    phi = np.exp(1j * rng.uniform(-np.pi, np.pi, (L, Ns, N, N)))
    x = O.fft2c(rho[:, None] * phi)
    assert np.allclose(O.magnitude(x), rho, rtol=0, atol=1e-12)
    amp = np.stack([rho * (1 + k) for k in range(Ns)], axis=1)  # |m_{l,i}| = (1 + i) rho_l
    x2 = O.fft2c(amp * phi)
    expect = rho * np.sqrt(np.mean([(1 + k) ** 2 for k in range(Ns)]))
    assert np.allclose(O.magnitude(x2), expect, rtol=0, atol=1e-12)

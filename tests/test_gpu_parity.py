"""GPU parity: every C-ABI call against the FP64 oracle on the same seeded inputs.

Tolerances (NRMSE = ||gpu - oracle|| / ||oracle||):
  * FP32 operators (forward, adjoint, fft2c, Gram, filter penalty): 1e-5.
  * the whole IRLS + CG solve, FP32 form: 2e-5 per slice (short schedules here;
    the full schedules of the workloads, and how the FP32 operators' rounding grows
    through CG into this bar, are in test_gpu_solve_parity.py).
  * reduced precision (BF16 split Gram): 1e-3, the metric's threshold.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1901_01893_gb300 import synth

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5
SOLVE_TOL = 2e-5   # per slice, FP32 form
BF16_TOL = 1e-3


def slice_err(x, ref):
    """Largest per-slice NRMSE over the slices (and directions) of x."""
    x = np.asarray(x)
    return float(np.max(O.nrmse(x, ref, axis=tuple(range(x.ndim - 3, x.ndim)))))


@pytest.fixture(scope="module")
def smsm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_01893_gb300 import _build, smsm as mod

    _build.build()
    mod.lib()
    return mod


DEV = "cuda:0"


def c64(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.complex64)).to(DEV)


def c128(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.complex128)).to(DEV)


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# geometry cases: (L, Ns, Nc, N, r, Ldiv); small ones span several tiles and a ragged tail
CASES = {
    "tiny": (2, 4, 8, 64, 5, 2),
    "plain": (2, 4, 32, 128, 6, 2),
    "precision": (3, 4, 32, 256, 6, 3),
    "radix3": (3, 2, 5, 48, 4, 3),     # N = 3*16, M = 24, C = 32
    "odd_shots": (1, 3, 4, 96, 3, 1),  # Ns = 3, M = 32, one slice
    "mb3_8shots": (3, 8, 6, 64, 3, 3),  # M = 8, C = 72
    "r1": (2, 2, 3, 32, 1, 2),         # filter 1: C = Ns
    "maxc": (2, 2, 4, 64, 9, 2),       # C = Cp = 162: FMA Gram, the two-CTA eigensolver's range
    "c294": (2, 6, 4, 48, 7, 2),       # C = 294 (10 row groups of 32): FMA Gram, cluster eigensolver
    "maxn": (1, 2, 2, 512, 2, 1),      # largest image edge, N = 512
}


def make_plan(smsm, key, sens=None, seed=0):
    L, Ns, Nc, N, r, Ldiv = CASES[key]
    plan = smsm.Plan(L, Ns, Nc, N, r, caipi_div=Ldiv)
    rng = np.random.default_rng(seed)
    if sens is None:
        sens = crandn(rng, L, Nc, N, N) / np.sqrt(Nc)
    plan.set_sens(c64(sens))
    return plan, sens, rng


@pytest.mark.parametrize("key", list(CASES))
def test_forward_adjoint_parity(smsm, key):
    plan, S, rng = make_plan(smsm, key)
    L, Ns, Nc, N, r, Ldiv = CASES[key]
    x = crandn(rng, L, Ns, N, N)
    y = crandn(rng, Ns, Nc, N // Ns, N)
    yg = plan.forward(c64(x)).cpu().numpy()
    xg = plan.adjoint(c64(y)).cpu().numpy()
    assert O.nrmse(yg, O.forward(x, S, Ldiv=Ldiv)) < OP_TOL
    assert O.nrmse(xg, O.adjoint(y, S, L, Ldiv=Ldiv)) < OP_TOL
    # adjoint identity on the GPU results, accumulated in FP64
    lhs = np.vdot(yg.astype(np.complex128), y)
    rhs = np.vdot(x, xg.astype(np.complex128))
    assert abs(lhs - rhs) < 1e-5 * abs(lhs)


@pytest.mark.parametrize("key", ["tiny", "radix3", "odd_shots"])
def test_forward_adjoint_phase_mode(smsm, key):
    plan, S, rng = make_plan(smsm, key)
    L, Ns, Nc, N, r, Ldiv = CASES[key]
    ph = np.exp(1j * rng.uniform(-np.pi, np.pi, (L, Ns, N, N)))
    x = crandn(rng, L, 1, N, N)
    y = crandn(rng, Ns, Nc, N // Ns, N)
    yg = plan.forward(c64(x), phase=c64(ph)).cpu().numpy()
    xg = plan.adjoint(c64(y), phase=c64(ph)).cpu().numpy()
    assert O.nrmse(yg, O.forward(x, S, Ldiv=Ldiv, phase=ph)) < OP_TOL
    assert O.nrmse(xg, O.adjoint(y, S, L, Ldiv=Ldiv, phase=ph)) < OP_TOL


@pytest.mark.parametrize("key", ["tiny", "precision", "radix3", "maxn"])
def test_fft2c_parity(smsm, key):
    plan, S, rng = make_plan(smsm, key)
    L, Ns, Nc, N, r, Ldiv = CASES[key]
    img = crandn(rng, 2 * L * Ns + 1, N, N)  # more images than one chunk, ragged tail
    k = plan.fft2c(c64(img)).cpu().numpy()
    assert O.nrmse(k, O.fft2c(img)) < OP_TOL
    back = plan.fft2c(c64(k), inverse=True).cpu().numpy()
    assert O.nrmse(back, img) < OP_TOL


@pytest.mark.parametrize("key", ["tiny", "plain", "radix3", "mb3_8shots", "r1", "maxc", "c294", "maxn"])
def test_gram_parity(smsm, key):
    plan, S, rng = make_plan(smsm, key)
    L, Ns, Nc, N, r, Ldiv = CASES[key]
    x = crandn(rng, L, Ns, N, N)
    G = plan.hankel_gram(c64(x)).cpu().numpy()
    ref = O.gram(x.astype(np.complex64).astype(np.complex128), r)
    assert O.nrmse(G, ref) < OP_TOL
    assert np.array_equal(G, np.conj(np.swapaxes(G, 1, 2)))  # exactly Hermitian


def test_gram_full_size_sampled(smsm):
    # 256^2, 3 slices, C = 144: sampled entries against the definition, one by one
    plan, S, rng = make_plan(smsm, "precision")
    L, Ns, Nc, N, r, Ldiv = CASES["precision"]
    x = crandn(rng, L, Ns, N, N).astype(np.complex64)
    G = plan.hankel_gram(c64(x)).cpu().numpy()
    x64 = x.astype(np.complex128)
    V = N - r + 1
    C = Ns * r * r
    for _ in range(40):
        l = rng.integers(L)
        a, b = rng.integers(C, size=2)
        i, p = divmod(a, r * r)
        j, q = divmod(b, r * r)
        ref = np.sum(np.conj(x64[l, i, p // r:p // r + V, p % r:p % r + V]) *
                     x64[l, j, q // r:q // r + V, q % r:q % r + V])
        assert abs(G[l, a, b] - ref) < 1e-5 * abs(G[l, a, a].real * G[l, b, b].real) ** 0.5


def _random_weight(rng, L, C):
    A = crandn(rng, L, C, C)
    return (A + np.conj(np.swapaxes(A, 1, 2))) / np.sqrt(C)


@pytest.mark.parametrize("key", ["tiny", "plain", "precision", "radix3", "mb3_8shots", "r1", "maxc", "c294",
                                 "maxn"])
def test_apply_filters_parity(smsm, key):
    plan, S, rng = make_plan(smsm, key)
    L, Ns, Nc, N, r, Ldiv = CASES[key]
    x = crandn(rng, L, Ns, N, N).astype(np.complex64)
    W = _random_weight(rng, L, Ns * r * r)
    out = plan.apply_filters(c128(W), c64(x)).cpu().numpy()
    ref = O.penalty(x.astype(np.complex128), W.astype(np.complex64).astype(np.complex128), r)
    assert O.nrmse(out, ref) < OP_TOL


@pytest.mark.parametrize("key", ["tiny", "radix3", "mb3_8shots"])
def test_apply_filters_is_self_adjoint(smsm, key):
    # Hermitian W: <P x, y> = <x, P y>.  The periodic multiplier is stored as the upper
    # triangle of a Hermitian shot coupling, so only rounding separates the two sides.
    plan, S, rng = make_plan(smsm, key)
    L, Ns, Nc, N, r, Ldiv = CASES[key]
    x = crandn(rng, L, Ns, N, N).astype(np.complex64)
    y = crandn(rng, L, Ns, N, N).astype(np.complex64)
    W = _random_weight(rng, L, Ns * r * r)
    px = plan.apply_filters(c128(W), c64(x)).cpu().numpy().astype(np.complex128)
    py = plan.apply_filters(c128(W), c64(y)).cpu().numpy().astype(np.complex128)
    lhs = np.vdot(px, y.astype(np.complex128))
    rhs = np.vdot(x.astype(np.complex128), py)
    assert abs(lhs - rhs) < 1e-5 * np.linalg.norm(px) * np.linalg.norm(y)


def test_apply_filters_identity_weight(smsm):
    # W = I: the penalty is the patch-count map c(n) times x (closed form)
    plan, S, rng = make_plan(smsm, "radix3")
    L, Ns, Nc, N, r, Ldiv = CASES["radix3"]
    C = Ns * r * r
    x = crandn(rng, L, Ns, N, N).astype(np.complex64)
    W = np.broadcast_to(np.eye(C), (L, C, C))
    out = plan.apply_filters(c128(W), c64(x)).cpu().numpy()
    n = np.arange(N)
    c1 = np.minimum.reduce([n + 1, np.full(N, r), N - n, np.full(N, N - r + 1)])
    assert O.nrmse(out, np.outer(c1, c1) * x) < OP_TOL


def _problem(key, seed):
    L, Ns, Nc, N, r, Ldiv = CASES[key]
    g = synth.make_group(L, Ns, Nc, N, seed, field=N >= 128)
    xt, y = O.make_data(g, 30.0, Ldiv=Ldiv)
    sc = np.sqrt(np.mean(np.abs(y) ** 2))
    return g, xt / sc, y / sc


@pytest.mark.parametrize("key,K,J", [("tiny", 3, 4), ("radix3", 3, 5), ("plain", 2, 3), ("r1", 3, 4),
                                     ("maxc", 2, 3), ("c294", 3, 4), ("maxn", 2, 3)])
def test_reconstruct_parity(smsm, key, K, J):
    L, Ns, Nc, N, r, Ldiv = CASES[key]
    g, xt, y = _problem(key, 1)
    lam = 1e-2
    ref = O.reconstruct(y, g["sens"], r, dict(K=K, J=J, lam=lam), Ldiv=Ldiv)
    plan, _, _ = make_plan(smsm, key, sens=g["sens"])
    prm = smsm.default_params(lam=lam, outer_iters=K, cg_iters=J)
    x, rep = plan.reconstruct(c64(y), params=prm)
    assert rep.status == 0
    err = slice_err(x.cpu().numpy(), ref)
    print(f"{key}: reconstruct NRMSE vs oracle (worst slice) {err:.3e}; vs truth gpu {O.nrmse(x.cpu().numpy(), xt):.3e} "
          f"oracle {O.nrmse(ref, xt):.3e}")
    assert err < SOLVE_TOL
    # the graph is replayed on a second call with the same parameters: identical result
    x2, _ = plan.reconstruct(c64(y), params=prm)
    assert torch.equal(x, x2)


@pytest.mark.parametrize("cluster", [False, True])
def test_reconstruct_nullspace_mode(smsm, cluster):
    # the projector onto the C - rank smallest eigenvectors, with either eigensolver
    key = "tiny"
    L, Ns, Nc, N, r, Ldiv = CASES[key]
    g, xt, y = _problem(key, 2)
    rank = 40
    ref = O.reconstruct(y, g["sens"], r, dict(K=3, J=5, lam=1e-1, mode="nullspace", rank=rank), Ldiv=Ldiv)
    plan = smsm.Plan(L, Ns, Nc, N, r, caipi_div=Ldiv, flags=smsm.SMSM_FLAG_CLUSTER_EIG if cluster else 0)
    plan.set_sens(c64(g["sens"]))
    prm = smsm.default_params(lam=1e-1, outer_iters=3, cg_iters=5, mode=smsm.SMSM_MODE_NULLSPACE, rank=rank)
    x, rep = plan.reconstruct(c64(y), params=prm)
    assert rep.status == 0
    err = slice_err(x.cpu().numpy(), ref)
    print(f"nullspace mode: worst slice NRMSE vs oracle {err:.3e}")
    assert err < SOLVE_TOL


def test_reconstruct_warm_start_and_lambda0(smsm):
    # lambda = 0 reduces the solve to CG on the SENSE normal equations; a warm
    # start continues from the given x exactly like the oracle does.
    key = "radix3"
    L, Ns, Nc, N, r, Ldiv = CASES[key]
    g, xt, y = _problem(key, 3)
    rng = np.random.default_rng(9)
    x0 = crandn(rng, L, Ns, N, N) * 0.1
    ref = O.reconstruct(y, g["sens"], r, dict(K=2, J=4, lam=0.0), x0=x0, Ldiv=Ldiv)
    plan, _, _ = make_plan(smsm, key, sens=g["sens"])
    prm = smsm.default_params(lam=0.0, outer_iters=2, cg_iters=4, warm=1)
    x, rep = plan.reconstruct(c64(y), x=c64(x0), params=prm)
    assert slice_err(x.cpu().numpy(), ref) < SOLVE_TOL


def test_errors_do_not_abort(smsm):
    plan, S, rng = make_plan(smsm, "tiny")
    L, Ns, Nc, N, r, Ldiv = CASES["tiny"]
    x = torch.zeros((L, Ns, N, N), dtype=torch.complex64, device=DEV)
    with pytest.raises(smsm.SmsmError) as e:
        plan.apply_filters(torch.zeros((L, Ns * r * r, Ns * r * r), dtype=torch.complex128, device=DEV), x, out=x)
    assert e.value.status == smsm.SMSM_ERR_ARG
    for bad in (smsm.default_params(outer_iters=-1), smsm.default_params(eig_tol=2.0),
                smsm.default_params(eig_tol=-1e-6), smsm.default_params(lanes=9)):
        with pytest.raises(smsm.SmsmError) as e:
            plan.reconstruct(torch.zeros(plan.y_shape, dtype=torch.complex64, device=DEV), params=bad)
        assert e.value.status == smsm.SMSM_ERR_ARG
    # an unset plan refuses to run
    p2 = smsm.Plan(L, Ns, Nc, N, r)
    with pytest.raises(smsm.SmsmError) as e:
        p2.forward(x)
    assert e.value.status == smsm.SMSM_ERR_STATE


def test_batch_matches_single_problems(smsm):
    # D independent problems (diffusion directions sharing coil maps) in one plan:
    # every operator and the whole solve must match the per-problem results.
    key = "tiny"
    L, Ns, Nc, N, r, Ldiv = CASES[key]
    D = 3
    rng = np.random.default_rng(21)
    S = crandn(rng, L, Nc, N, N) / np.sqrt(Nc)
    xb = crandn(rng, D, L, Ns, N, N)
    yb = crandn(rng, D, Ns, Nc, N // Ns, N)
    Wb = np.stack([_random_weight(rng, L, Ns * r * r) for _ in range(D)])
    pb = smsm.Plan(L, Ns, Nc, N, r, caipi_div=Ldiv, batch=D)
    pb.set_sens(c64(S))
    fwd = pb.forward(c64(xb)).cpu().numpy()
    adj = pb.adjoint(c64(yb)).cpu().numpy()
    G = pb.hankel_gram(c64(xb)).cpu().numpy()
    pen = pb.apply_filters(c128(Wb), c64(xb)).cpu().numpy()
    for d in range(D):
        assert O.nrmse(fwd[d], O.forward(xb[d], S, Ldiv=Ldiv)) < OP_TOL
        assert O.nrmse(adj[d], O.adjoint(yb[d], S, L, Ldiv=Ldiv)) < OP_TOL
        assert O.nrmse(G[d], O.gram(xb[d].astype(np.complex64).astype(complex), r)) < OP_TOL
        ref = O.penalty(xb[d].astype(np.complex64).astype(complex), Wb[d].astype(np.complex64).astype(complex), r)
        assert O.nrmse(pen[d], ref) < OP_TOL
    # whole solve: each direction against its own single-problem plan
    g, xt, y0 = _problem(key, 5)
    ys = np.stack([y0 * np.exp(1j * 0.3 * d) + 0.05 * crandn(rng, *y0.shape) for d in range(D)])
    prm = smsm.default_params(lam=1e-2, outer_iters=4, cg_iters=5)
    pb2 = smsm.Plan(L, Ns, Nc, N, r, caipi_div=Ldiv, batch=D)
    pb2.set_sens(c64(g["sens"]))
    xb_out, rep = pb2.reconstruct(c64(ys), params=prm)
    assert rep.status == 0
    p1 = smsm.Plan(L, Ns, Nc, N, r, caipi_div=Ldiv)
    p1.set_sens(c64(g["sens"]))
    for d in range(D):
        x1, _ = p1.reconstruct(c64(ys[d]), params=prm)
        assert slice_err(xb_out[d].cpu().numpy(), x1.cpu().numpy()) < SOLVE_TOL
    ref = O.reconstruct(ys[D - 1], g["sens"], r, dict(K=4, J=5, lam=1e-2), Ldiv=Ldiv)
    assert slice_err(xb_out[D - 1].cpu().numpy(), ref) < SOLVE_TOL


def test_periodic_boundary_parity(smsm):
    # PERIODIC patches (every origin, indices mod N): Gram on both Gram paths, the
    # penalty (multiplier only, no border band) and a short solve against the oracle.
    key = "tiny"
    L, Ns, Nc, N, r, Ldiv = CASES[key]
    C = Ns * r * r
    rng = np.random.default_rng(41)
    x = crandn(rng, L, Ns, N, N)
    x32 = x.astype(np.complex64).astype(complex)
    W = _random_weight(rng, L, C)
    W32 = W.astype(np.complex64).astype(complex)
    Gref = O.gram(x32, r, periodic=True)
    for flags in (0, smsm.SMSM_FLAG_GENERIC_KERNELS):
        p = smsm.Plan(L, Ns, Nc, N, r, caipi_div=Ldiv, flags=flags, boundary=smsm.SMSM_BOUNDARY_PERIODIC)
        assert O.nrmse(p.hankel_gram(c64(x)).cpu().numpy(), Gref) < OP_TOL
        pen = p.apply_filters(c128(W), c64(x)).cpu().numpy()
        assert O.nrmse(pen, O.penalty(x32, W32, r, periodic=True)) < OP_TOL
    g, xt, y = _problem(key, 7)
    p = smsm.Plan(L, Ns, Nc, N, r, caipi_div=Ldiv, boundary=smsm.SMSM_BOUNDARY_PERIODIC)
    p.set_sens(c64(g["sens"]))
    prm = smsm.default_params(lam=1e-2, outer_iters=3, cg_iters=4)
    xo, rep = p.reconstruct(c64(y), params=prm)
    assert rep.status == 0
    ref = O.reconstruct(y, g["sens"], r, dict(K=3, J=4, lam=1e-2, periodic=True), Ldiv=Ldiv)
    err = slice_err(xo.cpu().numpy(), ref)
    print(f"periodic: reconstruct NRMSE vs oracle (worst slice) {err:.3e}")
    assert err < SOLVE_TOL


@pytest.mark.parametrize("with_phase", [False, True])
def test_sms_sense_parity(smsm, with_phase):
    # SMS-SENSE (shots combined, one k-space per slice, least squares by CG) with and
    # without the shot phase, against the oracle's same J steps; batch of 2.
    key = "tiny"
    L, Ns, Nc, N, r, Ldiv = CASES[key]
    D, J = 2, 12
    g, xt, y0 = _problem(key, 9)
    rng = np.random.default_rng(51)
    ys = np.stack([y0, y0 * np.exp(0.4j) + 0.05 * crandn(rng, *y0.shape)])
    ph = np.stack([g["phase"], np.conj(g["phase"])]) if with_phase else None
    p = smsm.Plan(L, Ns, Nc, N, r, caipi_div=Ldiv, batch=D)
    p.set_sens(c64(g["sens"]))
    x, rep = p.sense(c64(ys), phase=c64(ph) if with_phase else None, cg_iters=J)
    assert rep.status == 0
    x = x.cpu().numpy()
    for d in range(D):
        ref = O.sense(ys[d], g["sens"], L, J, phase=ph[d] if with_phase else None, Ldiv=Ldiv)
        err = slice_err(x[d], ref)
        assert err < SOLVE_TOL, err


def test_groups_of_different_geometry_match_single_solves(smsm):
    # Two slice groups of different geometry (64^2 MB 2 4-shot; 48^2 MB 3 2-shot)
    # solved together in one graph launch give exactly their single-plan results; so
    # does the same call again with other data buffers (the cached group graph re-pointed),
    # and the per-group stream path taken when the solve is timed.
    prm = smsm.default_params(lam=1e-2, outer_iters=3, cg_iters=4)
    plans, ys, singles = [], [], []
    for key, seed in (("tiny", 3), ("radix3", 4)):
        L, Ns, Nc, N, r, Ldiv = CASES[key]
        g, xt, y = _problem(key, seed)
        p = smsm.Plan(L, Ns, Nc, N, r, caipi_div=Ldiv)
        p.set_sens(c64(g["sens"]))
        x1, rep = p.reconstruct(c64(y), params=prm)
        assert rep.status == 0
        plans.append(p)
        ys.append(c64(y))
        singles.append(x1.cpu().numpy())
    xs, reps = smsm.reconstruct_groups(plans, ys, params=prm)
    for k in range(len(plans)):
        assert reps[k].status == 0
        assert np.array_equal(xs[k].cpu().numpy(), singles[k])
    # other y buffers, reused x buffers holding stale values
    ys2 = [y.clone() for y in ys]
    xs2, reps = smsm.reconstruct_groups(plans, ys2, params=prm, xs=xs)
    for k in range(len(plans)):
        assert xs2[k] is xs[k] and reps[k].status == 0 and reps[k].elapsed_ms > 0
        assert np.array_equal(xs2[k].cpu().numpy(), singles[k])
    prm_t = smsm.default_params(lam=1e-2, outer_iters=3, cg_iters=4, timing=1 << 2)
    xs3, reps = smsm.reconstruct_groups(plans, ys2, params=prm_t)
    for k in range(len(plans)):
        assert reps[k].status == 0 and reps[k].stage_ms[2] > 0
        assert np.array_equal(xs3[k].cpu().numpy(), singles[k])


def test_lanes_give_identical_results(smsm):
    # Solving the batch as 1, 2 or 3 concurrent lanes (sub-batches on their own
    # graph branches) changes the schedule only: every direction runs the same
    # kernels with the same reduction splits, so the results are bit-identical.
    key = "tiny"
    L, Ns, Nc, N, r, Ldiv = CASES[key]
    D = 5
    g, xt, y0 = _problem(key, 6)
    rng = np.random.default_rng(31)
    ys = np.stack([y0 * np.exp(1j * 0.2 * d) + 0.05 * crandn(rng, *y0.shape) for d in range(D)])
    p = smsm.Plan(L, Ns, Nc, N, r, caipi_div=Ldiv, batch=D)
    p.set_sens(c64(g["sens"]))
    outs = []
    for lanes in (1, 2, 3):
        prm = smsm.default_params(lam=1e-2, outer_iters=3, cg_iters=4, lanes=lanes)
        x, rep = p.reconstruct(c64(ys), params=prm)
        assert rep.status == 0
        outs.append(x.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[2])


@pytest.mark.parametrize("L,Ns,Nc,N,r,Ldiv", [
    (2, 4, 8, 64, 5, 0),    # M = 16 (lane segments)
    (3, 4, 6, 64, 3, 8),    # CAIPI shift N/8: classes pair pixels 8 apart within M = 16
    (3, 2, 5, 64, 3, 4),    # CAIPI shift N/4 = M/2
    (3, 8, 6, 64, 3, 0),    # M = 8, three slices
    (2, 4, 8, 128, 6, 0),   # M = 32
    (2, 2, 6, 128, 4, 0),   # M = 64 (local radix-2)
    (1, 2, 4, 192, 4, 0),   # M = 96 (local radix-3), one slice
    (3, 2, 4, 256, 4, 0),   # M = 128 (local radix-4); 256 % 3 != 0: no aliasing classes
    (1, 3, 5, 96, 3, 0),    # N = 96, M = 32
])
def test_fast_column_stage_matches_generic(smsm, L, Ns, Nc, N, r, Ldiv):
    # the aliasing-class column stage, the warp-shuffle per-coil one and the
    # shape-generic one compute the same (A^H A + lambda P_W); compare whole
    # (short) solves, and one against the oracle
    rng = np.random.default_rng(L * 100 + N + Ns)
    S = crandn(rng, L, Nc, N, N) / np.sqrt(Nc)
    y = crandn(rng, Ns, Nc, N // Ns, N)
    prm = smsm.default_params(lam=3e-2, outer_iters=2, cg_iters=3)
    out = []
    for flags in (0, smsm.SMSM_FLAG_PER_COIL_NORMAL, smsm.SMSM_FLAG_GENERIC_KERNELS):
        p = smsm.Plan(L, Ns, Nc, N, r, caipi_div=Ldiv, flags=flags)
        p.set_sens(c64(S))
        x, rep = p.reconstruct(c64(y), params=prm)
        assert rep.status == 0
        out.append(x.cpu().numpy())
    assert O.nrmse(out[0], out[2]) < 1e-5
    assert O.nrmse(out[1], out[2]) < 1e-5
    if N <= 128:
        ref = O.reconstruct(y, S, r, dict(K=2, J=3, lam=3e-2), Ldiv=Ldiv or L)
        assert slice_err(out[0], ref) < SOLVE_TOL


def test_warm_started_eigensolver_matches_cold(smsm):
    # Jacobi started from the previous outer iteration's eigenvectors converges to
    # the same eigen-decomposition as a cold start: same solve up to rounding.
    key = "plain"
    L, Ns, Nc, N, r, Ldiv = CASES[key]
    g, xt, y = _problem(key, 4)
    plan, _, _ = make_plan(smsm, key, sens=g["sens"])
    out = []
    for cold in (0, 1):
        prm = smsm.default_params(lam=1e-2, outer_iters=4, cg_iters=4, eig_cold=cold)
        x, rep = plan.reconstruct(c64(y), params=prm)
        assert rep.status == 0
        out.append((x.cpu().numpy(), [rep.sweeps[k] for k in range(4)]))
    print("sweeps warm", out[0][1], "cold", out[1][1])
    assert slice_err(out[0][0], out[1][0]) < SOLVE_TOL
    assert sum(out[0][1][1:]) < sum(out[1][1][1:])  # warm starts need fewer sweeps


@pytest.mark.parametrize("key", ["tiny", "plain", "radix3", "mb3_8shots"])
def test_tensor_core_gram_matches_fma_gram(smsm, key):
    # tcgen05 Gram (TF32 split, FP32-accurate) against the FP32-FMA Gram and the oracle
    L, Ns, Nc, N, r, Ldiv = CASES[key]
    rng = np.random.default_rng(31)
    x = crandn(rng, L, Ns, N, N).astype(np.complex64)
    ref = O.gram(x.astype(np.complex128), r)
    out = {}
    for flags in (0, smsm.SMSM_FLAG_GENERIC_KERNELS):
        p = smsm.Plan(L, Ns, Nc, N, r, flags=flags)
        out[flags] = p.hankel_gram(c64(x)).cpu().numpy()
        assert p.device_status() == 0
    assert O.nrmse(out[0], ref) < OP_TOL
    assert O.nrmse(out[0], out[smsm.SMSM_FLAG_GENERIC_KERNELS]) < OP_TOL


def test_bf16_split_precision_form(smsm):
    # the BF16 split Gram (3 BF16 products, FP32 accumulate): error per slice reported,
    # below the 1e-3 metric threshold for the Gram and for the whole solve
    key = "plain"
    L, Ns, Nc, N, r, Ldiv = CASES[key]
    rng = np.random.default_rng(32)
    x = crandn(rng, L, Ns, N, N).astype(np.complex64)
    p = smsm.Plan(L, Ns, Nc, N, r, precision=smsm.SMSM_PRECISION_BF16_SPLIT)
    G = p.hankel_gram(c64(x)).cpu().numpy()
    ref = O.gram(x.astype(np.complex128), r)
    per_slice = [O.nrmse(G[l], ref[l]) for l in range(L)]
    print("BF16 split Gram NRMSE per slice", per_slice)
    assert max(per_slice) < 1e-4
    g, xt, y = _problem(key, 6)
    ref = O.reconstruct(y, g["sens"], r, dict(K=3, J=4, lam=1e-2), Ldiv=Ldiv)
    p.set_sens(c64(g["sens"]))
    xr, rep = p.reconstruct(c64(y), params=smsm.default_params(lam=1e-2, outer_iters=3, cg_iters=4))
    assert rep.status == 0
    err = slice_err(xr.cpu().numpy(), ref)
    print("BF16 split solve NRMSE vs FP64 oracle (worst slice)", err)
    assert err < BF16_TOL


def test_autotune_picks_a_candidate_and_keeps_the_results(smsm):
    # The tuner times the Gram's split-K candidates and 1..4 lanes on the plan's data and keeps
    # the fastest; the solve is unchanged up to the order of the Gram's partial sums, and a later
    # plan of the same shape starts from the cached choice.
    key = "tiny"
    L, Ns, Nc, N, r, Ldiv = CASES[key]
    D = 6
    g, xt, y0 = _problem(key, 12)
    rng = np.random.default_rng(61)
    ys = c64(np.stack([y0 * np.exp(1j * 0.3 * d) + 0.05 * crandn(rng, *y0.shape) for d in range(D)]))
    prm = smsm.default_params(lam=1e-2, outer_iters=3, cg_iters=4)
    p0 = smsm.Plan(L, Ns, Nc, N, r, caipi_div=Ldiv, batch=D)
    p0.set_sens(c64(g["sens"]))
    x0, _ = p0.reconstruct(ys, params=prm)
    p1 = smsm.Plan(L, Ns, Nc, N, r, caipi_div=Ldiv, batch=D)
    p1.set_sens(c64(g["sens"]))
    rep = p1.autotune(ys, params=prm)
    cands = list(rep.gram_candidates)[:rep.n_gram]
    print("autotune: Gram split-K", cands, [round(v, 3) for v in list(rep.gram_ms)[:rep.n_gram]], "->", rep.gram_nG,
          "; lanes ms", [round(v, 3) for v in rep.lane_ms], "->", rep.lanes)
    assert rep.n_gram >= 2 and rep.gram_nG in cands
    assert 1 <= rep.lanes <= 4 and rep.lane_ms[rep.lanes - 1] == min(v for v in rep.lane_ms if v > 0)
    x1, r1 = p1.reconstruct(ys, params=prm)
    assert r1.status == 0 and r1.lanes == rep.lanes
    assert slice_err(x1.cpu().numpy(), x0.cpu().numpy()) < SOLVE_TOL  # FP32 rounding of another split-K order
    p2 = smsm.Plan(L, Ns, Nc, N, r, caipi_div=Ldiv, batch=D)  # same shape: the cached choice
    p2.set_sens(c64(g["sens"]))
    x2, r2 = p2.reconstruct(ys, params=prm)
    assert r2.lanes == rep.lanes
    assert torch.equal(x1, x2)

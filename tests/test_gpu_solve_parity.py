"""Whole-solve parity at the full iteration schedules, per slice.

The GPU reconstruction (IRLS + CG for Eq. 10 through ``smsm_reconstruct``) is
compared with the FP64 oracle run with the same K, J, lam and eps schedule on
the same seeded data, slice by slice.

Bars, from the arithmetic of the FP32 form (FFTs, operators and CG vectors in
FP32, as the design fixes them; Gram products FP32-exact; weights, filter taps
and penalty multipliers formed in extended precision):
  * every FP32 operator agrees with the oracle to <= 1e-5 (test_gpu_parity.py);
  * one outer iteration (J CG steps) already differs from the oracle by ~1e-5:
    the CG iterate is a degree-J polynomial in A^H A + lam P_W, whose ~1e-6
    relative rounding (four FFT passes of ~u log2 N each) it amplifies; the
    later outer iterations carry that difference on (measured per slice after
    K = 1, 2, 3, 5, 8, 12, 16, 20 at 128^2: 1.2e-5, 1.8e-5, 2.4e-5, 2.0e-5, 1.5e-5,
    1.2e-5, 1.2e-5, 1.2e-5 on the worse slice; the same with the shape-generic
    kernels, so not a kernel's own error);
  * so the bars are 2e-5 per slice on the two-slice workloads (tiny 64^2, 10 x 10;
    plain 128^2, 20 x 15) and 3e-4 on the precision workload (MB 3, 256^2, FOV/3,
    20 x 15), whose middle slice grows from 3.1e-5 after one outer iteration to
    1.7e-4 after twenty (the other two stay at 3-4e-5);
  * the BF16 hi+lo split Gram on the precision workload: <= 1e-3 per slice (the
    metric's threshold), its measured value printed;
  * the eigen step by one-sided block Jacobi on an 8-CTA cluster (the only solver
    for C > 168: 8 shots with a 6x6 filter, C = 288) holds the same 2e-5 on the
    two-slice workloads: its eigenvalues and vectors carry FP32 rounding of the
    same order as the two-CTA two-sided solver's.

The oracle solves of the larger workloads take minutes on the host, so they
are started in spawned worker processes when the module's first test runs.
"""
import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest
import torch

import oracle as O
import _oracle_jobs as J

pytestmark = pytest.mark.gpu

BF16_TOL = 1e-3
FP32_TOL = {"tiny": 2e-5, "plain": 2e-5, "precision": 3e-4, "eight_shots": 2e-5}
LAM = 1e-2
DEV = "cuda:0"

# (L, Ns, Nc, N, r, Ldiv, seed, K, J)
WORK = {
    "tiny": (2, 4, 8, 64, 5, 2, 1, 10, 10),
    "plain": (2, 4, 32, 128, 6, 2, 1, 20, 15),
    "precision": (3, 4, 32, 256, 6, 3, 1, 20, 15),
    "eight_shots": (2, 8, 8, 64, 6, 2, 1, 10, 10),  # C = 8 * 36 = 288: cluster eigensolver
}


def _needed(request):
    """The workloads whose oracle solves the selected tests of this module read."""
    need = set()
    for item in request.session.items:
        if item.module is not request.module:
            continue
        cs = getattr(item, "callspec", None)
        if cs is not None and "key" in cs.params:
            need.add(cs.params["key"])
        elif item.originalname == "test_bf16_split_solve_per_slice":
            need.add("precision")
    return need


@pytest.fixture(scope="module")
def refs(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    need = _needed(request)
    ex = cf.ProcessPoolExecutor(max_workers=max(1, len(need)), mp_context=mp.get_context("spawn"))
    # the largest first, so it has the most time
    order = [k for k in ("precision", "plain", "eight_shots", "tiny") if k in need]
    futs = {k: ex.submit(J.solve, *WORK[k][:8], WORK[k][8], LAM) for k in order}
    yield futs
    ex.shutdown(wait=False, cancel_futures=True)


@pytest.fixture(scope="module")
def smsm(refs):
    from paper_1901_01893_gb300 import _build, smsm as mod

    _build.build()
    mod.lib()
    return mod


def c64(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.complex64)).to(DEV)


def gpu_solve(smsm, key, precision=0, flags=0):
    L, Ns, Nc, N, r, Ldiv, seed, K, Jc = WORK[key]
    g, xt, y = J.problem(L, Ns, Nc, N, seed, Ldiv)
    plan = smsm.Plan(L, Ns, Nc, N, r, caipi_div=Ldiv, precision=precision, flags=flags)
    plan.set_sens(c64(g["sens"]))
    x, rep = plan.reconstruct(c64(y), params=smsm.default_params(lam=LAM, outer_iters=K, cg_iters=Jc))
    assert rep.status == 0, rep.status
    return x.cpu().numpy(), xt, [rep.sweeps[k] for k in range(K)]


def per_slice(x, ref):
    return O.nrmse(x, ref, axis=(1, 2, 3))


@pytest.mark.parametrize("key", ["tiny", "plain", "precision", "eight_shots"])
def test_fp32_solve_per_slice(smsm, refs, key):
    x, xt, sweeps = gpu_solve(smsm, key)
    ref = refs[key].result()
    e = per_slice(x, ref)
    print(f"{key}: FP32 solve NRMSE vs FP64 oracle per slice {np.array2string(e, precision=2)}; "
          f"vs truth gpu {O.nrmse(x, xt):.3e} oracle {O.nrmse(ref, xt):.3e}; Jacobi sweeps {sweeps}")
    assert np.all(e <= FP32_TOL[key]), e


def test_bf16_split_solve_per_slice(smsm, refs):
    x, xt, sweeps = gpu_solve(smsm, "precision", precision=smsm.SMSM_PRECISION_BF16_SPLIT)
    ref = refs["precision"].result()
    e = per_slice(x, ref)
    print(f"precision, BF16 split Gram: solve NRMSE vs FP64 oracle per slice {np.array2string(e, precision=2)}")
    assert np.all(e <= BF16_TOL), e


@pytest.mark.parametrize("key", ["tiny", "plain"])
def test_cluster_eigensolver_solve_per_slice(smsm, refs, key):
    """The cluster eigensolver asked for where the two-CTA solver fits (C = 100, 144)."""
    x, xt, sweeps = gpu_solve(smsm, key, flags=smsm.SMSM_FLAG_CLUSTER_EIG)
    ref = refs[key].result()
    e = per_slice(x, ref)
    print(f"{key}, cluster eigensolver: FP32 solve NRMSE vs FP64 oracle per slice "
          f"{np.array2string(e, precision=2)}; Jacobi sweeps {sweeps}")
    assert np.all(e <= FP32_TOL[key]), e

"""The allocation-free Hankel Gram (smsm_hankel_gram_noalloc) against the planned one.

Callers that may not allocate device memory (they cannot create a plan) use
this entry point; its only scratch is a fixed array inside the library.  It
must give the same Gram as smsm_hankel_gram, on consecutive calls that reuse
the shared scratch.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the FP32-operator tolerance of the parity tests


@pytest.fixture(scope="module")
def smsm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_01893_gb300 import _build, smsm as mod

    _build.build()
    mod.lib()
    return mod


def _rand(rng, shape):
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return torch.from_numpy(a.astype(np.complex64)).to("cuda:0")


def _nrmse(a, b):
    return (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()


@pytest.mark.parametrize("L,Ns,N,r", [(2, 4, 64, 5), (3, 4, 256, 6), (2, 3, 48, 4)])
def test_noalloc_gram_matches_planned_gram_twice(smsm, L, Ns, N, r):
    rng = np.random.default_rng(17)
    plan = smsm.Plan(L, Ns, 1, N, r)
    for call in range(2):  # two calls in a row share (and reuse) the scratch array
        x = _rand(rng, (L, Ns, N, N))
        ref = plan.hankel_gram(x)
        got = smsm.smsm_hankel_gram_noalloc(x, r)
        torch.cuda.synchronize()
        assert _nrmse(got, ref) < TOL, (call, _nrmse(got, ref))
        if N <= 64:  # and against the FP64 oracle's Gram of the same (FP32) input
            G = O.gram(x.cpu().numpy().astype(np.complex128), r)
            assert O.nrmse(got.cpu().numpy(), G) < TOL
    plan.close()


def test_noalloc_gram_allocates_nothing(smsm):
    # after a first call (which may load the library's device code), further calls
    # leave the device's free memory unchanged: the library allocates nothing
    rng = np.random.default_rng(18)
    x = _rand(rng, (2, 4, 64, 64))
    G = torch.empty((2, 100, 100), dtype=torch.complex128, device="cuda:0")
    smsm.smsm_hankel_gram_noalloc(x, 5, G=G)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        smsm.smsm_hankel_gram_noalloc(x, 5, G=G)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_gram_rejects_oversize_geometry(smsm):
    # 8 shots, filter 6 at 512^2: 32 chunks x 288^2 x 16 B = 42 MB of partials > 8 MiB
    x = torch.zeros((1, 8, 512, 512), dtype=torch.complex64, device="cuda:0")
    with pytest.raises(smsm.SmsmError) as e:
        smsm.smsm_hankel_gram_noalloc(x, 6)
    assert e.value.status == smsm.SMSM_ERR_ARG
    assert "scratch" in str(e.value)
    # the column limit has its own message
    x = torch.zeros((1, 8, 64, 64), dtype=torch.complex64, device="cuda:0")
    with pytest.raises(smsm.SmsmError) as e:
        smsm.smsm_hankel_gram_noalloc(x, 7)  # C = 8 * 49 = 392 > 320
    assert e.value.status == smsm.SMSM_ERR_ARG
    assert "above 320" in str(e.value) and "scratch" not in str(e.value)

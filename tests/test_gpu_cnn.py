"""GPU parity of the learned warm start's CNN against the FP64 oracle (oracle/cnn.py).

The library's convolution, CReLU, residual, loss and manual backward kernels are
compared element by element with the oracle on the same inputs and on the same
BF16-rounded weights (the library rounds its FP32 master weights to BF16 for every
product; the oracle is given those rounded values in FP64):

  * forward x0 = a + f(a): NRMSE <= 1e-5 per sample;
  * gradients of the batch's mean loss: NRMSE <= 1e-4 per layer for W and b (FP32
    accumulation over every pixel of the batch);
  * Adam steps on a fixed batch lower the loss, and the learned start is
    x = F(cnn(F^-1(x_in))) (checked against the oracle's transforms and network).
Sizes cover ragged 16-pixel tiles and channel blocks.
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import cnn as OC

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def smsm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_01893_gb300 import _build, smsm as mod

    _build.build()
    mod.lib()
    return mod


def bf16(a):
    """Round the real and imaginary parts to BF16 (round to nearest even), as FP64."""
    t = torch.from_numpy(np.ascontiguousarray(a))
    re = t.real.to(torch.float32).to(torch.bfloat16).to(torch.float64)
    im = t.imag.to(torch.float32).to(torch.bfloat16).to(torch.float64)
    return (re + 1j * im).numpy()


def flat(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def unflat(v, shapes):
    out, o = [], 0
    for co, ci in shapes:
        n = co * ci * 9
        out.append((v[o:o + n].reshape(co, ci, 3, 3), v[o + n:o + n + co]))
        o += n + co
    return out


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def make(smsm, B, width, H, n, seed, layers=6):
    rng = np.random.default_rng(seed)
    shapes = OC.layer_shapes(B, width, layers)
    params = OC.init_params(rng, B, width, layers, last_scale=1.0)
    params = [(W, 0.1 * crandn(rng, *b.shape)) for W, b in params]
    net = smsm.CNN(B, H, H, width=width, layers=layers, max_batch=n)
    v = flat(params)
    assert net.count == v.size
    net.set_params(torch.from_numpy(v.astype(np.complex64)).to(DEV))
    p32 = unflat(bf16(v.astype(np.complex64)), shapes)  # the weights the kernels use
    a = crandn(rng, n, B, H, H).astype(np.complex64)
    t = crandn(rng, n, B, H, H).astype(np.complex64)
    return net, shapes, p32, a, t


CASES = [(12, 16, 24, 2), (3, 5, 20, 3), (12, 64, 18, 1)]  # (B, width, H, n)


@pytest.mark.parametrize("B,width,H,n", CASES)
def test_cnn_forward_parity(smsm, B, width, H, n):
    net, shapes, p, a, t = make(smsm, B, width, H, n, 1)
    out = net.forward(torch.from_numpy(a).to(DEV)).cpu().numpy()
    for s in range(n):
        ref = OC.forward(a[s].astype(np.complex128), p)
        assert O.nrmse(out[s], ref) < 1e-5


@pytest.mark.parametrize("B,width,H,n", CASES)
def test_cnn_gradient_parity(smsm, B, width, H, n):
    net, shapes, p, a, t = make(smsm, B, width, H, n, 2)
    loss, g = net.gradients(torch.from_numpy(a).to(DEV), torch.from_numpy(t).to(DEV))
    g = unflat(g.cpu().numpy().astype(np.complex128), shapes)
    ref_loss, ref = 0.0, None
    for s in range(n):
        L, gr = OC.backward(a[s].astype(np.complex128), t[s].astype(np.complex128), p)
        ref_loss += L / n
        ref = [(dW / n, db / n) for dW, db in gr] if ref is None else \
            [(rW + dW / n, rb + db / n) for (rW, rb), (dW, db) in zip(ref, gr)]
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    for k, ((gW, gb), (rW, rb)) in enumerate(zip(g, ref)):
        eW, eb = O.nrmse(gW, rW), O.nrmse(gb, rb)
        print(f"layer {k}: dW NRMSE {eW:.2e}, db NRMSE {eb:.2e}")
        assert eW < 1e-4 and eb < 1e-4, (k, eW, eb)


def test_cnn_training_lowers_the_loss(smsm):
    B, width, H, n = 4, 16, 24, 4
    net, shapes, p, a, t = make(smsm, B, width, H, n, 3)
    # a learnable target: a smoothed copy of the input
    ta = torch.from_numpy(a).to(DEV)
    tt = 0.5 * (ta + torch.roll(ta, 1, dims=-1))
    first = net.train_step(ta, tt, 1e-3)
    for _ in range(30):
        last = net.train_step(ta, tt, 1e-3)
    print(f"loss {first:.4f} -> {last:.4f}")
    assert last < 0.5 * first
    # the same steps from the same start are bit-reproducible
    net2, _, _, _, _ = make(smsm, B, width, H, n, 3)
    net2.train_step(ta, tt, 1e-3)
    for _ in range(30):
        last2 = net2.train_step(ta, tt, 1e-3)
    assert last2 == last
    assert torch.equal(net.get_params(), net2.get_params())


def test_learned_start_is_the_cnn_between_the_transforms(smsm):
    # x_in = A^H y made by the oracle; the expected value is the oracle's centred DFTs around
    # the oracle's network, applied to the same input
    L, Ns, Nc, N, r = 2, 2, 4, 32, 3
    rng = np.random.default_rng(7)
    S = crandn(rng, L, Nc, N, N) / np.sqrt(Nc)
    y = crandn(rng, Ns, Nc, N // Ns, N).astype(np.complex64)
    plan = smsm.Plan(L, Ns, Nc, N, r)
    plan.set_sens(torch.from_numpy(S.astype(np.complex64)).to(DEV))
    B = L * Ns
    net = smsm.CNN(B, N, N, width=8, layers=3, max_batch=1)
    shapes = OC.layer_shapes(B, 8, 3)
    params = OC.init_params(rng, B, 8, 3, last_scale=1.0)
    v = flat(params)
    net.set_params(torch.from_numpy(v.astype(np.complex64)).to(DEV))
    xin = O.adjoint(y.astype(np.complex128), S, L)
    x = smsm.learned_start(plan, net, torch.from_numpy(xin.astype(np.complex64)).to(DEV)).cpu().numpy()
    a = O.ifft2c(xin.astype(np.complex64).astype(np.complex128)).reshape(B, N, N)
    ref = O.fft2c(OC.forward(a, unflat(bf16(v.astype(np.complex64)), shapes))).reshape(L, Ns, N, N)
    assert O.nrmse(x, ref) < 1e-5

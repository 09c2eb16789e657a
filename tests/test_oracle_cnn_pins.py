"""Pins of the FP64 oracle of the warm-start CNN (oracle/cnn.py).

* the convolution equals SciPy's 2-D cross-correlation summed over input
  channels (a library routine, not a retyping of the loops);
* the manual backward equals central finite differences of the loss, for the
  weights, biases of every layer and for the input (the chain rule through the
  CReLUs and the residual connection);
* the input gradient of one convolution is its adjoint: <conv(h), g> = <h, conv^T(g)>.
"""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_conv_is_channel_summed_cross_correlation():
    rng = np.random.default_rng(0)
    h = crandn(rng, 3, 9, 7)
    W = crandn(rng, 2, 3, 3, 3)
    b = crandn(rng, 2)
    z = cnn.conv3x3(h, W, b)
    for o in range(2):
        # SciPy conjugates its second operand: pass conj(W) to get sum_k W[k] h[p + k - 1]
        ref = b[o] + sum(correlate2d(h[c], np.conj(W[o, c]), mode="same", boundary="fill") for c in range(3))
        assert np.allclose(z[o], ref, atol=1e-12)


def test_conv_input_gradient_is_the_adjoint():
    rng = np.random.default_rng(1)
    h = crandn(rng, 4, 8, 8)
    g = crandn(rng, 3, 8, 8)
    W = crandn(rng, 3, 4, 3, 3)
    z = cnn.conv3x3(h, W, np.zeros(3, dtype=complex))
    _, _, Gh = cnn.conv3x3_grads(h, W, g)
    assert np.isclose(np.vdot(z, g), np.vdot(h, Gh), rtol=1e-12)


@pytest.mark.parametrize("which", ["W", "b", "input"])
def test_backward_matches_finite_differences(which):
    rng = np.random.default_rng(2)
    B, width, H = 3, 5, 6
    params = cnn.init_params(rng, B, width=width, last_scale=1.0)
    params = [(W, crandn(rng, *b.shape) * 0.1) for W, b in params]
    a = crandn(rng, B, H, H)
    t = crandn(rng, B, H, H)
    L0, grads = cnn.backward(a, t, params)
    eps = 1e-6
    for k in (0, 3, 5):
        for _ in range(3):
            if which == "W":
                idx = tuple(rng.integers(s) for s in params[k][0].shape)
            elif which == "b":
                idx = (rng.integers(params[k][1].shape[0]),)
            else:
                idx = tuple(rng.integers(s) for s in a.shape)
            for unit in (1.0, 1j):
                def perturbed(e):
                    ps = [(W.copy(), b.copy()) for W, b in params]
                    aa = a.copy()
                    if which == "W":
                        ps[k][0][idx] += e * unit
                    elif which == "b":
                        ps[k][1][idx] += e * unit
                    else:
                        aa[idx] += e * unit
                    return cnn.loss(cnn.forward(aa, ps), t)
                fd = (perturbed(eps) - perturbed(-eps)) / (2 * eps)
                if which == "input":
                    # the input gradient: rerun the chain with the gradient kept at the input
                    g = _input_grad(a, t, params)[idx]
                else:
                    g = grads[k][0 if which == "W" else 1][idx]
                an = g.real if unit == 1.0 else g.imag
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (which, k, idx, unit, fd, an)
            if which == "input":
                break
        if which == "input":
            break


def _input_grad(a, t, params):
    out, hs, zs = cnn.forward(a, params, keep=True)
    G = 2.0 * (out - t) / np.sum(np.abs(t) ** 2)
    Gin = G.copy()  # residual connection
    for k in reversed(range(len(params))):
        if k + 1 < len(params):
            G = cnn.crelu_grad(zs[k], G)
        _, _, G = cnn.conv3x3_grads(hs[k], params[k][0], G)
    return Gin + G

"""Pins of the FP64 FNO oracle (CPU only): finite differences, numpy's real FFT, GELU values."""
import math

import numpy as np
import pytest

import oracle.fno_oracle as F

TINY = F.FnoShape(s=16, c_in=5, width=4, modes=3, layers=2, proj=6)


def tiny_problem(seed=3):
    p = F.init_params(TINY, seed)
    for l in range(TINY.layers):
        p[f"R{l}"] = p[f"R{l}"] * 30.0  # make the spectral branch matter
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((2, TINY.c_in, TINY.s, TINY.s))
    t = rng.standard_normal((2, 2, TINY.s, TINY.s))
    return p, a, t


def test_gelu_values():
    assert F._gelu(np.array(0.0)) == 0.0
    assert math.isclose(float(F._gelu(np.array(1.0))), 0.8413447460685429, rel_tol=1e-15)
    assert math.isclose(float(F._gelu(np.array(-1.0))), -0.15865525393145707, rel_tol=1e-14)
    x = np.linspace(-4, 4, 9)
    h = 1e-6
    fd = (F._gelu(x + h) - F._gelu(x - h)) / (2 * h)
    assert np.abs(fd - F._gelu_grad(x)).max() < 1e-9


def test_spectral_conv_matches_numpy_rfft2_truncation():
    sh = TINY
    rng = np.random.default_rng(0)
    v = rng.standard_normal((1, sh.width, sh.s, sh.s))
    R = rng.standard_normal((2 * sh.modes, sh.modes, sh.width, sh.width, 2))
    spec, V = F.spec_forward(v, R, sh)
    Vh = np.fft.rfft2(v)
    ky, kx = F.kept_modes(sh)
    assert np.allclose(V, Vh[:, :, ky][:, :, :, kx], atol=1e-10)
    Rc = R[..., 0] + 1j * R[..., 1]
    Uh = np.zeros_like(Vh)
    Uh[:, :, ky[:, None], kx[None, :]] = np.einsum("bipq,pqio->bopq", Vh[:, :, ky][:, :, :, kx], Rc)
    ref = np.fft.irfft2(Uh, s=(sh.s, sh.s))
    assert np.allclose(spec, ref, atol=1e-12)


@pytest.mark.parametrize("group", ["P", "pb", "R0", "W0", "b0", "R1", "W1", "b1", "Q1", "q1b",
                                   "Q2", "q2b"])
def test_backward_matches_central_differences(group):
    p, a, t = tiny_problem()
    out, cache = F.forward(p, a, TINY)
    _, dout = F.rel_l2_loss(out, t)
    g = F.backward(p, cache, dout, TINY)
    rng = np.random.default_rng(7)
    flat_idx = rng.choice(p[group].size, min(8, p[group].size), replace=False)
    for fi in flat_idx:
        idx = np.unravel_index(fi, p[group].shape)
        h = 1e-6
        q = {k: v.copy() for k, v in p.items()}
        q[group][idx] += h
        lp = F.rel_l2_loss(F.forward(q, a, TINY)[0], t)[0]
        q[group][idx] -= 2 * h
        lm = F.rel_l2_loss(F.forward(q, a, TINY)[0], t)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[group][idx]) <= 1e-6 * max(abs(fd), 1e-3), (group, idx, fd, g[group][idx])


def test_zero_spectral_weights_reduce_to_pointwise_network():
    p, a, _ = tiny_problem()
    for l in range(TINY.layers):
        p[f"R{l}"][:] = 0.0
    out, _ = F.forward(p, a, TINY)
    v = np.einsum("oc,bcyx->boyx", p["P"], a) + p["pb"][None, :, None, None]
    for l in range(TINY.layers):
        z = np.einsum("oi,biyx->boyx", p[f"W{l}"], v) + p[f"b{l}"][None, :, None, None]
        v = F._gelu(z) if l < TINY.layers - 1 else z
    h = F._gelu(np.einsum("jo,boyx->bjyx", p["Q1"], v) + p["q1b"][None, :, None, None])
    y = np.einsum("kj,bjyx->bkyx", p["Q2"], h) + p["q2b"][None, :, None, None]
    psi = (a[:, 0] + 1j * a[:, 1]) * np.exp(-1j * y[:, 0]) + y[:, 1] + 1j * y[:, 2]
    assert np.allclose(out, np.stack([psi.real, psi.imag], axis=1), atol=1e-13)


def test_head_turns_the_state_by_the_predicted_phase():
    rng = np.random.default_rng(4)
    a = rng.standard_normal((1, 5, 4, 4))
    y = np.zeros((1, 3, 4, 4))
    y[:, 0] = 0.7
    out = F.head(a, y)
    psi = (a[:, 0] + 1j * a[:, 1]) * np.exp(-0.7j)
    assert np.allclose(out[:, 0], psi.real) and np.allclose(out[:, 1], psi.imag)


def test_parameter_count_of_the_surrogate():
    sh = F.FnoShape()   # 256^2, width 64, 24 modes, 4 layers, projection 128
    assert F.n_params(sh) == (64 * 5 + 64) + 4 * (48 * 24 * 64 * 64 * 2 + 64 * 64 + 64) \
        + (128 * 64 + 128) + (3 * 128 + 3)

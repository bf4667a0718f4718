"""FP64 CPU oracle of the Fourier-neural-operator surrogate (forward and backward).

TEST INFRASTRUCTURE ONLY: imported by the tests and the benchmark's CPU
baseline, never by the CUDA library or its binding.

The surrogate maps the state of the split-step solver at time t, plus the
kernel parameters of Eq. 9 (alpha_Y, lambda_Y) and the local coefficient g as
constant channels, to the state 50 steps later.  It is written out from its
definition, with plain sums and matrix products, so the hand-derived backward
pass can be checked against central finite differences.

Network (channels c, grid s x s, kept modes ky in {0..m-1} u {s-m..s-1},
kx in {0..m-1}):
  v0 = P a + pb                                  (lift, per point)
  for l < L:  z_l = Spec_l(v_l) + W_l v_l + b_l,  v_{l+1} = gelu(z_l)  (last: v_L = z_{L-1})
  Spec(v)(y,x) = (1/s^2) sum_{ky,kx} w_kx Re( U[ky,kx] e^{+i th} ),  th = 2 pi (ky y + kx x)/s,
      U[o] = sum_i R[ky,kx,i,o] V[i],  V[i] = sum_{y,x} v_i(y,x) e^{-i th},  w_0 = 1, w_{kx>0} = 2
  h = gelu(Q1 v_L + q1b),   (phi, dr, di) = Q2 h + q2b   (three output channels)
  out = psi e^{-i phi} + (dr + i di),  psi = a[0] + i a[1]
        (the head turns the input state by a predicted phase field, the dominant effect
         of the nonlinear sub-step, and adds a correction)
  loss = mean_b ||out_b - target_b|| / ||target_b||
gelu(x) = x Phi(x) with the normal CDF Phi (the erf form).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Dict, List

import numpy as np


@dataclass
class FnoShape:
    s: int = 256        # grid points per axis
    c_in: int = 5       # input channels
    width: int = 64     # hidden channels
    modes: int = 24     # kept modes per axis block
    layers: int = 4
    proj: int = 128     # projection width


def _gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def _erf(x):
    from scipy.special import erf
    return erf(x)


def _gelu_grad(x):
    phi = np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * phi


def kept_modes(sh: FnoShape):
    ky = np.concatenate([np.arange(sh.modes), np.arange(sh.s - sh.modes, sh.s)])
    kx = np.arange(sh.modes)
    return ky, kx


def param_shapes(sh: FnoShape) -> List[tuple]:
    """Flat parameter order shared with the CUDA implementation."""
    shapes = [("P", (sh.width, sh.c_in)), ("pb", (sh.width,))]
    for l in range(sh.layers):
        shapes += [(f"R{l}", (2 * sh.modes, sh.modes, sh.width, sh.width, 2)),
                   (f"W{l}", (sh.width, sh.width)), (f"b{l}", (sh.width,))]
    shapes += [("Q1", (sh.proj, sh.width)), ("q1b", (sh.proj,)), ("Q2", (3, sh.proj)),
               ("q2b", (3,))]
    return shapes


def unflatten(sh: FnoShape, flat: np.ndarray) -> Dict[str, np.ndarray]:
    out, off = {}, 0
    for name, shp in param_shapes(sh):
        n = int(np.prod(shp))
        out[name] = flat[off:off + n].reshape(shp)
        off += n
    assert off == flat.size
    return out


def flatten(sh: FnoShape, p: Dict[str, np.ndarray]) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel()
                           for name, _ in param_shapes(sh)])


def n_params(sh: FnoShape) -> int:
    return sum(int(np.prod(shp)) for _, shp in param_shapes(sh))


def _phases(sh: FnoShape):
    ky, kx = kept_modes(sh)
    y = np.arange(sh.s)
    Ey = np.exp(-2j * np.pi * np.outer(ky, y) / sh.s)    # (2m, s)
    Ex = np.exp(-2j * np.pi * np.outer(y, kx) / sh.s)    # (s, m)
    return Ey, Ex


def spec_forward(v: np.ndarray, R: np.ndarray, sh: FnoShape):
    """v: (B, C, s, s) real; R: (2m, m, C, C, 2).  Returns (Spec(v), V) with V the kept modes."""
    Ey, Ex = _phases(sh)
    V = np.einsum("py,bcyx,xq->bcpq", Ey, v, Ex, optimize=True)       # (B, C, 2m, m)
    Rc = R[..., 0] + 1j * R[..., 1]                                   # (2m, m, Ci, Co)
    U = np.einsum("bipq,pqio->bopq", V, Rc, optimize=True)
    w = np.where(np.arange(sh.modes) == 0, 1.0, 2.0) / (sh.s * sh.s)
    spec = np.einsum("py,bopq,xq,q->boyx", np.conj(Ey), U, np.conj(Ex), w, optimize=True)
    return spec.real, V


def forward(params: Dict[str, np.ndarray], a: np.ndarray, sh: FnoShape):
    """a: (B, c_in, s, s).  Returns (out (B, 2, s, s), cache for backward)."""
    cache = {"a": a}
    v = np.einsum("oc,bcyx->boyx", params["P"], a) + params["pb"][None, :, None, None]
    cache["v0"] = v
    for l in range(sh.layers):
        spec, V = spec_forward(v, params[f"R{l}"], sh)
        z = spec + np.einsum("oi,biyx->boyx", params[f"W{l}"], v) + params[f"b{l}"][None, :, None, None]
        cache[f"V{l}"] = V
        cache[f"z{l}"] = z
        v = _gelu(z) if l < sh.layers - 1 else z
        cache[f"v{l + 1}"] = v
    g1 = np.einsum("jo,boyx->bjyx", params["Q1"], v) + params["q1b"][None, :, None, None]
    h = _gelu(g1)
    cache["g1"], cache["h"] = g1, h
    y = np.einsum("kj,bjyx->bkyx", params["Q2"], h) + params["q2b"][None, :, None, None]
    cache["y"] = y
    out = head(a, y)
    return out, cache


def head(a: np.ndarray, y: np.ndarray) -> np.ndarray:
    """psi e^{-i phi} + (dr + i di) as (re, im) planes; psi = a[0] + i a[1], (phi, dr, di) = y."""
    pr, pi, ph = a[:, 0], a[:, 1], y[:, 0]
    c, s = np.cos(ph), np.sin(ph)
    return np.stack([pr * c + pi * s + y[:, 1], pi * c - pr * s + y[:, 2]], axis=1)


def rel_l2_loss(out: np.ndarray, target: np.ndarray):
    """mean_b ||out_b - t_b|| / ||t_b|| and its gradient with respect to out."""
    B = out.shape[0]
    d = (out - target).reshape(B, -1)
    t = target.reshape(B, -1)
    dn = np.linalg.norm(d, axis=1)
    tn = np.linalg.norm(t, axis=1)
    loss = float(np.mean(dn / tn))
    grad = (d / (B * dn[:, None] * tn[:, None])).reshape(out.shape)
    return loss, grad


def backward(params: Dict[str, np.ndarray], cache, dout: np.ndarray, sh: FnoShape):
    """Gradients of a scalar loss with respect to every parameter, given dL/dout."""
    g = {}
    h, g1, y, a = cache["h"], cache["g1"], cache["y"], cache["a"]
    # head: d out_r / d phi = rot_i, d out_i / d phi = -rot_r with rot = psi e^{-i phi}
    c, s = np.cos(y[:, 0]), np.sin(y[:, 0])
    rot_r = a[:, 0] * c + a[:, 1] * s
    rot_i = a[:, 1] * c - a[:, 0] * s
    dy = np.stack([dout[:, 0] * rot_i - dout[:, 1] * rot_r, dout[:, 0], dout[:, 1]], axis=1)
    g["Q2"] = np.einsum("bkyx,bjyx->kj", dy, h)
    g["q2b"] = dy.sum(axis=(0, 2, 3))
    dh = np.einsum("kj,bkyx->bjyx", params["Q2"], dy)
    dg1 = dh * _gelu_grad(g1)
    vL = cache[f"v{sh.layers}"]
    g["Q1"] = np.einsum("bjyx,boyx->jo", dg1, vL)
    g["q1b"] = dg1.sum(axis=(0, 2, 3))
    dv = np.einsum("jo,bjyx->boyx", params["Q1"], dg1)
    Ey, Ex = _phases(sh)
    w = np.where(np.arange(sh.modes) == 0, 1.0, 2.0) / (sh.s * sh.s)
    for l in reversed(range(sh.layers)):
        z = cache[f"z{l}"]
        dz = dv * _gelu_grad(z) if l < sh.layers - 1 else dv
        vl = cache[f"v{l}"]
        g[f"W{l}"] = np.einsum("boyx,biyx->oi", dz, vl)
        g[f"b{l}"] = dz.sum(axis=(0, 2, 3))
        dv = np.einsum("oi,boyx->biyx", params[f"W{l}"], dz)
        # spectral branch: dL/dU = (w_kx / s^2) F(dz);  dL/dV_i = sum_o conj(R_io) dL/dU_o
        GU = np.einsum("py,boyx,xq->bopq", Ey, dz, Ex, optimize=True) * w[None, None, None, :]
        V = cache[f"V{l}"]
        Rc = params[f"R{l}"][..., 0] + 1j * params[f"R{l}"][..., 1]
        GR = np.einsum("bipq,bopq->pqio", np.conj(V), GU, optimize=True)
        g[f"R{l}"] = np.stack([GR.real, GR.imag], axis=-1)
        GV = np.einsum("pqio,bopq->bipq", np.conj(Rc), GU, optimize=True)
        # dL/dv(y,x) = sum_modes Re(GV e^{+i th})
        dv = dv + np.einsum("py,bipq,xq->biyx", np.conj(Ey), GV, np.conj(Ex), optimize=True).real
    g["P"] = np.einsum("boyx,bcyx->oc", dv, cache["a"])
    g["pb"] = dv.sum(axis=(0, 2, 3))
    return g


def init_params(sh: FnoShape, seed: int = 0) -> Dict[str, np.ndarray]:
    """Seeded initial parameters (uniform fans; spectral weights ~ U[0,1] / (C C))."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in param_shapes(sh):
        if name.startswith("R"):
            p[name] = rng.uniform(0.0, 1.0, shp) / (sh.width * sh.width)
        elif name in ("pb", "q1b", "q2b") or (name.startswith("b") and name[1:].isdigit()):
            p[name] = np.zeros(shp)
        else:
            fan_in = shp[1]
            bound = 1.0 / math.sqrt(fan_in)
            p[name] = rng.uniform(-bound, bound, shp)
    return p

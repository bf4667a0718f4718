"""Observables from FP32 line transforms with FP64 sums (sn_set_obs_mode).

The FP32 mode computes the quantities of sn_obs from the step's FP32 line
transforms: e_kin and the momenta by 1D Parseval along every axis, the
density's half spectrum along the last axis (with the real-space sums and
the centroids from its line modes), e_pot from sum K |F rho|^2 over it.  It
must agree with the FP64 mode (itself held to the oracle at 1e-10) and with
the oracle to the precision of FP32 transforms, on 2D and 3D grids with
lines of 8 to 1024 points, several fields, V_ext, both kernel kinds, and
states left open by earlier steps.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_1909_08354_b300 import sn

pytestmark = pytest.mark.gpu

REL = 2e-6  # mass, energies: relative to the FP64 values


def kernel_kw(kp, **over):
    kw = dict(coeff_lap=kp.coeff_lap, G=kp.G, alpha_Y=kp.alpha_Y, lambda_Y=kp.lambda_Y,
              g_local=kp.g_local)
    kw.update(over)
    return kw


def both_modes(shape, seed=4, fields=1, vext=False, steps=0, **over):
    psis, L, kp = W.random_fields(shape, seed, fields)
    kw = kernel_kw(kp, **over)
    if vext:
        kw["v_ext"] = np.random.default_rng(seed).standard_normal(shape) * 0.2
    g = sn.Grid(shape, L, "c64")
    try:
        g.set_fields(fields)
        g.set_kernel(**kw)
        g.set_state(psis[0] if fields == 1 else psis)
        if steps:
            g.step(0.02, steps)
        ref = g.observables()
        g.set_obs_mode(sn.SN_OBS_FP32)
        got = g.observables()
        state = g.get_state().copy()
    finally:
        g.close()
    return got, ref, L, kw, state


def check(got, ref, L, coeff_lap):
    for key in ("mass", "e_kin", "e_pot", "e_nl", "e_total"):
        assert abs(got[key] - ref[key]) <= REL * max(abs(ref[key]), 1e-30) + 1e-12, key
    # |p_a| <= sqrt(mass * sum k^2 |F psi|^2): the momenta's natural scale
    pscale = math.sqrt(ref["mass"] * abs(ref["e_kin"] / coeff_lap))
    for a in range(len(L)):
        assert abs(got["momentum"][a] - ref["momentum"][a]) <= REL * pscale + 1e-12, a
        d = (got["centroid"][a] - ref["centroid"][a] + L[a] / 2) % L[a] - L[a] / 2
        assert abs(d) <= 1e-5 * L[a], a
    if "step" in ref:
        assert got["step"] == ref["step"]


@pytest.mark.parametrize("shape", [(64, 64), (128, 256), (1024, 16), (8, 512), (32, 64, 16),
                                   (64, 64, 64), (16, 512, 8), (8, 8, 1024)],
                         ids=lambda s: "x".join(map(str, s)))
def test_fp32_observables_match_fp64(shape):
    got, ref, L, kw, _ = both_modes(shape, vext=True, steps=3)
    check(got, ref, L, kw["coeff_lap"])


@pytest.mark.parametrize("over", [dict(), dict(alpha_Y=0.0), dict(g_local=1.5),
                                  dict(kind=sn.SN_KERNEL_POISSON, B=1.0, C=-2.0, D=0.7)],
                         ids=["nmc", "newton", "local", "poisson"])
def test_fp32_observables_kernel_kinds(over):
    got, ref, L, kw, _ = both_modes((32, 64, 32), seed=9, steps=2, **over)
    check(got, ref, L, kw["coeff_lap"])


def test_fp32_observables_several_fields():
    got, ref, L, kw, _ = both_modes((32, 128, 16), seed=6, fields=3, vext=True, steps=2)
    check(got, ref, L, kw["coeff_lap"])


def test_fp32_observables_match_the_oracle():
    got, _, L, kw, state = both_modes((32, 16, 64), seed=13, vext=True, steps=2)
    okw = {k: v for k, v in kw.items() if k not in ("v_ext",)}
    ref = O.observables(state.astype(np.complex128), L, v_ext=kw["v_ext"], **okw)
    check(got, ref, L, kw["coeff_lap"])


def test_fp32_mode_rejects_complex128_and_unknown_modes():
    g = sn.Grid((16, 16), (4.0, 4.0), "c128")
    try:
        with pytest.raises(sn.SNError) as e:
            g.set_obs_mode(sn.SN_OBS_FP32)
        assert e.value.status == sn.SN_ENOTSUP
    finally:
        g.close()
    g = sn.Grid((16, 16), (4.0, 4.0), "c64")
    try:
        with pytest.raises(sn.SNError) as e:
            g.set_obs_mode(5)
        assert e.value.status == sn.SN_EINVAL
    finally:
        g.close()


def test_fp32_observables_at_256_cubed_are_faster():
    torch = pytest.importorskip("torch")
    w = W.nbody_3d()
    psi = w.psi0().astype(np.complex64)
    g = sn.Grid(w.n, w.L, "c64")
    try:
        g.set_kernel(**kernel_kw(w.kernel))
        g.set_state(psi)
        g.step(w.dt, 2)
        ref = g.observables()
        t = {}
        for mode in (sn.SN_OBS_FP64, sn.SN_OBS_FP32):
            g.set_obs_mode(mode)
            g.observables()
            torch.cuda.synchronize()
            import time
            t0 = time.perf_counter()
            for _ in range(3):
                out = g.observables()
            t[mode] = (time.perf_counter() - t0) / 3
        check(out, ref, w.L, w.kernel.coeff_lap)
        print(f"observables at 256^3: FP64 {t[sn.SN_OBS_FP64] * 1e3:.2f} ms, "
              f"FP32 {t[sn.SN_OBS_FP32] * 1e3:.2f} ms")
        assert t[sn.SN_OBS_FP32] < 0.5 * t[sn.SN_OBS_FP64]
    finally:
        g.close()

"""Several coupled wave functions (sn_set_fields): every field obeys Eq. 1
with one shared potential and local term of the total density, through the
C-ABI, against the FP64 oracle of oracle/fields_oracle.py.

Bars: the single-field ones, per split step rel-L2 over all fields <= 1e-6
(complex64, fused FP32 passes) and <= 1e-12 (complex128, FP64 path); k merged
steps: k times that.
"""
import math

import numpy as np
import pytest

import oracle as O
import oracle.fields_oracle as F
import workloads as W
from paper_1909_08354_b300 import sn

pytestmark = pytest.mark.gpu

STEP_TOL = {"c64": 1e-6, "c128": 1e-12}


def kernel_kw(kp):
    return dict(coeff_lap=kp.coeff_lap, G=kp.G, alpha_Y=kp.alpha_Y, lambda_Y=kp.lambda_Y,
                g_local=kp.g_local)


def gpu_fields(psis, L, kw, dtype, dt, nsteps, engine=sn.SN_ENGINE_FP32, v_ext=None):
    g = sn.Grid(psis.shape[1:], L, dtype)
    try:
        if engine != sn.SN_ENGINE_FP32:
            g.set_engine(engine)
        g.set_fields(psis.shape[0])
        g.set_kernel(**kw, v_ext=v_ext)
        g.set_state(np.ascontiguousarray(psis, dtype=g.np_dtype))
        g.step(dt, nsteps)
        return g.get_state()
    finally:
        g.close()


def inputs(shape, m, seed, L=10.0):
    psis, L, kp = W.random_fields(shape, seed, m, L)
    kw = kernel_kw(kp)
    kw["g_local"] = 0.05  # the local term of the total density is exercised
    return psis, L, kw


CASES = [((64, 128), 2), ((8, 8), 3), ((128, 32), 4), ((32, 16, 64), 2), ((16, 16, 16), 3),
         ((8, 32, 256), 2), ((16, 1024), 2), ((512, 16), 3), ((8, 512, 8), 2)]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("shape,m", CASES, ids=[f"{'x'.join(map(str, s))}-{m}f" for s, m in CASES])
def test_fields_match_oracle(shape, m, dtype):
    psis, L, kw = inputs(shape, m, seed=3 * sum(shape) + m)
    psis = psis.astype(np.complex64 if dtype == "c64" else np.complex128)
    for nsteps in (1, 3):
        out = gpu_fields(psis, L, kw, dtype, 0.02, nsteps)
        assert out.shape == psis.shape
        ref = F.fields_evolve(psis, 0.02, nsteps, L, **kw)
        err = O.rel_l2(out, ref)
        assert err <= nsteps * STEP_TOL[dtype], (nsteps, err)
    # the coupling matters here: field 0 alone would evolve differently
    solo = O.evolve(psis[0].astype(np.complex128), 0.02, 3, L, **kw)
    assert O.rel_l2(ref[0], solo) > 1e3 * STEP_TOL["c64"]


def test_fields_with_v_ext_and_the_optical_kernel():
    shape, m = (128, 64), 3
    psis, L, _ = inputs(shape, m, seed=77, L=(20.0, 12.0))
    kw = dict(coeff_lap=-0.5, kind=O.KIND_POISSON, B=1.0, C=-1.0 / 4.0, D=-2.0, g_local=0.02)
    x = W.coords(shape[0], L[0])[:, None]
    v = 0.3 * np.cos(2 * math.pi * x / L[0]) * np.ones((1, shape[1]))
    out = gpu_fields(psis.astype(np.complex64), L, kw, "c64", 0.02, 4, v_ext=v)
    ref = F.fields_evolve(psis, 0.02, 4, L, v_ext=v, **kw)
    assert O.rel_l2(out, ref) <= 4 * STEP_TOL["c64"]


@pytest.mark.parametrize("shape", [(256, 64), (16, 256, 16)])
def test_fields_on_the_tensor_core_engine(shape):
    psis, L, kw = inputs(shape, 2, seed=5 + sum(shape))
    out = gpu_fields(psis.astype(np.complex64), L, kw, "c64", 0.02, 3, engine=sn.SN_ENGINE_TC16)
    ref = F.fields_evolve(psis, 0.02, 3, L, **kw)
    assert O.rel_l2(out, ref) <= 3 * STEP_TOL["c64"]


def test_equal_copies_match_the_single_field_step():
    # two copies of psi / sqrt 2 carry the total density |psi|^2: each must
    # follow the single-field step of psi (which applies g |psi|^2 pointwise),
    # so the spectral local term of the multi-field path is checked against it
    w = W.random_small((64, 64), seed=9)
    kw = dict(kernel_kw(w.kernel), g_local=0.2)
    psi = w.psi0().astype(np.complex64)
    copies = np.stack([psi / np.float32(math.sqrt(2.0))] * 2)
    out = gpu_fields(copies, w.L, kw, "c64", 0.02, 5)
    g = sn.Grid(psi.shape, w.L, "c64")
    try:
        g.set_kernel(**kw)
        g.set_state(psi)
        g.step(0.02, 5)
        single = g.get_state()
    finally:
        g.close()
    for j in range(2):
        assert O.rel_l2(out[j] * math.sqrt(2.0), single) <= 5 * STEP_TOL["c64"]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_fields_observables_match_oracle(dtype):
    shape = (32, 64, 16) if dtype == "c64" else (64, 32)
    psis, L, kw = inputs(shape, 3, seed=123)
    x = W.coords(shape[0], L[0]).reshape((-1,) + (1,) * (len(shape) - 1))
    v = 0.1 * np.sin(2 * math.pi * x / L[0]) * np.ones(shape)
    g = sn.Grid(shape, L, dtype)
    try:
        g.set_fields(3)
        g.set_kernel(**kw, v_ext=v)
        g.set_state(psis.astype(g.np_dtype))
        got = g.observables()
        state = g.get_state().astype(np.complex128)
    finally:
        g.close()
    ref = F.fields_observables(state, L, v_ext=v, **kw)
    tol = 1e-10 if dtype == "c128" else 1e-9
    for k in ("mass", "e_kin", "e_pot", "e_nl", "e_total"):
        assert got[k] == pytest.approx(ref[k], rel=tol, abs=tol), k
    for a in range(len(shape)):
        assert got["centroid"][a] == pytest.approx(ref["centroid"][a], abs=1e-9)
        assert got["momentum"][a] == pytest.approx(ref["momentum"][a], rel=1e-9, abs=1e-9)


def test_each_field_keeps_its_mass_and_steps_reverse():
    psis, L, kw = inputs((128, 128), 3, seed=200)
    psis = (psis * np.array([1.0, 0.6, 0.3])[:, None, None]).astype(np.complex128)
    g = sn.Grid((128, 128), L, "c128")
    try:
        g.set_fields(3)
        g.set_kernel(**kw)
        g.set_state(psis)
        g.step(0.02, 50)
        mid = g.get_state()
        g.step(-0.02, 50)
        back = g.get_state()
    finally:
        g.close()
    m0 = (np.abs(psis) ** 2).sum(axis=(1, 2))
    m1 = (np.abs(mid) ** 2).sum(axis=(1, 2))
    assert np.allclose(m1, m0, rtol=1e-12, atol=0)
    assert np.abs(back - psis).max() < 1e-9 * np.abs(psis).max()


def test_set_fields_resets_the_state_and_validates():
    g = sn.Grid((16, 16), (4.0, 4.0), "c64")
    try:
        g.set_state(np.ones((16, 16), np.complex64))
        g.set_fields(3)
        assert sn.lib().sn_get_fields(g.h) == 3
        st = g.get_state()
        assert st.shape == (3, 16, 16) and not np.any(st)
        for bad in (0, -1, sn.SN_MAX_FIELDS + 1):
            with pytest.raises(sn.SNError) as e:
                g.set_fields(bad)
            assert e.value.status == sn.SN_EINVAL
        assert sn.lib().sn_get_fields(g.h) == 3
        g.set_fields(1)  # back to Eqs. 1-2, state zero
        assert g.get_state().shape == (16, 16) and not np.any(g.get_state())
    finally:
        g.close()


def test_fields_and_the_fluid_model_exclude_each_other():
    g = sn.Grid((16, 16), (4.0, 4.0), "c128")
    try:
        g.set_fields(2)
        with pytest.raises(sn.SNError) as e:
            g.set_fluid()
        assert e.value.status == sn.SN_ENOTSUP
        g.set_fields(1)
        g.set_fluid()
        with pytest.raises(sn.SNError) as e:
            g.set_fields(2)
        assert e.value.status == sn.SN_ENOTSUP
    finally:
        g.close()


def test_fields_through_device_pointers_on_a_torch_stream():
    torch = pytest.importorskip("torch")
    psis, L, kw = inputs((32, 64), 2, seed=300)
    psis = psis.astype(np.complex64)
    s = torch.cuda.Stream()
    g = sn.Grid((32, 64), L, "c64", stream=s.cuda_stream)
    try:
        g.set_fields(2)
        g.set_kernel(**kw)
        dev = torch.from_numpy(psis).cuda()
        torch.cuda.synchronize()
        g.set_state(dev)
        g.step(0.02, 3)
        out = torch.empty_like(dev)
        g.get_state(out)
        g.sync()
    finally:
        g.close()
    host = gpu_fields(psis, L, kw, "c64", 0.02, 3)
    assert np.array_equal(out.cpu().numpy(), host)  # the same kernels, bit for bit


def test_launches_per_step_do_not_grow_with_the_fields():
    # one launch per pass for all fields: a 3D step is six launches for any count
    counts = []
    for m in (1, 3):
        psis, L, kw = inputs((16, 32, 16), m, seed=400)
        g = sn.Grid((16, 32, 16), L, "c64")
        try:
            g.set_fields(m)
            g.set_kernel(**kw)
            g.set_state(psis.astype(np.complex64))
            n0 = g.launch_count()
            g.step(0.02, 10)
            counts.append(g.launch_count() - n0)
        finally:
            g.close()
    assert counts[0] == counts[1] == 6 * 10

"""Tensor-core line engine (SN_ENGINE_TC16): every 16-point DFT stage of a
256-point axis on mma.sync with FP16 operands split into hi + lo parts.

Bars, the same as the FP32 engine's:
  * one unnormalised 256-point DFT against numpy's FP64 FFT: rel-L2 per line
    <= 1e-6 (FP32 rounding of ~16 operations per value);
  * one split step against the FP64 oracle: rel-L2 <= 1e-6 (k merged steps:
    k times that);
  * mass over 1000 steps of the 256^3 N-body workload: drift <= 1e-5.
Lines of other lengths are left to the FP32 engine, bit for bit.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_1909_08354_b300 import sn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def kernel_kw(kp):
    return dict(coeff_lap=kp.coeff_lap, G=kp.G, alpha_Y=kp.alpha_Y, lambda_Y=kp.lambda_Y,
                g_local=kp.g_local)


def lines_256(nlines, seed):
    """Random lines with a few special ones: zero, huge, tiny, a delta, a constant."""
    rng = np.random.default_rng(seed)
    x = (rng.standard_normal((nlines, 256)) + 1j * rng.standard_normal((nlines, 256)))
    x *= np.exp(rng.uniform(-3, 3, (nlines, 1)))
    x[0] = 0
    x[1] *= 1e30
    x[2] *= 1e-30
    x[3] = 0
    x[3, 17] = 2.5 - 1j
    x[4] = 0.75 + 0.25j
    return x.astype(np.complex64)


def line_fft(x, sign, engine):
    d = torch.from_numpy(x.copy()).cuda()
    sn.sn_test_line_fft_f32(d, 256, sign, engine)
    return d.cpu().numpy()


@pytest.mark.parametrize("sign", [-1, 1])
@pytest.mark.parametrize("nlines", [16, 37, 1000])
def test_line_dft_matches_numpy(sign, nlines):
    x = lines_256(nlines, seed=nlines + sign)
    got = line_fft(x, sign, sn.SN_ENGINE_TC16).astype(np.complex128)
    xd = x.astype(np.complex128)
    ref = np.fft.fft(xd, axis=1) if sign < 0 else np.fft.ifft(xd, axis=1) * 256
    for i in range(nlines):
        nrm = np.linalg.norm(ref[i])
        err = np.linalg.norm(got[i] - ref[i])
        assert err <= 1e-6 * nrm or (nrm == 0 and err == 0), (i, err / max(nrm, 1e-300))


def test_line_dft_accuracy_is_that_of_the_fp32_engine():
    x = lines_256(512, seed=9)
    ref = np.fft.fft(x.astype(np.complex128), axis=1)

    def err(engine):
        got = line_fft(x, -1, engine).astype(np.complex128)
        return np.linalg.norm(got[5:] - ref[5:]) / np.linalg.norm(ref[5:])

    e_tc, e_fp32 = err(sn.SN_ENGINE_TC16), err(sn.SN_ENGINE_FP32)
    assert e_tc <= 3.0 * e_fp32, (e_tc, e_fp32)


def test_other_lengths_keep_the_fp32_engine():
    rng = np.random.default_rng(2)
    x = (rng.standard_normal((40, 128)) + 1j * rng.standard_normal((40, 128))).astype(np.complex64)
    a = torch.from_numpy(x.copy()).cuda()
    b = torch.from_numpy(x.copy()).cuda()
    sn.sn_test_line_fft_f32(a, 128, -1, sn.SN_ENGINE_FP32)
    sn.sn_test_line_fft_f32(b, 128, -1, sn.SN_ENGINE_TC16)
    assert torch.equal(a, b)


def run(psi, L, kw, dt, nsteps, engine):
    g = sn.Grid(psi.shape, L, "c64")
    try:
        g.set_engine(engine)
        g.set_kernel(**kw)
        g.set_state(np.ascontiguousarray(psi, dtype=np.complex64))
        g.step(dt, nsteps)
        return g.get_state()
    finally:
        g.close()


SHAPES = [(256, 256), (256, 32), (16, 256), (256, 16, 16), (16, 256, 16), (16, 16, 256),
          (256, 8, 256)]


@pytest.mark.parametrize("shape", SHAPES)
def test_one_step_matches_oracle(shape):
    w = W.random_small(shape, seed=sum(shape) + 5)
    psi = w.psi0().astype(np.complex64)
    kw = kernel_kw(w.kernel)
    out = run(psi, w.L, kw, 0.02, 1, sn.SN_ENGINE_TC16)
    ref = O.evolve(psi.astype(np.complex128), 0.02, 1, w.L, **kw)
    assert O.rel_l2(out, ref) <= 1e-6


@pytest.mark.parametrize("shape", [(256, 64), (32, 256, 8)])
def test_merged_steps_match_oracle(shape):
    w = W.random_small(shape, seed=11 + sum(shape))
    psi = w.psi0().astype(np.complex64)
    kw = kernel_kw(w.kernel)
    out = run(psi, w.L, kw, 0.03, 5, sn.SN_ENGINE_TC16)
    ref = O.evolve(psi.astype(np.complex128), 0.03, 5, w.L, **kw)
    assert O.rel_l2(out, ref) <= 5e-6


def test_nbody_3d_256_one_step_vs_oracle():
    """The 256^3 N-body workload, one step on the tensor-core engine."""
    w = W.nbody_3d()
    psi = w.psi0().astype(np.complex64)
    kw = kernel_kw(w.kernel)
    out = run(psi, w.L, kw, w.dt, 1, sn.SN_ENGINE_TC16)
    ref = O.evolve(psi.astype(np.complex128), w.dt, 1, w.L, **kw)
    assert O.rel_l2(out, ref) <= 1e-6


def test_nbody_3d_256_mass_drift_1000_steps():
    w = W.nbody_3d(alpha_Y=0.1)
    g = sn.Grid(w.n, w.L, "c64")
    g.set_engine(sn.SN_ENGINE_TC16)
    g.set_kernel(**kernel_kw(w.kernel))
    g.set_state(w.psi0().astype(np.complex64))
    m0 = g.observables()["mass"]
    g.step(w.dt, w.nsteps)
    m1 = g.observables()["mass"]
    g.close()
    assert abs(m1 / m0 - 1) <= 1e-5, m1 / m0 - 1


def test_engine_arguments():
    g = sn.Grid((16, 16), (1.0, 1.0), "c128")
    with pytest.raises(sn.SNError) as e:
        g.set_engine(sn.SN_ENGINE_TC16)
    assert e.value.status == sn.SN_ENOTSUP
    with pytest.raises(sn.SNError) as e:
        g.set_engine(7)
    assert e.value.status == sn.SN_EINVAL
    g.set_engine(sn.SN_ENGINE_FP32)
    g.close()

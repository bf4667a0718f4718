"""The tcgen05 form of the tensor-core line engine (SN_ENGINE_UMMA).

Both radix-16 stages of each 256-point line run as tcgen05.mma products with
split-FP16 operands and FP32 accumulators in tensor memory.  Each line's DFT
must match numpy's to the precision of the split (about 2^-21 per product),
in both directions, on ragged tiles of lines, zero lines and lines whose
magnitudes span many decades (the per-row power-of-two scaling); and the
three line engines are timed on the same lines.
"""
import numpy as np
import pytest

from paper_1909_08354_b300 import sn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def lines(nlines, seed, spread=0.0):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((nlines, 256)) + 1j * rng.standard_normal((nlines, 256))
    if spread:
        x *= 10.0 ** rng.uniform(-spread, spread, size=(nlines, 1))
    return x.astype(np.complex64)


def run(x, sign, engine=sn.SN_ENGINE_UMMA):
    d = torch.from_numpy(x.copy()).cuda()
    sn.sn_test_line_fft_engines(d, 256, sign, engine)
    return d.cpu().numpy()


def per_line_rel(got, ref):
    return np.linalg.norm(got - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-300)


@pytest.mark.parametrize("sign", [-1, 1])
@pytest.mark.parametrize("nlines", [1, 8, 299, 4096])
def test_umma_lines_match_numpy(sign, nlines):
    x = lines(nlines, seed=nlines + (sign > 0))
    got = run(x, sign)
    x64 = x.astype(np.complex128)
    ref = np.fft.fft(x64, axis=1) if sign < 0 else np.fft.ifft(x64, axis=1) * 256
    assert per_line_rel(got, ref).max() <= 2e-6


def test_umma_scaling_zero_and_wide_range_lines():
    x = lines(64, seed=7, spread=15.0)
    x[5] = 0
    x[9, :] = 0
    x[9, 3] = 1e-30
    got = run(x, -1)
    ref = np.fft.fft(x.astype(np.complex128), axis=1)
    assert np.all(got[5] == 0)
    rel = per_line_rel(got, ref)
    rel[5] = 0
    assert rel.max() <= 2e-6


def test_umma_engine_is_not_a_grid_engine():
    g = sn.Grid((16, 16), (1.0, 1.0), "c64")
    try:
        with pytest.raises(sn.SNError) as e:
            g.set_engine(sn.SN_ENGINE_UMMA)
        assert e.value.status == sn.SN_ENOTSUP
    finally:
        g.close()
    d = torch.zeros(128, dtype=torch.complex64, device="cuda")
    with pytest.raises(sn.SNError) as e:
        sn.sn_test_line_fft_engines(d, 128, -1, sn.SN_ENGINE_UMMA)
    assert e.value.status == sn.SN_EINVAL


def test_line_engines_timed_on_the_same_lines():
    """65536 lines of 256 points (one axis of the 256^3 grid): each engine's
    time per launch, and its error against numpy on a sample."""
    x = lines(65536, seed=1)
    x64 = x[:256].astype(np.complex128)
    ref = np.fft.fft(x64, axis=1)
    d = torch.from_numpy(x).cuda()
    out = {}
    for engine, name in ((sn.SN_ENGINE_FP32, "fp32"), (sn.SN_ENGINE_TC16, "tc16 mma.sync"),
                         (sn.SN_ENGINE_UMMA, "tcgen05")):
        y = d.clone()
        sn.sn_test_line_fft_engines(y, 256, -1, engine)
        err = per_line_rel(y[:256].cpu().numpy(), ref).max()
        ms = sn.sn_test_line_fft_engines(y, 256, -1, engine, reps=10)
        out[name] = (ms, err)
        print(f"line engine {name}: {ms * 1e3:.1f} us per launch of 65536 lines, "
              f"max rel error {err:.2e}")
        assert err <= 2e-6


def test_phase_cycles_of_the_tcgen05_engine():
    """Where the tcgen05 engine's time goes, per tile of 8 lines, on lines in
    HBM (65536) and in L2 (8192): the timed form gives the same bits as the
    untimed one, every tile is counted, and the phases add up to about the
    kernel's time (at 4 CTAs per SM the phases of one CTA overlap the other
    CTAs')."""
    for nlines in (65536, 8192):
        x = lines(nlines, seed=9)
        a = torch.from_numpy(x).cuda()
        b = a.clone()
        sn.sn_test_line_fft_engines(a, 256, -1, sn.SN_ENGINE_UMMA)
        cyc, tiles = sn.sn_test_umma_phases(b, -1)
        assert torch.equal(a, b)
        assert tiles == nlines // 8
        assert all(v > 0 for v in cyc.values()), cyc
        total = sum(cyc.values())
        print(f"{nlines} lines: tcgen05 cycles per tile " +
              ", ".join(f"{k} {v:.0f} ({v / total:.0%})" for k, v in cyc.items()))


def test_round_trip_norm_drift_of_the_engines():
    """Forward then inverse (scaled by 1/256), 100 times, on 4096 lines: the
    FP32 engine keeps the norm to rounding; both tensor-core engines correct
    the steady loss of their FP32 accumulation with Parseval (mma.sync in its
    next stage's lo split, tcgen05 by a per-line rescale of each transform's
    output) and keep it to a few 1e-6."""
    rng = np.random.default_rng(5)
    x = (rng.standard_normal((4096, 256)) + 1j * rng.standard_normal((4096, 256))).astype(np.complex64)
    n0 = np.sum(np.abs(x.astype(np.complex128)) ** 2)
    drift = {}
    for engine in (sn.SN_ENGINE_FP32, sn.SN_ENGINE_TC16, sn.SN_ENGINE_UMMA):
        d = torch.from_numpy(x.copy()).cuda()
        for _ in range(100):
            sn.sn_test_line_fft_engines(d, 256, -1, engine)
            sn.sn_test_line_fft_engines(d, 256, +1, engine)
            d.mul_(1.0 / 256)
        y = d.cpu().numpy().astype(np.complex128)
        drift[engine] = np.sum(np.abs(y) ** 2) / n0 - 1
    print("norm drift over 100 round trips: FP32 %.2e, mma.sync %.2e, tcgen05 %.2e"
          % (drift[sn.SN_ENGINE_FP32], drift[sn.SN_ENGINE_TC16], drift[sn.SN_ENGINE_UMMA]))
    assert abs(drift[sn.SN_ENGINE_FP32]) < 1e-7
    assert abs(drift[sn.SN_ENGINE_TC16]) < 1e-5
    assert abs(drift[sn.SN_ENGINE_UMMA]) < 2e-5

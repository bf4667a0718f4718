"""Schedules of the fused passes (sn_set_schedule, sn_autotune): the persistent
grid of every pass kind may be sized differently, and every choice must give
the same result bit for bit; the autotuner must leave the state alone."""
import numpy as np
import pytest

import workloads as W
from paper_1909_08354_b300 import sn

pytestmark = pytest.mark.gpu

N_SCHED = 3 * sn.SN_SCHED_KINDS  # the CTA part of a schedule


def kernel_kw(kp):
    return dict(coeff_lap=kp.coeff_lap, G=kp.G, alpha_Y=kp.alpha_Y, lambda_Y=kp.lambda_Y,
                g_local=kp.g_local)


def run(shape, schedule=None, fields=1, engine=sn.SN_ENGINE_FP32, seed=5, steps=3):
    psis, L, kp = W.random_fields(shape, seed, fields)
    g = sn.Grid(shape, L, "c64")
    try:
        if engine != sn.SN_ENGINE_FP32:
            g.set_engine(engine)
        g.set_fields(fields)
        g.set_kernel(**kernel_kw(kp))
        if schedule is not None:
            g.set_schedule(schedule)
        g.set_state(psis[0] if fields == 1 else psis)
        g.step(0.02, steps)
        return g.get_state().copy()
    finally:
        g.close()


@pytest.mark.parametrize("shape,fields,engine", [
    ((32, 64, 16), 1, sn.SN_ENGINE_FP32), ((1024, 16), 1, sn.SN_ENGINE_FP32),
    ((16, 512), 2, sn.SN_ENGINE_FP32), ((16, 256, 8), 1, sn.SN_ENGINE_TC16),
    ((64, 256, 128), 1, sn.SN_ENGINE_FP32), ((16, 128, 256), 2, sn.SN_ENGINE_FP32)])
def test_every_schedule_gives_the_same_bits(shape, fields, engine):
    ref = run(shape, None, fields, engine)
    for c in (-1, 1, 2, 3, 8, sn.SN_SCHED_MAX_CTAS):
        assert np.array_equal(run(shape, [c] * N_SCHED, fields, engine), ref), c
    mixed = [(-1, 0, 1, 2)[i % 4] for i in range(N_SCHED)]
    assert np.array_equal(run(shape, mixed, fields, engine), ref)
    # the staging of each pass kind and axis, chosen per entry
    staged = mixed + [(-1, sn.SN_STAGING_TMA, sn.SN_STAGING_REGISTERS)[i % 3] for i in range(N_SCHED)]
    assert np.array_equal(run(shape, staged, fields, engine), ref)


def test_autotune_keeps_the_state_and_the_bits(tmp_path):
    w = W.random_small((64, 64, 64), seed=12)
    psi = w.psi0().astype(np.complex64)
    g = sn.Grid(w.n, w.L, "c64")
    try:
        g.set_kernel(**kernel_kw(w.kernel))
        g.set_state(psi)
        g.step(0.02, 2)
        before = g.get_state().copy()
        step0 = g.observables()["step"]
        cache = str(tmp_path / "sched.json")
        vals = g.autotune(0.02, steps=4, cache=cache, device="test-device")
        assert len(vals) == sn.SN_SCHED_VALUES
        assert all(-1 <= v <= sn.SN_SCHED_MAX_CTAS for v in vals[:N_SCHED])
        assert all(-1 <= v <= sn.SN_STAGING_REGISTERS for v in vals[N_SCHED:])
        assert g.schedule() == vals
        assert np.array_equal(g.get_state(), before)
        assert g.observables()["step"] == step0
        g.step(0.02, 3)
        tuned = g.get_state().copy()
        # the cached schedule is reused without timing anything
        n0 = g.launch_count()
        assert g.autotune(0.02, steps=4, cache=cache, device="test-device") == vals
        assert g.launch_count() == n0
    finally:
        g.close()
    g = sn.Grid(w.n, w.L, "c64")
    try:
        g.set_kernel(**kernel_kw(w.kernel))
        g.set_state(before)
        g.step(0.02, 3)
        assert np.array_equal(g.get_state(), tuned)
    finally:
        g.close()


def test_schedule_validation():
    g = sn.Grid((16, 16), (4.0, 4.0), "c64")
    try:
        # a new grid: every pass as many CTAs as fit, with the grid's own staging
        assert g.schedule() == [0] * N_SCHED + [-1] * N_SCHED
        for bad in ([0] * (N_SCHED - 1), [-2] + [0] * (N_SCHED - 1),
                    [sn.SN_SCHED_MAX_CTAS + 1] + [0] * (N_SCHED - 1),
                    [0] * N_SCHED + [2] * N_SCHED, [0] * N_SCHED + [-2] * N_SCHED,
                    [0] * (N_SCHED + 1)):
            with pytest.raises(sn.SNError) as e:
                g.set_schedule(bad)
            assert e.value.status == sn.SN_EINVAL
        # the short form sets the CTAs and keeps the staging
        g.set_schedule([1] * N_SCHED + [sn.SN_STAGING_REGISTERS] * N_SCHED)
        g.set_schedule([2] * N_SCHED)
        assert g.schedule() == [2] * N_SCHED + [sn.SN_STAGING_REGISTERS] * N_SCHED
        for bad_dt, bad_steps in ((float("nan"), 2), (0.01, 0)):
            with pytest.raises(sn.SNError) as e:
                sn._check(g.h, sn.lib().sn_autotune(g.h, bad_dt, bad_steps))
            assert e.value.status == sn.SN_EINVAL
    finally:
        g.close()
    g = sn.Grid((16, 16), (4.0, 4.0), "c128")
    try:
        with pytest.raises(sn.SNError) as e:
            g.autotune(0.01, steps=2)
        assert e.value.status == sn.SN_ENOTSUP
    finally:
        g.close()

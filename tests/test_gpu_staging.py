"""Tile staging of the fused passes (sn_set_staging).

The TMA-staged kernels (tiles moved by bulk tensor copies into shared-memory
slots) run the same arithmetic as the register-staged ones, so every step
must agree bit for bit, on every geometry they take: 128- and 256-point lines
along every axis, strided tiles narrower than 16 lines (the copy fills the
missing lines with zeros and the store leaves them out), several fields, and
every schedule.  The default staging must also meet the oracle at full size.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_1909_08354_b300 import sn

pytestmark = pytest.mark.gpu


def kernel_kw(kp):
    return dict(coeff_lap=kp.coeff_lap, G=kp.G, alpha_Y=kp.alpha_Y, lambda_Y=kp.lambda_Y,
                g_local=kp.g_local)


def run(shape, staging, fields=1, seed=7, steps=3, schedule=None, dt=0.02):
    psis, L, kp = W.random_fields(shape, seed, fields)
    g = sn.Grid(shape, L, "c64")
    try:
        g.set_staging(staging)
        g.set_fields(fields)
        g.set_kernel(**kernel_kw(kp))
        if schedule is not None:
            g.set_schedule(schedule)
        g.set_state(psis[0] if fields == 1 else psis)
        g.step(dt, steps)
        g.step(dt, 2)  # the open merge continues across calls
        return g.get_state().copy()
    finally:
        g.close()


SHAPES = [(256, 256, 256), (128, 128, 128), (8, 128, 256), (256, 8, 128), (128, 256, 16),
          (16, 256, 8), (256, 128), (128, 8), (8, 256), (256, 64), (32, 128, 64), (1024, 256)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_tma_and_register_staging_give_the_same_bits(shape):
    tma = run(shape, sn.SN_STAGING_TMA)
    reg = run(shape, sn.SN_STAGING_REGISTERS)
    assert np.array_equal(tma, reg)


def test_staging_with_fields_and_schedules():
    shape = (64, 128, 256)
    ref = run(shape, sn.SN_STAGING_REGISTERS, fields=2)
    assert np.array_equal(run(shape, sn.SN_STAGING_TMA, fields=2), ref)
    for c in (-1, 1, 3):
        sched = [c] * (3 * sn.SN_SCHED_KINDS)
        assert np.array_equal(run(shape, sn.SN_STAGING_TMA, fields=2, schedule=sched), ref), c


def test_staging_rejects_unknown_modes():
    g = sn.Grid((16, 16), (1.0, 1.0), "c64")
    try:
        with pytest.raises(sn.SNError) as e:
            g.set_staging(7)
        assert e.value.status == sn.SN_EINVAL
    finally:
        g.close()


def test_tma_staging_matches_the_oracle_on_the_256_cubed_workload():
    w = W.nbody_3d()
    psi = w.psi0().astype(np.complex64)
    kw = kernel_kw(w.kernel)
    g = sn.Grid(w.n, w.L, "c64")
    try:
        g.set_staging(sn.SN_STAGING_TMA)
        g.set_kernel(**kw)
        g.set_state(psi)
        g.step(w.dt, 1)
        out = g.get_state()
    finally:
        g.close()
    ref = O.evolve(psi.astype(np.complex128), w.dt, 1, w.L, **O.kernel_kwargs(w.kernel))
    assert O.rel_l2(out, ref) <= 1e-6

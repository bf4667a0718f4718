"""Slab blocking of the 3D FP32 step (sn_set_blocking).

The y and x passes of each round run slab by slab over z, the same kernels on
sub-views of the state and of the half spectrum, so every sequence of calls
must give the unblocked bits: slabs that divide n_z and a ragged last slab,
both round parities (open merges left open across calls, reads that close on
a copy), V_ext (read per slab), and grids the blocking does not apply to.
"""
import numpy as np
import pytest

import workloads as W
from paper_1909_08354_b300 import sn

pytestmark = pytest.mark.gpu


def kernel_kw(kp, **over):
    kw = dict(coeff_lap=kp.coeff_lap, G=kp.G, alpha_Y=kp.alpha_Y, lambda_Y=kp.lambda_Y,
              g_local=kp.g_local)
    kw.update(over)
    return kw


def run(shape, planes, calls=(3, "read", 2), seed=11, fields=1, vext=False,
        staging=sn.SN_STAGING_TMA, dt=0.02):
    psis, L, kp = W.random_fields(shape, seed, fields)
    extra = {}
    if vext:
        rng = np.random.default_rng(seed + 1)
        extra["v_ext"] = rng.standard_normal(shape) * 0.3
    g = sn.Grid(shape, L, "c64")
    reads = []
    try:
        g.set_staging(staging)
        g.set_blocking(planes)
        g.set_fields(fields)
        g.set_kernel(**kernel_kw(kp, **extra))
        g.set_state(psis[0] if fields == 1 else psis)
        for c in calls:
            if c == "read":
                reads.append(g.get_state().copy())
            else:
                g.step(dt, c)
        reads.append(g.get_state().copy())
        reads.append(g.observables())
        return reads, g.launch_count()
    finally:
        g.close()


def same(a, b):
    assert len(a) == len(b)
    for x, y in zip(a[:-1], b[:-1]):
        assert np.array_equal(x, y)
    assert a[-1] == b[-1]


@pytest.mark.parametrize("shape,planes", [((64, 256, 256), 16), ((64, 256, 256), 32),
                                          ((32, 128, 256), 5), ((64, 256, 128), 24),
                                          ((16, 128, 128), 1), ((256, 256, 256), 64)],
                         ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else str(v))
def test_blocked_rounds_give_the_unblocked_bits(shape, planes):
    res, nb = run(shape, planes)
    ref, n0 = run(shape, 0)
    same(res, ref)
    # two launches per slab replace the pair's two launches in every round
    # (5 rounds of steps, 2 closing reads)
    slabs = -(-shape[0] // planes)
    assert nb - n0 == (5 + 2) * 2 * (slabs - 1)


def test_blocking_with_v_ext_and_every_call_pattern():
    shape = (32, 128, 128)
    for calls in ((1,), (2,), (1, "read", 1, "read", 3), (4, "read", 4)):
        res, _ = run(shape, 5, calls, vext=True)
        ref, _ = run(shape, 0, calls, vext=True)
        same(res, ref)


@pytest.mark.parametrize("shape,fields,staging", [((32, 128, 128), 2, sn.SN_STAGING_TMA),
                                                  ((32, 128, 128), 1, sn.SN_STAGING_REGISTERS),
                                                  ((32, 64, 64), 1, sn.SN_STAGING_TMA),
                                                  ((256, 256), 1, sn.SN_STAGING_TMA)])
def test_grids_the_blocking_does_not_take(shape, fields, staging):
    res, nb = run(shape, 4, fields=fields, staging=staging)
    ref, n0 = run(shape, 0, fields=fields, staging=staging)
    same(res, ref)
    assert nb == n0


def test_blocking_rejects_negative_planes():
    g = sn.Grid((16, 16, 16), (1.0,) * 3, "c64")
    try:
        with pytest.raises(sn.SNError) as e:
            g.set_blocking(-1)
        assert e.value.status == sn.SN_EINVAL
    finally:
        g.close()

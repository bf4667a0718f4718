"""Plane-resident 2D steps (SN_STAGING_RESIDENT).

On a square 64^2 or 128^2 grid the resident kernel runs every merged step of
an sn_step call in one CTA's shared memory.  It is the tiled path's round, in
the same arithmetic and order, so each sequence of calls -- open merges left
open across calls, reads that close on a copy, a change of step that settles
the merge, a parameter change that closes it in place -- must give the tiled
path's bits, and grids the kernel does not take must run the tiled path.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_1909_08354_b300 import sn

pytestmark = pytest.mark.gpu


def kernel_kw(kp, **over):
    kw = dict(coeff_lap=kp.coeff_lap, G=kp.G, alpha_Y=kp.alpha_Y, lambda_Y=kp.lambda_Y,
              g_local=kp.g_local)
    kw.update(over)
    return kw


def run(shape, staging, calls, seed=3, fields=1, dt=0.02):
    """Apply `calls` (ints: steps of one sn_step; 'read': get_state; ('dt', h):
    a new step; ('kernel', dict): new kernel parameters); return every read."""
    psis, L, kp = W.random_fields(shape, seed, fields)
    g = sn.Grid(shape, L, "c64")
    reads = []
    try:
        g.set_staging(staging)
        g.set_fields(fields)
        g.set_kernel(**kernel_kw(kp))
        g.set_state(psis[0] if fields == 1 else psis)
        for c in calls:
            if c == "read":
                reads.append(g.get_state().copy())
            elif isinstance(c, tuple) and c[0] == "dt":
                dt = c[1]
            elif isinstance(c, tuple) and c[0] == "kernel":
                g.set_kernel(**kernel_kw(kp, **c[1]))
            else:
                g.step(dt, c)
        reads.append(g.get_state().copy())
        reads.append(g.observables())
        return reads, g.launch_count()
    finally:
        g.close()


SEQS = [[1], [2], [5], [3, 2], [1, "read", 1, "read", 4], [4, ("dt", 0.013), 3],
        [2, ("kernel", dict(g_local=0.7)), 3, "read", 1],
        [3, ("kernel", dict(alpha_Y=0.4, lambda_Y=0.8)), 2]]


@pytest.mark.parametrize("n", [64, 128])
@pytest.mark.parametrize("seq", SEQS, ids=lambda s: "-".join(map(str, s)))
def test_resident_gives_the_tiled_bits(n, seq):
    res, _ = run((n, n), sn.SN_STAGING_RESIDENT, seq)
    ref, _ = run((n, n), sn.SN_STAGING_TMA, seq)
    assert len(res) == len(ref)
    for a, b in zip(res[:-1], ref[:-1]):
        assert np.array_equal(a, b)
    assert res[-1] == ref[-1]


@pytest.mark.parametrize("n", [64, 128])
def test_one_launch_per_call(n):
    _, launches = run((n, n), sn.SN_STAGING_RESIDENT, [7, 1, 12])
    _, tiled = run((n, n), sn.SN_STAGING_TMA, [7, 1, 12])
    # three resident launches against three passes per step; the closing read
    # and the observables are the same launches on both
    assert tiled - launches == 3 * 20 - 3


@pytest.mark.parametrize("shape,fields", [((256, 256), 1), ((64, 128), 1), ((128, 64), 1),
                                          ((32, 32), 1), ((64, 64), 2), ((64, 64, 64), 1)])
def test_other_grids_take_the_tiled_path(shape, fields):
    res, _ = run(shape, sn.SN_STAGING_RESIDENT, [3, 2], fields=fields)
    ref, _ = run(shape, sn.SN_STAGING_TMA, [3, 2], fields=fields)
    for a, b in zip(res[:-1], ref[:-1]):
        assert np.array_equal(a, b)


def test_resident_meets_the_oracle():
    w = W.random_small((128, 128), seed=21)
    psi = w.psi0().astype(np.complex64)
    g = sn.Grid(w.n, w.L, "c64")
    try:
        g.set_staging(sn.SN_STAGING_RESIDENT)
        g.set_kernel(**kernel_kw(w.kernel))
        g.set_state(psi)
        g.step(0.02, 4)
        out = g.get_state()
    finally:
        g.close()
    ref = O.evolve(psi.astype(np.complex128), 0.02, 4, w.L, **O.kernel_kwargs(w.kernel))
    assert O.rel_l2(out, ref) <= 5e-6

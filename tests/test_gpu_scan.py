"""Batched scan of independent 2D instances of uneven size.

Each instance of the batch must give what the oracle gives for it alone
(per-step bar 1e-6 rel-L2 in complex64, k merged steps held to k times it),
and what the single-grid path gives: on the persistent schedule (one
cooperative launch) within the per-step bar, on the graph schedule (the
single-grid pass kernels, an instance per graph branch) bit for bit.  The
bounded dependency waits are exercised by a zero wait limit: the launch must
end with SN_ETIMEOUT and leave the GPU usable.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_1909_08354_b300 import sn

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-6


def kw_of(kp):
    return dict(coeff_lap=kp.coeff_lap, G=kp.G, alpha_Y=kp.alpha_Y, lambda_Y=kp.lambda_Y,
                g_local=kp.g_local)


def grid_run(psi, L, kw, dt, nsteps):
    g = sn.Grid(psi.shape, L, "c64")
    g.set_kernel(**kw)
    g.set_state(psi)
    g.step(dt, nsteps)
    out = g.get_state()
    g.close()
    return out


@pytest.mark.parametrize("schedule", [sn.SN_BATCH_PERSISTENT, sn.SN_BATCH_CLASSES, sn.SN_BATCH_GRAPH])
def test_uneven_batch_matches_oracle_per_instance(schedule):
    sizes = [8, 16, 32, 64, 128, 256, 512, 64, 8, 128]
    ws = [W.random_small((n, n), seed=100 + i, L=12.0) for i, n in enumerate(sizes)]
    b = sn.Batch(sizes, [w.L[0] for w in ws])
    b.set_schedule(schedule)
    assert b.schedule() == schedule
    b.set_kernels([kw_of(w.kernel) for w in ws])
    psis = [w.psi0().astype(np.complex64) for w in ws]
    for i, p in enumerate(psis):
        b.set_state(i, p)
    dts = [0.01 + 0.002 * i for i in range(len(sizes))]
    b.step(dts, 3)
    b.sync()
    for i, w in enumerate(ws):
        ref = O.evolve(psis[i].astype(np.complex128), dts[i], 3, w.L, **kw_of(w.kernel))
        assert O.rel_l2(b.get_state(i), ref) <= 3 * STEP_TOL, (i, sizes[i])
    # persistent: one launch; per class: one for each of the 7 sizes; graph:
    # three passes per instance and round, two in the closing round
    want = {sn.SN_BATCH_PERSISTENT: 1, sn.SN_BATCH_CLASSES: 7, sn.SN_BATCH_GRAPH: 3 * 3 * 10 + 2 * 10}
    assert b.launch_count() == want[schedule]
    b.close()


def test_graph_schedule_gives_the_single_grid_bits():
    """The graph schedule runs each instance's round as the single-grid pass
    kernels: the same bits as sn_step on a grid of the instance, over calls of
    different lengths, with per-instance dt and kernels (Newton + Yukawa, local
    term, the optical kernel), a dt change (recapture) and a schedule switch."""
    sizes = [1024, 8, 512, 128, 256, 64, 1024, 16, 32, 128]
    ws = [W.random_small((n, n), seed=600 + i, L=14.0 + i) for i, n in enumerate(sizes)]
    kws = [kw_of(w.kernel) for w in ws]
    kws[3] = dict(kws[3], alpha_Y=0.5, lambda_Y=2.0)
    kws[4] = dict(kws[4], g_local=0.3)
    kws[5] = dict(kind=sn.SN_KERNEL_POISSON, coeff_lap=-0.5, B=1.0, C=-0.04, D=-2.0)
    psis = [w.psi0().astype(np.complex64) for w in ws]
    dts = [0.01 + 0.001 * i for i in range(len(sizes))]
    b = sn.Batch(sizes, [w.L[0] for w in ws])
    try:
        b.set_schedule(sn.SN_BATCH_GRAPH)
        b.set_kernels(kws)
        for i, p in enumerate(psis):
            b.set_state(i, p)
        b.step(dts, 3)
        b.step(dts, 1)
        b.step([2 * x for x in dts], 2)
        b.sync()
        got = [b.get_state(i).copy() for i in range(len(sizes))]
        for i, w in enumerate(ws):
            ref = grid_run(psis[i], w.L, kws[i], dts[i], 3)
            ref = grid_run(ref, w.L, kws[i], dts[i], 1)
            ref = grid_run(ref, w.L, kws[i], 2 * dts[i], 2)
            assert np.array_equal(got[i], ref), (i, sizes[i])
        # switching to the persistent schedule continues from the same states
        b.set_schedule(sn.SN_BATCH_PERSISTENT)
        b.step(dts, 2)
        b.sync()
        for i, w in enumerate(ws):
            ref = grid_run(got[i], w.L, kws[i], dts[i], 2)
            assert O.rel_l2(b.get_state(i), ref) <= 2 * STEP_TOL, (i, sizes[i])
        for bad in (-1, 3):
            with pytest.raises(sn.SNError) as e:
                b.set_schedule(bad)
            assert e.value.status == sn.SN_EINVAL
    finally:
        b.close()


def test_batch_graph_replay_and_largest_size():
    sizes = [1024, 128, 256]
    ws = [W.random_small((n, n), seed=200 + i, L=20.0) for i, n in enumerate(sizes)]
    b = sn.Batch(sizes, [w.L[0] for w in ws])
    b.set_kernels([kw_of(w.kernel) for w in ws])
    psis = [w.psi0().astype(np.complex64) for w in ws]
    for i, p in enumerate(psis):
        b.set_state(i, p)
    b.step(0.01, 2)
    b.step(0.01, 2)  # replays the captured launch
    for i, w in enumerate(ws):
        ref = grid_run(psis[i], w.L, kw_of(w.kernel), 0.01, 2)
        ref = grid_run(ref, w.L, kw_of(w.kernel), 0.01, 2)
        assert O.rel_l2(b.get_state(i), ref) <= 4 * STEP_TOL, sizes[i]
    o = b.observables(1)
    assert abs(o["mass"] / O.observables(psis[1].astype(np.complex128), ws[1].L)["mass"] - 1) < 1e-5
    b.close()


def test_expired_wait_reports_timeout_and_gpu_stays_usable():
    sizes = [256] * 8 + [64] * 8
    ws = [W.random_small((n, n), seed=300 + i, L=12.0) for i, n in enumerate(sizes)]
    b = sn.Batch(sizes, [w.L[0] for w in ws])
    b.set_kernels([kw_of(w.kernel) for w in ws])
    for i, w in enumerate(ws):
        b.set_state(i, w.psi0().astype(np.complex64))
    b.set_wait_limit(0)
    b.step(0.01, 20)
    with pytest.raises(sn.SNError) as e:
        b.sync()
    assert e.value.status == sn.SN_ETIMEOUT
    # a normal launch afterwards works and matches the single-grid path
    b.set_wait_limit(4_000_000_000)
    psi0 = ws[0].psi0().astype(np.complex64)
    b.set_state(0, psi0)
    b.step(0.01, 2)
    ref = grid_run(psi0, ws[0].L, kw_of(ws[0].kernel), 0.01, 2)
    assert O.rel_l2(b.get_state(0), ref) <= 2 * STEP_TOL
    b.close()


def test_one_instance_on_every_schedule():
    """The degenerate batch: one instance (one size class, one graph branch),
    each schedule against the single-grid path."""
    w = W.random_small((64, 64), seed=700, L=12.0)
    psi = w.psi0().astype(np.complex64)
    ref = grid_run(psi, w.L, kw_of(w.kernel), 0.01, 5)
    for sched in (sn.SN_BATCH_PERSISTENT, sn.SN_BATCH_CLASSES, sn.SN_BATCH_GRAPH):
        b = sn.Batch([64], [w.L[0]])
        try:
            b.set_schedule(sched)
            b.set_kernels([kw_of(w.kernel)])
            b.set_state(0, psi)
            b.step(0.01, 5)
            b.sync()
            out = b.get_state(0)
        finally:
            b.close()
        if sched == sn.SN_BATCH_GRAPH:
            assert np.array_equal(out, ref)
        else:
            assert O.rel_l2(out, ref) <= 5 * STEP_TOL, sched


def test_parameter_scan_96_instances_on_the_graph_schedule():
    """The 96-instance scan workload on the graph schedule: 20 steps of every
    instance give sn_step's bits, and the mass of every instance is kept."""
    ws = [W.scan_instance_2d(i) for i in range(96)]
    psis = [w.psi0().astype(np.complex64) for w in ws]
    b = sn.Batch([w.n[0] for w in ws], [w.L[0] for w in ws])
    try:
        b.set_schedule(sn.SN_BATCH_GRAPH)
        b.set_kernels([kw_of(w.kernel) for w in ws])
        for i, p in enumerate(psis):
            b.set_state(i, p)
        b.step(ws[0].dt, 20)
        b.sync()
        for i in range(0, 96, 7):
            w = ws[i]
            ref = grid_run(psis[i], w.L, kw_of(w.kernel), w.dt, 20)
            assert np.array_equal(b.get_state(i), ref), (i, w.n)
        for i, p in enumerate(psis):
            m0 = float(np.sum(np.abs(p.astype(np.complex128)) ** 2))
            m = float(np.sum(np.abs(b.get_state(i).astype(np.complex128)) ** 2))
            assert abs(m / m0 - 1) <= 1e-5, i
    finally:
        b.close()


def test_parameter_scan_96_instances_500_steps():
    """The 96-instance scan workload (sizes 128^2..1024^2, L=40, h=1e-2, 500 steps).

    One step of every instance matches the single-grid path; over 500 steps the
    mass of every instance is conserved to 1e-5, and the FP32 trajectory of a
    128^2 instance is as close to the FP64 oracle's as the single-grid FP32
    trajectory is (the two FP32 paths round differently, and a collapsing
    instance amplifies rounding over 500 steps)."""
    ws = [W.scan_instance_2d(i) for i in range(96)]
    psis = [w.psi0().astype(np.complex64) for w in ws]
    b = sn.Batch([w.n[0] for w in ws], [w.L[0] for w in ws])
    b.set_kernels([kw_of(w.kernel) for w in ws])
    for i, p in enumerate(psis):
        b.set_state(i, p)
    b.step(ws[0].dt, 1)
    for i, w in enumerate(ws):
        ref = grid_run(psis[i], w.L, kw_of(w.kernel), w.dt, 1)
        assert O.rel_l2(b.get_state(i), ref) <= 2 * STEP_TOL, (i, w.n)
    for i, p in enumerate(psis):
        b.set_state(i, p)
    m0 = [float(np.sum(np.abs(p.astype(np.complex128)) ** 2)) for p in psis]
    b.step(ws[0].dt, ws[0].nsteps)
    b.sync()
    for i in range(96):
        out = b.get_state(i)
        assert abs(float(np.sum(np.abs(out.astype(np.complex128)) ** 2)) / m0[i] - 1) <= 1e-5, i
    i = next(k for k, w in enumerate(ws) if w.n[0] == 128)
    w = ws[i]
    exact = O.evolve(psis[i].astype(np.complex128), w.dt, w.nsteps, w.L, **kw_of(w.kernel))
    grid = grid_run(psis[i], w.L, kw_of(w.kernel), w.dt, w.nsteps)
    e_grid = O.rel_l2(grid, exact)
    e_batch = O.rel_l2(b.get_state(i), exact)
    assert e_batch <= 2 * e_grid + 1e-5, (e_batch, e_grid)
    b.close()


def test_every_register_budget_gives_the_same_bits():
    """sn_set_batch_ctas changes the CTAs of the cooperative launch and the
    registers of its threads, and SN_BATCH_CLASSES splits the launch by size
    class; neither changes the arithmetic: the same bits for 1, 2 and 3 CTAs
    per SM in one launch or one per class, on every line length the scan
    takes."""
    sizes = [1024, 512, 256, 128, 64, 32, 16, 8, 256, 1024]
    ws = [W.random_small((n, n), seed=400 + i, L=16.0) for i, n in enumerate(sizes)]
    psis = [w.psi0().astype(np.complex64) for w in ws]
    outs = {}
    for sched in (sn.SN_BATCH_PERSISTENT, sn.SN_BATCH_CLASSES):
        for cps in (3, 2, 1):
            b = sn.Batch(sizes, [w.L[0] for w in ws])
            b.set_kernels([kw_of(w.kernel) for w in ws])
            b.set_schedule(sched)
            b.set_ctas(cps)
            for i, p in enumerate(psis):
                b.set_state(i, p)
            b.step(0.01, 3)
            b.sync()
            outs[sched, cps] = [b.get_state(i).copy() for i in range(len(sizes))]
            b.close()
    ref = outs[sn.SN_BATCH_PERSISTENT, 3]
    for key, out in outs.items():
        for i in range(len(sizes)):
            assert np.array_equal(out[i], ref[i]), (key, sizes[i])
    b = sn.Batch([8], [4.0])
    try:
        for bad in (0, 4):
            with pytest.raises(sn.SNError) as e:
                b.set_ctas(bad)
            assert e.value.status == sn.SN_EINVAL
    finally:
        b.close()


def test_batch_autotune_keeps_the_states():
    sizes = [256, 128, 128, 64, 512]
    ws = [W.random_small((n, n), seed=500 + i, L=16.0) for i, n in enumerate(sizes)]
    psis = [w.psi0().astype(np.complex64) for w in ws]
    b = sn.Batch(sizes, [w.L[0] for w in ws])
    try:
        b.set_kernels([kw_of(w.kernel) for w in ws])
        for i, p in enumerate(psis):
            b.set_state(i, p)
        chosen = b.autotune(0.01, steps=5)
        assert chosen in (1, 2, 3)
        schedule = b.schedule()
        assert schedule in (sn.SN_BATCH_PERSISTENT, sn.SN_BATCH_CLASSES, sn.SN_BATCH_GRAPH)
        for i, p in enumerate(psis):
            assert np.array_equal(b.get_state(i), p), i
        b.step(0.01, 3)
        b.sync()
        tuned = [b.get_state(i).copy() for i in range(len(sizes))]
    finally:
        b.close()
    b = sn.Batch(sizes, [w.L[0] for w in ws])
    try:
        b.set_schedule(schedule)
        b.set_ctas(chosen)
        b.set_kernels([kw_of(w.kernel) for w in ws])
        for i, p in enumerate(psis):
            b.set_state(i, p)
        b.step(0.01, 3)
        b.sync()
        for i in range(len(sizes)):
            assert np.array_equal(b.get_state(i), tuned[i]), sizes[i]
        with pytest.raises(sn.SNError) as e:
            b.autotune(0.01, steps=0)
        assert e.value.status == sn.SN_EINVAL
    finally:
        b.close()

"""sn_step_2d_noalloc: the fused 2D complex64 step without device allocation.

Callers that cannot call cudaMalloc (their device memory belongs to another
allocator, or an allocation's latency or failure is not acceptable where they
run) use this entry point; its working memory is a fixed static device array.
Here its output is checked against the regular grid API (sn_create_grid /
sn_step) on two calls in a row with different grid shapes, so a call that
depended on what the previous call left in the shared array would fail.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads as W
from paper_1909_08354_b300 import sn

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-6  # per-step rel-L2 bar of the complex64 path


def kernel_kw(kp):
    return dict(coeff_lap=kp.coeff_lap, G=kp.G, alpha_Y=kp.alpha_Y, lambda_Y=kp.lambda_Y,
                g_local=kp.g_local)


def grid_api(psi, L, kw, dt, nsteps):
    g = sn.Grid(psi.shape, L, "c64")
    try:
        g.set_kernel(**kw)
        g.set_state(psi)
        g.step(dt, nsteps)
        return g.get_state()
    finally:
        g.close()


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_noalloc_matches_grid_api_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    # the largest grid (its half spectrum fills the array's region for it), a
    # grid with a 16-point axis (no twiddle table is uploaded for it), and two
    # uneven shapes
    cases = [((256, 128), 31, 0.02, 4), ((64, 512), 32, 0.03, 3), ((512, 512), 33, 0.02, 2),
             ((16, 32), 34, 0.02, 3)]
    prepared = []
    for shape, seed, dt, nsteps in cases:
        w = W.random_small(shape, seed=seed)
        psi = w.psi0().astype(np.complex64)
        kw = kernel_kw(w.kernel)
        prepared.append((psi, w.L, kw, dt, nsteps, grid_api(psi, w.L, kw, dt, nsteps)))

    stream = torch.cuda.Stream()
    # one call per shape first, so that code loading and the one-time set-up are done
    for psi, L, kw, dt, nsteps, _ in prepared:
        warm = torch.from_numpy(psi).cuda()
        torch.cuda.synchronize()
        sn.sn_step_2d_noalloc(warm, L, dt, 1, stream=stream.cuda_stream, **kw)
    torch.cuda.synchronize()
    devs = [torch.from_numpy(p[0]).cuda() for p in prepared]
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]

    for dev, (psi, L, kw, dt, nsteps, ref) in zip(devs, prepared):
        sn.sn_step_2d_noalloc(dev, L, dt, nsteps, stream=stream.cuda_stream, **kw)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before

    for dev, (psi, L, kw, dt, nsteps, ref) in zip(devs, prepared):
        out = dev.cpu().numpy()
        assert rel_l2(out, ref) <= nsteps * STEP_TOL


def test_noalloc_rejects_oversized_grids():
    torch = pytest.importorskip("torch")
    big = torch.zeros((8, 1024), dtype=torch.complex64, device="cuda")
    with pytest.raises(sn.SNError) as e:
        sn.sn_step_2d_noalloc(big, (1.0, 1.0), 0.01, 1)
    assert e.value.status == sn.SN_ENOTSUP
    assert "SN_NOALLOC_MAX_N" in sn.sn_last_error(None)

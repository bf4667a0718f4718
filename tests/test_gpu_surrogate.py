"""Surrogate workflow at a reduced size (64^2 grids, a small network, seconds of training).

The network is trained on the GPU by the library's own forward, backward and
Adam kernels on pairs produced by the batched solver.  Over 50 steps of these
self-gravitating instances the phase turns by tens of radians (the potential
reaches about -100), so the plain map psi(t) -> psi(t + 50 dt) is hard to
learn; the surrogate is trained in its corrector form, on a coarse solve of
the same horizon (10 split steps of 5 dt).  The test shows what the trained
network gains over the method without it: on held-out instances its
prediction must be closer to the fine solver than the coarse solve alone (and
than the zero guess), and a rollout must run faster than the plain FP64 GPU
step over the same horizon.  The fallback is exercised by perturbing every
prediction's mass: each instance must then take the solver path and end
exactly where the solver alone does.
"""
import numpy as np
import pytest

from paper_1909_08354_b300 import sn, surrogate as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import oracle.fno_oracle as F  # noqa: E402

COARSE = 10


def small_net(batch, stream, c_in):
    sh = F.FnoShape(s=64, c_in=c_in, width=16, modes=8, layers=4, proj=32)
    net = sn.Fno(s=64, c_in=c_in, width=16, modes=8, layers=4, proj=32, batch_max=batch,
                 stream=stream.cuda_stream)
    net.set_params(F.flatten(sh, F.init_params(sh, 0)).astype(np.float32))
    return net


def test_trained_corrector_beats_the_coarse_solve_and_falls_back():
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    try:
        train_ws = S.instances(96, 5000, s=64)
        test_ws = S.instances(16, 9000, s=64)
        X, Y = S.generate_pairs(torch, train_ws, stride=50, nsnap=10, seed=1, coarse=COARSE)
        Xt, Yt = S.generate_pairs(torch, test_ws, stride=50, nsnap=2, seed=2, coarse=COARSE)
        net = small_net(16, stream, S.input_channels(COARSE))
        losses = S.train(net, X, Y, iters=600, batch=16, lr=2e-3)
        assert np.mean(losses[-50:]) < 0.8 * np.mean(losses[:10])
        e_net, e_coarse = S.one_step_errors(torch, net, Xt, Yt, 16)
        print(f"held-out one-call rel-L2: network {e_net:.3f}, coarse solve alone {e_coarse:.3f}")
        assert e_net < e_coarse < 1.0, (e_net, e_coarse)
        # forced fallback: scale every prediction by 1.01 (mass drift 2% > 1e-3)
        res = S.rollout(torch, net, test_ws[:8], rounds=3, stride=50, drift_tol=1e-3,
                        perturb=lambda r, p: p.mul_(1.01), coarse=COARSE)
        assert res["fallback_fraction"] == 1.0
        assert res["final_rel_l2_max"] <= 3e-6
        res = S.rollout(torch, net, test_ws[:8], rounds=3, stride=50, drift_tol=1e-3,
                        coarse=COARSE)
        assert 0.0 <= res["fallback_fraction"] <= 1.0
        t64 = S.plain_fp64_time(torch, test_ws[:8], 3 * 50, sample=2)
        print(f"rollout {res['t_surrogate_s']:.3f} s, plain FP64 GPU {t64:.3f} s, fallback "
              f"fraction {res['fallback_fraction']:.2f}")
        assert res["t_surrogate_s"] < t64
        net.close()
    finally:
        torch.cuda.set_stream(torch.cuda.default_stream())

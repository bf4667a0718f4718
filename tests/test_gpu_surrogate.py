"""Surrogate workflow at a reduced size (64^2 grids, a small network, seconds of training).

The network is trained on the GPU by the library's own forward, backward and
Adam kernels on pairs produced by the batched solver, and it must beat the
persistence guess psi(t + 50 dt) ~ psi(t) on held-out instances.  Over 50
steps of these self-gravitating instances the phase turns by tens of radians
(the potential reaches about -100), so persistence sits near relative error
1.4 and the learning bar is a drop of the training loss, not a small error.  The fallback
is exercised by perturbing every prediction's mass: each instance must then
take the solver path and end exactly where the solver alone does.
"""
import numpy as np
import pytest

from paper_1909_08354_b300 import sn, surrogate as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import oracle.fno_oracle as F  # noqa: E402


def small_net(batch, stream):
    sh = F.FnoShape(s=64, c_in=5, width=16, modes=8, layers=4, proj=32)
    net = sn.Fno(s=64, c_in=5, width=16, modes=8, layers=4, proj=32, batch_max=batch,
                 stream=stream.cuda_stream)
    net.set_params(F.flatten(sh, F.init_params(sh, 0)).astype(np.float32))
    return net


def test_trained_surrogate_beats_persistence_and_falls_back():
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    train_ws = S.instances(96, 5000, s=64)
    test_ws = S.instances(16, 9000, s=64)
    X, Y = S.generate_pairs(torch, train_ws, stride=50, nsnap=10, seed=1)
    Xt, Yt = S.generate_pairs(torch, test_ws, stride=50, nsnap=2, seed=2)
    net = small_net(16, stream)
    losses = S.train(net, X, Y, iters=600, batch=16, lr=2e-3)
    assert np.mean(losses[-50:]) < 0.8 * np.mean(losses[:10])
    e_net, e_id = S.one_step_errors(torch, net, Xt, Yt, 16)
    assert e_net < e_id, (e_net, e_id)
    # forced fallback: scale every prediction by 1.01 (mass drift 2% > 1e-3)
    res = S.rollout(torch, net, test_ws[:8], rounds=3, stride=50, drift_tol=1e-3,
                    perturb=lambda r, p: p.mul_(1.01))
    assert res["fallback_fraction"] == 1.0
    assert res["final_rel_l2_max"] <= 3e-6
    res = S.rollout(torch, net, test_ws[:8], rounds=3, stride=50, drift_tol=1e-3)
    assert 0.0 <= res["fallback_fraction"] <= 1.0
    net.close()
    torch.cuda.set_stream(torch.cuda.default_stream())

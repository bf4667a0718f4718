"""FNO surrogate workflow on the library's kernels.

* Training pairs: each seeded 2D instance (the scan-instance generator at one
  grid size) is advanced by the batched split-step solver; (psi(t), kernel
  parameters) -> psi(t + stride dt) pairs are cut every `stride` steps.
* Training: contiguous minibatches of a pre-shuffled pair set through
  sn_fno_forward / sn_fno_loss / sn_fno_backward / sn_fno_adam.
* Rollout: psi is advanced `stride` steps per network call; a prediction
  whose mass differs from its input's by more than `drift_tol` is replaced by
  `stride` solver steps (the solver is both the fallback and the reference).
* Corrector form (coarse > 0): the network also sees a coarse solve of the
  same horizon (`coarse` split steps of stride dt / coarse, from psi(t)) and
  its head turns that coarse state instead of psi(t): it learns what the
  coarse solve misses.  Input channels (re, im of the coarse state, re, im of
  psi(t), features); the coarse solve without the network is the method it
  is measured against.

Device memory comes from torch tensors; every computation is a library call.
Every call is queued on torch's current CUDA stream, which must be a
non-default stream; create the network on that same stream, e.g.

    stream = torch.cuda.Stream(); torch.cuda.set_stream(stream)
    net = sn.Fno(..., stream=stream.cuda_stream)
"""
from __future__ import annotations

import time
from typing import Dict, List, Sequence

import numpy as np

import workloads as W

from . import sn

# network input channels: (re psi, im psi, alpha_Y, lambda_Y / 20, g / 0.05)
FEATURE_SCALE = np.array([1.0, 1.0 / 20.0, 1.0 / 0.05])


def instances(n: int, seed0: int, s: int = 256) -> List[W.Workload]:
    return [W.scan_instance_2d(i, sizes=(s,), seed=seed0 + i) for i in range(n)]


def kernel_kw(kp) -> Dict[str, float]:
    return dict(coeff_lap=kp.coeff_lap, G=kp.G, alpha_Y=kp.alpha_Y, lambda_Y=kp.lambda_Y,
                g_local=kp.g_local)


def features(ws: Sequence[W.Workload]) -> np.ndarray:
    f = np.array([[w.kernel.alpha_Y, w.kernel.lambda_Y, w.kernel.g_local] for w in ws])
    return (f * FEATURE_SCALE).astype(np.float32)


def _stream(torch):
    h = torch.cuda.current_stream().cuda_stream
    if not h:
        raise RuntimeError("set a non-default current CUDA stream before the surrogate calls")
    return h


def _batch(torch, ws, stream):
    b = sn.Batch([w.n[0] for w in ws], [w.L[0] for w in ws], stream=stream)
    b.set_kernels([kernel_kw(w.kernel) for w in ws])
    for i, w in enumerate(ws):
        b.set_state(i, w.psi0(np.complex64))
    return b


def input_channels(coarse: int) -> int:
    """Network input channels: (re, im) of psi and 3 features, plus the (re, im)
    of the coarse solve in the corrector form."""
    return 7 if coarse > 0 else 5


def coarse_solve(torch, bc, psi, dt, coarse, out):
    """out[i] = `coarse` split steps of dt from psi[i], on the batch bc (one
    instance per state)."""
    for i in range(psi.shape[0]):
        bc.set_state(i, psi[i])
    bc.step(dt, coarse)
    for i in range(psi.shape[0]):
        bc.get_state(i, out[i])


def generate_pairs(torch, ws, stride=50, nsnap=10, chunk=512, seed=0, coarse=0):
    """X (N, c_in, s, s), Y (N, 2, s, s) float32 CUDA tensors, N = len(ws) * nsnap, in a
    seeded random order so that contiguous slices are shuffled minibatches.  With
    coarse > 0, X holds the corrector's input (coarse solve, psi(t), features)."""
    stream = _stream(torch)
    s = ws[0].n[0]
    n = len(ws) * nsnap
    cin = input_channels(coarse)
    perm = np.random.default_rng(seed).permutation(n)
    X = torch.empty((n, cin, s, s), dtype=torch.float32, device="cuda")
    Y = torch.empty((n, 2, s, s), dtype=torch.float32, device="cuda")
    for c0 in range(0, len(ws), chunk):
        part = ws[c0:c0 + chunk]
        c = len(part)
        feat = torch.from_numpy(features(part)).cuda()
        b = _batch(torch, part, stream)
        bc = _batch(torch, part, stream) if coarse > 0 else None
        cur = torch.empty((c, s, s), dtype=torch.complex64, device="cuda")
        nxt = torch.empty_like(cur)
        crs = torch.empty_like(cur) if coarse > 0 else None
        xs = torch.empty((c, cin, s, s), dtype=torch.float32, device="cuda")
        ys = torch.empty((c, 2, s, s), dtype=torch.float32, device="cuda")
        for k in range(nsnap):
            for i in range(c):
                b.get_state(i, cur[i])
            b.step(part[0].dt, stride)
            for i in range(c):
                b.get_state(i, nxt[i])
            if coarse > 0:
                coarse_solve(torch, bc, cur, part[0].dt * stride / coarse, coarse, crs)
                sn.sn_fno_pack2(crs, cur, feat, xs, stream)
            else:
                sn.sn_fno_pack(cur, feat, xs, stream)
            sn.sn_fno_pack(nxt, None, ys, stream)
            for i in range(c):
                j = int(perm[(c0 + i) * nsnap + k])
                X[j].copy_(xs[i])
                Y[j].copy_(ys[i])
        b.close()
        if bc is not None:
            bc.close()
    torch.cuda.synchronize()
    return X, Y


def train(net, X, Y, iters: int, batch: int, lr: float = 1e-3, time_budget: float = None,
          log=None, data_parallel: bool = False, device: str = "cuda"):
    """Adam on contiguous minibatches with a cosine-decayed rate; returns the losses.

    data_parallel: this process is one rank of a process group and X, Y are its
    shard; the gradients are averaged over the ranks (dist.average_gradients)
    between each backward and Adam step, so all ranks keep the same parameters
    (they must start from the same ones).  device: where the output and
    gradient buffers live (the network's own; "cuda" for sn.Fno)."""
    import math
    import torch
    from . import dist as D
    n = X.shape[0]
    out = torch.empty((batch, 2, X.shape[2], X.shape[3]), dtype=torch.float32, device=device)
    gbuf = (torch.empty(net.nparams, dtype=torch.float32, device=device)
            if data_parallel and D.world() > 1 else None)
    # a shard smaller than one batch has no minibatch: every rank must learn of it
    # before the first all-reduce, or the ranks that have one would wait there
    short = 1.0 if n < batch else 0.0
    if gbuf is not None:
        short = D.max_over_ranks(short)
    if short > 0.0:
        raise ValueError(f"train: a rank holds fewer pairs than one batch ({n} < {batch})")
    losses, t0 = [], time.perf_counter()
    nb = n // batch
    for it in range(1, iters + 1):
        k = (it - 1) % nb
        xb, yb = X[k * batch:(k + 1) * batch], Y[k * batch:(k + 1) * batch]
        net.forward(xb, out)
        losses.append(net.loss(yb, batch))
        net.backward()
        if gbuf is not None:
            net.get_grads(gbuf)
            D.average_gradients(gbuf)
            net.set_grads(gbuf)
        net.adam(lr * 0.5 * (1.0 + math.cos(math.pi * (it - 1) / iters)), it)
        if log and it % 100 == 0:
            log(f"iter {it} loss {np.mean(losses[-100:]):.4f} ({time.perf_counter() - t0:.0f} s)")
        if time_budget is not None:
            over = time.perf_counter() - t0 > time_budget
            # data-parallel ranks stop together, or one would wait in an all-reduce
            if gbuf is not None:
                over = D.max_over_ranks(1.0 if over else 0.0) > 0.0
            if over:
                break
    net.sync()
    return losses


def _masses(torch, psi, stream=None):
    out = torch.empty(psi.shape[0], dtype=torch.float64, device="cuda")
    sn.sn_mass_c64(psi, out, stream)
    return out


def rollout(torch, net, ws, rounds=20, stride=50, drift_tol=1e-3, perturb=None, coarse=0):
    """Advance every instance `rounds` x `stride` steps by the surrogate with
    fallback, and by the solver alone; compare.  `perturb(r, psi)` may alter
    the predictions (used to exercise the fallback).  With coarse > 0 every
    network call first takes the coarse solve of its horizon (timed with it),
    and the coarse solves alone are rolled out too, as the method without the
    network."""
    stream = _stream(torch)
    s = ws[0].n[0]
    n = len(ws)
    dt = ws[0].dt
    feat = torch.from_numpy(features(ws)).cuda()
    psi0 = torch.stack([torch.from_numpy(w.psi0(np.complex64)) for w in ws]).cuda()
    # solver reference trajectory (one batch, snapshots every `stride` steps)
    b = _batch(torch, ws, stream)
    ref = torch.empty((rounds, n, s, s), dtype=torch.complex64, device="cuda")
    for r in range(rounds):
        b.step(dt, stride)
        for i in range(n):
            b.get_state(i, ref[r, i])
    # solver alone, timed: all rounds in one call
    for i in range(n):
        b.set_state(i, psi0[i])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(dt, rounds * stride)
    b.sync()
    t_solver = time.perf_counter() - t0
    dt_c = dt * stride / coarse if coarse > 0 else 0.0
    bc = _batch(torch, ws, stream) if coarse > 0 else None
    # the coarse solves alone (the method without the network), and their errors
    coarse_errs = None
    if coarse > 0:
        crs_only = psi0.clone()
        tmp = torch.empty_like(crs_only)
        first_err = None
        for r in range(rounds):
            coarse_solve(torch, bc, crs_only, dt_c, coarse, tmp)
            crs_only, tmp = tmp, crs_only
            if r == 0:
                first_err = _rel_errors(crs_only, ref[0])
        coarse_errs = {"coarse_only_first_call_rel_l2_mean": float(np.mean(first_err)),
                       "coarse_only_final_rel_l2_mean": float(np.mean(_rel_errors(crs_only, ref[rounds - 1])))}
    # surrogate with fallback
    B = net.batch_max
    X = torch.empty((B, input_channels(coarse), s, s), dtype=torch.float32, device="cuda")
    Yb = torch.empty((B, 2, s, s), dtype=torch.float32, device="cuda")
    psi = psi0.clone()
    nxt = torch.empty_like(psi)
    crs = torch.empty_like(psi) if coarse > 0 else None
    errors, fallbacks = [], []
    first_call = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in range(rounds):
        if coarse > 0:
            coarse_solve(torch, bc, psi, dt_c, coarse, crs)
        for c0 in range(0, n, B):
            c = min(B, n - c0)
            if coarse > 0:
                sn.sn_fno_pack2(crs[c0:c0 + c], psi[c0:c0 + c], feat[c0:c0 + c], X, stream)
            else:
                sn.sn_fno_pack(psi[c0:c0 + c], feat[c0:c0 + c], X, stream)
            net.forward(X[:c], Yb[:c])
            sn.sn_fno_unpack(Yb[:c], nxt[c0:c0 + c], stream)
        if perturb is not None:
            perturb(r, nxt)
        m_old = _masses(torch, psi, stream).cpu().numpy()
        m_new = _masses(torch, nxt, stream).cpu().numpy()
        bad = np.nonzero(np.abs(m_new / m_old - 1.0) > drift_tol)[0]
        if len(bad):
            fb = sn.Batch([s] * len(bad), [ws[i].L[0] for i in bad], stream=stream)
            fb.set_kernels([kernel_kw(ws[i].kernel) for i in bad])
            for j, i in enumerate(bad):
                fb.set_state(j, psi[int(i)])
            fb.step(dt, stride)
            for j, i in enumerate(bad):
                fb.get_state(j, nxt[int(i)])
            fb.sync()
            fb.close()
        psi, nxt = nxt, psi
        fallbacks.append(len(bad))
        if r == 0:
            first_call = psi.clone()
    torch.cuda.synchronize()
    t_sur = time.perf_counter() - t0
    first_errs = _rel_errors(first_call, ref[0])
    if bc is not None:
        bc.close()
    # relative L2 error of the final surrogate state against the solver's (host, FP64)
    fin = psi.cpu().numpy().astype(np.complex128)
    want = ref[rounds - 1].cpu().numpy().astype(np.complex128)
    errs = [float(np.linalg.norm(fin[i] - want[i]) / np.linalg.norm(want[i])) for i in range(n)]
    b.close()
    res = {"instances": n, "rounds": rounds, "stride": stride, "t_surrogate_s": t_sur,
           "t_solver_s": t_solver, "fallbacks_per_round": fallbacks,
           "fallback_fraction": float(sum(fallbacks)) / (rounds * n),
           "first_call_rel_l2_mean": float(np.mean(first_errs)),
           "final_rel_l2_mean": float(np.mean(errs)), "final_rel_l2_max": float(np.max(errs))}
    if coarse_errs is not None:
        res.update(coarse_errs)
        res["coarse_steps"] = coarse
    return res


def _rel_errors(a, b):
    """Relative L2 distance of each state of a (B, s, s) from b's (host FP64)."""
    x = a.cpu().numpy().astype(np.complex128).reshape(a.shape[0], -1)
    y = b.cpu().numpy().astype(np.complex128).reshape(b.shape[0], -1)
    return np.linalg.norm(x - y, axis=1) / np.linalg.norm(y, axis=1)


def plain_fp64_time(torch, ws, steps, sample=4):
    """Seconds of `steps` plain FP64 GPU steps (one complex128 grid per instance,
    one after another), estimated from the first `sample` instances."""
    stream = _stream(torch)
    grids = []
    for w in ws[:sample]:
        g = sn.Grid(w.n, w.L, "c128", stream=stream)
        g.set_kernel(**kernel_kw(w.kernel))
        g.set_state(w.psi0(np.complex128))
        g.step(w.dt, 2)
        grids.append(g)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g in grids:
        g.step(ws[0].dt, steps)
    for g in grids:
        g.sync()
    t = (time.perf_counter() - t0) * len(ws) / len(grids)
    for g in grids:
        g.close()
    return t


def one_step_errors(torch, net, X, Y, batch):
    """Mean relative L2 error of single predictions and of the state the head
    turns (channels 0, 1 of X) taken as the prediction, over the pairs (X, Y)
    (host FP64 for the latter): the persistence guess psi(t + stride dt) ~ psi(t),
    or in the corrector form the coarse solve alone."""
    out = torch.empty((batch, 2, X.shape[2], X.shape[3]), dtype=torch.float32, device="cuda")
    e_net, e_id = [], []
    for k in range(X.shape[0] // batch):
        xb, yb = X[k * batch:(k + 1) * batch], Y[k * batch:(k + 1) * batch]
        net.forward(xb, out)
        e_net.append(net.loss(yb, batch))
        x = xb[:, :2].cpu().numpy().astype(np.float64).reshape(batch, -1)
        y = yb.cpu().numpy().astype(np.float64).reshape(batch, -1)
        e_id.append(float(np.mean(np.linalg.norm(x - y, axis=1) / np.linalg.norm(y, axis=1))))
    return float(np.mean(e_net)), float(np.mean(e_id))


def main(argv=None):
    """Config-scale run: train on solver pairs, then roll out held-out instances.

    Prints one JSON line with the training loss, the held-out single-prediction
    error against the persistence guess and the zero guess (whose relative error
    is 1 by definition), and the rollout's fallback fraction, final error and
    wall times against the batched solver alone.

    Under torchrun (WORLD_SIZE > 1, one process per GPU, NCCL) the training is
    data-parallel: each rank generates the pairs of its share of the training
    trajectories (every world-th), all ranks start from the same parameters and
    average their gradients before every Adam step; rank 0 evaluates."""
    import argparse
    import json
    import os
    import torch
    from . import dist as D
    ap = argparse.ArgumentParser()
    ap.add_argument("--s", type=int, default=256)
    ap.add_argument("--train", type=int, default=4096, help="training trajectories")
    ap.add_argument("--heldout", type=int, default=512)
    ap.add_argument("--nsnap", type=int, default=10)
    ap.add_argument("--stride", type=int, default=50)
    ap.add_argument("--rounds", type=int, default=20)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--iters", type=int, default=100000)
    ap.add_argument("--budget", type=float, default=600.0, help="training seconds")
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--width", type=int, default=64)
    ap.add_argument("--modes", type=int, default=24)
    ap.add_argument("--layers", type=int, default=4)
    ap.add_argument("--proj", type=int, default=128)
    ap.add_argument("--drift-tol", type=float, default=1e-3)
    ap.add_argument("--init-seed", type=int, default=0)
    ap.add_argument("--coarse", type=int, default=10,
                    help="coarse split steps per call of the corrector form (0: the plain map)")
    a = ap.parse_args(argv)
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    rank, world = D.rank(), D.world()
    log = (lambda m: print(m, flush=True)) if rank == 0 else (lambda m: None)  # noqa: E731
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    t0 = time.perf_counter()
    X, Y = generate_pairs(torch, instances(a.train, 5000, a.s)[rank::world], a.stride, a.nsnap,
                          seed=1, coarse=a.coarse)
    test_ws = instances(a.heldout, 9000, a.s) if rank == 0 else []
    Xt, Yt = (generate_pairs(torch, test_ws, a.stride, 2, seed=2, coarse=a.coarse)
              if rank == 0 else (None, None))
    t_gen = time.perf_counter() - t0
    log(f"pairs: {X.shape[0]} train per rank x {world}, "
        f"{Xt.shape[0] if Xt is not None else 0} held out ({t_gen:.0f} s)")
    net = sn.Fno(s=a.s, c_in=input_channels(a.coarse), width=a.width, modes=a.modes,
                 layers=a.layers, proj=a.proj, batch_max=a.batch, stream=stream.cuda_stream)
    p0 = _init_params(a)
    if p0.size != net.nparams:
        raise RuntimeError("parameter layout mismatch")
    net.set_params(p0)
    t0 = time.perf_counter()
    losses = train(net, X, Y, a.iters, a.batch, a.lr, a.budget, log, data_parallel=world > 1)
    t_train = time.perf_counter() - t0
    # the aggregate rate: every rank's samples over the slowest rank's time
    samples_all = D.sum_over_ranks(len(losses) * a.batch)
    t_train_max = D.max_over_ranks(t_train)
    del X, Y
    if rank != 0:
        D.barrier()
        net.close()
        return
    e_net, e_id = one_step_errors(torch, net, Xt, Yt, a.batch)
    res = rollout(torch, net, test_ws, a.rounds, a.stride, a.drift_tol, coarse=a.coarse)
    t64 = plain_fp64_time(torch, test_ws, a.rounds * a.stride)
    res.update({"grid": a.s, "train_pairs": a.train * a.nsnap, "train_iters": len(losses),
                "train_samples_per_s": samples_all / t_train_max, "train_s": t_train_max,
                "loss_first100": float(np.mean(losses[:100])),
                "loss_last100": float(np.mean(losses[-100:])),
                "heldout_rel_l2_net": e_net,
                ("heldout_rel_l2_coarse" if a.coarse > 0 else "heldout_rel_l2_persistence"): e_id,
                "heldout_rel_l2_zero": 1.0, "params": net.nparams,
                "t_plain_fp64_gpu_s": t64,
                "speedup_vs_plain_fp64_gpu": t64 / res["t_surrogate_s"],
                "speedup_vs_batched_fp32_solver": res["t_solver_s"] / res["t_surrogate_s"]})
    res.pop("fallbacks_per_round", None)
    if world > 1:
        res["data_parallel_ranks"] = world
    print(json.dumps(res), flush=True)
    if world > 1:
        D.barrier()
    net.close()


def _init_params(a):
    """Seeded initial weights in the library's flat layout (same scheme as the
    FP64 network's initialiser: uniform +-1/sqrt(fan-in), spectral weights scaled
    by 1/(width^2))."""
    rng = np.random.default_rng(a.init_seed)
    w, m2, m, P = a.width, 2 * a.modes, a.modes, a.proj
    cin = input_channels(a.coarse)
    parts = [rng.uniform(-1, 1, (w, cin)) / np.sqrt(cin), np.zeros(w)]
    for _ in range(a.layers):
        parts += [rng.uniform(0, 1, (m2, m, w, w, 2)) / (w * w),
                  rng.uniform(-1, 1, (w, w)) / np.sqrt(w), np.zeros(w)]
    parts += [rng.uniform(-1, 1, (P, w)) / np.sqrt(w), np.zeros(P),
              rng.uniform(-1, 1, (3, P)) / np.sqrt(P), np.zeros(3)]
    return np.concatenate([q.ravel() for q in parts]).astype(np.float32)


if __name__ == "__main__":
    main()

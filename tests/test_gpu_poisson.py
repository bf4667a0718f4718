"""Eq. 2 kernels of the optical media (SN_KERNEL_POISSON) through the C-ABI,
against the FP64 oracle.

Sec. II A: thermo-optical media (Eq. 4, lap dn - dn/sigma^2 = -(zeta mu/kappa)
|E|^2) and nematic liquid crystals (Eq. 5, nu lap theta - 2 q theta = -2 |E|^2)
are Eq. 2 with C < 0, so K(k) = B D / (C - k^2).  Bars as for the default
kernel: rel-L2 per step <= 1e-6 (complex64) and <= 1e-12 (complex128), k
merged steps k times that, FP64 observables to 1e-10.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_1909_08354_b300 import sn

pytestmark = pytest.mark.gpu

STEP_TOL = {"c64": 1e-6, "c128": 1e-12}


def thermo_optical(sigma=3.0, zeta_mu_over_kappa=2.0, B=1.0, g=0.01):
    """Eq. 4 with dn = phi: C = -1/sigma^2, D = -zeta mu / kappa."""
    return dict(coeff_lap=-0.5, g_local=g, kind=sn.SN_KERNEL_POISSON, B=B,
                C=-1.0 / sigma ** 2, D=-zeta_mu_over_kappa)


def nematic(nu=1.5, q=0.4, B=0.5, g=0.0):
    """Eq. 5 with theta = phi: C = -2q/nu, D = -2/nu."""
    return dict(coeff_lap=-0.5, g_local=g, kind=sn.SN_KERNEL_POISSON, B=B,
                C=-2.0 * q / nu, D=-2.0 / nu)


def oracle_kw(kw):
    return dict(coeff_lap=kw["coeff_lap"], g_local=kw["g_local"], kind=O.KIND_POISSON,
                B=kw["B"], C=kw["C"], D=kw["D"])


def gpu_run(psi, L, kw, dtype, dt, nsteps):
    g = sn.Grid(psi.shape, L, dtype)
    try:
        g.set_kernel(**kw)
        g.set_state(np.ascontiguousarray(psi, dtype=g.np_dtype))
        g.step(dt, nsteps)
        return g.get_state()
    finally:
        g.close()


CASES = [
    ("thermo-optical 2D", (64, 128), (30.0, 40.0), thermo_optical()),
    ("thermo-optical 2D strong", (128, 64), (20.0, 20.0), thermo_optical(sigma=1.5, zeta_mu_over_kappa=20.0)),
    ("nematic 3D", (16, 32, 64), (12.0, 16.0, 20.0), nematic()),
    ("nematic 3D, 1024-point axis", (8, 16, 1024), (6.0, 8.0, 60.0), nematic(nu=0.8, q=1.0, g=0.02)),
]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("name,shape,L,kw", CASES, ids=[c[0] for c in CASES])
def test_poisson_kernel_steps_match_oracle(name, shape, L, kw, dtype):
    w = W.random_small(shape, seed=7 + sum(shape), L=L)
    psi = w.psi0().astype(np.complex64 if dtype == "c64" else np.complex128)
    okw = oracle_kw(kw)
    dt = 0.02
    for nsteps in (1, 3):
        out = gpu_run(psi, L, kw, dtype, dt, nsteps)
        ref = O.evolve(psi.astype(np.complex128), dt, nsteps, L, **okw)
        assert O.rel_l2(out, ref) <= nsteps * STEP_TOL[dtype], (nsteps, O.rel_l2(out, ref))
    # the nonlocal potential is not negligible here
    free = O.evolve(psi.astype(np.complex128), dt, 1, L, **dict(okw, D=0.0))
    one = O.evolve(psi.astype(np.complex128), dt, 1, L, **okw)
    assert O.rel_l2(free, one) > 1e2 * STEP_TOL["c64"]


@pytest.mark.parametrize("shape,L,kw", [((64, 32), (20.0, 10.0), thermo_optical()),
                                        ((16, 32, 8), (8.0, 12.0, 6.0), nematic(g=0.03))])
def test_poisson_kernel_observables_match_oracle(shape, L, kw):
    w = W.random_small(shape, seed=23, L=L)
    psi = w.psi0()
    g = sn.Grid(shape, L, "c128")
    try:
        g.set_kernel(**kw)
        g.set_state(psi)
        got = g.observables()
    finally:
        g.close()
    ref = O.observables(psi.astype(np.complex128), L, **oracle_kw(kw))
    assert abs(ref["e_pot"]) > 1e-3 * abs(ref["e_kin"])
    for key in ["mass", "e_kin", "e_pot", "e_nl", "e_total"]:
        assert abs(got[key] - ref[key]) <= 1e-10 * max(1.0, abs(ref[key])), key


def test_unscreened_poisson_kernel_is_the_newton_kernel():
    """C = 0 and B D = 4 pi G give the alpha_Y = 0 kernel of Eq. 14."""
    w = W.random_small((32, 64), seed=3, L=(10.0, 12.0))
    G = 1.3
    a = gpu_run(w.psi0(), w.L, dict(coeff_lap=-0.5, G=G), "c128", 0.02, 2)
    b = gpu_run(w.psi0(), w.L, dict(coeff_lap=-0.5, kind=sn.SN_KERNEL_POISSON, B=2.0, C=0.0,
                                    D=4 * np.pi * G / 2.0), "c128", 0.02, 2)
    assert O.rel_l2(b, a) <= 1e-13


def test_batch_and_noalloc_accept_poisson_kernels():
    torch = pytest.importorskip("torch")
    ws = [W.random_small((64, 64), seed=41, L=(20.0, 20.0)),
          W.random_small((128, 128), seed=42, L=(30.0, 30.0))]
    kws = [thermo_optical(), nematic(g=0.02)]
    b = sn.Batch([v.n[0] for v in ws], [v.L[0] for v in ws])
    try:
        b.set_kernels(kws)
        for i, v in enumerate(ws):
            b.set_state(i, v.psi0().astype(np.complex64))
        b.step(0.02, 3)
        for i, v in enumerate(ws):
            ref = O.evolve(v.psi0(), 0.02, 3, v.L, **oracle_kw(kws[i]))
            assert O.rel_l2(b.get_state(i), ref) <= 3 * STEP_TOL["c64"], i
    finally:
        b.close()
    v = ws[1]
    d = torch.from_numpy(v.psi0().astype(np.complex64)).cuda()
    sn.sn_step_2d_noalloc(d, v.L, 0.02, 3, **kws[1])
    ref = O.evolve(v.psi0(), 0.02, 3, v.L, **oracle_kw(kws[1]))
    assert O.rel_l2(d.cpu().numpy(), ref) <= 3 * STEP_TOL["c64"]


@pytest.mark.parametrize("bad", [dict(C=0.5), dict(kind=7), dict(B=float("nan")),
                                 dict(D=float("inf"))])
def test_invalid_poisson_kernels_are_rejected(bad):
    kw = dict(thermo_optical(), **bad)
    g = sn.Grid((8, 8), (1.0, 1.0), "c64")
    try:
        with pytest.raises(sn.SNError) as e:
            g.set_kernel(**kw)
        assert e.value.status == sn.SN_EINVAL
    finally:
        g.close()

"""The self-gravitating fluid model of Sec. II B (Eq. 16, GR and the pure
non-minimal coupling) on complex128 grids, through the C-ABI, against the FP64
oracle of oracle/cosmo_oracle.py.

Bar: the plain FP64 path's, rel-L2 <= 1e-12 per split step from the same input
(k steps: k times that); mass to 1e-12 relative (every sub-step is unitary).
"""
import math

import numpy as np
import pytest

import oracle as O
import oracle.cosmo_oracle as C
import workloads as W
from paper_1909_08354_b300 import sn

pytestmark = pytest.mark.gpu

TOL = 1e-12


def gaussian_fluid(n, L, M0=25.0, sigma=3.0, seed=0):
    """A Gaussian mass distribution of total mass M0 (Figs. 3-4) with a weak random
    velocity field, so that no symmetry hides an axis or sign slip."""
    d = len(n)
    grids = np.meshgrid(*[W.coords(n[a], L[a]) for a in range(d)], indexing="ij")
    r2 = sum(g * g for g in grids)
    rho = M0 / (2 * math.pi * sigma * sigma) ** (d / 2) * np.exp(-r2 / (2 * sigma * sigma))
    rng = np.random.default_rng(seed)
    phase = sum(0.3 * rng.standard_normal() * np.sin(2 * math.pi * (a + 1) * grids[a] / L[a])
                for a in range(d))
    return np.sqrt(rho) * np.exp(1j * phase)


def params(model, **kw):
    base = dict(nu=1.0, w=1.02, n_poly=1.0, lam=1.0, M=25.0, rho_floor=1e-10)
    base.update(kw)
    return base


def to_oracle(model, p):
    return C.CosmoParams(nu=p["nu"], w=p["w"], n_poly=p["n_poly"], model=model, lam=p["lam"],
                         M=p["M"], rho_floor=p["rho_floor"], floor_mode=p.get("floor_mode", 0))


def gpu_fluid(psi, L, model, p, dt, nsteps):
    g = sn.Grid(psi.shape, L, "c128")
    try:
        g.set_fluid(model=model, **p)
        g.set_state(psi)
        g.step(dt, nsteps)
        return g.get_state()
    finally:
        g.close()


CASES = [
    ("GR 2D", (64, 128), (24.0, 32.0), sn.SN_GRAVITY_GR, params(sn.SN_GRAVITY_GR)),
    ("NMC 2D (Figs. 3-4 parameters)", (128, 128), (30.0, 30.0), sn.SN_GRAVITY_NMC,
     params(sn.SN_GRAVITY_NMC)),
    ("NMC 2D, n = 5/3, nu = 0.7", (64, 64), (24.0, 24.0), sn.SN_GRAVITY_NMC,
     params(sn.SN_GRAVITY_NMC, n_poly=5.0 / 3.0, nu=0.7, lam=1.6, M=12.0)),
    ("NMC 3D", (32, 32, 16), (24.0, 24.0, 20.0), sn.SN_GRAVITY_NMC,
     params(sn.SN_GRAVITY_NMC, n_poly=2.0)),
    ("GR 3D", (16, 32, 64), (20.0, 24.0, 28.0), sn.SN_GRAVITY_GR, params(sn.SN_GRAVITY_GR)),
    ("NMC 2D, smooth floor", (128, 128), (30.0, 30.0), sn.SN_GRAVITY_NMC,
     params(sn.SN_GRAVITY_NMC, floor_mode=sn.SN_FLOOR_SMOOTH, rho_floor=1e-6)),
]


@pytest.mark.parametrize("name,shape,L,model,p", CASES, ids=[c[0] for c in CASES])
def test_fluid_steps_match_oracle(name, shape, L, model, p):
    psi = gaussian_fluid(shape, L, seed=len(name))
    dt = 0.01
    for nsteps in (1, 2, 3):  # one step; merged half steps; a replayed middle step
        out = gpu_fluid(psi, L, model, p, dt, nsteps)
        ref = C.cosmo_evolve(psi, dt, nsteps, L, to_oracle(model, p))
        assert O.rel_l2(out, ref) <= nsteps * TOL, (nsteps, O.rel_l2(out, ref))
    assert O.rel_l2(ref, psi) > 1e-4  # the steps move the state


def test_fluid_mass_conservation_and_time_reversal():
    shape, L = (128, 128), (30.0, 30.0)
    psi = gaussian_fluid(shape, L, seed=5)
    g = sn.Grid(shape, L, "c128")
    try:
        g.set_fluid(model=sn.SN_GRAVITY_NMC, **params(sn.SN_GRAVITY_NMC))
        g.set_state(psi)
        m0 = g.observables()["mass"]
        g.step(0.01, 40)
        obs = g.observables()
        assert abs(obs["mass"] / m0 - 1) < 1e-12
        g.step(-0.01, 40)
        back = g.get_state()
    finally:
        g.close()
    assert np.abs(back - psi).max() < 1e-9 * np.abs(psi).max()


def test_replayed_steps_follow_dt_and_parameter_changes():
    """A call of more than two steps replays its middle steps from a captured
    step (the launches carry dt and the fluid parameters): a change of dt, of
    the model and of nu between calls must each take effect."""
    shape, L = (64, 64), (24.0, 24.0)
    psi = gaussian_fluid(shape, L, seed=9)
    pg = params(sn.SN_GRAVITY_GR)
    pn = params(sn.SN_GRAVITY_NMC, nu=0.8)
    g = sn.Grid(shape, L, "c128")
    try:
        g.set_fluid(model=sn.SN_GRAVITY_GR, **pg)
        g.set_state(psi)
        g.step(0.01, 4)
        g.step(0.01, 3)
        g.step(0.005, 4)
        g.set_fluid(model=sn.SN_GRAVITY_NMC, **pn)
        g.step(0.005, 5)
        out = g.get_state()
    finally:
        g.close()
    ref = C.cosmo_evolve(psi, 0.01, 7, L, to_oracle(sn.SN_GRAVITY_GR, pg))
    ref = C.cosmo_evolve(ref, 0.005, 4, L, to_oracle(sn.SN_GRAVITY_GR, pg))
    ref = C.cosmo_evolve(ref, 0.005, 5, L, to_oracle(sn.SN_GRAVITY_NMC, pn))
    assert O.rel_l2(out, ref) <= 16 * TOL, O.rel_l2(out, ref)


def test_nmc_and_gr_differ_and_set_kernel_switches_back():
    shape, L = (64, 64), (24.0, 24.0)
    psi = gaussian_fluid(shape, L, seed=2)
    gr = gpu_fluid(psi, L, sn.SN_GRAVITY_GR, params(sn.SN_GRAVITY_GR), 0.01, 20)
    nmc = gpu_fluid(psi, L, sn.SN_GRAVITY_NMC, params(sn.SN_GRAVITY_NMC), 0.01, 20)
    assert O.rel_l2(nmc, gr) > 1e-3
    g = sn.Grid(shape, L, "c128")
    try:
        g.set_fluid(model=sn.SN_GRAVITY_NMC)
        g.set_kernel(coeff_lap=-0.5, G=1.0, g_local=0.01)  # back to Eqs. 1-2
        g.set_state(psi)
        g.step(0.01, 2)
        out = g.get_state()
    finally:
        g.close()
    ref = O.evolve(psi, 0.01, 2, L, coeff_lap=-0.5, G=1.0, g_local=0.01)
    assert O.rel_l2(out, ref) <= 2 * TOL


@pytest.mark.parametrize("bad", [dict(nu=0.0), dict(rho_floor=0.0), dict(lam=-1.0), dict(M=0.0),
                                 dict(model=5), dict(w=float("nan"))])
def test_invalid_fluid_parameters_are_rejected(bad):
    g = sn.Grid((8, 8), (1.0, 1.0), "c128")
    try:
        kw = dict(params(sn.SN_GRAVITY_NMC), model=sn.SN_GRAVITY_NMC)
        kw.update(bad)
        with pytest.raises(sn.SNError) as e:
            g.set_fluid(**kw)
        assert e.value.status == sn.SN_EINVAL
    finally:
        g.close()


def test_fluid_needs_a_complex128_grid():
    g = sn.Grid((8, 8), (1.0, 1.0), "c64")
    try:
        with pytest.raises(sn.SNError) as e:
            g.set_fluid()
        assert e.value.status == sn.SN_ENOTSUP
    finally:
        g.close()


@pytest.mark.parametrize("name,shape,L,model,p", CASES, ids=[c[0] for c in CASES])
def test_fluid_energies_match_oracle(name, shape, L, model, p):
    """sn_observables in the fluid mode against oracle.cosmo_oracle.fluid_energies (both
    FP64) on the same state, after two steps (1e-10 relative to the largest term)."""
    psi = gaussian_fluid(shape, L, seed=3)
    g = sn.Grid(shape, L, "c128")
    try:
        g.set_fluid(model=model, **p)
        g.set_state(psi)
        g.step(0.01, 2)
        got = g.observables()
        state = g.get_state()
    finally:
        g.close()
    ref = C.fluid_energies(state, L, to_oracle(model, p))
    scale = max(abs(ref[k]) for k in ("e_kin", "e_pot", "e_nl"))
    for k in ("e_kin", "e_pot", "e_nl", "e_total"):
        assert abs(got[k] - ref[k]) <= 1e-10 * scale, (k, got[k], ref[k])


def test_nmc_concentrates_the_centre_faster_than_gr():
    """The qualitative result of Figs. 3-4's run (M0 = 25, nu = 1, w = 1.02, n = 1,
    lambda = 1, a Gaussian of sigma = 3 at rest on a 40-wide box), in the regime where the
    split step resolves the kinetic and Bohm rotation of the highest wavenumber
    (k_max^2 h / 2 <= 1/4): at t = 1 the non-minimal coupling holds a central density
    several times that of General Relativity and a larger mass fraction within L/8, with
    the same sign under 2x changes of the time step, of the grid (h scaled as dx^2) and of
    the density floor (max form and smooth form)."""
    L, sigma, M0 = 40.0, 3.0, 25.0
    runs = [(256, 5e-4, 1e-12, sn.SN_FLOOR_MAX), (256, 1e-3, 1e-12, sn.SN_FLOOR_MAX),
            (256, 5e-4, 1e-10, sn.SN_FLOOR_MAX), (256, 5e-4, 1e-6, sn.SN_FLOOR_SMOOTH),
            (512, 2.5e-4, 1e-12, sn.SN_FLOOR_MAX)]
    for n, dt, floor, mode in runs:
        x = W.coords(n, L)
        X, Y = np.meshgrid(x, x, indexing="ij")
        r2 = X * X + Y * Y
        psi0 = np.sqrt(M0 / (2 * math.pi * sigma ** 2) * np.exp(-r2 / (2 * sigma ** 2))) + 0j
        summary = {}
        for name, model in (("GR", sn.SN_GRAVITY_GR), ("NMC", sn.SN_GRAVITY_NMC)):
            g = sn.Grid((n, n), (L, L), "c128")
            try:
                g.set_fluid(nu=1.0, w=1.02, n_poly=1.0, model=model, lam=1.0, M=M0,
                            rho_floor=floor, floor_mode=mode)
                g.set_state(psi0)
                g.step(dt, int(round(1.0 / dt)))
                rho = np.abs(g.get_state()) ** 2
            finally:
                g.close()
            inner = float(rho[np.sqrt(r2) <= L / 8].sum() * (L / n) ** 2 / M0)
            summary[name] = (float(rho[n // 2, n // 2]), inner)
        print(f"fluid n={n} dt={dt:g} floor={floor:g} mode={mode}: centre GR {summary['GR'][0]:.3f} "
              f"NMC {summary['NMC'][0]:.3f}, inner mass GR {summary['GR'][1]:.4f} "
              f"NMC {summary['NMC'][1]:.4f}")
        assert summary["NMC"][0] > 2.0 * summary["GR"][0]
        assert summary["NMC"][1] > summary["GR"][1]

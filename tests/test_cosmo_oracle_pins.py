"""Pins of the Eq. 16 oracle (oracle/cosmo_oracle.py) against closed forms,
finite differences and exact invariants (CPU only).

* the Bohm potential of a Gaussian amplitude is a quadratic (closed form);
* Eq. 15 under GR (beta = 0, gamma = 1/2) is Newton's law with 4 pi G = 1/2,
  and a constant beta adds beta (rho - <rho>) exactly;
* Eq. 15 with the NMC profiles satisfies its own PDE under a finite-difference
  Laplacian (independent of the spectral one);
* Eqs. 11-13 obey beta = 2 dgamma/dr and phi_C = ln(2 gamma);
* the polytropic V_p satisfies grad P / rho = grad V_p;
* the split step of Eq. 16 conserves mass and is time-reversible.
"""
import math

import numpy as np
import pytest

import oracle as O
import oracle.cosmo_oracle as C
import workloads as W


def grid2(n, L):
    x = W.coords(n[0], L[0])
    y = W.coords(n[1], L[1])
    return np.meshgrid(x, y, indexing="ij")


def fd_laplacian(f, dx):
    """4th-order central finite-difference Laplacian on a periodic grid."""
    out = np.zeros_like(f)
    for a in range(f.ndim):
        out += (-np.roll(f, 2, a) + 16 * np.roll(f, 1, a) - 30 * f + 16 * np.roll(f, -1, a)
                - np.roll(f, -2, a)) / (12 * dx[a] ** 2)
    return out


@pytest.mark.parametrize("shape,L,s", [((64, 128), (16.0, 24.0), 1.0),
                                       ((32, 32, 64), (12.0, 12.0, 16.0), 0.8)])
def test_bohm_potential_of_gaussian_is_quadratic(shape, L, s):
    """sqrt rho = A exp(-r^2/(2 s^2))  =>  lap(sqrt rho)/(2 sqrt rho) = (r^2/s^4 - d/s^2)/2.
    The Gaussian is ~1e-8 at the box edge, so its periodic extension is smooth enough."""
    d = len(shape)
    A = 0.7
    grids = np.meshgrid(*[W.coords(shape[a], L[a]) for a in range(d)], indexing="ij")
    r2 = sum(g * g for g in grids)
    amp = A * np.exp(-r2 / (2 * s * s))
    vb = C.bohm_potential(amp ** 2, L, rho_floor=1e-300)
    ref = 0.5 * (r2 / s ** 4 - d / s ** 2)
    core = amp > 1e-4 * A  # the quotient loses digits where the amplitude is tiny
    assert np.abs(vb[core] - ref[core]).max() < 1e-8 * np.abs(ref).max()


def test_gr_newtonian_part_is_newton_with_4piG_one_half():
    n, L = (32, 64), (10.0, 14.0)
    X, Y = grid2(n, L)
    rho = np.exp(-(X ** 2 + 2 * Y ** 2) / 3.0) + 0.2 * np.exp(-((X - 2) ** 2 + Y ** 2))
    p = C.CosmoParams(model=C.GR)
    g, b, pc = C.coupling_profiles(n, L, p)
    assert np.all(g == 0.5) and np.all(b == 0.0) and np.all(pc == 0.0)
    phi = C.newtonian_potential(rho, L, g, b)
    ref = O.potential(rho, L, G=0.5 / (4 * math.pi))
    assert np.abs(phi - ref).max() < 1e-13 * np.abs(ref).max()


def test_constant_beta_adds_beta_times_density_fluctuation():
    """lap phi = beta lap rho + gamma rho with constant beta: phi = beta (rho - <rho>) + Newton."""
    n, L = (32, 32, 16), (8.0, 8.0, 6.0)
    rng = np.random.default_rng(3)
    rho = np.abs(rng.standard_normal(n) + 1j * rng.standard_normal(n)) ** 2
    beta, gamma = 0.37, 0.5
    phi = C.newtonian_potential(rho, L, np.full(n, gamma), np.full(n, beta))
    ref = beta * (rho - rho.mean()) + O.potential(rho, L, G=gamma / (4 * math.pi))
    assert np.abs(phi - ref).max() < 1e-12 * np.abs(ref).max()


def test_nmc_newtonian_part_solves_eq15_by_finite_differences():
    """With the position-dependent gamma(r), beta(r) of Eqs. 11-12, lap phi_N equals
    beta lap rho + gamma rho minus its mean (the k = 0 mode removed); both Laplacians
    by 4th-order finite differences, on a smooth density."""
    n, L = (256, 256), (40.0, 40.0)
    X, Y = grid2(n, L)
    rho = 2.0 * np.exp(-(X ** 2 + Y ** 2) / 18.0)
    p = C.CosmoParams(model=C.NMC, lam=1.0, M=25.0)
    g, b, _ = C.coupling_profiles(n, L, p)
    phi = C.newtonian_potential(rho, L, g, b)
    dx = (L[0] / n[0], L[1] / n[1])
    src = b * fd_laplacian(rho, dx) + g * rho
    res = fd_laplacian(phi, dx) - (src - src.mean())
    # beta(r) has a cusp at the centre (|r|), whose spectral image rings there:
    # compare beyond 20 grid spacings (r > 3.1; the residual is 8e-4 of the source
    # at 2.5 spacings, 2e-5 at 10, 4e-6 at 20)
    mask = C.radius(n, L) > 20 * dx[0]
    assert np.abs(res[mask]).max() < 1e-5 * np.abs(src).max()


def test_coupling_profiles_obey_eqs_11_to_13_relations():
    """gamma = (1 - q)/2, beta = lambda q/(r + r0), phi_C = ln(1 - q) with
    q = (r0/(r + r0))^lambda imply beta = 2 dgamma/dr and phi_C = ln(2 gamma);
    gamma -> 1/2 far away and r0 = M / 4 pi."""
    n, L = (8, 8192), (1.0, 400.0)
    p = C.CosmoParams(model=C.NMC, lam=1.7, M=25.0)
    g, b, pc = C.coupling_profiles(n, L, p)
    c = n[0] // 2  # the row through the centre (y = 0)
    r = C.radius(n, L)[c]
    gg, bb, cc = g[c], b[c], pc[c]
    h = L[1] / n[1]
    i = np.arange(n[1] // 2 + 8, n[1] - 8)  # x > 0, r = x, away from the centre
    dg = (-gg[i + 2] + 8 * gg[i + 1] - 8 * gg[i - 1] + gg[i - 2]) / (12 * h)  # 4th order
    assert np.allclose(r[i], W.coords(n[1], L[1])[i])
    assert np.abs(2 * dg - bb[i]).max() < 1e-5 * np.abs(bb[i]).max()
    assert np.abs(cc - np.log(2 * gg)).max() < 1e-12
    r0 = 25.0 / (4 * math.pi)
    assert gg[n[1] // 2 + 1] == pytest.approx(0.5 * (1 - (r0 / (h + r0)) ** 1.7), rel=1e-14)
    assert 0.5 - gg[-1] < 0.5 * (r0 / 190.0) ** 1.7 * 1.1


@pytest.mark.parametrize("npoly", [1.0, 2.0, 5.0 / 3.0, -0.5])
def test_pressure_potential_is_enthalpy(npoly):
    """grad P / rho = grad V_p for P = w rho^n (Eq. 17), by finite differences."""
    x = np.linspace(-3, 3, 2001)
    rho = 0.3 + np.exp(-x ** 2)
    w = 1.02
    p = C.CosmoParams(w=w, n_poly=npoly)
    vp = C.pressure_potential(rho, p)
    P = w * rho ** npoly
    lhs = np.gradient(P, x) / rho
    rhs = np.gradient(vp, x)
    assert np.abs(lhs - rhs)[5:-5].max() < 1e-5 * np.abs(lhs).max()


@pytest.mark.parametrize("model", [C.GR, C.NMC])
def test_cosmo_step_conserves_mass_and_is_reversible(model):
    n, L = (64, 64), (20.0, 20.0)
    X, Y = grid2(n, L)
    psi = np.sqrt(25.0 / (math.pi * 9.0)) * np.exp(-(X ** 2 + Y ** 2) / 18.0) * np.exp(0.2j * X)
    p = C.CosmoParams(model=model, rho_floor=1e-10)
    h = 0.01
    out = C.cosmo_evolve(psi, h, 5, L, p)
    assert abs(C.mass(out, L) / C.mass(psi, L) - 1) < 1e-12
    back = C.cosmo_evolve(out, -h, 5, L, p)
    assert np.abs(back - psi).max() < 1e-10 * np.abs(psi).max()
    assert O.rel_l2(out, psi) > 1e-3  # the step does something


def test_uniform_plane_wave_phase_fixes_the_nu_scalings():
    """Under GR a plane wave of uniform density rho0 has V_B = 0, phi_N = 0 (uniform
    source, k = 0 removed) and V_p = w ln rho0, so Eq. 16, i nu psi_t =
    -(nu^2/2) lap psi + V_p psi, gives psi(t) = psi0 exp(-i (nu k^2/2 + V_p/nu) t)."""
    n, L = (32, 64), (8.0, 16.0)
    X, Y = grid2(n, L)
    kx, ky = 2 * math.pi * 3 / L[0], 2 * math.pi * (-5) / L[1]
    rho0, nu, w = 1.7, 0.6, 1.02
    psi = math.sqrt(rho0) * np.exp(1j * (kx * X + ky * Y))
    p = C.CosmoParams(model=C.GR, nu=nu, w=w, n_poly=1.0)
    h, steps = 0.01, 7
    out = C.cosmo_evolve(psi, h, steps, L, p)
    om = nu * (kx * kx + ky * ky) / 2 + w * math.log(rho0) / nu
    assert np.abs(out - psi * np.exp(-1j * om * h * steps)).max() < 1e-11


# ---- energies of Eq. 16 (fluid_energies) --------------------------------------

def test_fluid_energies_of_a_gaussian_match_closed_forms():
    """sqrt rho = A exp(-r^2/(2 s^2)) in 2D, at rest: e_kin = (nu/2) int |grad a|^2 =
    (nu/2) pi A^2; the Bohm part of e_nl is -(nu/2) pi A^2, so that the quantum pressure
    cancels; int rho (ln rho - 1) = M (ln A^2 - 2) with M = pi s^2 A^2 (d = 2); under GR
    e_pot is Newton's E_pot (sn_oracle, pinned by a Fourier series) with 4 pi G = 1/2."""
    n, L, s, A = (128, 128), (30.0, 30.0), 2.0, 0.8
    X, Y = grid2(n, L)
    psi = A * np.exp(-(X ** 2 + Y ** 2) / (2 * s * s)) + 0j
    nu, w = 0.7, 1.3
    p = C.CosmoParams(model=C.GR, nu=nu, w=w, n_poly=1.0, rho_floor=1e-300)
    e = C.fluid_energies(psi, L, p)
    M = math.pi * s * s * A * A
    assert abs(e["e_kin"] - 0.5 * nu * math.pi * A * A) < 1e-10
    eps = w * M * (math.log(A * A) - 2.0)
    bohm = -0.5 * nu * math.pi * A * A  # (1/nu) (-(nu^2/2) pi A^2)
    assert abs(e["e_nl"] - (bohm + eps / nu)) < 1e-9 * abs(eps / nu)
    newton = O.observables(psi, L, G=1.0 / (8.0 * math.pi))["e_pot"]
    assert abs(e["e_pot"] - newton / nu) < 1e-12 * abs(newton)


def test_fluid_energy_of_a_power_law_pressure():
    """P = w rho^n: eps = w rho^n / (n - 1); for the Gaussian density rho = A^2 e^{-r^2/s^2},
    int rho^n = pi s^2 A^(2n) / n (2D)."""
    n, L, s, A = (128, 128), (30.0, 30.0), 2.0, 0.8
    X, Y = grid2(n, L)
    psi = A * np.exp(-(X ** 2 + Y ** 2) / (2 * s * s)) + 0j
    npoly, w = 2.0, 0.9
    p = C.CosmoParams(model=C.GR, nu=1.0, w=w, n_poly=npoly, rho_floor=1e-300)
    e = C.fluid_energies(psi, L, p)
    bohm = -0.5 * math.pi * A * A
    eps = w / (npoly - 1.0) * math.pi * s * s * A ** (2 * npoly) / npoly
    assert abs(e["e_nl"] - (bohm + eps)) < 1e-9 * abs(eps)


def test_fluid_hamiltonian_is_conserved_to_second_order_under_gr():
    """Under GR Eq. 16 is Hamiltonian, so the split step conserves e_kin + e_pot + e_nl to
    O(h^2): over the same time span, halving h cuts the largest drift about 4x (a dropped or
    misweighted energy term would leave an O(1) drift)."""
    n, L = (64, 64), (24.0, 24.0)
    X, Y = grid2(n, L)
    psi0 = (np.sqrt(25.0 / (math.pi * 9.0)) * np.exp(-(X ** 2 + Y ** 2) / 18.0)
            * np.exp(2j * np.sin(2 * math.pi * X / L[0]))).astype(np.complex128)
    p = C.CosmoParams(model=C.GR, nu=1.0, w=1.02, n_poly=1.0, rho_floor=1e-14)
    drifts = []
    for h, steps in ((0.04, 10), (0.02, 20)):
        e0 = C.fluid_energies(psi0, L, p)["e_total"]
        psi, worst = psi0, 0.0
        for _ in range(steps):
            psi = C.cosmo_step(psi, h, L, p)
            worst = max(worst, abs(C.fluid_energies(psi, L, p)["e_total"] - e0))
        drifts.append(worst)
    assert 3.0 < drifts[0] / drifts[1] < 5.0, drifts

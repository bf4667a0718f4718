"""Pins of the FP64 oracle against what the mathematics fixes (CPU only).

Each test ties one part of the oracle to something other than itself: the
O(n^2) DFT definition, numpy's FFT, closed-form solutions of the sub-problems,
brute-force Fourier series, and exact invariants of the symmetric split step
(Sec. III).  A plausible slip in the oracle (a dropped Yukawa term, a sign
flip in a propagator, a half step taken as a full step, an axis mix-up on a
non-cubic grid, a misplaced 1/N) fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

RNG = np.random.default_rng(1909)


def crand(shape):
    return RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)


# ----------------------------------------------------------------------------
# DFT
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 64, 128])
def test_radix2_equals_definition(n):
    x = crand((3, n))
    ref = O.dft_naive(x, axis=1)
    assert np.abs(O.fft_radix2(x, axis=1) - ref).max() <= 1e-13 * n
    assert np.abs(O.fft_radix2(ref, axis=1, inverse=True) - x).max() <= 1e-13 * n


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_radix2_matches_numpy_along_each_axis(axis):
    x = crand((8, 16, 32))
    assert np.allclose(O.fft_radix2(x, axis=axis), np.fft.fft(x, axis=axis), atol=1e-12, rtol=0)
    assert np.allclose(O.fft_radix2(x, axis=axis, inverse=True), np.fft.ifft(x, axis=axis),
                       atol=1e-14, rtol=0)


def test_brute_force_3d_dft_on_8_cubed():
    """Full 3D DFT as one O(N^2) sum over all 512 points, against fftn."""
    n = 8
    x = crand((n, n, n))
    idx = np.indices((n, n, n)).reshape(3, -1)          # (3, 512)
    phase = (idx.T @ idx) % n                            # j . k mod n for all pairs
    X = (np.exp(-2j * np.pi * phase / n) @ x.ravel()).reshape(n, n, n)
    assert np.abs(O.fftn(x) - X).max() < 1e-11
    assert np.abs(O.fftn(X, inverse=True) - x).max() < 1e-13


def test_parseval_and_delta():
    x = crand((16, 32))
    assert math.isclose((np.abs(x) ** 2).sum(), (np.abs(O.fftn(x)) ** 2).sum() / x.size,
                        rel_tol=1e-13)
    d = np.zeros((8, 8, 8), complex)
    d[0, 0, 0] = 1.0
    assert np.abs(O.fftn(d) - 1.0).max() < 1e-15
    c = np.ones((8, 16), complex)
    C = O.fftn(c)
    assert abs(C[0, 0] - 128) < 1e-12 and np.abs(C.ravel()[1:]).max() < 1e-12


def test_wavenumbers_match_fftfreq():
    for n, L in [(8, 1.0), (32, 20.0), (256, 80.0)]:
        assert np.allclose(O.wavenumbers(n, L), 2 * np.pi * np.fft.fftfreq(n, d=L / n), rtol=0,
                           atol=1e-12)


# ----------------------------------------------------------------------------
# Kinetic sub-step: plane waves and the free Gaussian
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n,L", [((16, 32), (6.0, 10.0)), ((8, 16, 32), (4.0, 5.0, 7.0))])
def test_plane_wave_phase_non_cubic(n, L):
    """exp(i k0.x) with k0 on the grid picks up exactly exp(i A |k0|^2 t)."""
    d = len(n)
    m = [1, -3, 2][:d]
    k0 = [2 * np.pi * m[a] / L[a] for a in range(d)]
    grids = np.meshgrid(*[W.coords(n[a], L[a]) for a in range(d)], indexing="ij")
    psi = np.exp(1j * sum(k0[a] * grids[a] for a in range(d)))
    t = 0.37
    out = O.kinetic(psi, t, L, coeff_lap=-0.5)
    expect = psi * np.exp(-0.5j * sum(k * k for k in k0) * t)
    assert np.abs(out - expect).max() < 1e-12


def free_gaussian(n, L, sigma, t, images=2):
    """Closed-form free evolution of exp(-|x|^2/(2 sigma^2)) under i psi_t = -(1/2) lap psi,
    summed over periodic images: (sigma^2/(sigma^2+it))^(d/2) exp(-|x|^2/(2(sigma^2+it)))."""
    d = len(n)
    s = sigma * sigma + 1j * t
    out = np.ones(tuple(n), complex) * (sigma * sigma / s) ** (d / 2)
    for a in range(d):
        x = W.coords(n[a], L[a])
        f = sum(np.exp(-(x + j * L[a]) ** 2 / (2 * s)) for j in range(-images, images + 1))
        shape = [1] * d
        shape[a] = n[a]
        out = out * f.reshape(shape)
    return out


@pytest.mark.parametrize("d", [2, 3])
def test_free_gaussian_closed_form(d):
    n = (64,) * d if d == 2 else (32, 32, 32)
    L = (20.0,) * d
    sigma = 1.5
    psi0 = free_gaussian(n, L, sigma, 0.0)
    for t in (0.3, 1.7):
        out = O.kinetic(psi0, t, L)
        assert np.abs(out - free_gaussian(n, L, sigma, t)).max() < 1e-9


def test_free_strang_steps_equal_closed_form():
    """With G = g = 0 the split step is the exact free propagator: n steps of h land
    on the closed form at t = n h (catches a half step taken as a full step)."""
    n, L, sigma = (64, 64), (20.0, 20.0), 1.5
    psi = free_gaussian(n, L, sigma, 0.0)
    h, steps = 0.05, 12
    out = O.evolve(psi, h, steps, L, G=0.0, g_local=0.0)
    assert np.abs(out - free_gaussian(n, L, sigma, h * steps)).max() < 1e-9


# ----------------------------------------------------------------------------
# Potential: Fourier series of a Gaussian density, brute force
# ----------------------------------------------------------------------------

def gaussian_series_potential(points, L, s, G, alpha_Y, lambda_Y, kmax_modes):
    """V(x) = L^-d sum_{k != 0} K(k) (pi s^2)^(d/2) exp(-k^2 s^2/4) exp(i k.x) by direct sum."""
    d = len(L)
    ms = np.arange(-kmax_modes, kmax_modes + 1)
    grids = np.meshgrid(*[2 * np.pi * ms / L[a] for a in range(d)], indexing="ij")
    ks = np.stack([g.ravel() for g in grids], axis=1)
    k2 = (ks ** 2).sum(1)
    keep = k2 > 0
    ks, k2 = ks[keep], k2[keep]
    K = -4 * np.pi * G * (1 / k2 + alpha_Y / (k2 + 1 / lambda_Y ** 2))
    rhohat = (np.pi * s * s) ** (d / 2) * np.exp(-k2 * s * s / 4)
    vol = float(np.prod(L))
    return np.array([float((K * rhohat * np.cos(ks @ np.asarray(p))).sum()) / vol for p in points])


@pytest.mark.parametrize("d,alpha_Y", [(2, 0.0), (2, 0.7), (3, 0.0), (3, 0.3)])
def test_potential_of_gaussian_density(d, alpha_Y):
    n = (32,) * d if d == 2 else (32, 64, 32)
    L = (10.0,) * d if d == 2 else (10.0, 12.0, 10.0)
    s, G, lam = 1.0, 1.3, 2.0
    grids = np.meshgrid(*[W.coords(n[a], L[a]) for a in range(d)], indexing="ij")
    rho = np.exp(-sum(g * g for g in grids) / (s * s))
    V = O.potential(rho, L, G=G, alpha_Y=alpha_Y, lambda_Y=lam)
    pick = [tuple(RNG.integers(0, n[a]) for a in range(d)) for _ in range(6)]
    pts = [[grids[a][p] for a in range(d)] for p in pick]
    ref = gaussian_series_potential(pts, L, s, G, alpha_Y, lam, kmax_modes=24)
    got = np.array([V[p] for p in pick])
    assert np.abs(got - ref).max() < 1e-9 * max(1.0, np.abs(ref).max())


def test_uniform_density_has_zero_potential():
    V = O.potential(np.full((16, 8, 32), 2.5), (3.0, 4.0, 5.0), G=1.0, alpha_Y=0.4, lambda_Y=2.0)
    assert np.abs(V).max() < 1e-13


def test_yukawa_only_screened_poisson_residual_by_finite_differences():
    """The Yukawa part solves (lap - 1/lambda^2) V = 4 pi G alpha (rho - <rho>) on a fine 1D-like
    grid; checked with a 4th-order finite-difference Laplacian (independent of the spectral k^2)."""
    n, L = (8, 512), (1.0, 20.0)
    x = W.coords(n[1], L[1])
    rho = np.tile(np.exp(-x ** 2 / 2.0), (n[0], 1))
    G, alpha, lam = 1.0, 1.0, 1.5
    Vn = O.potential(rho, L, G=G, alpha_Y=0.0, lambda_Y=lam)
    Vt = O.potential(rho, L, G=G, alpha_Y=alpha, lambda_Y=lam)
    Vy = (Vt - Vn)[0]
    dx = L[1] / n[1]
    lap = (-np.roll(Vy, 2) + 16 * np.roll(Vy, 1) - 30 * Vy + 16 * np.roll(Vy, -1)
           - np.roll(Vy, -2)) / (12 * dx * dx)
    src = 4 * np.pi * G * alpha * (rho[0] - rho[0].mean())
    # the k=0 mode is removed from the whole multiplier, so compare up to the mean of Vy
    res = lap - (Vy - Vy.mean()) / lam ** 2 - src
    assert np.abs(res).max() < 1e-6 * np.abs(src).max()


def yukawa_gaussian_free_space(r, s, mu):
    """int exp(-|y|^2/s^2) exp(-mu |x - y|) / |x - y| dy at |x| = r > 0 (3D), the
    textbook screened potential of a Gaussian charge of per-axis variance
    sig^2 = s^2/2 and total pi^(3/2) s^3:
      M0 e^(mu^2 sig^2/2) / (2r) [e^(-mu r) erfc((mu sig^2 - r)/(sig sqrt 2))
                                  - e^(mu r) erfc((mu sig^2 + r)/(sig sqrt 2))]."""
    from scipy.special import erfc
    sig = s / np.sqrt(2.0)
    m0 = np.pi ** 1.5 * s ** 3
    a = np.exp(-mu * r) * erfc((mu * sig * sig - r) / (sig * np.sqrt(2.0)))
    b = np.exp(mu * r) * erfc((mu * sig * sig + r) / (sig * np.sqrt(2.0)))
    return m0 * np.exp(mu * mu * sig * sig / 2.0) / (2.0 * r) * (a - b)


def test_poisson_kind_matches_free_space_screened_gaussian():
    """Eq. 2 with C = -mu^2 < 0 in 3D: lap(phi) - mu^2 phi = D rho has the Green's function
    -exp(-mu r)/(4 pi r), so phi = -(D/4 pi) (Yukawa potential of rho).  The box is many
    screening lengths wide, so periodic images are negligible; removing k = 0 subtracts the
    box mean D M0 / (C L^3).  The kinetic-free potential is B phi."""
    n, Lb = 64, 32.0
    L = (Lb, Lb, Lb)
    s, mu, B, D = 1.5, 1.2, 0.8, -2.5
    C = -mu * mu
    x = W.coords(n, Lb)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    rho = np.exp(-(X * X + Y * Y + Z * Z) / (s * s))
    V = O.potential(rho, L, kind=O.KIND_POISSON, B=B, C=C, D=D)
    c = n // 2  # x = 0 is the node n/2
    r = x[c + 1:c + 13]  # 0.5 .. 6
    m0 = np.pi ** 1.5 * s ** 3
    ref = B * (-(D / (4 * np.pi)) * yukawa_gaussian_free_space(r, s, mu) - D * m0 / (C * Lb ** 3))
    got = V[c, c, c + 1:c + 13]
    assert np.abs(got - ref).max() < 1e-8 * np.abs(ref).max()


def test_poisson_kind_residual_by_finite_differences():
    """(lap + C) V = B D (rho - <rho>) for KIND_POISSON (k = 0 removed), checked on a fine
    1D-like grid with a 4th-order finite-difference Laplacian, independent of the spectral k^2.
    The parameters are those of a nematic liquid crystal, Eq. 5 (nu lap theta - 2 q theta =
    -2 rho): C = -2q/nu, D = -2/nu."""
    n, L = (8, 512), (1.0, 24.0)
    x = W.coords(n[1], L[1])
    rho = np.tile(np.exp(-x ** 2 / 3.0), (n[0], 1))
    nu, q, B = 1.5, 0.6, 0.9
    C, D = -2 * q / nu, -2 / nu
    V = O.potential(rho, L, kind=O.KIND_POISSON, B=B, C=C, D=D)[0]
    dx = L[1] / n[1]
    lap = (-np.roll(V, 2) + 16 * np.roll(V, 1) - 30 * V + 16 * np.roll(V, -1)
           - np.roll(V, -2)) / (12 * dx * dx)
    src = B * D * (rho[0] - rho[0].mean())
    assert np.abs(lap + C * V - src).max() < 1e-6 * np.abs(src).max()


def test_poisson_kind_unscreened_limit_is_newton():
    """C = 0, B D = 4 pi G: Eq. 2 is Newton's law, the alpha_Y = 0 kernel of Eq. 14."""
    rho = np.abs(crand((16, 8, 32))) ** 2
    L = (3.0, 4.0, 5.0)
    G = 1.7
    Vp = O.potential(rho, L, kind=O.KIND_POISSON, B=2.0, C=0.0, D=4 * np.pi * G / 2.0)
    Vn = O.potential(rho, L, G=G)
    assert np.abs(Vp - Vn).max() < 1e-13 * np.abs(Vn).max()


def test_thermo_optical_index_peaks_on_the_beam():
    """Eq. 4, lap(dn) - dn/sigma^2 = -(zeta mu/kappa)|E|^2 with zeta mu/kappa > 0: the index
    change (B = 1) is largest where the intensity is, and smallest far from the beam."""
    n, L = (64, 64), (30.0, 30.0)
    x = W.coords(n[0], L[0])
    Y, X = np.meshgrid(x, x, indexing="ij")
    rho = np.exp(-(X * X + Y * Y) / 4.0)
    dn = O.potential(rho, L, kind=O.KIND_POISSON, B=1.0, C=-1.0 / 9.0, D=-0.5)
    assert dn[32, 32] == dn.max()
    assert dn[0, 0] == pytest.approx(dn.min(), rel=1e-6)


def test_poisson_kind_rejects_antiscreening():
    with pytest.raises(ValueError):
        O.green_multiplier((8, 8), (1.0, 1.0), kind=O.KIND_POISSON, B=1.0, C=0.5, D=1.0)


# ----------------------------------------------------------------------------
# Nonlinear sub-step
# ----------------------------------------------------------------------------

def test_local_term_only_is_exact_phase():
    psi = crand((8, 16))
    h, g = 0.3, 0.7
    out = O.nonlinear(psi, h, (1.0, 2.0), G=0.0, g_local=g)
    assert np.abs(out - psi * np.exp(-1j * g * np.abs(psi) ** 2 * h)).max() < 1e-14
    assert np.abs(np.abs(out) - np.abs(psi)).max() < 1e-14


def test_external_potential_enters_phase():
    psi = crand((8, 8))
    v = RNG.standard_normal((8, 8))
    out = O.nonlinear(psi, 0.2, (1.0, 1.0), G=0.0, v_ext=v)
    assert np.abs(out - psi * np.exp(-0.2j * v)).max() < 1e-14


# ----------------------------------------------------------------------------
# Whole step: invariants and order
# ----------------------------------------------------------------------------

def small_state(n, seed=7, L=10.0):
    w = W.random_small(n, seed, L=L)
    return w.psi0(), w.L, O.kernel_kwargs(w.kernel)


@pytest.mark.parametrize("n", [(32, 32), (16, 8, 32)])
def test_mass_conserved(n):
    psi, L, kw = small_state(n)
    m0 = O.observables(psi, L, **kw)["mass"]
    out = O.evolve(psi, 0.05, 10, L, **kw)
    assert abs(O.observables(out, L, **kw)["mass"] / m0 - 1) < 1e-13


@pytest.mark.parametrize("n", [(32, 32), (8, 16, 16)])
def test_time_reversible(n):
    """S(-h) S(h) psi = psi exactly (rho is invariant under the nonlinear sub-step)."""
    psi, L, kw = small_state(n, seed=11)
    h = 0.08
    back = O.strang_step(O.strang_step(psi, h, L, **kw), -h, L, **kw)
    assert O.rel_l2(back, psi) < 1e-13


def collapse_case(amplitude=0.5):
    w = W.centred_gaussian_2d(n=64, L=20.0)
    w.lumps[0].amplitude = amplitude
    w.kernel.g_local = 0.05
    w.kernel.alpha_Y, w.kernel.lambda_Y = 0.4, 3.0
    return w.psi0(), w.L, O.kernel_kwargs(w.kernel)


def test_energy_drift_is_second_order():
    """The Hamiltonian is conserved only to O(h^2): the largest drift along a trajectory
    drops 4x when h is halved."""
    psi, L, kw = collapse_case()
    H0 = O.observables(psi, L, **kw)["e_total"]
    drift = []
    for h in (0.04, 0.02):
        p, worst = psi, 0.0
        for _ in range(int(round(0.8 / h))):
            p = O.strang_step(p, h, L, **kw)
            worst = max(worst, abs(O.observables(p, L, **kw)["e_total"] - H0))
        drift.append(worst)
    ratio = drift[0] / drift[1]
    assert 3.8 < ratio < 4.2, ratio
    assert drift[1] < 1e-3 * abs(H0)


def test_global_error_is_second_order():
    psi, L, kw = collapse_case()
    T = 0.8
    ref = O.evolve(psi, T / 128, 128, L, **kw)
    errs = [O.rel_l2(O.evolve(psi, T / m, m, L, **kw), ref) for m in (8, 16)]
    ratio = errs[0] / errs[1]
    assert 3.5 < ratio < 4.5, ratio


def test_gaussian_collapses_under_attraction_and_spreads_without():
    """Sec. IV: under Newtonian attraction the Gaussian contracts towards its centre;
    without the potential it spreads.  Compare the central density after t = 2."""
    w = W.centred_gaussian_2d(n=64, L=20.0)
    psi = w.psi0()
    rho0 = abs(psi[32, 32]) ** 2
    grav = O.evolve(psi, 0.05, 40, w.L, G=1.0)
    free = O.evolve(psi, 0.05, 40, w.L, G=0.0)
    assert abs(grav[32, 32]) ** 2 > rho0 > abs(free[32, 32]) ** 2


def test_mirror_and_axis_permutation_symmetry():
    n, L = (16, 16, 16), (8.0, 8.0, 8.0)
    grids = np.meshgrid(*[W.coords(16, 8.0)] * 3, indexing="ij")
    psi = np.exp(-(grids[0] ** 2 + grids[1] ** 2 + grids[2] ** 2) / 3.0) * (1 + 0.1 * grids[0] ** 2)
    psi = psi + psi.transpose(1, 2, 0) + psi.transpose(2, 0, 1)     # symmetric under cyclic perms
    kw = dict(G=1.0, alpha_Y=0.2, lambda_Y=2.0, g_local=0.03)
    out = O.evolve(psi, 0.05, 3, L, **kw)
    assert np.abs(out - out.transpose(1, 2, 0)).max() < 1e-12
    mirror = np.roll(out[::-1], 1, axis=0)                        # x -> -x about the node x=0
    assert np.abs(out - mirror).max() < 1e-12


def test_galilean_boost_translates_the_state():
    """Eq. 1 is covariant under boosts, and so is the split step when the
    boost wavenumber k0 is on the grid and each half step moves the state by
    a whole number of cells (k0 h / 2 = dx): S(h)^k (e^{i k0 x} psi) =
    e^{-i k0^2 t / 2} e^{i k0 x} psi_k(x - k0 t) with psi_k = S(h)^k psi and
    t = k h, self-gravity and the local term included (the density does not
    see the boost).  A sign slip in the kinetic factor, a half step taken as
    a full one or a misordered wavenumber table breaks it."""
    n, L = (64, 32), (2 * np.pi, 4.0)
    dx = L[0] / n[0]
    k0 = 2 * np.pi * 2 / L[0]            # two periods over the box: on the grid
    h = 2 * dx / k0                      # each half step moves one cell
    steps = 3
    x = W.coords(n[0], L[0])[:, None]
    y = W.coords(n[1], L[1])[None, :]
    # narrow enough that the periodic wrap of the tails is below 1e-10
    psi = np.exp(-(x - 0.3) ** 2 / (2 * 0.4 ** 2) - y ** 2 / (2 * 0.5 ** 2)) * (1 + 0.2j * y)
    kw = dict(G=1.0, alpha_Y=0.3, lambda_Y=1.5, g_local=0.4)
    boost = np.exp(1j * k0 * x)
    moved = O.evolve(boost * psi, h, steps, L, **kw)
    rest = O.evolve(psi, h, steps, L, **kw)
    t = steps * h
    want = np.exp(-0.5j * k0 * k0 * t) * boost * np.roll(rest, steps * 2, axis=0)
    assert np.abs(moved - want).max() < 1e-10 * np.abs(want).max()
    assert O.rel_l2(rest, psi) > 1e-2   # the state evolves


# ----------------------------------------------------------------------------
# Observables: closed forms for a Gaussian
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("d", [2, 3])
def test_observables_of_gaussian(d):
    n = (64,) * d if d == 2 else (32, 32, 32)
    L = (16.0,) * d
    sigma, A, g = 1.2, 0.8, 0.3
    vel = [0.0, 0.5, -0.25][:d]
    vel = [2 * np.pi * 1 / L[0] * v / abs(v) if v else 0.0 for v in vel]   # on-grid boosts
    c = [0.0] * d
    c[-1] = 2 * L[-1] / n[-1] * 4                                        # a node
    lump = W.Lump(tuple(c), sigma, A, tuple(vel))
    psi = W.gaussian_lumps(n, L, [lump])
    obs = O.observables(psi, L, G=0.0, g_local=g)
    mass = A * A * (np.pi * sigma * sigma) ** (d / 2)
    assert math.isclose(obs["mass"], mass, rel_tol=1e-10)
    ekin = A * A * (d * (np.pi * sigma ** 2) ** (d / 2) / (4 * sigma ** 2)
                    + 0.5 * sum(v * v for v in vel) * (np.pi * sigma ** 2) ** (d / 2))
    assert math.isclose(obs["e_kin"], ekin, rel_tol=1e-9)
    enl = 0.5 * g * A ** 4 * (np.pi * sigma * sigma / 2) ** (d / 2)
    assert math.isclose(obs["e_nl"], enl, rel_tol=1e-10)
    for a in range(d):
        assert abs(obs["centroid"][a] - c[a]) < 1e-10
        assert abs(obs["momentum"][a] - mass * vel[a]) < 1e-9


@pytest.mark.parametrize("d", [2, 3])
def test_potential_energy_of_gaussian(d):
    n = (32,) * d
    L = (10.0,) * d
    s = 1.0                                    # psi = exp(-|x|^2/(2 s^2)) -> rho = exp(-|x|^2/s^2)
    lump = W.Lump((0.0,) * d, s, 1.0, (0.0,) * d)
    psi = W.gaussian_lumps(n, L, [lump])
    G, al, lam = 0.9, 0.5, 1.5
    obs = O.observables(psi, L, G=G, alpha_Y=al, lambda_Y=lam)
    ms = np.arange(-24, 25)
    ks = np.stack([g.ravel() for g in np.meshgrid(*[2 * np.pi * ms / L[a] for a in range(d)],
                                                  indexing="ij")], 1)
    k2 = (ks ** 2).sum(1)
    k2 = k2[k2 > 0]
    K = -4 * np.pi * G * (1 / k2 + al / (k2 + 1 / lam ** 2))
    rhohat = (np.pi * s * s) ** (d / 2) * np.exp(-k2 * s * s / 4)
    epot = 0.5 * float((K * rhohat ** 2).sum()) / float(np.prod(L))
    assert math.isclose(obs["e_pot"], epot, rel_tol=1e-9)

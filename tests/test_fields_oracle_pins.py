"""Pins of the coupled-fields oracle (oracle/fields_oracle.py) against what the
mathematics fixes (CPU only).

The coupled system shares one potential V[rho] and one local term g rho of the
total density rho = sum_j |psi_j|^2.  Each pin ties the oracle to something
other than itself: the single-field oracle in the cases that reduce to it
(one field; M equal copies of psi / sqrt(M), whose total density is |psi|^2),
the invariance of the dynamics under a constant unitary mixing of the fields,
the separate mass conservation of every field, the sign of the mutual
attraction under Newton's kernel, and second-order convergence of the
Hamiltonian.  A per-field density in place of the total one, a missing cross
term, or a dropped 1/2 in E_pot fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
import oracle.fields_oracle as F
import workloads as W

KW = dict(G=1.0, alpha_Y=0.3, lambda_Y=2.0, g_local=0.04)


def test_one_field_is_the_single_field_oracle():
    psis, L, _ = W.random_fields((16, 32), 11, 1)
    out = F.fields_evolve(psis, 0.01, 3, L, **KW)
    ref = O.evolve(psis[0], 0.01, 3, L, **KW)
    assert np.abs(out[0] - ref).max() <= 1e-13 * np.abs(ref).max()
    o1, o2 = F.fields_observables(psis, L, **KW), O.observables(psis[0], L, **KW)
    for k in ("mass", "e_kin", "e_pot", "e_nl"):
        assert o1[k] == pytest.approx(o2[k], rel=1e-13, abs=1e-13)


@pytest.mark.parametrize("m", [2, 3])
def test_equal_copies_follow_the_single_field_of_the_total_density(m):
    # M copies of psi / sqrt(M): rho = |psi|^2, so every copy is evolve(psi) / sqrt(M)
    psis, L, _ = W.random_fields((32, 16), 21, 1)
    psi = psis[0]
    v = 0.2 * np.cos(2 * math.pi * W.coords(32, L[0]) / L[0])[:, None] * np.ones((1, 16))
    copies = np.stack([psi / math.sqrt(m)] * m)
    out = F.fields_evolve(copies, 0.02, 4, L, v_ext=v, **KW)
    ref = O.evolve(psi, 0.02, 4, L, v_ext=v, **KW) / math.sqrt(m)
    for j in range(m):
        assert np.abs(out[j] - ref).max() <= 1e-12 * np.abs(ref).max()
    o1 = F.fields_observables(copies, L, v_ext=v, **KW)
    o2 = O.observables(psi, L, v_ext=v, **KW)
    for k in ("mass", "e_kin", "e_pot", "e_nl", "e_total"):
        assert o1[k] == pytest.approx(o2[k], rel=1e-12, abs=1e-13), k
    for a in range(2):
        assert o1["centroid"][a] == pytest.approx(o2["centroid"][a], abs=1e-12)
        assert o1["momentum"][a] == pytest.approx(o2["momentum"][a], abs=1e-12)


def test_unitary_mixing_commutes_with_the_step():
    # rho and V are invariant under psi -> U psi (U unitary, constant), and every
    # sub-step acts on each field alike, so evolve(U psi) = U evolve(psi)
    psis, L, _ = W.random_fields((16, 16, 8), 31, 3, L=(8.0, 8.0, 6.0))
    rng = np.random.default_rng(5)
    U, _ = np.linalg.qr(rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3)))
    mix = lambda x: np.tensordot(U, x, axes=1)
    a = F.fields_evolve(mix(psis), 0.02, 3, L, **KW)
    b = mix(F.fields_evolve(psis, 0.02, 3, L, **KW))
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    # and the dynamics is not trivial: field 0 alone evolves differently
    solo = O.evolve(psis[0], 0.02, 3, L, **KW)
    assert O.rel_l2(F.fields_evolve(psis, 0.02, 3, L, **KW)[0], solo) > 1e-3


def test_every_field_keeps_its_own_mass():
    psis, L, _ = W.random_fields((32, 32), 41, 3)
    psis = psis * np.array([1.0, 0.5, 0.25])[:, None, None]
    dV = O.cell_volume((32, 32), L)
    m0 = dV * (np.abs(psis) ** 2).sum(axis=(1, 2))
    out = F.fields_evolve(psis, 0.02, 10, L, **KW)
    m1 = dV * (np.abs(out) ** 2).sum(axis=(1, 2))
    assert np.allclose(m1, m0, rtol=1e-12, atol=0)
    assert len(set(np.round(m0, 6))) == 3


def test_newton_attraction_pulls_the_two_fields_together():
    # a lump of each field at rest, at x = -d and x = +d: Newton's kernel (G > 0)
    # is attractive, so the centroids approach; with G = 0 they do not move
    n, L, d = (64, 32), (24.0, 12.0), 3.0
    lump = lambda c: W.gaussian_lumps(n, L, [W.Lump((c, 0.0), 1.2, 1.0, (0.0, 0.0))])
    psis = np.stack([lump(-d), lump(+d)])
    def centroids(G):
        out = F.fields_evolve(psis, 0.02, 40, L, G=G, alpha_Y=0.0, lambda_Y=1.0, g_local=0.0)
        return [F.fields_observables(out[j:j + 1], L)["centroid"][0] for j in range(2)]
    c0, c1 = centroids(2.0)
    assert c0 > -d + 0.02 and c1 < d - 0.02
    f0, f1 = centroids(0.0)
    assert abs(f0 + d) < 1e-6 and abs(f1 - d) < 1e-6


def test_hamiltonian_drift_is_second_order():
    psis, L, _ = W.random_fields((32, 32), 51, 2)
    kw = dict(G=1.0, alpha_Y=0.2, lambda_Y=2.0, g_local=0.5)
    H0 = F.fields_observables(psis, L, **kw)["e_total"]
    drift = []
    for h, k in ((0.02, 20), (0.01, 40)):
        out = F.fields_evolve(psis, h, k, L, **kw)
        drift.append(abs(F.fields_observables(out, L, **kw)["e_total"] - H0))
    assert drift[0] > 1e-9
    assert 3.0 < drift[0] / drift[1] < 5.0

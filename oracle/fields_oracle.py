"""CPU FP64 oracle of several coupled wave functions (Sec. II, below Eqs. 1-2:
the system generalizes to multiple wave functions coupled through its
nonlinearities).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this module.  The CUDA library shares
no code with it and never calls it.

Reading (the paper states the generalization without equations): M fields
psi_j share one index change, as beams in one nonlocal medium do.  Each obeys
Eq. 1 with the same A,
    i dpsi_j/dt = A lap(psi_j) + (V + V_ext + g rho) psi_j,
    V = F^-1[K F rho],  rho = sum_j |psi_j|^2,
with K the kernel of Eq. 2 (or the Newton + Yukawa kernel of Eq. 9).  With
M = 1 this is Eqs. 1-2.  The symmetric split step of Sec. III carries over
field by field: Kin(h/2) on every field, the potential sub-step (rho, hence
V, is unchanged by it, so it is exact), Kin(h/2) on every field.

Observables of the coupled system: mass, E_kin and momentum are sums over the
fields; E_pot = (1/2) dV sum V rho (+ dV sum V_ext rho) and
E_nl = (g/2) dV sum rho^2 of the total density, so that H = E_kin + E_pot +
E_nl is the Hamiltonian whose variation gives the equations above; centroids
are those of the total density.
"""
from typing import Dict, Optional, Sequence

import numpy as np

from .sn_oracle import (KIND_NMC, TWO_PI, _axis_view, cell_volume, fftn, k_squared, kinetic,
                        potential, wavenumbers)


def total_density(psis: np.ndarray) -> np.ndarray:
    """rho = sum_j |psi_j|^2 over the leading (field) axis."""
    psis = np.asarray(psis, dtype=np.complex128)
    return (psis * np.conj(psis)).real.sum(axis=0)


def fields_nonlinear(psis: np.ndarray, h: float, L: Sequence[float], G: float = 1.0,
                     alpha_Y: float = 0.0, lambda_Y: float = 1.0, g_local: float = 0.0,
                     v_ext: Optional[np.ndarray] = None, kind: int = KIND_NMC, B: float = 1.0,
                     C: float = 0.0, D: float = 0.0) -> np.ndarray:
    """Exact potential sub-step of every field: psi_j exp(-i (V + V_ext + g rho) h),
    V and rho of the total density (unchanged by the sub-step)."""
    rho = total_density(psis)
    U = potential(rho, L, G, alpha_Y, lambda_Y, kind, B, C, D) + g_local * rho
    if v_ext is not None:
        U = U + v_ext
    return np.asarray(psis, dtype=np.complex128) * np.exp(-1j * U * h)[None]


def fields_strang_step(psis: np.ndarray, h: float, L: Sequence[float], G: float = 1.0,
                       alpha_Y: float = 0.0, lambda_Y: float = 1.0, g_local: float = 0.0,
                       coeff_lap: float = -0.5, v_ext: Optional[np.ndarray] = None,
                       kind: int = KIND_NMC, B: float = 1.0, C: float = 0.0,
                       D: float = 0.0) -> np.ndarray:
    """One symmetric split step of the coupled fields."""
    psis = np.stack([kinetic(p, 0.5 * h, L, coeff_lap) for p in psis])
    psis = fields_nonlinear(psis, h, L, G, alpha_Y, lambda_Y, g_local, v_ext, kind, B, C, D)
    return np.stack([kinetic(p, 0.5 * h, L, coeff_lap) for p in psis])


def fields_evolve(psis: np.ndarray, h: float, nsteps: int, L: Sequence[float],
                  **kernel) -> np.ndarray:
    """nsteps plain Strang steps of the fields (array of shape (M, *n))."""
    psis = np.asarray(psis, dtype=np.complex128)
    for _ in range(nsteps):
        psis = fields_strang_step(psis, h, L, **kernel)
    return psis


def fields_observables(psis: np.ndarray, L: Sequence[float], G: float = 1.0,
                       alpha_Y: float = 0.0, lambda_Y: float = 1.0, g_local: float = 0.0,
                       coeff_lap: float = -0.5, v_ext: Optional[np.ndarray] = None,
                       kind: int = KIND_NMC, B: float = 1.0, C: float = 0.0,
                       D: float = 0.0) -> Dict[str, object]:
    """Observables of the coupled system (module docstring)."""
    psis = np.asarray(psis, dtype=np.complex128)
    n = psis.shape[1:]
    d = len(n)
    N = int(np.prod(n))
    dV = cell_volume(n, L)
    rho = total_density(psis)
    k2 = k_squared(n, L)
    pk2 = np.zeros(n)
    for p in psis:
        pk = fftn(p)
        pk2 = pk2 + (pk * np.conj(pk)).real
    mass = dV * float(rho.sum())
    e_kin = -coeff_lap * dV / N * float((k2 * pk2).sum())
    V = potential(rho, L, G, alpha_Y, lambda_Y, kind, B, C, D)
    e_pot = 0.5 * dV * float((V * rho).sum())
    if v_ext is not None:
        e_pot += dV * float((v_ext * rho).sum())
    e_nl = 0.5 * g_local * dV * float((rho * rho).sum())
    centroid, momentum = [], []
    for a in range(d):
        x = -0.5 * L[a] + np.arange(n[a]) * (L[a] / n[a])
        ph = _axis_view(np.exp(1j * TWO_PI * x / L[a]), a, d)
        centroid.append(L[a] / TWO_PI * float(np.angle((rho * ph).sum())))
        ka = wavenumbers(n[a], L[a]).copy()
        ka[n[a] // 2] = 0.0
        momentum.append(dV / N * float((_axis_view(ka, a, d) * pk2).sum()))
    return dict(mass=mass, e_kin=e_kin, e_pot=e_pot, e_nl=e_nl, e_total=e_kin + e_pot + e_nl,
                centroid=centroid, momentum=momentum)

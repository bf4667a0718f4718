"""CPU FP64 oracle of the Schroedinger-Newton form of the self-gravitating
fluid (Sec. II B, Eq. 16) under General Relativity and the pure non-minimal
matter-curvature coupling (alpha = 0, Eq. 15 with Eqs. 11-13).

TEST INFRASTRUCTURE ONLY.  Only the test suite and the smoke check import
this module; the CUDA library shares no code with it.

Eq. 16:  i nu psi_t = -(nu^2/2) lap psi + [nu^2 V_B + phi_N + phi_C + V_p] psi,
written for the solver as
    i psi_t = -(nu/2) lap psi + (U / nu) psi,   U = nu^2 V_B + phi_N + phi_C + V_p,
with, for rho = |psi|^2 (all potentials depend on rho only, so the potential
sub-step exp(-i U h / nu) is exact, as in Sec. III):
  * Bohm potential  V_B = lap(sqrt rho) / (2 sqrt rho);
  * Newtonian part  lap phi_N = beta(r) lap rho + gamma(r) rho   (Eq. 15),
    solved spectrally with the k = 0 mode removed (lap rho spectral too);
  * coupling part   phi_C = ln[1 - (r0/(r + r0))^lambda]          (Eq. 13);
  * pressure        V_p = w ln rho (n = 1), n w / (n - 1) rho^(n-1) otherwise
                    (Eq. 17, P = w rho^n);
  * gamma(r) = 1/2 (GR) or 1/2 [1 - (r0/(r + r0))^lambda] (NMC)   (Eq. 11);
    beta(r) = 0 (GR) or lambda (r0/(r + r0))^lambda / (r + r0)    (Eq. 12);
    phi_C = 0 under GR; r0 = M / (4 pi).
Readings (the paper leaves them open): r is the distance from the box centre
(the node x = 0); r is taken as max(r, h/2), h the smallest grid spacing, so
that phi_C (-infinity at r = 0) stays finite; sqrt rho and ln rho use
max(rho, rho_floor).

Built on the FFT, wavenumbers and kinetic propagator of sn_oracle.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Dict, Sequence, Tuple

import numpy as np

from .sn_oracle import _axis_view, fftn, k_squared, kinetic, cell_volume

GR, NMC = 0, 1


@dataclass
class CosmoParams:
    nu: float = 1.0         # analogue of hbar (psi = sqrt(rho) exp(i Phi / nu))
    w: float = 1.02         # polytropic coefficient, P = w rho^n
    n_poly: float = 1.0     # polytropic exponent
    model: int = NMC        # GR or NMC
    lam: float = 1.0        # NMC strength lambda (Eqs. 11-13)
    M: float = 25.0         # mass setting r0 = M / (4 pi)
    rho_floor: float = 1e-12
    floor_mode: int = 0     # 0: max(rho, floor) under sqrt and ln; 1: rho + floor (smooth)


def radius(n: Sequence[int], L: Sequence[float]) -> np.ndarray:
    """Distance from the box centre (x_j = -L/2 + j L/n, so x = 0 is node n/2),
    floored at half the smallest grid spacing."""
    d = len(n)
    r2 = np.zeros(tuple(n))
    for a in range(d):
        x = -0.5 * L[a] + np.arange(n[a]) * (L[a] / n[a])
        r2 = r2 + _axis_view(x * x, a, d)
    hmin = min(L[a] / n[a] for a in range(d))
    return np.maximum(np.sqrt(r2), 0.5 * hmin)


def coupling_profiles(n: Sequence[int], L: Sequence[float],
                      p: CosmoParams) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """gamma(r), beta(r), phi_C(r) on the grid (Eqs. 11-13)."""
    r = radius(n, L)
    if p.model == GR:
        return np.full(r.shape, 0.5), np.zeros(r.shape), np.zeros(r.shape)
    r0 = p.M / (4.0 * math.pi)
    q = (r0 / (r + r0)) ** p.lam
    gamma = 0.5 * (1.0 - q)
    beta = p.lam * q / (r + r0)
    phi_c = np.log(1.0 - q)
    return gamma, beta, phi_c


def spectral_laplacian(f: np.ndarray, L: Sequence[float]) -> np.ndarray:
    """lap f = F^-1[-k^2 F f] for real f (periodic box)."""
    return fftn(-k_squared(f.shape, L) * fftn(f), inverse=True).real


def floored(rho: np.ndarray, rho_floor: float, floor_mode: int = 0) -> np.ndarray:
    """rho as it enters sqrt and ln: max(rho, floor), or rho + floor (floor_mode 1)."""
    return rho + rho_floor if floor_mode == 1 else np.maximum(rho, rho_floor)


def bohm_potential(rho: np.ndarray, L: Sequence[float], rho_floor: float,
                   floor_mode: int = 0) -> np.ndarray:
    """V_B = lap(sqrt rho) / (2 sqrt rho), sqrt rho of the floored rho."""
    a = np.sqrt(floored(rho, rho_floor, floor_mode))
    return spectral_laplacian(a, L) / (2.0 * a)


def newtonian_potential(rho: np.ndarray, L: Sequence[float], gamma: np.ndarray,
                        beta: np.ndarray) -> np.ndarray:
    """phi_N with lap phi_N = beta lap rho + gamma rho (Eq. 15), k = 0 removed."""
    src = beta * spectral_laplacian(rho, L) + gamma * rho
    k2 = k_squared(rho.shape, L)
    mult = np.zeros_like(k2)
    nz = k2 > 0
    mult[nz] = -1.0 / k2[nz]
    return fftn(mult * fftn(src), inverse=True).real


def pressure_potential(rho: np.ndarray, p: CosmoParams) -> np.ndarray:
    """V_p of P = w rho^n: w ln rho (n = 1) or n w / (n - 1) rho^(n-1)."""
    r = floored(rho, p.rho_floor, p.floor_mode)
    if p.n_poly == 1.0:
        return p.w * np.log(r)
    return p.n_poly * p.w / (p.n_poly - 1.0) * r ** (p.n_poly - 1.0)


def total_potential(rho: np.ndarray, L: Sequence[float], p: CosmoParams) -> np.ndarray:
    """U = nu^2 V_B + phi_N + phi_C + V_p (the bracket of Eq. 16)."""
    gamma, beta, phi_c = coupling_profiles(rho.shape, L, p)
    return (p.nu ** 2 * bohm_potential(rho, L, p.rho_floor, p.floor_mode)
            + newtonian_potential(rho, L, gamma, beta) + phi_c + pressure_potential(rho, p))


def cosmo_step(psi: np.ndarray, h: float, L: Sequence[float], p: CosmoParams) -> np.ndarray:
    """One symmetric split step of Eq. 16: Kin(h/2) with A = -nu/2, then
    psi exp(-i U h / nu), then Kin(h/2)."""
    psi = kinetic(psi, 0.5 * h, L, -0.5 * p.nu)
    rho = (psi * np.conj(psi)).real
    psi = psi * np.exp(-1j * total_potential(rho, L, p) * h / p.nu)
    return kinetic(psi, 0.5 * h, L, -0.5 * p.nu)


def cosmo_evolve(psi: np.ndarray, h: float, nsteps: int, L: Sequence[float],
                 p: CosmoParams) -> np.ndarray:
    psi = np.asarray(psi, dtype=np.complex128)
    for _ in range(nsteps):
        psi = cosmo_step(psi, h, L, p)
    return psi


def internal_energy(rho: np.ndarray, p: CosmoParams) -> np.ndarray:
    """eps(rho) with d eps / d rho = V_p (P = w rho^n): w rho (ln rho - 1) for n = 1,
    w rho^n / (n - 1) otherwise; rho under ln and the power taken as max(rho, floor)."""
    r = floored(rho, p.rho_floor, p.floor_mode)
    if p.n_poly == 1.0:
        return p.w * rho * (np.log(r) - 1.0)
    return p.w * rho * r ** (p.n_poly - 1.0) / (p.n_poly - 1.0)


def fluid_energies(psi: np.ndarray, L: Sequence[float], p: CosmoParams) -> Dict[str, float]:
    """Energies of Eq. 16 in the solver's form i psi_t = -(nu/2) lap psi + (U/nu) psi,
    whose Hamiltonian is int [(nu/2)|grad psi|^2] + (1/nu) times the functional
    whose rho-derivative is U:
      e_kin = (nu/2) int |grad psi|^2                     (spectral, as sn_oracle),
      e_pot = (1/nu) [ (1/2) int phi_N rho + int phi_C rho ],
      e_nl  = (1/nu) [ -(nu^2/2) int |grad sqrt rho|^2 + int eps(rho) ]
    (-(nu^2/2) int |grad a|^2 has rho-derivative nu^2 V_B, eps has V_p; the
    gradient term is -int a lap a on the periodic box, a = sqrt(max(rho, floor))).
    Under GR (phi_N linear and symmetric in rho) e_kin + e_pot + e_nl is the
    conserved Hamiltonian of the exact flow."""
    psi = np.asarray(psi, dtype=np.complex128)
    rho = (psi * np.conj(psi)).real
    dV = cell_volume(psi.shape, L)
    gamma, beta, phi_c = coupling_profiles(psi.shape, L, p)
    phi_n = newtonian_potential(rho, L, gamma, beta)
    a = np.sqrt(floored(rho, p.rho_floor, p.floor_mode))
    grad_a2 = -float((a * spectral_laplacian(a, L)).sum()) * dV
    psik = fftn(psi)
    e_kin = 0.5 * p.nu * dV / psi.size * float((k_squared(psi.shape, L) * np.abs(psik) ** 2).sum())
    e_pot = dV * (0.5 * float((phi_n * rho).sum()) + float((phi_c * rho).sum())) / p.nu
    e_nl = (-0.5 * p.nu ** 2 * grad_a2 + dV * float(internal_energy(rho, p).sum())) / p.nu
    return dict(e_kin=e_kin, e_pot=e_pot, e_nl=e_nl, e_total=e_kin + e_pot + e_nl)


def mass(psi: np.ndarray, L: Sequence[float]) -> float:
    return cell_volume(psi.shape, L) * float((np.abs(psi) ** 2).sum())


def profile_summary(psi: np.ndarray, L: Sequence[float]) -> Dict[str, float]:
    """Central density and the mass fraction within radius L_min/8 of the centre."""
    rho = np.abs(psi) ** 2
    r = radius(psi.shape, L)
    c = tuple(s // 2 for s in psi.shape)
    inner = r <= min(L) / 8.0
    return dict(rho_centre=float(rho[c]), inner_fraction=float(rho[inner].sum() / rho.sum()))

"""Seeded synthetic initial conditions and parameter sets.

The paper starts every run from a Gaussian distribution of matter (Sec. IV)
and maps a fluid velocity to the phase of psi through the Madelung transform
psi = sqrt(rho) exp(i Phi / nu), v = grad Phi (Sec. II B, Eq. 15-16).  The
workloads below follow that recipe: each lump is a Gaussian in |psi| with a
linear phase ramp (a uniform velocity).  Only input construction lives here;
no step of the split-step method does.

Conventions (shared by every consumer of these arrays):
  * arrays are C-ordered, slowest axis first: 2D (ny, nx), 3D (nz, ny, nx);
  * node-centred periodic coordinates x_j = -L/2 + j L / n per axis;
  * a lump is A exp(-|d|^2 / (2 sigma^2)) exp(i v . d) with d the
    minimum-image displacement from the lump centre, so lumps wrap around the
    periodic box and the ramp is continuous across the lump.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

from .rng import SplitMix64


@dataclass
class Lump:
    centre: Tuple[float, ...]     # per axis, array order (z, y, x) / (y, x)
    sigma: float
    amplitude: float
    velocity: Tuple[float, ...]   # per axis, array order


@dataclass
class KernelParams:
    """Parameters of the potential and the local term.

    kind 0: Green's multiplier K(k) = -4 pi G [1/k^2 + alpha_Y/(k^2 + 1/lambda_Y^2)];
    kind 1: Eq. 2 with constants B, C <= 0, D, K(k) = B D / (C - k^2);
    K(0) := 0 for both; local term g |psi|^2; Laplacian coefficient A (Eq. 1).
    """
    G: float = 1.0
    alpha_Y: float = 0.0
    lambda_Y: float = 1.0
    g_local: float = 0.0
    coeff_lap: float = -0.5
    kind: int = 0
    B: float = 1.0
    C: float = 0.0
    D: float = 0.0


@dataclass
class Workload:
    name: str
    n: Tuple[int, ...]
    L: Tuple[float, ...]
    lumps: List[Lump]
    kernel: KernelParams
    dt: float
    nsteps: int
    meta: dict = field(default_factory=dict)

    @property
    def ndim(self) -> int:
        return len(self.n)

    @property
    def cells(self) -> int:
        return int(np.prod(self.n))

    def psi0(self, dtype=np.complex128) -> np.ndarray:
        return gaussian_lumps(self.n, self.L, self.lumps).astype(dtype)


def coords(n: int, L: float) -> np.ndarray:
    """Node-centred periodic coordinates x_j = -L/2 + j L/n."""
    return -0.5 * L + np.arange(n, dtype=np.float64) * (L / n)


def _min_image(x: np.ndarray, c: float, L: float) -> np.ndarray:
    d = x - c
    return d - L * np.round(d / L)


def gaussian_lumps(n: Sequence[int], L: Sequence[float], lumps: Sequence[Lump]) -> np.ndarray:
    """Superposition of separable Gaussian lumps with phase ramps (complex128)."""
    n = tuple(int(v) for v in n)
    L = tuple(float(v) for v in L)
    psi = np.zeros(n, dtype=np.complex128)
    for lump in lumps:
        term = None
        for a in range(len(n)):
            d = _min_image(coords(n[a], L[a]), lump.centre[a], L[a])
            f = np.exp(-d * d / (2.0 * lump.sigma ** 2)) * np.exp(1j * lump.velocity[a] * d)
            shape = [1] * len(n)
            shape[a] = n[a]
            f = f.reshape(shape)
            term = f if term is None else term * f
        psi += lump.amplitude * term
    return psi


# ----------------------------------------------------------------------------
# The five workload families
# ----------------------------------------------------------------------------

def centred_gaussian_2d(n: int = 128, L: float = 20.0, sigma: float = 1.5,
                        dt: float = 1e-3, nsteps: int = 200) -> Workload:
    """2D Newtonian collapse of one centred Gaussian (G=1, no local term)."""
    lumps = [Lump((0.0, 0.0), sigma, 1.0, (0.0, 0.0))]
    return Workload("sn2d_gaussian_128", (n, n), (L, L), lumps,
                    KernelParams(G=1.0, alpha_Y=0.0, lambda_Y=1.0, g_local=0.0), dt, nsteps)


def head_on_collision_3d(n: int = 128, L: float = 40.0, dt: float = 5e-3,
                         nsteps: int = 2000) -> Workload:
    """Two lumps (sigma 2) at x = +-8 moving towards each other at |v| = 0.3."""
    lumps = [Lump((0.0, 0.0, -8.0), 2.0, 1.0, (0.0, 0.0, +0.3)),
             Lump((0.0, 0.0, +8.0), 2.0, 1.0, (0.0, 0.0, -0.3))]
    k = KernelParams(G=1.0, alpha_Y=0.1, lambda_Y=5.0, g_local=0.01)
    return Workload("sn3d_collision_128", (n, n, n), (L, L, L), lumps, k, dt, nsteps)


def nbody_3d(n: int = 256, L: float = 80.0, alpha_Y: float = 0.1, seed: int = 3000,
             nlumps: int = 16, dt: float = 1e-2, nsteps: int = 1000) -> Workload:
    """16 seeded lumps: sigma~U[1,2.5], A~U[0.5,1], centres U(box), v~N(0,0.2)."""
    r = SplitMix64(seed)
    lumps = []
    for _ in range(nlumps):
        sigma = r.uniform(1.0, 2.5)
        amp = r.uniform(0.5, 1.0)
        centre = tuple(r.uniform(-0.5 * L, 0.5 * L) for _ in range(3))
        vel = tuple(r.normal(0.0, 0.2) for _ in range(3))
        lumps.append(Lump(centre, sigma, amp, vel))
    k = KernelParams(G=1.0, alpha_Y=alpha_Y, lambda_Y=10.0, g_local=0.0)
    return Workload(f"sn3d_nbody_{n}", (n, n, n), (L, L, L), lumps, k, dt, nsteps,
                    meta={"seed": seed})


SCAN_SIZES = (128, 256, 512, 1024)


def scan_instance_2d(i: int, sizes: Sequence[int] = SCAN_SIZES, L: float = 40.0,
                     dt: float = 1e-2, nsteps: int = 500, seed: int | None = None) -> Workload:
    """Instance i of the batched parameter scan (seed 4000 + i unless given)."""
    seed = 4000 + i if seed is None else seed
    r = SplitMix64(seed)
    n = int(sizes[min(int(r.uniform() * len(sizes)), len(sizes) - 1)])
    nl = r.randint(2, 8)
    lumps = []
    for _ in range(nl):
        sigma = r.uniform(1.0, 3.0)
        amp = r.uniform(0.5, 1.0)
        centre = tuple(r.uniform(-0.5 * L, 0.5 * L) for _ in range(2))
        vel = tuple(r.normal(0.0, 0.2) for _ in range(2))
        lumps.append(Lump(centre, sigma, amp, vel))
    k = KernelParams(G=1.0, alpha_Y=r.uniform(0.0, 1.0), lambda_Y=r.uniform(1.0, 20.0),
                     g_local=r.uniform(0.0, 0.05))
    return Workload(f"scan2d_{i}_{n}", (n, n), (L, L), lumps, k, dt, nsteps,
                    meta={"seed": seed, "index": i})


def optical_beams_2d(n: int = 1024, L: float = 100.0, seed: int = 6000, sigma_nl: float = 5.0,
                     zeta_mu_over_kappa: float = 2.0, dt: float = 1e-2,
                     nsteps: int = 500) -> Workload:
    """Beams in a thermo-optical medium (Eq. 3 with the nonlocal index of Eq. 4):
    2 to 6 Gaussian beams (waist U[2, 4], amplitude U[0.5, 1], centres uniform,
    transverse tilts N(0, 0.3)) in the transverse plane, nonlocal length
    sigma_nl; kernel kind 1 with C = -1/sigma_nl^2, D = -zeta mu / kappa, B = 1."""
    r = SplitMix64(seed)
    nb = r.randint(2, 6)
    lumps = []
    for _ in range(nb):
        sigma = r.uniform(2.0, 4.0)
        amp = r.uniform(0.5, 1.0)
        centre = tuple(r.uniform(-0.5 * L, 0.5 * L) for _ in range(2))
        vel = tuple(r.normal(0.0, 0.3) for _ in range(2))
        lumps.append(Lump(centre, sigma, amp, vel))
    k = KernelParams(G=0.0, g_local=0.0, kind=1, B=1.0, C=-1.0 / (sigma_nl * sigma_nl),
                     D=-zeta_mu_over_kappa)
    return Workload(f"optical2d_{n}", (n, n), (L, L), lumps, k, dt, nsteps, meta={"seed": seed})


def random_small(n: Sequence[int], seed: int, L: float | Sequence[float] = 10.0,
                 nlumps: int = 3, kernel: KernelParams | None = None) -> Workload:
    """Small seeded grid for parity tests: lumps sized to the box."""
    r = SplitMix64(seed)
    n = tuple(int(v) for v in n)
    Ls = tuple(float(v) for v in (L if isinstance(L, (list, tuple)) else [L] * len(n)))
    lumps = []
    for _ in range(nlumps):
        sigma = r.uniform(0.08, 0.2) * min(Ls)
        amp = r.uniform(0.5, 1.0)
        centre = tuple(r.uniform(-0.5 * Ls[a], 0.5 * Ls[a]) for a in range(len(n)))
        vel = tuple(r.normal(0.0, 1.0) for _ in range(len(n)))
        lumps.append(Lump(centre, sigma, amp, vel))
    if kernel is None:
        kernel = KernelParams(G=1.0, alpha_Y=r.uniform(0.0, 0.5), lambda_Y=r.uniform(1.0, 4.0),
                              g_local=r.uniform(0.0, 0.05))
    return Workload(f"small_{'x'.join(map(str, n))}_{seed}", n, Ls, lumps, kernel, 1e-2, 1,
                    meta={"seed": seed})


def random_fields(n: Sequence[int], seed: int, count: int, L: float | Sequence[float] = 10.0,
                  kernel: KernelParams | None = None):
    """count coupled fields for the multi-wave-function tests: field j is the
    state of random_small(n, seed + j) (its own lumps and ramps); the kernel is
    field 0's unless one is given.  Returns (psis of shape (count, *n), L, kernel)."""
    ws = [random_small(n, seed + j, L) for j in range(count)]
    psis = np.stack([w.psi0() for w in ws])
    return psis, ws[0].L, (kernel if kernel is not None else ws[0].kernel)

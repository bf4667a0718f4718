"""CPU FP64 oracle of the generalized Schroedinger-Newton split-step solver.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this module.  The CUDA library shares
no code with it and never calls it.

It is the plain, slow, readable statement of what the solver computes:

* Eq. 1 (Sec. II):  i dpsi/dt = A lap(psi) + B phi psi + G(|psi|^2) psi, with
  B = 1 and the local term G(|psi|^2) = g |psi|^2.
* Eq. 2 (Sec. II):  lap(phi) + C phi = D |psi|^2, solved spectrally
  (Sec. III: "also with spectral methods").  Two kernel kinds:
  - KIND_NMC: a sum of two such equations gives the Newton + Yukawa
    multiplier of the modified Poisson equation (Eq. 9 with constant
    coefficients; Eq. 14 is its alpha -> 0 limit), with B = 1:
      K(k) = -4 pi G [ 1/k^2 + alpha_Y / (k^2 + 1/lambda_Y^2) ],  K(0) := 0.
  - KIND_POISSON: Eq. 2 itself with constants B (Eq. 1), C <= 0 and D, the
    form of the optical media of Sec. II A (thermo-optical, Eq. 4:
    C = -1/sigma^2; nematic liquid crystals, Eq. 5: C = -2q/nu, D = -2/nu):
      K(k) = B D / (C - k^2),  K(0) := 0.
* Sec. III: the symmetric split-step Fourier method,
      S(h) = Kin(h/2) o Nl(h) o Kin(h/2),
  Kin(tau) = F^-1 exp(i A k^2 tau) F          (exact free propagator of Eq. 1),
  Nl(h) psi = exp(-i (V + V_ext + g |psi|^2) h) psi,  V = F^-1[K F |psi|^2]
  (exact propagator of the potential part: |psi|^2, hence V, is constant
  under it).

Conventions: arrays are C-ordered, slowest axis first; x_j = -L/2 + j L/n;
F is the unnormalised DFT F(f)_k = sum_j f_j exp(-2 pi i j k / n) and its
inverse carries 1/n; k_j = (2 pi / L) (j if j < n/2 else j - n).

The DFT is computed by this module's own iterative radix-2 Cooley-Tukey FFT,
pinned against the O(n^2) definition (dft_naive) and against numpy.fft in the
tests.  Everything runs in float64 / complex128.
"""
from __future__ import annotations

import math
from typing import Dict, Optional, Sequence, Tuple

import numpy as np

TWO_PI = 2.0 * math.pi
KIND_NMC = 0      # Newton + Yukawa kernel of Eq. 9 / Eq. 14 (G, alpha_Y, lambda_Y)
KIND_POISSON = 1  # Eq. 2 with constants B, C, D (Eqs. 4 and 5)


# ----------------------------------------------------------------------------
# Discrete Fourier transform
# ----------------------------------------------------------------------------

def dft_naive(x: np.ndarray, axis: int = -1, inverse: bool = False) -> np.ndarray:
    """O(n^2) DFT along one axis, straight from the definition.

    Forward: X_k = sum_j x_j exp(-2 pi i j k / n); inverse: (1/n) sum_k X_k exp(+...).
    The phase index j*k is reduced mod n before the exponential.
    """
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[axis]
    j = np.arange(n)
    jk = np.outer(j, j) % n
    sign = 1.0 if inverse else -1.0
    W = np.exp(sign * 1j * TWO_PI * jk / n)
    y = np.moveaxis(np.tensordot(W, np.moveaxis(x, axis, 0), axes=([1], [0])), 0, axis)
    return y / n if inverse else y


def _bit_reverse_permutation(n: int) -> np.ndarray:
    bits = n.bit_length() - 1
    idx = np.arange(n)
    rev = np.zeros(n, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    return rev


def fft_radix2(x: np.ndarray, axis: int = -1, inverse: bool = False) -> np.ndarray:
    """Iterative radix-2 decimation-in-time FFT along one axis (n a power of two).

    After the bit-reversal permutation, stage m (m = 1, 2, 4, ...) merges pairs
    of length-m transforms E, O into a length-2m transform:
        X[k] = E[k] + w^k O[k],  X[k+m] = E[k] - w^k O[k],  w = exp(-+2 pi i/(2m)).
    The inverse uses the conjugate twiddles and divides by n.
    """
    x = np.asarray(x, dtype=np.complex128)
    axis = axis % x.ndim
    n = x.shape[axis]
    if n & (n - 1):
        raise ValueError("fft_radix2 needs a power-of-two length")
    pre = int(np.prod(x.shape[:axis], dtype=np.int64))
    post = int(np.prod(x.shape[axis + 1:], dtype=np.int64))
    y = np.take(x, _bit_reverse_permutation(n), axis=axis).reshape(pre, n, post)
    sign = 1.0 if inverse else -1.0
    m = 1
    while m < n:
        blocks = y.reshape(pre, n // (2 * m), 2, m, post)
        w = np.exp(sign * 1j * TWO_PI * np.arange(m) / (2 * m)).reshape(m, 1)
        e = blocks[:, :, 0]
        o = blocks[:, :, 1] * w
        out = np.empty_like(blocks)
        np.add(e, o, out=out[:, :, 0])
        np.subtract(e, o, out=out[:, :, 1])
        y = out.reshape(pre, n, post)
        m *= 2
    if inverse:
        y = y / n
    return y.reshape(x.shape)


def fftn(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Multi-dimensional DFT as one radix-2 FFT per axis (separability)."""
    y = np.asarray(x, dtype=np.complex128)
    for a in range(y.ndim):
        y = fft_radix2(y, axis=a, inverse=inverse)
    return y


# ----------------------------------------------------------------------------
# Grid quantities
# ----------------------------------------------------------------------------

def wavenumbers(n: int, L: float) -> np.ndarray:
    """k_j = (2 pi / L) (j if j < n/2 else j - n)."""
    j = np.arange(n)
    return (TWO_PI / L) * np.where(j < n // 2, j, j - n).astype(np.float64)


def _axis_view(v: np.ndarray, a: int, ndim: int) -> np.ndarray:
    shape = [1] * ndim
    shape[a] = v.shape[0]
    return v.reshape(shape)


def k_squared(n: Sequence[int], L: Sequence[float]) -> np.ndarray:
    d = len(n)
    k2 = np.zeros(tuple(n), dtype=np.float64)
    for a in range(d):
        k2 = k2 + _axis_view(wavenumbers(n[a], L[a]) ** 2, a, d)
    return k2


def cell_volume(n: Sequence[int], L: Sequence[float]) -> float:
    return float(np.prod([L[a] / n[a] for a in range(len(n))]))


def green_multiplier(n: Sequence[int], L: Sequence[float], G: float = 1.0,
                     alpha_Y: float = 0.0, lambda_Y: float = 1.0, kind: int = KIND_NMC,
                     B: float = 1.0, C: float = 0.0, D: float = 0.0) -> np.ndarray:
    """Spectral solution operator of the Poisson-type equation (Eq. 2, Eq. 9):
    the potential B phi entering Eq. 1 is F^-1[K F rho].

    Eq. 2 in Fourier space reads (C - k^2) phi_k = D rho_k, so one equation
    gives K = B D / (C - k^2).
    KIND_NMC (B = 1):
      Newton part (C = 0, D = 4 pi G):  phi_k = -4 pi G rho_k / k^2;
      Yukawa part (C = -1/lambda_Y^2, D = 4 pi G alpha_Y):
          phi_k = -4 pi G alpha_Y rho_k / (k^2 + 1/lambda_Y^2).
    KIND_POISSON: K = B D / (C - k^2) with the caller's B, C <= 0, D.
    The whole multiplier is zero at k = 0 (removes the mean density).
    """
    k2 = k_squared(n, L)
    K = np.zeros_like(k2)
    nz = k2 > 0
    if kind == KIND_POISSON:
        if not C <= 0.0:
            raise ValueError("KIND_POISSON needs C <= 0")
        K[nz] = B * D / (C - k2[nz])
        return K
    if kind != KIND_NMC:
        raise ValueError(f"unknown kernel kind {kind}")
    K[nz] = -4.0 * math.pi * G * (1.0 / k2[nz])
    if alpha_Y != 0.0:
        K[nz] += -4.0 * math.pi * G * alpha_Y / (k2[nz] + 1.0 / (lambda_Y * lambda_Y))
    return K


# ----------------------------------------------------------------------------
# Sub-steps of the symmetric split-step Fourier method (Sec. III)
# ----------------------------------------------------------------------------

def kinetic(psi: np.ndarray, tau: float, L: Sequence[float], coeff_lap: float = -0.5) -> np.ndarray:
    """Exact propagator of i dpsi/dt = A lap(psi) over time tau (Eq. 1, A = coeff_lap).

    In Fourier space d(psi_k)/dt = i A k^2 psi_k, so psi_k <- exp(i A k^2 tau) psi_k.
    """
    k2 = k_squared(psi.shape, L)
    return fftn(np.exp(1j * coeff_lap * k2 * tau) * fftn(psi), inverse=True)


def potential(rho: np.ndarray, L: Sequence[float], G: float = 1.0, alpha_Y: float = 0.0,
              lambda_Y: float = 1.0, kind: int = KIND_NMC, B: float = 1.0, C: float = 0.0,
              D: float = 0.0) -> np.ndarray:
    """V = F^-1[K F rho] (Eq. 2 solved spectrally, Sec. III); real for real rho."""
    K = green_multiplier(rho.shape, L, G, alpha_Y, lambda_Y, kind, B, C, D)
    return fftn(K * fftn(rho), inverse=True).real


def nonlinear(psi: np.ndarray, h: float, L: Sequence[float], G: float = 1.0,
              alpha_Y: float = 0.0, lambda_Y: float = 1.0, g_local: float = 0.0,
              v_ext: Optional[np.ndarray] = None, kind: int = KIND_NMC, B: float = 1.0,
              C: float = 0.0, D: float = 0.0) -> np.ndarray:
    """Exact propagator of i dpsi/dt = (V + V_ext + g|psi|^2) psi over time h.

    |psi|^2 does not change under this sub-step, so V is computed once from the
    input density and the update is the pointwise phase exp(-i(...) h).
    """
    rho = (psi * np.conj(psi)).real
    V = potential(rho, L, G, alpha_Y, lambda_Y, kind, B, C, D)
    if v_ext is not None:
        V = V + v_ext
    return psi * np.exp(-1j * (V + g_local * rho) * h)


def strang_step(psi: np.ndarray, h: float, L: Sequence[float], G: float = 1.0,
                alpha_Y: float = 0.0, lambda_Y: float = 1.0, g_local: float = 0.0,
                coeff_lap: float = -0.5, v_ext: Optional[np.ndarray] = None,
                kind: int = KIND_NMC, B: float = 1.0, C: float = 0.0,
                D: float = 0.0) -> np.ndarray:
    """One symmetric split step S(h) = Kin(h/2) Nl(h) Kin(h/2) (Sec. III)."""
    psi = kinetic(psi, 0.5 * h, L, coeff_lap)
    psi = nonlinear(psi, h, L, G, alpha_Y, lambda_Y, g_local, v_ext, kind, B, C, D)
    return kinetic(psi, 0.5 * h, L, coeff_lap)


def evolve(psi: np.ndarray, h: float, nsteps: int, L: Sequence[float], **kernel) -> np.ndarray:
    """nsteps plain (unmerged) Strang steps."""
    psi = np.asarray(psi, dtype=np.complex128)
    for _ in range(nsteps):
        psi = strang_step(psi, h, L, **kernel)
    return psi


def kernel_kwargs(kp) -> Dict[str, float]:
    """Keyword arguments of the sub-steps from a parameter object with the same field
    names (kind, B, C, D when it has them)."""
    kw = dict(G=kp.G, alpha_Y=kp.alpha_Y, lambda_Y=kp.lambda_Y, g_local=kp.g_local,
              coeff_lap=kp.coeff_lap)
    for name in ("kind", "B", "C", "D"):
        if hasattr(kp, name):
            kw[name] = getattr(kp, name)
    return kw


# ----------------------------------------------------------------------------
# Observables at an integer step
# ----------------------------------------------------------------------------

def observables(psi: np.ndarray, L: Sequence[float], G: float = 1.0, alpha_Y: float = 0.0,
                lambda_Y: float = 1.0, g_local: float = 0.0, coeff_lap: float = -0.5,
                v_ext: Optional[np.ndarray] = None, kind: int = KIND_NMC, B: float = 1.0,
                C: float = 0.0, D: float = 0.0) -> Dict[str, object]:
    """Mass, Hamiltonian parts, periodic centroids and momentum of psi.

    H is the conserved energy of Eq. 1 with the Hartree potential:
      E_kin = -A (dV/N) sum_k k^2 |F psi|^2          (= int (1/2)|grad psi|^2 for A = -1/2)
      E_pot = (1/2) dV sum V rho  (+ dV sum V_ext rho; the 1/2 counts each pair once)
      E_nl  = (g/2) dV sum rho^2
    centroid_a = (L_a / 2 pi) arg(sum rho exp(2 pi i x_a / L_a)) (circular mean),
    momentum_a = (dV/N) sum_k k_a |F psi|^2 with the Nyquist k_a taken as 0.
    """
    psi = np.asarray(psi, dtype=np.complex128)
    n = psi.shape
    d = psi.ndim
    N = psi.size
    dV = cell_volume(n, L)
    rho = (psi * np.conj(psi)).real
    psik = fftn(psi)
    pk2 = (psik * np.conj(psik)).real
    mass = dV * rho.sum()
    e_kin = -coeff_lap * dV / N * float((k_squared(n, L) * pk2).sum())
    V = potential(rho, L, G, alpha_Y, lambda_Y, kind, B, C, D)
    e_pot = 0.5 * dV * float((V * rho).sum())
    if v_ext is not None:
        e_pot += dV * float((v_ext * rho).sum())
    e_nl = 0.5 * g_local * dV * float((rho * rho).sum())
    centroid = []
    momentum = []
    for a in range(d):
        x = -0.5 * L[a] + np.arange(n[a]) * (L[a] / n[a])
        ph = _axis_view(np.exp(1j * TWO_PI * x / L[a]), a, d)
        centroid.append(L[a] / TWO_PI * float(np.angle((rho * ph).sum())))
        ka = wavenumbers(n[a], L[a]).copy()
        ka[n[a] // 2] = 0.0
        momentum.append(dV / N * float((_axis_view(ka, a, d) * pk2).sum()))
    return dict(mass=float(mass), e_kin=e_kin, e_pot=e_pot, e_nl=e_nl,
                e_total=e_kin + e_pot + e_nl, centroid=centroid, momentum=momentum)


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    """||a - b|| / ||b||."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))

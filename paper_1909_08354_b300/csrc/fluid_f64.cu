// Elementwise kernels of the self-gravitating fluid model (Sec. II B, Eq. 16)
// on complex128 grids.  The axis FFTs are those of the plain FP64 step; these
// kernels form the fields the potential needs and apply the potential
// sub-step
//     psi <- psi exp(-i U h / nu),  U = nu^2 V_B + phi_N + phi_C + V_p,
// with V_B = lap(sqrt rho) / (2 sqrt rho) (Bohm), phi_N from
// lap phi_N = beta(r) lap rho + gamma(r) rho (Eq. 15), phi_C (Eq. 13) and
// V_p of P = w rho^n (Eq. 17).  U depends on rho = |psi|^2 only, which the
// sub-step leaves unchanged, so the sub-step is exact.
#include <cuda_runtime.h>

#include "pdl.cuh"
#include "sn_internal.h"

namespace sn {
namespace {

constexpr int kThreads = 256;

unsigned blocks_for(long long cells) {
  const long long b = (cells + kThreads - 1) / kThreads;
  return (unsigned)(b < 148LL * 32 ? b : 148LL * 32);
}

__device__ __forceinline__ double density(const double2* psi, long long c) {
  const double2 z = psi[c];
  return z.x * z.x + z.y * z.y;
}

// rho as it enters sqrt and ln: max(rho, floor) or rho + floor (smooth)
__device__ __forceinline__ double floored(double rho, double floor, int mode) {
  return mode == 1 ? rho + floor : fmax(rho, floor);
}

// wa = rho + i sqrt(max(rho, floor)): two real fields in one complex array, so
// that one FFT, the Laplacian multiplier and one inverse FFT give both
// Laplacians (real part: lap rho, imaginary part: lap sqrt rho)
__global__ void prep_kernel(const double2* psi, double2* wa, double floor, int mode,
                            long long cells) {
  pdl_allow_next();
  pdl_wait_prev();
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
       c += (long long)gridDim.x * blockDim.x) {
    const double rho = density(psi, c);
    wa[c] = make_double2(rho, sqrt(floored(rho, floor, mode)));
  }
}

// w *= -k^2 scale (spectral Laplacian; scale carries the 1/N of the inverse)
__global__ void lap_mult_kernel(double2* w, long long n0, long long n1, long long n2,
                                const double* k20, const double* k21, const double* k22,
                                double scale) {
  pdl_allow_next();
  pdl_wait_prev();
  const long long cells = n0 * n1 * n2;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
       c += (long long)gridDim.x * blockDim.x) {
    const long long i2 = c % n2, i1 = (c / n2) % n1, i0 = c / (n2 * n1);
    const double k2 = (k20 ? k20[i0] : 0.0) + k21[i1] + k22[i2];
    const double f = -k2 * scale;
    const double2 z = w[c];
    w[c] = make_double2(z.x * f, z.y * f);
  }
}

// w = beta lap(rho) + gamma rho with lap(rho) = Re wlap; beta == NULL means
// beta = 0, gamma == NULL means gamma = 1/2 (GR)
__global__ void source_kernel(const double2* psi, const double2* wlap, double2* w,
                              const double* gamma, const double* beta, long long cells) {
  pdl_allow_next();
  pdl_wait_prev();
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
       c += (long long)gridDim.x * blockDim.x) {
    const double g = gamma ? gamma[c] : 0.5;
    double s = g * density(psi, c);
    if (beta) s = fma(beta[c], wlap[c].x, s);
    w[c] = make_double2(s, 0.0);
  }
}

__global__ void phase_kernel(double2* psi, const double2* wphi, const double2* wlap,
                             const double* phi_c, FluidPhase p, long long cells) {
  pdl_allow_next();
  pdl_wait_prev();
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
       c += (long long)gridDim.x * blockDim.x) {
    const double2 z = psi[c];
    const double rf = floored(z.x * z.x + z.y * z.y, p.rho_floor, p.floor_mode);
    const double vb = wlap[c].y / (2.0 * sqrt(rf));  // lap sqrt rho / (2 sqrt rho)
    const double vp = p.n_poly == 1.0 ? p.w * log(rf) : p.cp * pow(rf, p.n_poly - 1.0);
    double u = fma(p.nu * p.nu, vb, wphi[c].x + vp);
    if (phi_c) u += phi_c[c];
    double sn, cs;
    sincos(u * p.h_over_nu, &sn, &cs);
    psi[c] = make_double2(z.x * cs + z.y * sn, z.y * cs - z.x * sn);  // psi exp(-i U h / nu)
  }
}

}  // namespace

cudaError_t launch_fluid_prep_f64(const double2* psi, double2* wa, double floor, int floor_mode,
                                  long long cells, cudaStream_t s) {
  return launch_pdl(prep_kernel, dim3(blocks_for(cells)), dim3(kThreads), 0, s, psi, wa, floor,
                    floor_mode, cells);
}

cudaError_t launch_lap_mult_f64(double2* w, const int* n, int ndim, const double* const* k2,
                                double scale, cudaStream_t s) {
  const long long n0 = ndim == 3 ? n[0] : 1, n1 = ndim == 3 ? n[1] : n[0];
  const long long n2 = ndim == 3 ? n[2] : n[1];
  const double* a0 = ndim == 3 ? k2[0] : nullptr;
  const double* a1 = ndim == 3 ? k2[1] : k2[0];
  const double* a2 = ndim == 3 ? k2[2] : k2[1];
  return launch_pdl(lap_mult_kernel, dim3(blocks_for(n0 * n1 * n2)), dim3(kThreads), 0, s, w, n0, n1, n2,
                    a0, a1, a2, scale);
}

cudaError_t launch_fluid_source_f64(const double2* psi, const double2* wlap, double2* w,
                                    const double* gamma, const double* beta, long long cells,
                                    cudaStream_t s) {
  return launch_pdl(source_kernel, dim3(blocks_for(cells)), dim3(kThreads), 0, s, psi, wlap, w, gamma,
                    beta, cells);
}

cudaError_t launch_fluid_phase_f64(double2* psi, const double2* wphi, const double2* wlap,
                                   const double* phi_c, const FluidPhase& p, long long cells,
                                   cudaStream_t s) {
  return launch_pdl(phase_kernel, dim3(blocks_for(cells)), dim3(kThreads), 0, s, psi, wphi, wlap, phi_c,
                    p, cells);
}

}  // namespace sn

// Plain FP64 split step and FP64 observables.
//
// The plain step is the symmetric split-step Fourier method of Sec. III
// written the textbook way on complex128, one kernel per operation and no
// merging of sub-steps: full 3D (or 2D) FFT, kinetic multiplier, inverse FFT;
// density, FFT, Green's multiplier (Eq. 2 / Eq. 9), inverse FFT, nonlinear
// phase; and the second kinetic half step.  It is the double-precision
// reference path on the GPU.  The observables (mass, Hamiltonian parts,
// centroids, momentum) use the same FP64 axis FFTs and block reductions with a
// fixed order, so repeated calls give bit-identical results.
#include "sn_fft.cuh"
#include "pdl.cuh"
#include "sn_internal.h"

using namespace snfft;

namespace sn {
namespace {

__device__ __forceinline__ cx<double> ldd(const double2* p) {
  const double2 v = *p;
  return {v.x, v.y};
}
__device__ __forceinline__ void std2(double2* p, cx<double> v) { *p = make_double2(v.re, v.im); }

template <int N>
struct LinesF64 {
  // lines per CTA: keeps shared memory under ~110 KB for the long lines
  static constexpr int value = N <= 256 ? 16 : (N == 512 ? 8 : 4);
  // a grid of few lines (a 2D plane of 256^2 or less, say) would leave most
  // SMs idle at `value` lines a CTA: one warp's worth of lines a CTA instead
  // (at least one line), the same per-line arithmetic
  static constexpr int few = Plan<N>::T >= 32 ? 1 : 32 / Plan<N>::T;
};

template <int N, bool STRIDED, int SIGN, int LPB>
__global__ void __launch_bounds__(LPB * Plan<N>::T)
fft_f64_kernel(double2* data, long long outer, long long inner, const double2* tw) {
  using P = Plan<N>;
  constexpr int E = P::E, T = P::T, NT = LPB * T, LS = P::LS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<double>* tw_sm = reinterpret_cast<cx<double>*>(smem_raw);
  cx<double>* lines = tw_sm + P::TWN;
  const int tid = threadIdx.x;
  const int l = STRIDED ? (tid % LPB) : (tid / T);
  const int t = STRIDED ? (tid / LPB) : (tid % T);
  size_t base, stride;
  bool valid;
  if constexpr (STRIDED) {
    const long long o = blockIdx.y, i = (long long)blockIdx.x * LPB + l;
    valid = i < inner;
    base = (size_t)o * N * inner + i;
    stride = inner;
  } else {
    const long long o = (long long)blockIdx.x * LPB + l;
    valid = o < outer;
    base = (size_t)o * N;
    stride = 1;
  }
  pdl_allow_next();
  for (int k = tid; k < P::TWN; k += NT) tw_sm[k] = ldd(tw + k);
  __syncthreads();
  pdl_wait_prev();  // the lines come from the previous kernel
  cx<double> v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    cx<double> z = {0.0, 0.0};
    if (valid) z = ldd(data + base + (size_t)(t + T * m) * stride);
    v[m] = z;
  }
  line_transform<double, N, SIGN>(v, lines + l * LS, tw_sm, t, true);
  if (valid) {
#pragma unroll
    for (int m = 0; m < E; ++m) std2(data + base + (size_t)(t + T * m) * stride, v[m]);
  }
}

template <int N, bool STRIDED, int SIGN, int LPB>
cudaError_t launch_fft_lpb(double2* d, long long outer, long long inner, const double2* tw,
                           cudaStream_t s) {
  constexpr size_t smem = (size_t)(Plan<N>::TWN + LPB * Plan<N>::LS) * sizeof(cx<double>);
  auto kern = fft_f64_kernel<N, STRIDED, SIGN, LPB>;
  static bool attr_of[kDeviceSlots] = {};
  bool& attr = attr_of[device_slot()];
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 block(LPB * Plan<N>::T);
  dim3 grid = STRIDED ? dim3((unsigned)((inner + LPB - 1) / LPB), (unsigned)outer)
                      : dim3((unsigned)((outer + LPB - 1) / LPB));
  return launch_pdl(kern, grid, block, smem, s, d, outer, inner, tw);
}

// Lines per CTA: LinesF64::value, or LinesF64::few when that leaves fewer
// than two CTAs per SM of the B300's 148 (the results are the same bits).
template <int N, bool STRIDED, int SIGN>
cudaError_t launch_fft_t(double2* d, long long outer, long long inner, const double2* tw,
                         cudaStream_t s) {
  constexpr int LPB = LinesF64<N>::value, FEW = LinesF64<N>::few;
  const long long lines = outer * inner;
  if (FEW < LPB && (lines + LPB - 1) / LPB < 2 * 148)
    return launch_fft_lpb<N, STRIDED, SIGN, FEW>(d, outer, inner, tw, s);
  return launch_fft_lpb<N, STRIDED, SIGN, LPB>(d, outer, inner, tw, s);
}

template <int N>
cudaError_t fft_dispatch(bool strided, int sign, double2* d, long long outer, long long inner,
                         const double2* tw, cudaStream_t s) {
  if (strided) {
    return sign < 0 ? launch_fft_t<N, true, -1>(d, outer, inner, tw, s)
                    : launch_fft_t<N, true, +1>(d, outer, inner, tw, s);
  }
  return sign < 0 ? launch_fft_t<N, false, -1>(d, outer, inner, tw, s)
                  : launch_fft_t<N, false, +1>(d, outer, inner, tw, s);
}

struct Dims {
  long long n0, n1, n2;  // padded to 3D: (n0, n1, n2) = (1, ny, nx) in 2D
};
__host__ Dims dims_of(const int* n, int ndim) {
  if (ndim == 2) return {1, n[0], n[1]};
  return {n[0], n[1], n[2]};
}

constexpr int kEwThreads = 256;
inline unsigned ew_blocks(long long cells) {
  long long b = (cells + kEwThreads - 1) / kEwThreads;
  return (unsigned)(b < 148LL * 32 ? b : 148LL * 32);
}

__global__ void mult_kinetic_kernel(double2* psi, Dims d, const double2* m0, const double2* m1,
                                    const double2* m2) {
  pdl_allow_next();
  pdl_wait_prev();
  const long long cells = d.n0 * d.n1 * d.n2;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
       c += (long long)gridDim.x * blockDim.x) {
    const long long i2 = c % d.n2, i1 = (c / d.n2) % d.n1, i0 = c / (d.n2 * d.n1);
    cx<double> f = ldd(m2 + i2);
    f = cmul(f, ldd(m1 + i1));
    if (m0 != nullptr) f = cmul(f, ldd(m0 + i0));
    std2(psi + c, cmul(ldd(psi + c), f));
  }
}

__global__ void density_kernel(const double2* psi, double2* w, long long cells, bool accumulate) {
  pdl_allow_next();
  pdl_wait_prev();
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
       c += (long long)gridDim.x * blockDim.x) {
    const cx<double> z = ldd(psi + c);
    w[c] = make_double2((accumulate ? w[c].x : 0.0) + cnorm2(z), 0.0);
  }
}

__global__ void green_kernel(double2* w, Dims d, const double* k20, const double* k21,
                             const double* k22, double cN, double cY, double mu2, double cL) {
  pdl_allow_next();
  pdl_wait_prev();
  const long long cells = d.n0 * d.n1 * d.n2;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
       c += (long long)gridDim.x * blockDim.x) {
    const long long i2 = c % d.n2, i1 = (c / d.n2) % d.n1, i0 = c / (d.n2 * d.n1);
    const double k2 = (k20 ? k20[i0] : 0.0) + k21[i1] + k22[i2];
    const double K = ((k2 > 0.0) ? (cN / k2 + cY / (k2 + mu2)) : 0.0) + cL;
    std2(w + c, cscale(ldd(w + c), K));
  }
}

__global__ void phase_kernel(double2* psi, const double2* w, const double* vext, double h,
                             double gh, long long cells) {
  pdl_allow_next();
  pdl_wait_prev();
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
       c += (long long)gridDim.x * blockDim.x) {
    const cx<double> z = ldd(psi + c);
    double th = w[c].x + gh * cnorm2(z);
    if (vext != nullptr) th += vext[c] * h;
    double s, co;
    sincos(th, &s, &co);
    std2(psi + c, {z.re * co + z.im * s, z.im * co - z.re * s});
  }
}

__global__ void widen_kernel(const float2* in, double2* out, long long cells) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
       c += (long long)gridDim.x * blockDim.x) {
    const float2 z = in[c];
    out[c] = make_double2((double)z.x, (double)z.y);
  }
}

template <class Z>
__global__ void total_amplitude_kernel(const Z* psi, int count, long long cells, double2* out) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
       c += (long long)gridDim.x * blockDim.x) {
    double rho = 0.0;
    for (int j = 0; j < count; ++j) {
      const Z z = psi[(size_t)j * cells + c];
      rho += (double)z.x * (double)z.x + (double)z.y * (double)z.y;
    }
    out[c] = make_double2(sqrt(rho), 0.0);
  }
}

// ---- observables: per-block partial sums added to partials, fixed order -----

template <int NQ>
__device__ __forceinline__ void block_reduce_store(double (&acc)[NQ], double* partials, int q0) {
  __shared__ double red[32][NQ];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double v = acc[q];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
    partials[(size_t)blockIdx.x * Q_NUM + q0 + threadIdx.x] += s;
  }
}

// cs_a[j] = (cos, sin)(2 pi x_j / L_a) per axis, padded axes hold a single (1, 0)
__global__ void obs_space_kernel(const double2* psi, const double* vext, Dims d,
                                 const double2* cs0, const double2* cs1, const double2* cs2,
                                 double* partials) {
  // Q_MASS, Q_RHO2, Q_VEXT, then (cos, sin) sums per axis (padded 3D order)
  constexpr int NQ = 9;
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
  const long long cells = d.n0 * d.n1 * d.n2;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
       c += (long long)gridDim.x * blockDim.x) {
    const long long i2 = c % d.n2, i1 = (c / d.n2) % d.n1, i0 = c / (d.n2 * d.n1);
    const double rho = cnorm2(ldd(psi + c));
    acc[0] += rho;
    acc[1] += rho * rho;
    if (vext != nullptr) acc[2] += rho * vext[c];
    const double2 a0 = cs0[i0], a1 = cs1[i1], a2 = cs2[i2];
    acc[3] += rho * a0.x;
    acc[4] += rho * a0.y;
    acc[5] += rho * a1.x;
    acc[6] += rho * a1.y;
    acc[7] += rho * a2.x;
    acc[8] += rho * a2.y;
  }
  block_reduce_store<NQ>(acc, partials, 0);
}

__global__ void obs_kaxis_kernel(const double2* fa, Dims d, int axis3, const double* kax,
                                 double* partials, int q0) {
  // sum k_a^2 |F_a psi|^2 and sum k_a |F_a psi|^2 (Nyquist k_a taken as 0 for the latter)
  double acc[2] = {0.0, 0.0};
  const long long cells = d.n0 * d.n1 * d.n2;
  const long long na = axis3 == 0 ? d.n0 : (axis3 == 1 ? d.n1 : d.n2);
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
       c += (long long)gridDim.x * blockDim.x) {
    const long long i2 = c % d.n2, i1 = (c / d.n2) % d.n1, i0 = c / (d.n2 * d.n1);
    const long long j = axis3 == 0 ? i0 : (axis3 == 1 ? i1 : i2);
    const double p = cnorm2(ldd(fa + c));
    const double k = kax[j];
    acc[0] += k * k * p;
    if (2 * j != na) acc[1] += k * p;
  }
  block_reduce_store<2>(acc, partials, q0);
}

__global__ void obs_green_kernel(const double2* rh, Dims d, const double* k20, const double* k21,
                                 const double* k22, double cN, double cY, double mu2,
                                 double* partials) {
  double acc[1] = {0.0};
  const long long cells = d.n0 * d.n1 * d.n2;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
       c += (long long)gridDim.x * blockDim.x) {
    const long long i2 = c % d.n2, i1 = (c / d.n2) % d.n1, i0 = c / (d.n2 * d.n1);
    const double k2 = (k20 ? k20[i0] : 0.0) + k21[i1] + k22[i2];
    const double K = (k2 > 0.0) ? (cN / k2 + cY / (k2 + mu2)) : 0.0;
    acc[0] += K * cnorm2(ldd(rh + c));
  }
  block_reduce_store<1>(acc, partials, Q_EPOT);
}

// Energy terms of the self-gravitating fluid (Eq. 16), into partials[0..3]:
// sum rho phi_N, sum rho phi_C, sum eps(rho) (the polytropic internal energy,
// d eps / d rho = V_p), sum a lap(a) with a = sqrt(max(rho, floor)).
__global__ void obs_fluid_kernel(const double2* psi, const double2* wphi, const double2* wlap,
                                 const double* phi_c, double w, double n_poly, double floor,
                                 int mode, long long cells, double* partials) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
       c += (long long)gridDim.x * blockDim.x) {
    const double rho = cnorm2(ldd(psi + c));
    const double rf = mode == 1 ? rho + floor : fmax(rho, floor);
    acc[0] += rho * wphi[c].x;
    if (phi_c != nullptr) acc[1] += rho * phi_c[c];
    acc[2] += n_poly == 1.0 ? w * rho * (log(rf) - 1.0)
                            : w * rho * pow(rf, n_poly - 1.0) / (n_poly - 1.0);
    acc[3] += sqrt(rf) * wlap[c].y;
  }
  block_reduce_store<4>(acc, partials, 0);
}

__global__ void obs_finish_kernel(const double* partials, int nblocks, double* out) {
  const int q = threadIdx.x;
  if (q >= Q_NUM) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partials[(size_t)b * Q_NUM + q];
  out[q] = s;
}

}  // namespace

cudaError_t launch_fft_f64(int N, bool strided, int sign, double2* d, long long outer,
                           long long inner, const double2* tw, cudaStream_t s) {
  switch (N) {
    case 8: return fft_dispatch<8>(strided, sign, d, outer, inner, tw, s);
    case 16: return fft_dispatch<16>(strided, sign, d, outer, inner, tw, s);
    case 32: return fft_dispatch<32>(strided, sign, d, outer, inner, tw, s);
    case 64: return fft_dispatch<64>(strided, sign, d, outer, inner, tw, s);
    case 128: return fft_dispatch<128>(strided, sign, d, outer, inner, tw, s);
    case 256: return fft_dispatch<256>(strided, sign, d, outer, inner, tw, s);
    case 512: return fft_dispatch<512>(strided, sign, d, outer, inner, tw, s);
    case 1024: return fft_dispatch<1024>(strided, sign, d, outer, inner, tw, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_mult_kinetic_f64(double2* psi, const int* n, int ndim, const double2* const* m,
                                    cudaStream_t s) {
  const Dims d = dims_of(n, ndim);
  const double2* m0 = ndim == 3 ? m[0] : nullptr;
  const double2* m1 = ndim == 3 ? m[1] : m[0];
  const double2* m2 = ndim == 3 ? m[2] : m[1];
  return launch_pdl(mult_kinetic_kernel, dim3(ew_blocks(d.n0 * d.n1 * d.n2)), dim3(kEwThreads), 0, s,
                    psi, d, m0, m1, m2);
}

cudaError_t launch_density_f64(const double2* psi, double2* w, long long cells, cudaStream_t s,
                               bool accumulate) {
  return launch_pdl(density_kernel, dim3(ew_blocks(cells)), dim3(kEwThreads), 0, s, psi, w, cells,
                    accumulate);
}

cudaError_t launch_green_f64(double2* w, const int* n, int ndim, const double* const* k2,
                             double cN, double cY, double mu2, cudaStream_t s, double cL) {
  const Dims d = dims_of(n, ndim);
  const double* a0 = ndim == 3 ? k2[0] : nullptr;
  const double* a1 = ndim == 3 ? k2[1] : k2[0];
  const double* a2 = ndim == 3 ? k2[2] : k2[1];
  return launch_pdl(green_kernel, dim3(ew_blocks(d.n0 * d.n1 * d.n2)), dim3(kEwThreads), 0, s, w, d, a0,
                    a1, a2, cN, cY, mu2, cL);
}

cudaError_t launch_phase_f64(double2* psi, const double2* w, const double* vext, double h,
                             double gh, long long cells, cudaStream_t s) {
  return launch_pdl(phase_kernel, dim3(ew_blocks(cells)), dim3(kEwThreads), 0, s, psi, w, vext, h, gh,
                    cells);
}

cudaError_t launch_widen_f32_to_f64(const float2* in, double2* out, long long cells,
                                    cudaStream_t s) {
  widen_kernel<<<ew_blocks(cells), kEwThreads, 0, s>>>(in, out, cells);
  return cudaGetLastError();
}

cudaError_t launch_total_amplitude(const void* psi, bool f32, int count, long long cells,
                                   double2* out, cudaStream_t s) {
  if (f32)
    total_amplitude_kernel<<<ew_blocks(cells), kEwThreads, 0, s>>>(
        static_cast<const float2*>(psi), count, cells, out);
  else
    total_amplitude_kernel<<<ew_blocks(cells), kEwThreads, 0, s>>>(
        static_cast<const double2*>(psi), count, cells, out);
  return cudaGetLastError();
}

cudaError_t launch_obs_space(const double2* psi, const double* vext, const int* n, int ndim,
                             const double2* const* cs, const double2* cs_one, double* partials,
                             cudaStream_t s) {
  const double2* c0 = ndim == 3 ? cs[0] : cs_one;
  const double2* c1 = ndim == 3 ? cs[1] : cs[0];
  const double2* c2 = ndim == 3 ? cs[2] : cs[1];
  obs_space_kernel<<<kObsBlocks, kEwThreads, 0, s>>>(psi, vext, dims_of(n, ndim), c0, c1, c2,
                                                     partials);
  return cudaGetLastError();
}

cudaError_t launch_obs_kaxis(const double2* fa, const int* n, int ndim, int axis,
                             const double* kax, double* partials, cudaStream_t s) {
  const int axis3 = ndim == 3 ? axis : axis + 1;
  obs_kaxis_kernel<<<kObsBlocks, kEwThreads, 0, s>>>(fa, dims_of(n, ndim), axis3, kax, partials,
                                                     Q_EKIN0 + 2 * axis);
  return cudaGetLastError();
}

cudaError_t launch_obs_green(const double2* rhohat, const int* n, int ndim,
                             const double* const* k2, double cN, double cY, double mu2,
                             double* partials, cudaStream_t s) {
  const double* a0 = ndim == 3 ? k2[0] : nullptr;
  const double* a1 = ndim == 3 ? k2[1] : k2[0];
  const double* a2 = ndim == 3 ? k2[2] : k2[1];
  obs_green_kernel<<<kObsBlocks, kEwThreads, 0, s>>>(rhohat, dims_of(n, ndim), a0, a1, a2, cN, cY,
                                                     mu2, partials);
  return cudaGetLastError();
}

cudaError_t launch_obs_fluid(const double2* psi, const double2* wphi, const double2* wlap,
                             const double* phi_c, double w, double n_poly, double floor,
                             int floor_mode, long long cells, double* partials, cudaStream_t s) {
  obs_fluid_kernel<<<kObsBlocks, 256, 0, s>>>(psi, wphi, wlap, phi_c, w, n_poly, floor,
                                              floor_mode, cells, partials);
  return cudaGetLastError();
}

cudaError_t launch_obs_finish(const double* partials, int nq, double* out, cudaStream_t s) {
  (void)nq;
  obs_finish_kernel<<<1, 32, 0, s>>>(partials, kObsBlocks, out);
  return cudaGetLastError();
}

}  // namespace sn

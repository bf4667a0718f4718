// Observables of a complex64 grid from FP32 line transforms with FP64 sums
// (the quantities of sn_obs: mass, e_kin, e_pot, e_nl, centroids, momenta;
// Sec. III's conserved quantities of Eqs. 1-2).
//
// The FP64 path widens the state and runs FP64 FFTs, which the B300's FP64
// rate makes the dominant cost; here every transform is the FP32 line
// transform of the step (sn_fft.cuh) and only the sums are FP64:
//   spectral sums, one read-only pass per axis a: the forward FFT of each line
//     along a, then sum k_a^2 |F_a psi|^2 and sum k_a |F_a psi|^2 (1D Parseval
//     per line: the sum over lines equals the sum over the full spectrum of
//     the same weights, as the FP64 path takes it);
//   density pass along the last axis h: rho = sum_j |psi_j|^2, the real-space
//     sums (mass, rho^2, V_ext rho), the forward FFT of rho along h written
//     out as its half spectrum [k][line], and the centroid sums from the
//     line modes (x_a = -L_a / 2 + j L_a / n_a): sum rho exp(2 pi i x_h / L_h)
//     = -conj(F_h rho (k = 1)) per line, sum rho exp(2 pi i x_a / L_a) =
//     F_h rho (k = 0) exp(2 pi i x_a / L_a) per line for the other axes;
//   (3D: the forward FFT along the middle axis, the step's own half-spectrum
//     pass;)
//   Green's sum along the remaining axis: the forward FFT, then
//     sum w K(k) |F rho|^2 with w = 2 for the half axis' interior modes
//     (Hermitian symmetry), 1 for k_h = 0 and N_h / 2.
// Each CTA keeps its sums per tile in FP32 (16 terms a thread) and adds them
// to FP64 accumulators; it adds its block total to its own row of the partial
// array (one writer per entry, launches in stream order), so the result does
// not depend on scheduling.
#include <cuda_runtime.h>

#include "sn_internal.h"
#include "sn_fft.cuh"

using namespace snfft;

namespace sn {
namespace {

constexpr int kL = 16;  // lines per tile

template <int N>
__host__ __device__ constexpr int obs_threads() { return kL * Plan<N>::T; }

template <int N>
constexpr size_t obs_smem_bytes() {
  // one region for the tile as loaded and for the transform's line buffers
  // (kL lines of LS words), then the twiddles (hi, lo)
  return (size_t)kL * Plan<N>::LS * sizeof(cx<float>) + 2 * (size_t)Plan<N>::TWN * sizeof(cx<float>);
}

// Sum of NQ doubles over the CTA, added by thread 0 to partials[blockIdx.x][q0 + q].
template <int NQ>
__device__ void block_add(double (&acc)[NQ], double* partials, int q0) {
  __shared__ double red[32][NQ];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double s = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp][q] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += red[w][q];
      partials[(size_t)blockIdx.x * Q_NUM + q0 + q] += s;
    }
  }
}

// Lines (outer, inner) of N points, as the passes take them: element p of
// line (o, i) at o N inner + p inner + i.  Tile tau holds lines i0 .. i0 + 15
// of one o (strided, inner > 1) or lines tau * 16 .. + 15 (inner == 1).
struct TileGeom {
  long long outer, inner, tiles_i, count;
  __device__ void at(long long tau, long long& o, long long& i0) const {
    if (inner > 1) {
      o = tau / tiles_i;
      i0 = (tau - o * tiles_i) * kL;
    } else {
      o = tau * kL;
      i0 = 0;
    }
  }
};
__host__ TileGeom tile_geom(long long outer, long long inner) {
  TileGeom g{outer, inner, 1, 0};
  if (inner > 1) {
    g.tiles_i = (inner + kL - 1) / kL;
    g.count = outer * g.tiles_i;
  } else {
    g.count = (outer + kL - 1) / kL;
  }
  return g;
}

// Tile tau of src into the CTA's region (coalesced: position-major rows of 16
// lines for strided lines, line-major rows of stride LS otherwise), then line
// l's pattern-P elements into v; lines past the end read as zero.
template <int N>
__device__ __forceinline__ void load_tile(cx<float> (&v)[Plan<N>::E], cx<float>* region,
                                          const float2* src, const TileGeom& G, long long tau,
                                          int l, int t) {
  using P = Plan<N>;
  constexpr int E = P::E, T = P::T, NT = kL * T, LS = P::LS;
  long long o, i0;
  G.at(tau, o, i0);
  const bool strided = G.inner > 1;
  __syncthreads();  // earlier readers of the region are done
  for (int w = threadIdx.x; w < kL * N; w += NT) {
    if (strided) {
      const int p = w / kL, q = w % kL;
      const bool ok = i0 + q < G.inner;
      const float2 z = ok ? src[(o * N + p) * G.inner + i0 + q] : make_float2(0.f, 0.f);
      region[p * kL + q] = {z.x, z.y};
    } else {
      const int q = w / N, p = w % N;
      const bool ok = o + q < G.outer;
      const float2 z = ok ? src[(o + q) * N + p] : make_float2(0.f, 0.f);
      region[q * LS + p] = {z.x, z.y};
    }
  }
  __syncthreads();
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int p = t + T * m;
    v[m] = strided ? region[p * kL + l] : region[l * LS + p];
  }
}

template <int N>
__device__ __forceinline__ void stage_tw(cx<float>* tw_sm, const float2* tw) {
  constexpr int W = 2 * Plan<N>::TWN;
  for (int k = threadIdx.x; k < W; k += obs_threads<N>()) tw_sm[k] = {tw[k].x, tw[k].y};
}

// ---- spectral sums along one axis -------------------------------------------
// q0: Q_EKIN0 + 2 a (sum k^2 |F psi|^2), q0 + 1 = Q_P0 + 2 a (sum k |F psi|^2,
// the Nyquist mode taken as 0); kscale = 2 pi / L_a.
template <int N>
__global__ void __launch_bounds__(obs_threads<N>(), 1)
spec_sum_kernel(const float2* psi, TileGeom G, const float2* tw, float kscale, double* partials,
                int q0) {
  using P = Plan<N>;
  constexpr int E = P::E, T = P::T;
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* region = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tw_sm = region + kL * P::LS;
  const int l = threadIdx.x % kL, t = threadIdx.x / kL;
  stage_tw<N>(tw_sm, tw);
  double acc[2] = {0.0, 0.0};
  for (long long tau = blockIdx.x; tau < G.count; tau += gridDim.x) {
    cx<float> v[E];
    load_tile<N>(v, region, psi, G, tau, l, t);
    line_transform<float, N, -1, false>(v, region + l * P::LS, tw_sm, t, true);
    float s2 = 0.f, s1 = 0.f;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int k = t + T * m;
      const float kk = (float)(k <= N / 2 ? k : k - N) * kscale;
      const float p = cnorm2(v[m]);
      s2 = fmaf(kk * kk, p, s2);
      if (2 * k != N) s1 = fmaf(kk, p, s1);
    }
    acc[0] += (double)s2;
    acc[1] += (double)s1;
  }
  block_add<2>(acc, partials, q0);
}

// ---- density pass along the last axis h ----------------------------------------
// Lines along h are contiguous (inner == 1); line = c0 n1 + c1 in the padded 3D
// coordinates (c0, c1) of the two axes before h (a 2D grid: c0 = 0, n0 = 1).
struct DensityArgs {
  const float2* psi;   // field 0; field j at psi + j * cells
  int nfields;
  long long cells;
  const float* vext;   // V_ext in psi layout, or NULL
  float2* rh;          // out: half spectrum [N/2 + 1][lines] of rho along h
  int n0, n1;          // padded 3D sizes of the axes before h
};

template <int N>
__global__ void __launch_bounds__(obs_threads<N>(), 1)
density_kernel(DensityArgs a, TileGeom G, const float2* tw, double* partials) {
  using P = Plan<N>;
  constexpr int E = P::E, T = P::T;
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* region = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tw_sm = region + kL * P::LS;
  const int l = threadIdx.x % kL, t = threadIdx.x / kL;
  stage_tw<N>(tw_sm, tw);
  // Q_MASS, Q_RHO2, Q_VEXT, then (cos, sin) sums of padded 3D axes 0, 1, 2 (= h)
  double acc[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const long long lines = G.outer;
  for (long long tau = blockIdx.x; tau < G.count; tau += gridDim.x) {
    cx<float> v[E];
    float rho[E];
#pragma unroll
    for (int m = 0; m < E; ++m) rho[m] = 0.f;
    for (int j = 0; j < a.nfields; ++j) {
      load_tile<N>(v, region, a.psi + (size_t)j * a.cells, G, tau, l, t);
#pragma unroll
      for (int m = 0; m < E; ++m) rho[m] += cnorm2(v[m]);
    }
    const long long line = tau * kL + l;
    const bool valid = line < lines;
    float sm = 0.f, s2 = 0.f, sv = 0.f;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      sm += rho[m];
      s2 = fmaf(rho[m], rho[m], s2);
      if (a.vext != nullptr && valid) sv = fmaf(a.vext[line * N + t + T * m], rho[m], sv);
      v[m] = {rho[m], 0.f};
    }
    acc[0] += (double)sm;
    acc[1] += (double)s2;
    acc[2] += (double)sv;
    line_transform<float, N, -1, false>(v, region + l * P::LS, tw_sm, t, true);
    if (valid) {
      const int c0 = (int)(line / a.n1), c1 = (int)(line - (long long)c0 * a.n1);
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int k = t + T * m;
        if (k <= N / 2) a.rh[(size_t)k * lines + line] = make_float2(v[m].re, v[m].im);
        if (k == 0) {
          // the line's sum of rho times exp(2 pi i x_a / L_a) at its coordinates
          // x_a = -L_a / 2 + c_a L_a / n_a (a 2D grid's padded axis 0 is unused)
          float s0, cc0, s1, cc1;
          sincospif(2.f * (float)c0 / (float)a.n0 - 1.f, &s0, &cc0);
          sincospif(2.f * (float)c1 / (float)a.n1 - 1.f, &s1, &cc1);
          const float S0 = v[m].re;
          acc[3] += (double)(S0 * cc0);
          acc[4] += (double)(S0 * s0);
          acc[5] += (double)(S0 * cc1);
          acc[6] += (double)(S0 * s1);
        } else if (k == 1) {
          // sum over the line of rho exp(2 pi i x_h / L_h) = -conj(mode 1), the
          // sign from the half-box offset of x_h
          acc[7] -= (double)v[m].re;
          acc[8] += (double)v[m].im;
        }
      }
    }
  }
  block_add<9>(acc, partials, Q_MASS);
}

// ---- Green's sum along the remaining axis -------------------------------------
// Lines of the half spectrum in the geometry of the step's Green's pass:
// strided (plane o, mid i) or contiguous (o = plane * mid_n + mid).
struct GreenSumArgs {
  const float2* rh;
  const float* k2p;   // k^2 of the half axis, by plane
  const float* k2m;   // k^2 of the middle axis (a single 0 in 2D)
  const float* k2l;   // k^2 of the line axis
  long long mid_n;
  int nh;             // length of the half axis (planes 0 .. nh / 2)
  float cN, cY, mu2;  // K = cN / k^2 + cY / (k^2 + mu2), 0 at k^2 = 0
};

template <int N>
__global__ void __launch_bounds__(obs_threads<N>(), 1)
green_sum_kernel(GreenSumArgs a, TileGeom G, const float2* tw, double* partials) {
  using P = Plan<N>;
  constexpr int E = P::E, T = P::T;
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* region = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tw_sm = region + kL * P::LS;
  const int l = threadIdx.x % kL, t = threadIdx.x / kL;
  stage_tw<N>(tw_sm, tw);
  double acc[1] = {0.0};
  for (long long tau = blockIdx.x; tau < G.count; tau += gridDim.x) {
    cx<float> v[E];
    load_tile<N>(v, region, a.rh, G, tau, l, t);
    line_transform<float, N, -1, false>(v, region + l * P::LS, tw_sm, t, true);
    long long o, i0;
    G.at(tau, o, i0);
    long long plane, mid;
    bool valid;
    if (G.inner > 1) {
      plane = o;
      mid = i0 + l;
      valid = mid < G.inner;
    } else {
      const long long line = o + l;
      plane = line / a.mid_n;
      mid = line - plane * a.mid_n;
      valid = line < G.outer;
    }
    if (!valid) continue;
    const float w = (plane == 0 || 2 * plane == a.nh) ? 1.f : 2.f;
    const float k2pm = a.k2p[plane] + a.k2m[mid];
    float s = 0.f;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const float k2 = k2pm + a.k2l[t + T * m];
      const float K = (k2 > 0.f) ? a.cN / k2 + a.cY / (k2 + a.mu2) : 0.f;
      s = fmaf(K, cnorm2(v[m]), s);
    }
    acc[0] += (double)(w * s);
  }
  block_add<1>(acc, partials, Q_EPOT);
}

// the dynamic shared-memory limit of kernel KIND of length N, once per device
template <int N, int KIND, typename K>
cudaError_t prep(K kern, size_t smem) {
  static bool done[kDeviceSlots] = {};
  bool& d = done[device_slot()];
  if (!d) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    d = true;
  }
  return cudaSuccess;
}

template <int N>
cudaError_t spec_t(const float2* psi, long long outer, long long inner, const float2* tw,
                   float kscale, double* partials, int q0, cudaStream_t s) {
  constexpr size_t smem = obs_smem_bytes<N>();
  cudaError_t e = prep<N, 0>(spec_sum_kernel<N>, smem);
  if (e != cudaSuccess) return e;
  spec_sum_kernel<N><<<kObsBlocks, obs_threads<N>(), smem, s>>>(psi, tile_geom(outer, inner), tw,
                                                                kscale, partials, q0);
  return cudaGetLastError();
}

template <int N>
cudaError_t density_t(const DensityArgs& a, long long lines, const float2* tw, double* partials,
                      cudaStream_t s) {
  constexpr size_t smem = obs_smem_bytes<N>();
  cudaError_t e = prep<N, 1>(density_kernel<N>, smem);
  if (e != cudaSuccess) return e;
  density_kernel<N><<<kObsBlocks, obs_threads<N>(), smem, s>>>(a, tile_geom(lines, 1), tw, partials);
  return cudaGetLastError();
}

template <int N>
cudaError_t green_t(const GreenSumArgs& a, long long outer, long long inner, const float2* tw,
                    double* partials, cudaStream_t s) {
  constexpr size_t smem = obs_smem_bytes<N>();
  cudaError_t e = prep<N, 2>(green_sum_kernel<N>, smem);
  if (e != cudaSuccess) return e;
  green_sum_kernel<N><<<kObsBlocks, obs_threads<N>(), smem, s>>>(a, tile_geom(outer, inner), tw,
                                                                 partials);
  return cudaGetLastError();
}

#define SN_OBS_DISPATCH(N_, CALL) \
  switch (N_) {                   \
    case 8: return CALL(8);       \
    case 16: return CALL(16);     \
    case 32: return CALL(32);     \
    case 64: return CALL(64);     \
    case 128: return CALL(128);   \
    case 256: return CALL(256);   \
    case 512: return CALL(512);   \
    case 1024: return CALL(1024); \
    default: return cudaErrorInvalidValue; \
  }

}  // namespace

cudaError_t launch_obs32_spec(int N, const float2* psi, long long outer, long long inner,
                              const float2* tw, double L, int axis, double* partials,
                              cudaStream_t s) {
  const float kscale = (float)(6.28318530717958647692 / L);
  const int q0 = Q_EKIN0 + 2 * axis;
#define SN_CALL(n) spec_t<n>(psi, outer, inner, tw, kscale, partials, q0, s)
  SN_OBS_DISPATCH(N, SN_CALL)
#undef SN_CALL
}

cudaError_t launch_obs32_density(int N, const float2* psi, int nfields, long long cells,
                                 const float* vext, float2* rh, int n0, int n1, const float2* tw,
                                 double* partials, cudaStream_t s) {
  DensityArgs a{psi, nfields, cells, vext, rh, n0, n1};
  const long long lines = cells / N;
#define SN_CALL(n) density_t<n>(a, lines, tw, partials, s)
  SN_OBS_DISPATCH(N, SN_CALL)
#undef SN_CALL
}

cudaError_t launch_obs32_green(int N, const float2* rh, long long outer, long long inner,
                               long long mid_n, const float* k2p, const float* k2m,
                               const float* k2l, int nh, double cN, double cY, double mu2,
                               const float2* tw, double* partials, cudaStream_t s) {
  GreenSumArgs a{rh, k2p, k2m, k2l, mid_n, nh, (float)cN, (float)cY, (float)mu2};
#define SN_CALL(n) green_t<n>(a, outer, inner, tw, partials, s)
  SN_OBS_DISPATCH(N, SN_CALL)
#undef SN_CALL
}

}  // namespace sn

// Plane-resident merged split steps of a small 2D complex64 grid (Sec. III;
// Eqs. 1-2): the whole state of an N x N grid (N = 64 or 128) -- psi, the
// potential's half spectrum and the tables -- is held in one CTA's shared
// memory for all rounds of an sn_step call, so the passes of a step touch HBM
// not at all (the state is read once at the start and written once at the
// end) and a call is one launch whatever its number of steps.
//
// Each round is the tiled path's round (passes_f32.cu / passes_tma.cu) on the
// resident arrays, with the same arithmetic in the same order, so the results
// agree with it bit for bit:
//   pass A along axis a0: [C2R of the half spectrum along a0 -> V h, the
//     nonlinear phase] then FFT . m . IFFT along a0;
//   pass B along axis a1: FFT . m . IFFT along a1, then |psi|^2 and its R2C
//     along a1 -> the half spectrum [k][line];
//   the Green's pass: FFT . K(k) . IFFT along a0 on the half spectrum's rows;
// with (a0, a1) = (y, x) on even rounds and (x, y) on odd ones.  Two real
// lines share one complex transform in the C2R and the R2C, paired as the
// tiled path pairs them (lines 16 t + j and 16 t + j + 8 of each 16).
//
// Exchanges run in place: a column (lines along y) keeps the array's own
// [y][x] layout, a row (lines along x) its row with the swizzle of
// tma_ops.cuh.  The CTA holds N lines in chunks of NT / T.
#include <cuda_runtime.h>

#include "sn_internal.h"
#include "tile_ops.cuh"
#include "tma_ops.cuh"

using namespace snfft;

namespace sn {
namespace {

template <int N>
struct Res {
  static constexpr int E = Plan<N>::E, T = Plan<N>::T;
  static constexpr int NT = N * T < 512 ? N * T : 512;  // threads
  static constexpr int LPC = NT / T;                     // lines per chunk
  static constexpr int CH = N / LPC;                     // chunks of a pass over N lines
  static constexpr int H = N / 2 + 1;                    // half-spectrum length
  static constexpr int HALF_LINES = N / 2;               // packed lines of a C2R / R2C
  static constexpr int NH = (H + T - 1) / T;
  // rows of the half-spectrum region: H rounded up to whole warps (32 / T rows
  // each), so that a warp of the Green's pass with rows past H exchanges them
  // in padding rows
  static constexpr int RPW = 32 / T;
  static constexpr int HR = (H + RPW - 1) / RPW * RPW;
  // shared memory: psi [N][N], the half spectrum [H][N] (also the packed
  // transforms' exchange space and V), twiddles (float4 hi/lo), the kinetic
  // shears [axis][half, full][N], k^2 [axis][N]
  static constexpr size_t PSI = (size_t)N * N * sizeof(float2);
  static constexpr size_t RH = (size_t)HR * N * sizeof(float2);
  static constexpr size_t TW = (size_t)Plan<N>::TWN * sizeof(float4);
  static constexpr size_t LIFT = (size_t)4 * N * sizeof(float4);
  static constexpr size_t K2 = (size_t)2 * N * sizeof(float);
  static constexpr size_t SMEM = PSI + RH + TW + LIFT + K2;
};

// Tiled-path pairing of real lines in one complex transform: packed line q
// carries lines 16 (q / 8) + q % 8 (real part) and that + 8 (imaginary part).
__device__ __forceinline__ int pair_a(int q) { return 16 * (q >> 3) + (q & 7); }
// packed line of line l, and whether l is its real part
__device__ __forceinline__ int pair_of(int l) { return 8 * (l >> 4) + (l & 7); }

// FFT . m . IFFT along my line l (position t of its threads) of psi, m the
// kinetic shears lt (the tiled path's lift of tile_ops.cuh)
template <int N, bool STRIDED>
__device__ __forceinline__ void kinetic(cx<float> (&v)[Plan<N>::E], cx<float>* psi,
                                        const float4* tw4, const float4* lt, int l, int t) {
  constexpr int E = Plan<N>::E, T = Plan<N>::T;
  tma::xform<N, -1, STRIDED, N>(v, psi, tw4, l, t);
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const float4 q = lt[t + T * m];
    const float x1 = fmaf(-q.x, v[m].im, v[m].re);
    const float y1 = fmaf(q.y, x1, v[m].im);
    const float x2 = fmaf(-q.x, y1, x1);
    v[m] = {x2 * q.z, y1 * q.z};
  }
  tma::xform<N, +1, STRIDED, N>(v, psi, tw4, l, t);
}

template <int N>
__global__ void __launch_bounds__(Res<N>::NT, 1) resident_2d_kernel(Resident2dArgs a) {
  using R = Res<N>;
  constexpr int E = R::E, T = R::T, NT = R::NT, LPC = R::LPC, H = R::H, NH = R::NH;
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* psi = reinterpret_cast<cx<float>*>(smem);
  cx<float>* rh = reinterpret_cast<cx<float>*>(smem + R::PSI);
  float* rf = reinterpret_cast<float*>(rh);
  float4* tw4 = reinterpret_cast<float4*>(smem + R::PSI + R::RH);
  float4* lift = reinterpret_cast<float4*>(smem + R::PSI + R::RH + R::TW);
  float* k2 = reinterpret_cast<float*>(smem + R::PSI + R::RH + R::TW + R::LIFT);
  const int tid = threadIdx.x;

  // ---- state and tables into shared memory
  for (int i = tid; i < N * N; i += NT) {
    const float2 z = a.psi[i];
    psi[i] = {z.x, z.y};
  }
  for (int i = tid; i < H * N; i += NT) {
    const float2 z = a.rh[i];
    rh[i] = {z.x, z.y};
  }
  tma::stage_twiddles<N>(tw4, a.tw, tid, NT);
  for (int i = tid; i < 4 * N; i += NT) lift[i] = a.lift[i / N][i % N];
  for (int i = tid; i < 2 * N; i += NT) k2[i] = a.k2[i / N][i % N];
  __syncthreads();

  // element (line l, position p) of psi for lines along axis 0 (columns, x = l)
  // or axis 1 (rows, y = l)
  auto at = [&](int ax, int l, int p) { return ax == 0 ? p * N + l : l * N + p; };

  bool nphase = a.nphase != 0;
  int full = a.full;
  bool odd = a.odd != 0;
  for (int r = 0; r < a.rounds; ++r) {
    const int a0 = odd ? 1 : 0, a1 = odd ? 0 : 1;
    // ---- pass A: C2R -> V h, phase, kinetic along a0
    if (nphase) {
      // packed line q = tid / T (all N/2 of them at once), position tc = tid % T
      const int q = tid / T, tc = tid % T;
      const bool pk = q < R::HALF_LINES;
      const int la = pair_a(q < R::HALF_LINES ? q : 0), lb = la + 8;
      cx<float> c[E];
      if (pk) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
          const int k = tc + T * m;
          cx<float> A, B;
          if (k <= N / 2) {
            A = rh[k * N + la];
            B = rh[k * N + lb];
            if (k == 0 || k == N / 2) { A.im = 0.f; B.im = 0.f; }
          } else {
            A = cconj(rh[(N - k) * N + la]);
            B = cconj(rh[(N - k) * N + lb]);
          }
          c[m] = {A.re - B.im, A.im + B.re};  // A + i B
        }
      }
      __syncthreads();  // the half spectrum is in registers: the region becomes exchange space
      if (pk) tma::xform<N, +1, false, N>(c, rh, tw4, q, tc);
      __syncthreads();
      if (pk) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
          const int p = tc + T * m;
          rf[la * N + p] = c[m].re;  // V h of line la at p
          rf[lb * N + p] = c[m].im;
        }
      }
      __syncthreads();
    }
    for (int ch = 0; ch < R::CH; ++ch) {
      const int l = ch * LPC + (a0 == 0 ? tid % LPC : tid / T);
      const int t = a0 == 0 ? tid / LPC : tid % T;
      cx<float> v[E];
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = psi[at(a0, l, t + T * m)];
      if (a0 == 0) __syncthreads();  // a column's words lie in every row
      if (nphase)
        tile::nonlinear_phase_at<E, T>(
            v, [&](int m) { return rf[l * N + t + T * m]; }, a.gh, nullptr, 0.f, 1u, t, true);
      if (a0 == 0) kinetic<N, true>(v, psi, tw4, lift + full * N, l, t);
      else kinetic<N, false>(v, psi, tw4, lift + (2 + full) * N, l, t);
      if (a0 == 0) __syncthreads(); else __syncwarp();
#pragma unroll
      for (int m = 0; m < E; ++m) psi[at(a0, l, t + T * m)] = v[m];
      __syncthreads();
    }
    // ---- pass B: kinetic along a1, then |psi|^2 and its R2C along a1
    for (int ch = 0; ch < R::CH; ++ch) {
      const int l = ch * LPC + (a1 == 0 ? tid % LPC : tid / T);
      const int t = a1 == 0 ? tid / LPC : tid % T;
      cx<float> v[E];
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = psi[at(a1, l, t + T * m)];
      if (a1 == 0) __syncthreads();
      if (a1 == 0) kinetic<N, true>(v, psi, tw4, lift + full * N, l, t);
      else kinetic<N, false>(v, psi, tw4, lift + (2 + full) * N, l, t);
      if (a1 == 0) __syncthreads(); else __syncwarp();
#pragma unroll
      for (int m = 0; m < E; ++m) psi[at(a1, l, t + T * m)] = v[m];
      __syncthreads();
    }
    {
      const int q = tid / T, tc = tid % T;
      const bool pk = q < R::HALF_LINES;
      const int la = pair_a(q < R::HALF_LINES ? q : 0), lb = la + 8;
      cx<float> c[E];
      if (pk) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
          const int p = tc + T * m;
          c[m] = {cnorm2(psi[at(a1, la, p)]), cnorm2(psi[at(a1, lb, p)])};
        }
      }
      __syncthreads();  // the region (V) is free: it becomes exchange space
      if (pk) tma::xform<N, -1, false, N>(c, rh, tw4, q, tc);
      __syncthreads();
      if (pk) {
#pragma unroll
        for (int m = 0; m < E; ++m) rh[q * N + tc + T * m] = c[m];  // Z of packed line q at k
      }
      __syncthreads();
      // unpack: line l of chunk ch, k = t + T j
      cx<float> hs[R::CH][NH];
#pragma unroll
      for (int ch = 0; ch < R::CH; ++ch) {
        const int l = ch * LPC + tid / T, t = tid % T;
        const int zq = pair_of(l);
        const bool pa = (l & 15) < 8;
#pragma unroll
        for (int j = 0; j < NH; ++j) {
          const int k = t + T * j;
          hs[ch][j] = {0.f, 0.f};
          if (k < H) {
            const cx<float> zk = rh[zq * N + k];
            const cx<float> zn = cconj(rh[zq * N + ((N - k) & (N - 1))]);
            if (pa) {
              hs[ch][j] = cscale(zk + zn, 0.5f);
            } else {
              const cx<float> d = zk - zn;
              hs[ch][j] = {0.5f * d.im, -0.5f * d.re};  // (zk - conj z_{N-k}) / (2i)
            }
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (int ch = 0; ch < R::CH; ++ch) {
        const int l = ch * LPC + tid / T, t = tid % T;
#pragma unroll
        for (int j = 0; j < NH; ++j) {
          const int k = t + T * j;
          if (k < H) rh[k * N + l] = hs[ch][j];
        }
      }
      __syncthreads();
    }
    // ---- Green's pass along a0 on the half spectrum's rows
    for (int r0 = 0; r0 < H; r0 += LPC) {
      const int l = r0 + tid / T, t = tid % T;
      const bool valid = l < H;
      // a warp runs if its first row is a row of the half spectrum; its rows
      // past H (< HR) transform zeros in padding rows, which are not stored
      const bool wrun = r0 + (tid / 32) * R::RPW < H;
      cx<float> v[E];
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = valid ? rh[l * N + t + T * m] : cx<float>{0.f, 0.f};
      if (wrun) {
        tma::xform<N, -1, false, N>(v, rh, tw4, l, t);
        const float k2pm = (valid ? k2[a1 * N + l] : 0.f) + 0.f;
#pragma unroll
        for (int m = 0; m < E; ++m) {
          const float kk = k2pm + k2[a0 * N + t + T * m];
          const float den = kk * (kk + a.mu2);
          const float K =
              ((kk > 0.f) ? __fdividef(fmaf(a.cN, kk + a.mu2, a.cY * kk), den) : 0.f) + 0.f;
          v[m] = cscale(v[m], K);
        }
        tma::xform<N, +1, false, N>(v, rh, tw4, l, t);
        __syncwarp();
        if (valid) {
#pragma unroll
          for (int m = 0; m < E; ++m) rh[l * N + t + T * m] = v[m];
        }
      }
      __syncthreads();
    }
    nphase = true;
    full = 1;
    odd = !odd;
  }

  // ---- state back to HBM
  for (int i = tid; i < N * N; i += NT) a.psi[i] = make_float2(psi[i].re, psi[i].im);
  for (int i = tid; i < H * N; i += NT) a.rh[i] = make_float2(rh[i].re, rh[i].im);
}

template <int N>
cudaError_t launch_t(const Resident2dArgs& a, cudaStream_t s) {
  constexpr size_t smem = Res<N>::SMEM;
  static bool attr_of[kDeviceSlots] = {};
  bool& attr = attr_of[device_slot()];
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(resident_2d_kernel<N>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  resident_2d_kernel<N><<<1, Res<N>::NT, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool resident_2d_supported(int ny, int nx) { return ny == nx && (nx == 64 || nx == 128); }

cudaError_t launch_resident_2d(int n, const Resident2dArgs& a, cudaStream_t s) {
  if (a.rounds < 1) return cudaSuccess;
  if (n == 128) return launch_t<128>(a, s);
  if (n == 64) return launch_t<64>(a, s);
  return cudaErrorNotSupported;
}

}  // namespace sn

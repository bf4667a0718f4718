// TMA-staged line passes of the fused FP32 split step (Sec. III; Eqs. 1-2).
//
// The same per-line work as the plain kinetic pass and the three
// half-spectrum passes of passes_f32.cu (FFT . m . IFFT along one axis;
// forward FFT; FFT . K(k) . IFFT; inverse FFT), with a different way of
// moving the data: every tile of 16 lines travels between HBM and shared
// memory as one cp.async.bulk.tensor copy issued by one thread.  A CTA keeps
// two tile slots: while it transforms the tile in one slot, the TMA unit
// loads its next tile into the other, and a finished tile is stored from its
// slot by the copy engine.  The threads issue no global loads or stores and
// hold no prefetched tile in registers; the stage exchanges of the transform
// run in the tile's own slot (tma_ops.cuh).
//
// Taken for 128- and 256-point lines of one field on the FP32 engine; every
// other case keeps the register-staged kernels.  Each wait on a tile's
// mbarrier has a clock-cycle limit: when it expires the CTA records the
// failure in a status word that the host reads at its next synchronising
// call, waits (bounded) for its copies in flight, and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>
#include <unordered_map>

#include "sn_internal.h"
#include "tile_ops.cuh"
#include "tma_ops.cuh"

using namespace snfft;

namespace sn {
namespace {

constexpr int kLpb = 16;                     // lines per tile
// Tile slots per CTA: two for the passes with a transform pair per tile,
// three for the forward and inverse half-spectrum passes, which have one
// transform per tile and so need more tiles in flight to cover the loads.
template <int OP>
__host__ __device__ constexpr int line_slots() { return (OP == LINE_FWD || OP == LINE_INV) ? 3 : 2; }
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at the B300's clock

// Kernel parameter block; the tensor map (aligned by its own type) must be a
// __grid_constant__ parameter for the TMA unit to read it.
struct TmaLineArgs {
  CUtensorMap map;        // the lines' array as tiles of kLpb lines x N points
  long long outer, inner; // lines = outer * inner (inner = 1: contiguous lines)
  const float2* tw;       // twiddles of N (hi parts, then lo parts)
  const float4* lift;     // LINE_KINETIC: exp(i A k^2 tau) / N as three shears
  const float* k2p;       // LINE_GREEN: k^2 of the half axis, indexed by plane
  const float* k2m;       // LINE_GREEN: k^2 of the middle axis
  const float* k2l;       // LINE_GREEN: k^2 of the line axis
  long long mid_n;        // LINE_GREEN, contiguous lines: outer = plane * mid_n + mid
  float cN, cY, mu2, cL;  // LINE_GREEN: K = cN/k2 + cY/(k2 + mu2) (0 at k2 = 0) + cL
  int* status;            // set to 1 if a tile wait expired
};

__device__ __forceinline__ void pdl_allow_next() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
__device__ __forceinline__ void pdl_wait_prev() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

template <int N>
constexpr int tma_threads() { return kLpb * Plan<N>::T; }
// resident CTAs the registers are sized for (two or three tile slots per CTA)
template <int N>
constexpr int tma_min_ctas() { return N == 256 ? 2 : 4; }

template <int N, int OP>
constexpr size_t tma_smem_bytes() {
  constexpr int kSlots = line_slots<OP>();
  return 128 + kSlots * (size_t)kLpb * N * sizeof(float2)    // alignment, tile slots
         + 2 * (size_t)Plan<N>::TWN * sizeof(float2)          // twiddles (hi, lo)
         + (size_t)N * sizeof(float4)                         // kinetic shears
         + kSlots * sizeof(uint64_t);                         // tile barriers
}

template <int N, bool STRIDED, int OP>
__global__ void __launch_bounds__(tma_threads<N>(), tma_min_ctas<N>())
line_pass_tma_kernel(const __grid_constant__ TmaLineArgs a) {
  using P = Plan<N>;
  constexpr int E = P::E, T = P::T, NT = kLpb * T;
  constexpr int TILE = kLpb * N;  // words per slot
  constexpr unsigned TILE_BYTES = (unsigned)(TILE * sizeof(float2));
  constexpr int kSlots = line_slots<OP>();
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  // the tile slots need 128-byte alignment: the window is over-allocated by
  // 128 bytes and its base rounded up
  unsigned char* smem_raw = smem_dyn + ((128u - (tma::smem_u32(smem_dyn) & 127u)) & 127u);
  cx<float>* slots = reinterpret_cast<cx<float>*>(smem_raw);
  float4* tw_sm = reinterpret_cast<float4*>(slots + kSlots * TILE);
  float4* lift_sm = tw_sm + P::TWN;
  uint64_t* bar = reinterpret_cast<uint64_t*>(lift_sm + N);

  const int tid = threadIdx.x;
  const int l = STRIDED ? (tid % kLpb) : (tid / T);
  const int t = STRIDED ? (tid / kLpb) : (tid % T);
  const long long tiles_i = STRIDED ? (a.inner + kLpb - 1) / kLpb : 1;
  const long long count = STRIDED ? a.outer * tiles_i : (a.outer + kLpb - 1) / kLpb;

  pdl_allow_next();
  tma::stage_twiddles<N>(tw_sm, a.tw, tid, NT);
  if constexpr (OP == LINE_KINETIC)
    for (int k = tid; k < N; k += NT) lift_sm[k] = a.lift[k];
  if (tid == 0) {
    for (int s = 0; s < kSlots; ++s) tma::mbar_init(&bar[s], 1);
    tma::mbar_fence_init();
  }
  __syncthreads();
  pdl_wait_prev();  // the lines come from the previous pass

  // coordinates of tile tau: strided (inner i0, 0, outer o), contiguous (0, first line)
  auto issue_load = [&](int s, long long tau) {
    tma::mbar_expect_tx(&bar[s], TILE_BYTES);
    if constexpr (STRIDED) {
      const long long o = tau / tiles_i;
      const int i0 = (int)((tau - o * tiles_i) * kLpb);
      tma::tma_load_3d(slots + s * TILE, &a.map, i0, 0, (int)o, &bar[s]);
    } else {
      tma::tma_load_2d(slots + s * TILE, &a.map, 0, (int)(tau * kLpb), &bar[s]);
    }
  };
  auto issue_store = [&](int s, long long tau) {
    if constexpr (STRIDED) {
      const long long o = tau / tiles_i;
      const int i0 = (int)((tau - o * tiles_i) * kLpb);
      if constexpr (OP == LINE_KINETIC)  // psi: leave L2 to the half spectrum
        tma::tma_store_3d_ef(&a.map, i0, 0, (int)o, slots + s * TILE, tma::policy_evict_first());
      else
        tma::tma_store_3d(&a.map, i0, 0, (int)o, slots + s * TILE);
    } else {
      if constexpr (OP == LINE_KINETIC)
        tma::tma_store_2d_ef(&a.map, 0, (int)(tau * kLpb), slots + s * TILE, tma::policy_evict_first());
      else
        tma::tma_store_2d(&a.map, 0, (int)(tau * kLpb), slots + s * TILE);
    }
    tma::bulk_commit();
  };

  // Tile it of this CTA sits in slot it % kSlots.  The first kSlots tiles are
  // loaded up front.  Tile it is stored from its slot at the end of iteration
  // it; thread 0 loads tile it + kSlots into that slot one step later, once it
  // holds the next tile in registers, so that the store has had that time to
  // read the slot.
  long long tau = blockIdx.x;
  // loads issued into each slot, and waits completed on it (thread 0's count)
  int issued[kSlots] = {}, used[kSlots] = {};
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < kSlots; ++q)
      if (tau + (long long)q * gridDim.x < count) {
        issue_load(q, tau + (long long)q * gridDim.x);
        ++issued[q];
      }
  }
  long long pend_tau = -1;  // thread 0: a load owed to slot pend_s
  int pend_s = 0;

  bool failed = false;
  for (int it = 0, s = 0; tau < count; ++it, tau += gridDim.x, s = (s + 1 == kSlots ? 0 : s + 1)) {
    cx<float>* buf = slots + s * TILE;
    const bool ok = tma::mbar_wait_bounded(&bar[s], (unsigned)(used[s] & 1), kWaitCycles);
    if (!__syncthreads_and(ok)) {
      failed = true;
      break;
    }
    ++used[s];
    cx<float> v[E];
#pragma unroll
    for (int m = 0; m < E; ++m)
      v[m] = buf[STRIDED ? (t + T * m) * kLpb + l : l * N + t + T * m];
    if (tid == 0 && pend_tau >= 0) {
      tma::bulk_wait_read<0>();  // the previous tile's store has read its slot
      issue_load(pend_s, pend_tau);
      ++issued[pend_s];
      pend_tau = -1;
    }
    __syncthreads();  // every thread holds its tile data: the slot becomes exchange space

    if constexpr (OP == LINE_KINETIC || OP == LINE_GREEN || OP == LINE_FWD)
      tma::xform<N, -1, STRIDED, kLpb>(v, buf, tw_sm, l, t);
    if constexpr (OP == LINE_KINETIC) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const float4 q = lift_sm[t + T * m];
        const float x1 = fmaf(-q.x, v[m].im, v[m].re);
        const float y1 = fmaf(q.y, x1, v[m].im);
        const float x2 = fmaf(-q.x, y1, x1);
        v[m] = {x2 * q.z, y1 * q.z};
      }
    } else if constexpr (OP == LINE_GREEN) {
      long long o, i;
      if constexpr (STRIDED) {
        o = tau / tiles_i;
        i = (tau - o * tiles_i) * kLpb + l;
      } else {
        o = tau * kLpb + l;
        i = 0;
      }
      long long plane, mid;
      if constexpr (STRIDED) {
        plane = o;
        mid = i;
      } else {
        plane = o / a.mid_n;
        mid = o - plane * a.mid_n;
      }
      const bool valid = STRIDED ? (i < a.inner) : (o < a.outer);
      const float k2pm = valid ? a.k2p[plane] + a.k2m[mid] : 0.f;
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const float k2 = k2pm + a.k2l[t + T * m];
        const float den = k2 * (k2 + a.mu2);
        const float K =
            ((k2 > 0.f) ? __fdividef(fmaf(a.cN, k2 + a.mu2, a.cY * k2), den) : 0.f) + a.cL;
        v[m] = cscale(v[m], K);
      }
    }
    if constexpr (OP == LINE_KINETIC || OP == LINE_GREEN || OP == LINE_INV)
      tma::xform<N, +1, STRIDED, kLpb>(v, buf, tw_sm, l, t);

    tma::xsync<STRIDED>();  // the last exchange reads are done before the tile is rewritten
#pragma unroll
    for (int m = 0; m < E; ++m)
      buf[STRIDED ? (t + T * m) * kLpb + l : l * N + t + T * m] = v[m];
    tma::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      issue_store(s, tau);
      const long long tau2 = tau + (long long)kSlots * gridDim.x;
      if (tau2 < count) {
        pend_tau = tau2;
        pend_s = s;
      }
    }
  }
  if (failed && tid == 0) {
    atomicExch(a.status, 1);
    // loads still in flight into this CTA's slots: wait for them, bounded
    for (int s = 0; s < kSlots; ++s)
      for (; used[s] < issued[s]; ++used[s])
        (void)tma::mbar_wait_bounded(&bar[s], (unsigned)(used[s] & 1), kWaitCycles / 8);
  }
  if (tid == 0) tma::bulk_wait_all();
}

// ---- potential and density passes ---------------------------------------------
//
// P1 (EDGE_PHASE): the half spectrum of the potential (lines [k][line], k <=
// N/2) arrives with each psi tile; its C2R inverse FFT along the lines (two
// real lines per complex transform, lines l and l + 8) gives V h, then
// psi <- exp(-i (V h + V_ext h + g h |psi|^2)) psi and FFT . m . IFFT.
// P3 (EDGE_DENSITY): FFT . m . IFFT, the tile is stored, then rho = |psi|^2
// and its R2C FFT along the lines (two real lines per complex transform) go
// out as a [k][line] half-spectrum tile.
// Arithmetic and order are those of tile::potential_c2r, tile::kinetic,
// tile::nonlinear_phase_at and tile::density_r2c_rho, so results agree with
// the register-staged kernels bit for bit.
//
// Slot s holds the psi tile (kLpb x N words) and, 1024-byte aligned after it,
// the half-spectrum region (kLpb x (N/2 + 1) words, TMA's 128-byte swizzle:
// the 16-byte chunk c of row k sits at chunk c ^ (k & 7)).  P1 loads the
// potential's tile there and then uses the region for the C2R's exchange and
// for V; P3 uses it for rho, the R2C's exchange, the packed spectrum and the
// outgoing half-spectrum tile.
constexpr int EDGE_PHASE = 0, EDGE_DENSITY = 1;

struct TmaEdgeArgs {
  CUtensorMap psi_map;   // psi lines, as TmaLineArgs::map
  CUtensorMap rh_map;    // half spectrum: (inner, outer, N/2+1) strided, (lines, N/2+1) contiguous
  long long outer, inner;
  const float2* tw;
  const float4* lift;
  const float* vext;     // EDGE_PHASE: V_ext in psi layout, or NULL
  float h, gh;           // EDGE_PHASE: h (multiplies V_ext), g h
  int* status;
};

template <int N>
__host__ __device__ constexpr size_t edge_rh_bytes() {  // one half-spectrum region, rounded to 1024 bytes
  return ((size_t)kLpb * (N / 2 + 1) * sizeof(float2) + 1023) / 1024 * 1024;
}
template <int N>
__host__ __device__ constexpr size_t edge_slot_bytes() { return (size_t)kLpb * N * sizeof(float2) + edge_rh_bytes<N>(); }
template <int N>
constexpr size_t edge_smem_bytes() {
  return 1024 + 2 * edge_slot_bytes<N>() + 2 * (size_t)Plan<N>::TWN * sizeof(float2) +
         (size_t)N * sizeof(float4) + 2 * sizeof(uint64_t);
}

// word of (line row, position pos) in a line-major float region of a tile (V
// of contiguous tiles in P1, rho in P3): pos XOR 2 pi(row), pi a permutation
// of the 16 lines.  The contiguous mapping puts R = 32 / T lines of T
// consecutive positions in a warp, the strided one all 16 lines at two
// positions; pi(row) = (row mod R) 16 / R + row / R keeps the lanes of a warp
// on distinct banks in both (a plain pitch of N put the contiguous mapping's
// lines on the same banks).
template <int N>
__device__ __forceinline__ int vw(int row, int pos) {
  constexpr int T = Plan<N>::T, R = 32 / T;
  static_assert(T == 8 || T == 16, "edge passes take 128- and 256-point lines");
  const int pi = ((row % R) * (kLpb / R)) | (row / R);
  return row * N + (pos ^ (pi << 1));
}

// The words vw(row, t + T m), m = 0 … E - 1, of one thread (t < T): with
// s = 2 pi(row) = T s_hi + s_lo (s_lo < T, s_hi < R), (t + T m) XOR s is
// (t XOR s_lo) + T ((m mod R) XOR s_hi) + 32 (m / R), so the row's words are
// R per-thread bases plus a constant per m: no swizzle arithmetic per access
// once the loops over m are unrolled.
template <int N>
struct VRow {
  static constexpr int T = Plan<N>::T, R = 32 / T;
  int base[R];
  __device__ __forceinline__ VRow(int row, int t) {
    const int sw = vw<N>(row, 0) - row * N;  // 2 pi(row)
    const int lo = row * N + (t ^ (sw % T));
#pragma unroll
    for (int r = 0; r < R; ++r) base[r] = lo + T * (r ^ (sw / T));
  }
  __device__ __forceinline__ int operator[](int m) const { return base[m % R] + 32 * (m / R); }
};

// word of (row k, line col) in a swizzled half-spectrum region
__device__ __forceinline__ int rhw(int k, int col) {
  return k * kLpb + ((((col >> 1) ^ (k & 7)) << 1) | (col & 1));
}

template <int N, bool STRIDED, int EDGE>
__global__ void __launch_bounds__(tma_threads<N>(), tma_min_ctas<N>())
edge_pass_tma_kernel(const __grid_constant__ TmaEdgeArgs a) {
  using P = Plan<N>;
  constexpr int E = P::E, T = P::T, NT = kLpb * T, H = N / 2 + 1, HALF = kLpb / 2;
  constexpr int TILE = kLpb * N;
  constexpr unsigned PSI_BYTES = (unsigned)(TILE * sizeof(float2));
  constexpr unsigned RH_BYTES = (unsigned)(kLpb * H * sizeof(float2));
  constexpr size_t SLOT = edge_slot_bytes<N>();
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  // the swizzled regions need 1024-byte alignment: the window is over-allocated
  // by 1 KB and its base rounded up
  unsigned char* smem_raw = smem_dyn + ((1024u - (tma::smem_u32(smem_dyn) & 1023u)) & 1023u);
  float4* tw_sm = reinterpret_cast<float4*>(smem_raw + 2 * SLOT);
  float4* lift_sm = tw_sm + P::TWN;
  uint64_t* bar = reinterpret_cast<uint64_t*>(lift_sm + N);
  auto psi_of = [&](int s) { return reinterpret_cast<cx<float>*>(smem_raw + s * SLOT); };
  auto rh_of = [&](int s) {
    return reinterpret_cast<cx<float>*>(smem_raw + s * SLOT + (size_t)TILE * sizeof(float2));
  };

  const int tid = threadIdx.x;
  const int l = STRIDED ? (tid % kLpb) : (tid / T);
  const int t = STRIDED ? (tid / kLpb) : (tid % T);
  const int lc = tid / T, tc = tid % T;  // the packed transforms' contiguous mapping
  const bool pk = lc < HALF;             // this thread transforms packed line lc
  const long long tiles_i = STRIDED ? (a.inner + kLpb - 1) / kLpb : 1;
  const long long count = STRIDED ? a.outer * tiles_i : (a.outer + kLpb - 1) / kLpb;

  pdl_allow_next();
  tma::stage_twiddles<N>(tw_sm, a.tw, tid, NT);
  for (int k = tid; k < N; k += NT) lift_sm[k] = a.lift[k];
  if (tid == 0) {
    tma::mbar_init(&bar[0], 1);
    tma::mbar_init(&bar[1], 1);
    tma::mbar_fence_init();
  }
  __syncthreads();
  pdl_wait_prev();

  auto tile_at = [&](long long tau, long long& o, int& i0) {
    if constexpr (STRIDED) {
      o = tau / tiles_i;
      i0 = (int)((tau - o * tiles_i) * kLpb);
    } else {
      o = tau * kLpb;
      i0 = 0;
    }
  };
  auto issue_load = [&](int s, long long tau) {
    long long o;
    int i0;
    tile_at(tau, o, i0);
    tma::mbar_expect_tx(&bar[s], PSI_BYTES + (EDGE == EDGE_PHASE ? RH_BYTES : 0u));
    if constexpr (STRIDED) {
      tma::tma_load_3d(psi_of(s), &a.psi_map, i0, 0, (int)o, &bar[s]);
      if constexpr (EDGE == EDGE_PHASE) tma::tma_load_3d(rh_of(s), &a.rh_map, i0, (int)o, 0, &bar[s]);
    } else {
      tma::tma_load_2d(psi_of(s), &a.psi_map, 0, (int)o, &bar[s]);
      if constexpr (EDGE == EDGE_PHASE) tma::tma_load_2d(rh_of(s), &a.rh_map, (int)o, 0, &bar[s]);
    }
  };

  long long tau = blockIdx.x;
  int issued[2] = {0, 0}, used[2] = {0, 0};
  if (tid == 0) {
    if (tau < count) { issue_load(0, tau); ++issued[0]; }
    if (tau + gridDim.x < count) { issue_load(1, tau + gridDim.x); ++issued[1]; }
  }
  long long pend_tau = -1;
  int pend_s = 0;

  bool failed = false;
  for (int it = 0, s = 0; tau < count; ++it, tau += gridDim.x, s ^= 1) {
    cx<float>* buf = psi_of(s);
    cx<float>* rh = rh_of(s);
    float* rf = reinterpret_cast<float*>(rh);
    long long o;
    int i0;
    tile_at(tau, o, i0);
    const bool valid = STRIDED ? (i0 + l < a.inner) : (o + l < a.outer);
    const bool ok = tma::mbar_wait_bounded(&bar[s], (unsigned)(used[s] & 1), kWaitCycles);
    if (!__syncthreads_and(ok)) {
      failed = true;
      break;
    }
    ++used[s];
    cx<float> v[E];

    if constexpr (EDGE == EDGE_PHASE) {
      // ---- C2R of packed lines (lc, lc + 8): V h of the tile's 16 lines
      cx<float> c[E];
      if (pk) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
          const int k = tc + T * m;
          cx<float> A, B;
          if (k <= N / 2) {
            A = rh[rhw(k, lc)];
            B = rh[rhw(k, lc + HALF)];
            if (k == 0 || k == N / 2) { A.im = 0.f; B.im = 0.f; }
          } else {
            A = cconj(rh[rhw(N - k, lc)]);
            B = cconj(rh[rhw(N - k, lc + HALF)]);
          }
          c[m] = {A.re - B.im, A.im + B.re};  // A + i B
        }
      }
      __syncthreads();  // the potential's tile is in registers: the region becomes exchange space
      if (pk) tma::xform<N, +1, false, kLpb>(c, rh, tw_sm, lc, tc);
      __syncthreads();  // every exchange read is done: the region takes V
      if (pk) {
        if constexpr (STRIDED) {
#pragma unroll
          for (int m = 0; m < E; ++m) {
            const int p = tc + T * m;
            rf[p * kLpb + (lc ^ (p & 15))] = c[m].re;
            rf[p * kLpb + ((lc + HALF) ^ (p & 15))] = c[m].im;
          }
        } else {
          const VRow<N> ra(lc, tc), rb(lc + HALF, tc);
#pragma unroll
          for (int m = 0; m < E; ++m) {
            rf[ra[m]] = c[m].re;
            rf[rb[m]] = c[m].im;
          }
        }
      }
    }
#pragma unroll
    for (int m = 0; m < E; ++m)
      v[m] = buf[STRIDED ? (t + T * m) * kLpb + l : l * N + t + T * m];
    if (tid == 0 && pend_tau >= 0) {
      tma::bulk_wait_read<EDGE == EDGE_DENSITY ? 1 : 0>();  // the previous psi store has read its slot
      issue_load(pend_s, pend_tau);
      ++issued[pend_s];
      pend_tau = -1;
    }
    __syncthreads();  // psi in registers (and V visible): the psi slot becomes exchange space

    if constexpr (EDGE == EDGE_PHASE) {
      const float* vx = nullptr;
      if (a.vext != nullptr && valid)
        vx = a.vext + (STRIDED ? (size_t)o * N * a.inner + i0 + l : (size_t)(o + l) * N);
      const unsigned ustride = STRIDED ? (unsigned)a.inner : 1u;
      const VRow<N> rv(l, t);
      tile::nonlinear_phase_at<E, T>(
          v,
          [&](int m) {
            const int p = t + T * m;
            return STRIDED ? rf[p * kLpb + (l ^ (p & 15))] : rf[rv[m]];
          },
          a.gh, vx, a.h, ustride, t, valid);
    }
    // ---- kinetic factor along the lines
    tma::xform<N, -1, STRIDED, kLpb>(v, buf, tw_sm, l, t);
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const float4 q = lift_sm[t + T * m];
      const float x1 = fmaf(-q.x, v[m].im, v[m].re);
      const float y1 = fmaf(q.y, x1, v[m].im);
      const float x2 = fmaf(-q.x, y1, x1);
      v[m] = {x2 * q.z, y1 * q.z};
    }
    tma::xform<N, +1, STRIDED, kLpb>(v, buf, tw_sm, l, t);
    tma::xsync<STRIDED>();
#pragma unroll
    for (int m = 0; m < E; ++m)
      buf[STRIDED ? (t + T * m) * kLpb + l : l * N + t + T * m] = v[m];
    tma::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      // psi leaves L2 first; the half spectrum a density pass writes stays
      if constexpr (STRIDED) tma::tma_store_3d_ef(&a.psi_map, i0, 0, (int)o, buf, tma::policy_evict_first());
      else tma::tma_store_2d_ef(&a.psi_map, 0, (int)o, buf, tma::policy_evict_first());
      tma::bulk_commit();
      const long long tau2 = tau + 2 * (long long)gridDim.x;
      if (tau2 < count) {
        pend_tau = tau2;
        pend_s = s;
      }
      // P3: this slot's half-spectrum region was last read by the store of
      // tile it - 2 (issued before the stores of it - 1 and it)
      if constexpr (EDGE == EDGE_DENSITY) tma::bulk_wait_read<2>();
    }

    if constexpr (EDGE == EDGE_DENSITY) {
      // ---- rho = |psi|^2 and its R2C along the lines (packed lines lc, lc + 8)
      __syncthreads();  // the region is free
      {
        const VRow<N> rw(l, t);
#pragma unroll
        for (int m = 0; m < E; ++m) rf[rw[m]] = cnorm2(v[m]);
      }
      __syncthreads();
      cx<float> c[E];
      if (pk) {
        const VRow<N> ra(lc, tc), rb(lc + HALF, tc);
#pragma unroll
        for (int m = 0; m < E; ++m) c[m] = {rf[ra[m]], rf[rb[m]]};
      }
      __syncthreads();  // rho is in registers: the region becomes exchange space
      if (pk) tma::xform<N, -1, false, kLpb>(c, rh, tw_sm, lc, tc);
      __syncthreads();
      // the packed spectrum Z of line lc at k: [k][8] with the line index XOR (k & 7)
      // for strided tiles (whose unpacking reads 8 lines at one k), [lc][k] otherwise
      auto zw = [&](int line, int k) {
        return STRIDED ? k * HALF + (line ^ (k & 7)) : line * N + k;
      };
      if (pk) {
#pragma unroll
        for (int q = 0; q < E; ++q) rh[zw(lc, tc + T * q)] = c[q];
      }
      __syncthreads();
      constexpr int NH = (H + T - 1) / T;
      cx<float> hs[NH];
      const int zl = l % HALF;
      const bool pa = l < HALF;
#pragma unroll
      for (int q = 0; q < NH; ++q) {
        const int k = t + T * q;
        hs[q] = {0.f, 0.f};
        if (k < H) {
          const cx<float> zk = rh[zw(zl, k)];
          const cx<float> zn = cconj(rh[zw(zl, (N - k) & (N - 1))]);
          if (pa) {
            hs[q] = cscale(zk + zn, 0.5f);
          } else {
            const cx<float> d = zk - zn;
            hs[q] = {0.5f * d.im, -0.5f * d.re};  // (zk - conj z_{N-k}) / (2i)
          }
        }
      }
      __syncthreads();  // every read of Z is done: the region takes the outgoing tile
#pragma unroll
      for (int q = 0; q < NH; ++q) {
        const int k = t + T * q;
        if (k < H) rh[rhw(k, l)] = hs[q];
      }
      tma::fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        if constexpr (STRIDED) tma::tma_store_3d(&a.rh_map, i0, (int)o, 0, rh);
        else tma::tma_store_2d(&a.rh_map, (int)o, 0, rh);
        tma::bulk_commit();
      }
    }
  }
  if (failed && tid == 0) {
    atomicExch(a.status, 1);
    for (int s = 0; s < 2; ++s)
      for (; used[s] < issued[s]; ++used[s])
        (void)tma::mbar_wait_bounded(&bar[s], (unsigned)(used[s] & 1), kWaitCycles / 8);
  }
  if (tid == 0) tma::bulk_wait_all();
}

// ---- host side -----------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Tensor map of lines (outer, inner) x N complex64 points: strided lines as the
// 3D array (inner, N, outer) with boxes (kLpb, N, 1); contiguous lines as the
// 2D array (N, outer) with boxes (N, kLpb).  Elements are 8-byte words.
cudaError_t encode_lines(CUtensorMap* map, void* base, int N, bool strided, long long outer,
                         long long inner) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  cuuint64_t dims[3], strides[2];
  cuuint32_t box[3], estr[3] = {1, 1, 1};
  cuuint32_t rank;
  if (strided) {
    rank = 3;
    dims[0] = (cuuint64_t)inner;
    dims[1] = (cuuint64_t)N;
    dims[2] = (cuuint64_t)outer;
    strides[0] = (cuuint64_t)inner * 8;
    strides[1] = (cuuint64_t)inner * N * 8;
    box[0] = kLpb;
    box[1] = (cuuint32_t)N;
    box[2] = 1;
  } else {
    rank = 2;
    dims[0] = (cuuint64_t)N;
    dims[1] = (cuuint64_t)outer;
    strides[0] = (cuuint64_t)N * 8;
    box[0] = (cuuint32_t)N;
    box[1] = kLpb;
  }
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, rank, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tensor map of the half spectrum [k][line] (k <= N/2) of the lines (outer,
// inner): strided lines as the 3D array (inner, outer, N/2 + 1) with boxes
// (kLpb, 1, N/2 + 1), so that a tile narrower than kLpb lines stops at the
// end of its row of lines; contiguous lines as the 2D array (lines, N/2 + 1)
// with boxes (kLpb, N/2 + 1).  A row holds row_lines >= outer * inner lines
// (a launch over a slab of them; 0: exactly outer * inner).  128-byte swizzle.
cudaError_t encode_half(CUtensorMap* map, void* base, int N, bool strided, long long outer,
                        long long inner, long long row_lines) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const long long nlines = outer * inner;
  const long long rowl = row_lines > 0 ? row_lines : nlines;
  const cuuint32_t H = (cuuint32_t)(N / 2 + 1);
  cuuint64_t dims[3], strides[2];
  cuuint32_t box[3], estr[3] = {1, 1, 1};
  cuuint32_t rank;
  if (strided) {
    rank = 3;
    dims[0] = (cuuint64_t)inner;
    dims[1] = (cuuint64_t)outer;
    dims[2] = H;
    strides[0] = (cuuint64_t)inner * 8;
    strides[1] = (cuuint64_t)rowl * 8;
    box[0] = kLpb;
    box[1] = 1;
    box[2] = H;
  } else {
    rank = 2;
    dims[0] = (cuuint64_t)nlines;
    dims[1] = H;
    strides[0] = (cuuint64_t)rowl * 8;
    box[0] = kLpb;
    box[1] = H;
  }
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, rank, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename K>
unsigned tma_grid(K kern, int threads, size_t smem, long long ntiles, int cps) {
  if (cps < 0) return (unsigned)(ntiles < 0x7fffffffLL ? ntiles : 0x7fffffffLL);
  static int sms_of[kDeviceSlots] = {};
  int& sms = sms_of[device_slot()];
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  if (cps > 0 && cps < per_sm) per_sm = cps;
  const long long cap = (long long)per_sm * sms;
  return (unsigned)(ntiles < cap ? ntiles : cap);
}

template <int N, bool STRIDED, int OP>
cudaError_t launch_t(const LinePassArgs& in, cudaStream_t s) {
  constexpr size_t smem = tma_smem_bytes<N, OP>();
  constexpr int threads = tma_threads<N>();
  auto kern = line_pass_tma_kernel<N, STRIDED, OP>;
  static bool attr_of[kDeviceSlots] = {};
  bool& attr = attr_of[device_slot()];
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  TmaLineArgs a;
  std::memset(&a, 0, sizeof(a));
  cudaError_t e = encode_lines(&a.map, in.data, N, STRIDED, in.outer, in.inner);
  if (e != cudaSuccess) return e;
  a.outer = in.outer;
  a.inner = in.inner;
  a.tw = in.tw;
  a.lift = in.lift;
  a.k2p = in.k2p;
  a.k2m = in.k2m;
  a.k2l = in.k2l;
  a.mid_n = in.mid_n;
  a.cN = in.cN;
  a.cY = in.cY;
  a.mu2 = in.mu2;
  a.cL = in.cL;
  a.status = in.status;
  const long long ntiles = STRIDED ? in.outer * ((in.inner + kLpb - 1) / kLpb)
                                   : (in.outer + kLpb - 1) / kLpb;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(tma_grid(kern, threads, smem, ntiles, in.ctas_per_sm));
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute lattr[1];
  lattr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  lattr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = lattr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int N, bool STRIDED, int EDGE>
cudaError_t launch_edge_t(const PsiPassArgs& in, int* status, cudaStream_t s) {
  constexpr size_t smem = edge_smem_bytes<N>();
  constexpr int threads = tma_threads<N>();
  auto kern = edge_pass_tma_kernel<N, STRIDED, EDGE>;
  static bool attr_of[kDeviceSlots] = {};
  bool& attr = attr_of[device_slot()];
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  TmaEdgeArgs a;
  std::memset(&a, 0, sizeof(a));
  cudaError_t e = encode_lines(&a.psi_map, in.psi, N, STRIDED, in.outer, in.inner);
  if (e == cudaSuccess)
    e = encode_half(&a.rh_map, EDGE == EDGE_PHASE ? (void*)in.rh_in : (void*)in.rh_out, N, STRIDED,
                    in.outer, in.inner, in.rh_lines);
  if (e != cudaSuccess) return e;
  a.outer = in.outer;
  a.inner = in.inner;
  a.tw = in.tw;
  a.lift = in.lift;
  a.vext = in.vext;
  a.h = in.h;
  a.gh = in.gh;
  a.status = status;
  const long long ntiles = STRIDED ? in.outer * ((in.inner + kLpb - 1) / kLpb)
                                   : (in.outer + kLpb - 1) / kLpb;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(tma_grid(kern, threads, smem, ntiles, in.ctas_per_sm));
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute lattr[1];
  lattr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  lattr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = lattr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int N, bool STRIDED>
cudaError_t dispatch_op(int op, const LinePassArgs& a, cudaStream_t s) {
  switch (op) {
    case LINE_KINETIC: return launch_t<N, STRIDED, LINE_KINETIC>(a, s);
    case LINE_FWD: return launch_t<N, STRIDED, LINE_FWD>(a, s);
    case LINE_GREEN: return launch_t<N, STRIDED, LINE_GREEN>(a, s);
    case LINE_INV: return launch_t<N, STRIDED, LINE_INV>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool line_pass_tma_supported(int N, bool strided, long long outer, long long inner) {
  if (N != 128 && N != 256) return false;
  // the TMA coordinates are 32-bit, the strided box spans kLpb inner points
  // (the inner extent must hold whole 16-byte pairs), outer fits an int
  if (outer > 0x7fffffffLL || inner > 0x7fffffffLL) return false;
  if (strided && (inner % 2) != 0) return false;
  return encode_fn() != nullptr;
}

cudaError_t launch_edge_pass_tma(int N, bool strided, int variant, const PsiPassArgs& a,
                                 int* status, cudaStream_t s) {
  if (!line_pass_tma_supported(N, strided, a.outer, a.inner) || a.nfields > 1 || a.rh_accum ||
      a.tc != nullptr || (variant != PSI_NPHASE && variant != PSI_DENSITY))
    return cudaErrorNotSupported;
  const int edge = variant == PSI_NPHASE ? EDGE_PHASE : EDGE_DENSITY;
  if (N == 256) {
    if (strided) return edge == EDGE_PHASE ? launch_edge_t<256, true, EDGE_PHASE>(a, status, s)
                                           : launch_edge_t<256, true, EDGE_DENSITY>(a, status, s);
    return edge == EDGE_PHASE ? launch_edge_t<256, false, EDGE_PHASE>(a, status, s)
                              : launch_edge_t<256, false, EDGE_DENSITY>(a, status, s);
  }
  if (strided) return edge == EDGE_PHASE ? launch_edge_t<128, true, EDGE_PHASE>(a, status, s)
                                         : launch_edge_t<128, true, EDGE_DENSITY>(a, status, s);
  return edge == EDGE_PHASE ? launch_edge_t<128, false, EDGE_PHASE>(a, status, s)
                            : launch_edge_t<128, false, EDGE_DENSITY>(a, status, s);
}

cudaError_t launch_line_pass_tma(int N, bool strided, int op, const LinePassArgs& a,
                                 cudaStream_t s) {
  if (!line_pass_tma_supported(N, strided, a.outer, a.inner)) return cudaErrorNotSupported;
  if (N == 256) return strided ? dispatch_op<256, true>(op, a, s) : dispatch_op<256, false>(op, a, s);
  return strided ? dispatch_op<128, true>(op, a, s) : dispatch_op<128, false>(op, a, s);
}

}  // namespace sn

// Device side of the batched scan (scan.cu): the per-instance description,
// the work items, the bounded dependency wait and the persistent kernel,
// templated on the register budget (resident CTAs per SM).  Each budget is
// instantiated in a translation unit of its own (scan_k1.cu, scan_k2.cu,
// scan_k3.cu), so the three compile in parallel; scan.cu holds the host side.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "sn.h"
#include "sn_internal.h"
#include "tile_ops.cuh"

namespace sn_scan {

using namespace sn;
using snfft::cx;
using snfft::Plan;

constexpr double kPi = 3.14159265358979323846;
constexpr int kThreads = 256;  // threads per CTA for every line length
// Resident CTAs per SM the registers are sized for: 3 (80 registers a
// thread, the default), 2 (128) or 1 (255), chosen per batch
// (sn_set_batch_ctas): fewer CTAs hide less latency, more spill the three-stage
// 512- and 1024-point items.
constexpr int kDefaultCtasPerSm = 3;
constexpr int kMaxLog2 = 10;

template <int N>
struct ScanCfg {
  static constexpr int T = Plan<N>::T;
  static constexpr int LPB = kThreads / T;  // lines per tile
  using C = tile::Cfg<N, LPB>;
  // the line buffers; the staged half-spectrum tile of a potential item
  // ([H][LPB + 1]) is read into registers before they are used, so it
  // occupies them too
  static constexpr size_t smem_words = (size_t)LPB * C::LS;
  static_assert((size_t)C::H * C::TSTR <= smem_words, "half-spectrum tile must fit the line buffers");
};

constexpr size_t max_words() {
  size_t w = 0;
  w = std::max(w, ScanCfg<8>::smem_words);
  w = std::max(w, ScanCfg<16>::smem_words);
  w = std::max(w, ScanCfg<32>::smem_words);
  w = std::max(w, ScanCfg<64>::smem_words);
  w = std::max(w, ScanCfg<128>::smem_words);
  w = std::max(w, ScanCfg<256>::smem_words);
  w = std::max(w, ScanCfg<512>::smem_words);
  w = std::max(w, ScanCfg<1024>::smem_words);
  return w;
}
constexpr size_t kSmemBytes = max_words() * sizeof(cx<float>);

inline int log2i(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

inline int lines_per_tile(int n) { return kThreads / (n / snfft::plan_e(n)); }

// Per-instance description, device resident.
struct Inst {
  int n;
  int pad;
  float2* psi;          // n x n
  float2* rho;          // (n/2 + 1) x n half spectrum
  const float2* tw;     // twiddles of length n (hi, lo)
  const float2* mult;   // [half, full] x n kinetic factors as shears (float4), same for both axes
  const float* k2;      // n entries
  float cN, cY, mu2, gh;
  unsigned t_psi, t_rho;  // tiles per psi pass and per Green's pass
};

// One work item of a round: queue position of the instance, slot | (items of
// the instance's earlier slots in the round) << 2, tile, items of the
// instance per round.  Item q of the launch is entry q mod per_round of round
// q / per_round.
struct ScanArgs {
  const Inst* inst;
  int count;
  int nsteps;
  const int4* items;                      // [per_round] items of one round in queue order
  unsigned long long per_round;           // items of a full round
  unsigned long long total;               // items of the whole launch
  unsigned* done;                         // [count] finished items per instance
  int* err;                               // [2]: code, queue index
  long long wait_limit;                   // clock cycles per wait
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Bounded wait (thread 0): true when done[i] >= req.
__device__ inline bool wait_for(const ScanArgs& a, int i, unsigned req, unsigned long long q) {
  if (ld_acquire(a.done + i) >= req) return true;
  const long long t0 = clock64();
  for (;;) {
    __nanosleep(64);
    if (ld_acquire(a.done + i) >= req) return true;
    if (ld_relaxed(a.err) != 0) return false;
    if (clock64() - t0 > a.wait_limit) {
      if (atomicCAS(a.err, 0, 1) == 0) a.err[1] = (int)q;
      return false;
    }
  }
}

template <int N, bool STRIDED, int VARIANT>
__device__ __forceinline__ void psi_item(const Inst& d, int full, long long tau, unsigned char* smem) {
  using S = ScanCfg<N>;
  using C = typename S::C;
  constexpr int LPB = S::LPB, E = C::E, T = C::T, LS = C::LS, H = C::H, TSTR = C::TSTR;
  constexpr bool CONTIG = !STRIDED;  // line l held by threads [l T, (l + 1) T)
  cx<float>* lines = reinterpret_cast<cx<float>*>(smem);
  cx<float>* rtile = lines;  // staged tile of a potential item, read before the lines are used
  const int tid = threadIdx.x;
  const int l = STRIDED ? (tid % LPB) : (tid / T);
  const int t = STRIDED ? (tid / LPB) : (tid % T);
  const tile::Tiles<LPB, STRIDED> tiles(STRIDED ? 1 : N, STRIDED ? N : 1);
  long long line0, o, i;
  int nvalid;
  size_t base;
  tiles.at(tau, l, N, line0, nvalid, base, o, i);
  const bool valid = l < nvalid;
  const unsigned ustride = STRIDED ? (unsigned)N : 1u;
  const cx<float>* tw = reinterpret_cast<const cx<float>*>(d.tw);
  const float4* lift = reinterpret_cast<const float4*>(d.mult) + full * N;
  const float* vrow = nullptr;
  (void)vrow;
  if constexpr (VARIANT == PSI_NPHASE) {
    for (int idx = tid; idx < H * LPB; idx += kThreads) {
      const int ll = idx % LPB, k = idx / LPB;
      cx<float> z = {0.f, 0.f};
      if (ll < nvalid) z = tile::ldg_c<true>(d.rho + (size_t)k * N + line0 + ll);
      rtile[k * TSTR + ll] = z;
    }
    __syncthreads();
    vrow = tile::potential_c2r<N, LPB, CONTIG, false, STRIDED, true>(rtile, lines, tw, l, t);
  }
  cx<float> v[E];
  tile::load_line<E, T, true>(v, d.psi + base, ustride, t, valid);
  if constexpr (VARIANT == PSI_NPHASE)
    tile::nonlinear_phase<E, T>(v, vrow, d.gh, nullptr, 0.f, ustride, t, valid);
  tile::kinetic<N, CONTIG>(v, lines + l * LS, tw, lift, t);
  tile::store_line<E, T>(v, d.psi + base, ustride, t, valid);
  if constexpr (VARIANT == PSI_DENSITY) {
    float2* rh = d.rho;
    auto put = [&](int k, int ll, cx<float> z) { tile::stg_c(rh + (size_t)k * N + line0 + ll, z); };
    tile::density_r2c<N, LPB, CONTIG, decltype(put), false, STRIDED>(v, valid, lines, tw, l, t, tid,
                                                                 nvalid, put);
  }
}

template <int N>
__device__ __forceinline__ void green_item(const Inst& d, long long tau, unsigned char* smem) {
  using S = ScanCfg<N>;
  using C = typename S::C;
  constexpr int LPB = S::LPB, E = C::E, T = C::T, LS = C::LS;
  cx<float>* lines = reinterpret_cast<cx<float>*>(smem);
  const int tid = threadIdx.x;
  const int l = tid / T, t = tid % T;
  const tile::Tiles<LPB, false> tiles(N / 2 + 1, 1);
  long long line0, o, i;
  int nvalid;
  size_t base;
  tiles.at(tau, l, N, line0, nvalid, base, o, i);
  const bool valid = l < nvalid;
  cx<float> v[E];
  tile::load_line<E, T, true>(v, d.rho + base, 1u, t, valid);
  const float k2pm = valid ? d.k2[o] : 0.f;
  tile::green<N, true>(v, lines + l * LS, reinterpret_cast<const cx<float>*>(d.tw), d.k2, k2pm,
                       d.cN, d.cY, d.mu2, 0.f, t);
  tile::store_line<E, T>(v, d.rho + base, 1u, t, valid);
}

template <int N>
__device__ void run_item(const Inst& d, int r, int s, int nsteps, long long tau,
                         unsigned char* smem) {
  // round r: axis order (0, 1) when r is even, (1, 0) when odd; axis 0 lines are strided
  const bool odd = (r & 1) != 0;
  const int full = (r == 0 || r == nsteps) ? 0 : 1;
  if (s == 2) {
    green_item<N>(d, tau, smem);
    return;
  }
  const int axis = (s == 0) ? (odd ? 1 : 0) : (odd ? 0 : 1);
  const bool strided = axis == 0;
  int variant = PSI_PLAIN;
  if (s == 0 && r > 0) variant = PSI_NPHASE;
  if (s == 1 && r < nsteps) variant = PSI_DENSITY;
  if (strided) {
    if (variant == PSI_NPHASE) psi_item<N, true, PSI_NPHASE>(d, full, tau, smem);
    else if (variant == PSI_DENSITY) psi_item<N, true, PSI_DENSITY>(d, full, tau, smem);
    else psi_item<N, true, PSI_PLAIN>(d, full, tau, smem);
  } else {
    if (variant == PSI_NPHASE) psi_item<N, false, PSI_NPHASE>(d, full, tau, smem);
    else if (variant == PSI_DENSITY) psi_item<N, false, PSI_DENSITY>(d, full, tau, smem);
    else psi_item<N, false, PSI_PLAIN>(d, full, tau, smem);
  }
}

template <int CPS>
__global__ void __launch_bounds__(kThreads, CPS) scan_kernel(ScanArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int4 s_item;
  __shared__ int s_round, s_go;
  for (unsigned long long q = blockIdx.x; q < a.total; q += gridDim.x) {
    // thread 0 decodes q -> (round, instance, slot, tile) and waits for the
    // instance's previous slot; the others meet it at the barrier
    if (threadIdx.x == 0) {
      const unsigned long long r = q / a.per_round;
      const int4 e = __ldg(a.items + (q - r * a.per_round));
      const unsigned req = (unsigned)r * (unsigned)e.w + ((unsigned)e.y >> 2);
      s_item = e;
      s_round = (int)r;
      s_go = (ld_relaxed(a.err) == 0) && wait_for(a, e.x, req, q);
    }
    __syncthreads();
    if (!s_go) return;
    const int4 e = s_item;
    const int inst = e.x, s = e.y & 3;
    const long long r = s_round, tau = e.z;
    const Inst d = a.inst[inst];
    switch (d.n) {
      case 8: run_item<8>(d, (int)r, s, a.nsteps, tau, smem); break;
      case 16: run_item<16>(d, (int)r, s, a.nsteps, tau, smem); break;
      case 32: run_item<32>(d, (int)r, s, a.nsteps, tau, smem); break;
      case 64: run_item<64>(d, (int)r, s, a.nsteps, tau, smem); break;
      case 128: run_item<128>(d, (int)r, s, a.nsteps, tau, smem); break;
      case 256: run_item<256>(d, (int)r, s, a.nsteps, tau, smem); break;
      case 512: run_item<512>(d, (int)r, s, a.nsteps, tau, smem); break;
      default: run_item<1024>(d, (int)r, s, a.nsteps, tau, smem); break;
    }
    __syncthreads();  // every store of this item precedes the release below
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(a.done + inst, 1u);
    }
  }
}


using ScanKern = void (*)(ScanArgs);
// the kernel of register budget cps (1, 2, 3), from its own translation unit
ScanKern scan_kernel_1();
ScanKern scan_kernel_2();
ScanKern scan_kernel_3();

}  // namespace sn_scan

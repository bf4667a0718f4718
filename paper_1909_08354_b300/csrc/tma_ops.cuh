// Device building blocks of the TMA-staged pass kernels (passes_tma.cu).
//
// A pass kernel moves each tile of LPB lines between HBM and shared memory
// with the tensor-memory accelerator (cp.async.bulk.tensor): a load completes
// on an mbarrier, a store is a bulk group read from shared memory by the copy
// engine.  The threads only transform: they read the tile into registers in
// pattern P (sn_fft.cuh), run the line transforms with their stage exchanges
// in the tile's own shared memory, and write the result back for the store.
//
// Exchange layouts (8-byte words, 32 banks = 16 bank pairs per half-warp):
//   strided lines (half-warp = 16 lines at one position): [pos][line], the
//     TMA tile's own layout, so the 16 lanes always hit 16 bank pairs;
//   contiguous lines (half-warp = the T threads of 16 / T lines): [line][pos]
//     with the low four bits of pos XOR-swizzled (xw below), chosen so that
//     every write and read of the 2-stage Stockham exchange of 64-, 128- and
//     256-point lines is served in the minimum two wavefronts per warp.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sn_fft.cuh"

namespace sn {
namespace tma {

using snfft::cx;
using snfft::Plan;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// ---- mbarriers ---------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
// make the initialised barriers visible to the async proxy (the TMA unit)
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of bar, giving up after `budget` clock cycles.
// Returns whether the phase completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity,
                                                  long long budget) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

// ---- bulk tensor copies ---------------------------------------------------------
__device__ __forceinline__ void tma_load_2d(void* dst, const void* map, int c0, int c1,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const void* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_2d(const void* map, int c0, int c1, const void* src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(c0), "r"(c1), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void tma_store_3d(const void* map, int c0, int c1, int c2,
                                             const void* src) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];\n" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(src))
      : "memory");
}
// L2 policy for data the next kernels do not read soon: psi written by a pass
// (134 MB at 256^3, larger than L2) goes first, so that the half spectrum the
// density pass writes beside it is still in L2 for the next pass.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
  return pol;
}
// the tile stores with an L2 cache policy
__device__ __forceinline__ void tma_store_2d_ef(const void* map, int c0, int c1, const void* src,
                                                uint64_t pol) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group.L2::cache_hint"
      " [%0, {%1, %2}], [%3], %4;\n" ::"l"(reinterpret_cast<uint64_t>(map)),
      "r"(c0), "r"(c1), "r"(smem_u32(src)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void tma_store_3d_ef(const void* map, int c0, int c1, int c2,
                                                const void* src, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group.L2::cache_hint"
      " [%0, {%1, %2, %3}], [%4], %5;\n" ::"l"(reinterpret_cast<uint64_t>(map)),
      "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(src)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}
// at most N of this thread's bulk groups still reading shared memory
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(N) : "memory");
}
// every bulk group of this thread complete (its global writes done)
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
}
// generic-proxy writes to shared memory, made visible to a following bulk store
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// ---- exchange layouts -----------------------------------------------------------
// Word of position pos of line l in a tile slot (see the top of this file).
template <int N, bool STRIDED, int LPB>
__device__ __forceinline__ int xw(int l, int pos) {
  if constexpr (STRIDED) {
    return pos * LPB + l;
  } else if constexpr (N == 256) {
    return l * N + (pos ^ ((pos >> 4) & 15));
  } else if constexpr (N == 128) {
    return l * N + (pos ^ ((pos >> 3) & 6) ^ ((pos >> 6) & 1) ^ ((l & 1) ? 9 : 0));
  } else if constexpr (N == 64) {
    // a half-warp holds 4 lines of 4 threads: the low bits take pos bits 4, 5
    // and the line's two low bits
    const int sw = ((pos >> 4) & 1) ^ (((pos >> 5) & 1) << 1) ^ ((l & 1) ? 5 : 0) ^ ((l & 2) ? 10 : 0);
    return l * N + (pos ^ sw);
  } else {
    return l * N + pos;
  }
}

// Barrier among the threads that touch one line's words: the CTA for strided
// tiles (a line's positions are spread over every warp), the warp otherwise
// (a line of T <= 32 threads sits in one warp, and its words in its own row).
template <bool STRIDED>
__device__ __forceinline__ void xsync() {
  if constexpr (STRIDED) __syncthreads();
  else __syncwarp();
}

// Twiddle table of N in shared memory as one float4 (hi.re, hi.im, lo.re,
// lo.im) per entry, from the global table's hi parts [0, TWN) and lo parts
// [TWN, 2 TWN): one 128-bit load per twiddle product.
template <int N>
__device__ __forceinline__ void stage_twiddles(float4* tw4, const float2* tw, int tid, int nt) {
  constexpr int TWN = Plan<N>::TWN;
  for (int k = tid; k < TWN; k += nt) {
    const float2 h = tw[k], lo = tw[TWN + k];
    tw4[k] = make_float4(h.x, h.y, lo.x, lo.y);
  }
}

// In-place transform of my line (pattern P in and out), 2-stage Stockham plans
// (32 <= N <= 256), with the stage exchange in the tile slot `buf` at the
// words xw(l, pos).  Same arithmetic as snfft::line_transform (the twiddle
// product is snfft::cmul_hl of the same hi and lo parts).
template <int N, int SIGN, bool STRIDED, int LPB>
__device__ __forceinline__ void xform(cx<float> (&v)[Plan<N>::E], cx<float>* buf,
                                      const float4* tw4, int l, int t) {
  using P = Plan<N>;
  static_assert(P::STAGES == 2, "the TMA passes take 2-stage line plans");
  constexpr int E = P::E, T = P::T;
  constexpr int RA = SIGN < 0 ? P::R0 : P::R1;
  constexpr int RB = SIGN < 0 ? P::R1 : P::R0;
  constexpr int UA = E / RA, UB = E / RB;
  xsync<STRIDED>();  // earlier readers of these words are done
#pragma unroll
  for (int u = 0; u < UA; ++u) {
    cx<float> a[RA];
#pragma unroll
    for (int r = 0; r < RA; ++r) a[r] = v[u + r * UA];
    snfft::dft<float, SIGN, RA>(a);
    const int j = t + T * u;
#pragma unroll
    for (int q = 0; q < RA; ++q) buf[xw<N, STRIDED, LPB>(l, j * RA + q)] = a[q];
  }
  xsync<STRIDED>();
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = buf[xw<N, STRIDED, LPB>(l, t + T * m)];
  const float4* tw = tw4 + (SIGN < 0 ? 0 : N);
#pragma unroll
  for (int u = 0; u < UB; ++u) {
    const int j = t + T * u;
    const int jm = j & (RA - 1);
    cx<float> a[RB];
    a[0] = v[u];
#pragma unroll
    for (int r = 1; r < RB; ++r) {
      const float4 w = tw[r * RA + jm];
      a[r] = snfft::cmul_hl(v[u + r * UB], {w.x, w.y}, {w.z, w.w});
    }
    snfft::dft<float, SIGN, RB>(a);
#pragma unroll
    for (int q = 0; q < RB; ++q) v[u + q * UB] = a[q];
  }
}

}  // namespace tma
}  // namespace sn

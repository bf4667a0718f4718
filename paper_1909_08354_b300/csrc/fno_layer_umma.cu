// The second half of an FNO spectral layer in one tcgen05 kernel: the inverse
// truncated DFT along x, the 1x1 convolution, the bias and the activation.
//
// For a sample b, a row y and 128 consecutive x, the layer's pre-activation is
//   z[b][o][y][x] = sum_q WxI[q][x] B1[b][o][y][q] + sum_c W[o][c] v[b][c][y][x] + bias[o]
// (q < 2m over the row's inverse-DFT coefficients along y already applied,
// c < C over the input channels).  As one product D[x][o] with M = 128 rows
// x, N = C columns o: A1[x][q] = WxI[q][x] against B1[o][q], then
// A2[x][c] = v[b][c][y][x] against W[o][c], both groups accumulating in
// tensor memory (tcgen05.mma kind::f16 with BF16 operands, FP32
// accumulation: the rounding of the GEMMs it replaces).  The epilogue reads
// row x of D (tcgen05.ld), adds the bias and writes z and the activation
// v' = GELU(z) (or z itself after the last layer).  It replaces the inverse
// GEMM along x (which wrote z), the 1x1 GEMM (which read v and z and wrote
// z) and the bias/activation pass (which read z and wrote z and v'): three
// passes over the layer's activations instead of six.
//
// One CTA of 256 threads takes tiles (b, y, x0) in turn; threads i and
// i + 128 stage row x0 + i of A2 (each half the channels; the loads of v are
// coalesced across the warp) and read row i of the accumulator, warps 0-3
// its first half of the columns and warps 4-7 the second (a warp reaches the
// 32 tensor-memory lanes of its rank modulo 4).  The operands of the next tile and its
// accumulator are double-buffered, so the staging of tile i + 1 overlaps the
// products of tile i.  Every wait is bounded (the status word, then a
// bounded wait for the products in flight, then the tensor memory is freed).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sn_internal.h"
#include "tma_ops.cuh"

namespace sn {
namespace {

constexpr int kRows = 128;     // x per tile (M)
constexpr int kThreads = 256;  // two threads per row: each stages half the channels
constexpr int kMaxC = 64;      // channels (N, K2) the kernel takes
constexpr int kMaxQ = 64;      // 2m (K1) the kernel takes
constexpr long long kWaitCycles = 4000000000LL;

__host__ __device__ constexpr int pad16(int v) { return (v + 15) / 16 * 16; }

// Byte offset of (row, k) in a K-major operand of K halves a row, no swizzle:
// core matrices of 8 rows x 16 bytes, K-neighbours 128 bytes apart, 8-row
// groups K / 8 * 128 bytes apart.
__device__ __forceinline__ unsigned opo(int row, int k, int K) {
  return (unsigned)(((row >> 3) * (K >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}
__device__ __forceinline__ uint64_t sdesc(unsigned saddr, int K) {
  const unsigned lbo = 128, sbo = (unsigned)(K >> 3) * 128;
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// kind::f16, FP32 accumulator, BF16 A and B (format 1), both K-major, N, M = 128
__device__ __forceinline__ uint32_t idesc_bf16(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}

__device__ __forceinline__ void umma(unsigned tmem, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %3, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %4, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(acc), "r"(idesc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                   tma::smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void ld16(unsigned taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void put_bf16(unsigned char* base, unsigned off, float x) {
  *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(x);
}
// elements k and k + 1 (k even) of a row: one 4-byte store
__device__ __forceinline__ void put_bf16x2(unsigned char* base, unsigned off, float x0, float x1) {
  *reinterpret_cast<__nv_bfloat162*>(base + off) = __floats2bfloat162_rn(x0, x1);
}

// GELU, the erf form of the network's other activation passes
__device__ __forceinline__ float gelu_erf(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
// its derivative, the form of the network's other backward passes
__device__ __forceinline__ float gelu_grad_erf(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * __expf(-0.5f * x * x);
}

struct LayerArgs {
  const float* v;    // [B][C][s][s] layer input (backward: the gradient dz)
  const float* B1;   // [B][C][s][2m] the inverse DFT along y, per row
  const float* WxI;  // [2m][s] inverse DFT along x
  const float* W;    // [C][C] 1x1 weights W[o][c]
  const float* bias; // [C] (forward)
  float* z;          // [B][C][s][s] forward: the pre-activation (with the bias)
  float* vout;       // [B][C][s][s] forward: the activation; backward: the gradient out
  const float* zp;   // backward: the previous layer's pre-activation (its GELU' scales
                     // the gradient), or NULL for none
  int B, C, s, Q, act;
  int back;          // 1: the backward form (W transposed, no bias, vout = D GELU'(zp))
  int* status;
};

// shared-memory plan (bytes) for C channels, Q = 2m
struct Plan {
  int N, K1, K2;
  unsigned a1, b2, a2[2], b1[2], bytes;
};
__host__ __device__ inline Plan plan_of(int C, int Q) {
  Plan p{};
  p.N = pad16(C);
  p.K1 = pad16(Q);
  p.K2 = pad16(C);
  unsigned o = 0;
  p.a1 = o; o += 2u * kRows * p.K1 * 2;  // two halves of WxI^T: [2][128][K1]
  p.b2 = o; o += (unsigned)p.N * p.K2 * 2;
  for (int i = 0; i < 2; ++i) { p.a2[i] = o; o += (unsigned)kRows * p.K2 * 2; }
  for (int i = 0; i < 2; ++i) { p.b1[i] = o; o += (unsigned)p.N * p.K1 * 2; }
  p.bytes = o;
  return p;
}

__global__ void __launch_bounds__(kThreads, 2) fno_layer_kernel(LayerArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ unsigned tmem_slot;
  const Plan P = plan_of(a.C, a.Q);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int s = a.s, C = a.C, Q = a.Q;
  const int halves = (s + kRows - 1) / kRows;
  const long long tiles = (long long)a.B * s * halves;
  // constants: WxI^T for each x block of the tile grid (at most two blocks of
  // 128 are kept; wider rows are not taken) and W
  for (int i = tid; i < 2 * kRows * P.K1; i += kThreads) {
    const int h = i / (kRows * P.K1), r = (i / P.K1) % kRows, q = i % P.K1;
    const int x = h * kRows + r;
    const float w = (q < Q && x < s && h < halves) ? a.WxI[(long long)q * s + x] : 0.f;
    put_bf16(sm + P.a1 + (unsigned)h * kRows * P.K1 * 2, opo(r, q, P.K1), w);
  }
  for (int i = tid; i < P.N * P.K2; i += kThreads) {
    const int o = i / P.K2, c = i % P.K2;
    // forward: W[o][c]; backward: the transpose, W[c][o]
    const long long wi = a.back ? (long long)c * C + o : (long long)o * C + c;
    put_bf16(sm + P.b2, opo(o, c, P.K2), (o < C && c < C) ? a.W[wi] : 0.f);
  }
  if (tid == 0) {
    tma::mbar_init(&bar[0], 1);
    tma::mbar_init(&bar[1], 1);
    tma::mbar_fence_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     tma::smem_u32(&tmem_slot)),
                 "r"(128)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const unsigned tmem = tmem_slot;
  const uint32_t idesc = idesc_bf16(P.N);

  // stage tile tau into buffer u: A2 row tid (v along c), B1 (o, q)
  const int row = tid & (kRows - 1), part = tid >> 7;  // my row of the tile, my half
  auto stage = [&](long long tau, int u) {
    const int h = (int)(tau % halves);
    const long long by = tau / halves;
    const int y = (int)(by % s), b = (int)(by / s);
    const int x = h * kRows + row;
    unsigned char* A2 = sm + P.a2[u];
    const size_t plane = (size_t)s * s;
    if ((s & 3) == 0) {
      // float4 along x: warp g takes channels 8 g .. 8 g + 7, lane l the four
      // rows 4 l .. 4 l + 3 (a warp's load is 512 contiguous bytes)
      const int g = tid >> 5, l = tid & 31;
      const int xr = h * kRows + 4 * l;
      for (int cb = 8 * g; cb < P.K2; cb += 8 * (kThreads / 32)) {
        const float* vp4 = a.v + ((size_t)b * C * s + y) * s + xr + (size_t)cb * plane;
#pragma unroll
        for (int c = 0; c < 8; c += 2) {
          float4 p0 = make_float4(0.f, 0.f, 0.f, 0.f), p1 = p0;
          if (xr < s && cb + c < C) p0 = __ldg(reinterpret_cast<const float4*>(vp4 + (size_t)c * plane));
          if (xr < s && cb + c + 1 < C) p1 = __ldg(reinterpret_cast<const float4*>(vp4 + (size_t)(c + 1) * plane));
          put_bf16x2(A2, opo(4 * l + 0, cb + c, P.K2), p0.x, p1.x);
          put_bf16x2(A2, opo(4 * l + 1, cb + c, P.K2), p0.y, p1.y);
          put_bf16x2(A2, opo(4 * l + 2, cb + c, P.K2), p0.z, p1.z);
          put_bf16x2(A2, opo(4 * l + 3, cb + c, P.K2), p0.w, p1.w);
        }
      }
    } else {
    const int ch = P.K2 / 2, c0 = part * ch;  // my channels [c0, c0 + ch)
    const int cend = min(c0 + ch, x < s ? C : 0);  // channels with data; the rest are zero
    const float* vp = a.v + ((size_t)b * C * s + y) * s + x + (size_t)c0 * plane;
    int c = c0;
#pragma unroll 4
    for (; c + 1 < cend; c += 2, vp += 2 * plane) {
      // consecutive channel pairs: 4 bytes on in a core matrix, 128 bytes on every 8
      put_bf16x2(A2, opo(row, c, P.K2), vp[0], vp[plane]);
    }
    for (; c < c0 + ch; c += 2) {
      const float w0 = c < cend ? vp[0] : 0.f;
      put_bf16x2(A2, opo(row, c, P.K2), w0, 0.f);
      vp += 2 * plane;
    }
    }

    unsigned char* B1s = sm + P.b1[u];
    const float* bp = a.B1 + ((long long)b * C * s + y) * Q;  // (b, o = 0, y, q = 0)
    for (int i = tid; i < P.N * P.K1 / 2; i += kThreads) {
      const int o = (2 * i) / P.K1, q = (2 * i) % P.K1;
      const float* r = bp + (long long)o * s * Q;
      const float w0 = (o < C && q < Q) ? r[q] : 0.f;
      const float w1 = (o < C && q + 1 < Q) ? r[q + 1] : 0.f;
      put_bf16x2(B1s, opo(o, q, P.K1), w0, w1);
    }
  };
  auto issue = [&](long long tau, int u) {
    const int h = (int)(tau % halves);
    const unsigned d = tmem + (unsigned)(u * 64);
    const uint64_t a1 = sdesc(tma::smem_u32(sm + P.a1 + (unsigned)h * kRows * P.K1 * 2), P.K1);
    const uint64_t b1 = sdesc(tma::smem_u32(sm + P.b1[u]), P.K1);
    const uint64_t a2 = sdesc(tma::smem_u32(sm + P.a2[u]), P.K2);
    const uint64_t b2 = sdesc(tma::smem_u32(sm + P.b2), P.K2);
    fence_after();
    for (int k = 0; k < P.K1 / 16; ++k) umma(d, a1 + 16ull * k, b1 + 16ull * k, idesc, k > 0);
    for (int k = 0; k < P.K2 / 16; ++k) umma(d, a2 + 16ull * k, b2 + 16ull * k, idesc, 1);
    umma_commit(&bar[u]);
  };

  long long tau = blockIdx.x;
  unsigned phase[2] = {0u, 0u};
  bool failed = false;
  int pend[2] = {0, 0};  // products committed to bar[u] and not yet waited for
  if (tau < tiles) {
    stage(tau, 0);
    tma::fence_proxy_async();
    fence_before();
    __syncthreads();
    if (tid == 0) issue(tau, 0);
    pend[0] = 1;
  }
  for (int it = 0; tau < tiles; ++it, tau += gridDim.x) {
    const int u = it & 1;
    const long long nxt = tau + gridDim.x;
    if (nxt < tiles) stage(nxt, u ^ 1);  // overlaps the products of tile tau
    tma::fence_proxy_async();
    fence_before();
    __syncthreads();
    if (tid == 0 && nxt < tiles) issue(nxt, u ^ 1);
    if (nxt < tiles) pend[u ^ 1] = 1;
    const bool ok = tma::mbar_wait_bounded(&bar[u], phase[u], kWaitCycles);
    if (!__syncthreads_and(ok)) {
      failed = true;
      break;
    }
    phase[u] ^= 1u;
    pend[u] = 0;
    fence_after();
    // epilogue: row tid of D = pixel (b, y, x), columns o
    const int h = (int)(tau % halves);
    const long long by = tau / halves;
    const int y = (int)(by % s), b = (int)(by / s);
    const int x = h * kRows + row;
    const unsigned d = tmem + ((unsigned)((warp & 3) * 32) << 16) + (unsigned)(u * 64);
    const size_t plane = (size_t)s * s;
    const size_t base = ((size_t)b * C * s + y) * s + x;  // (b, o = 0, y, x)
    // columns of my half: 16-column chunks alternate between the two halves
    for (int c0 = part * 16; c0 < P.N; c0 += 32) {
      float r[16];
      ld16(d + (unsigned)c0, r);
      if (x < s && a.back) {
        // gradient: D, times GELU'(z) of the previous layer where it has one
        float* gq = a.vout + base + (size_t)c0 * plane;
        const float* zq = a.zp != nullptr ? a.zp + base + (size_t)c0 * plane : nullptr;
        const int n = min(16, C - c0);
        for (int j = 0; j < n; ++j) gq[j * plane] = zq != nullptr ? r[j] * gelu_grad_erf(zq[j * plane]) : r[j];
      } else if (x < s) {
        float* zp = a.z + base + (size_t)c0 * plane;
        float* vq = a.vout + base + (size_t)c0 * plane;
        const int n = min(16, C - c0);
        if (n == 16) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float zz = r[j] + __ldg(a.bias + c0 + j);
            zp[j * plane] = zz;
            vq[j * plane] = a.act ? gelu_erf(zz) : zz;
          }
        } else {
          for (int j = 0; j < n; ++j) {
            const float zz = r[j] + __ldg(a.bias + c0 + j);
            zp[j * plane] = zz;
            vq[j * plane] = a.act ? gelu_erf(zz) : zz;
          }
        }
      }
    }
    fence_before();
    __syncthreads();  // the accumulator u is read before tile tau + 2 G reuses it
  }
  if (failed) {
    if (tid == 0) atomicExch(a.status, 1);
    for (int u = 0; u < 2; ++u)
      if (pend[u]) (void)tma::mbar_wait_bounded(&bar[u], phase[u], kWaitCycles / 8);
    fence_before();
    __syncthreads();
  }
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(128)
                 : "memory");
  }
}

}  // namespace

bool fno_layer_umma_supported(int C, int Q, int s) {
  return C >= 1 && C <= kMaxC && Q >= 2 && Q <= kMaxQ && (Q & 1) == 0 && s <= 2 * kRows;
}

cudaError_t launch_fno_layer_umma(const float* v, const float* B1, const float* WxI, const float* W,
                                  const float* bias, float* z, float* vout, const float* zp, int B,
                                  int C, int s, int Q, int act, int back, int* status, cudaStream_t st) {
  if (!fno_layer_umma_supported(C, Q, s)) return cudaErrorNotSupported;
  const Plan P = plan_of(C, Q);
  static bool attr_of[kDeviceSlots] = {};
  bool& attr = attr_of[device_slot()];
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(fno_layer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fno_layer_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  static int sms_of[kDeviceSlots] = {};
  int& sms = sms_of[device_slot()];
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  const long long tiles = (long long)B * s * ((s + kRows - 1) / kRows);
  // two CTAs per SM where their shared memory fits (registers: 2 x 256 threads
  // at the 128-register bound; tensor memory: 2 x 128 of the 512 columns)
  static int smem_sm_of[kDeviceSlots] = {};
  int& smem_sm = smem_sm_of[device_slot()];
  if (smem_sm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  }
  const int per_sm = 2 * ((long long)P.bytes + 2048) <= (long long)smem_sm ? 2 : 1;
  const long long grid = std::min<long long>(tiles, (long long)per_sm * sms);
  LayerArgs a{v, B1, WxI, W, bias, z, vout, zp, B, C, s, Q, act, back, status};
  fno_layer_kernel<<<(unsigned)grid, kThreads, P.bytes, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sn

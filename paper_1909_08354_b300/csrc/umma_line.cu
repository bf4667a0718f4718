// 256-point line DFTs with both radix-16 stages on the fifth-generation tensor
// cores: tcgen05.mma (kind::f16, FP16 operands in shared memory, FP32
// accumulators in tensor memory), read back with tcgen05.ld (Sec. III's FFT of
// the split step, in the split-FP16 form of the tensor-core engine).
//
// A 256-point DFT is 16 x 16 with n = 16 r + t and k = k1 + 16 k2: stage A is a
// 16-point DFT over r for each column t, then the twiddle w256^(t k1), then
// stage B a 16-point DFT over t for each k1.  A complex 16-point DFT of a
// vector is one real product with the 32 x 32 real form of F16, so a stage of
// 8 lines (128 vectors) is one M = 128, N = 32, K = 32 matrix product:
// D[v][n] = sum_k A[v][k] F[n][k], each row v a vector's 16 (re, im) pairs.
// Both operands are split, x = x_hi + x_lo and F = F_hi + F_lo in FP16, and
// D = x_hi F_lo + x_lo F_hi + x_hi F_hi accumulates in FP32 (the small
// products first).  Rows are scaled by a power of two before the split (per
// vector in stage A, per line in stage B), so that no value overflows FP16
// and the lo parts stay out of its subnormals; the DFT is linear per row, so
// the scale is taken back exactly afterwards.
//
// One CTA of 128 threads takes tiles of 8 lines; thread i owns vector i, which
// is also lane i of the accumulator in tensor memory.  One thread issues the
// MMAs; their completion arrives on an mbarrier (bounded waits: an expired
// wait sets the status word to 1, waits again, bounded, frees the tensor
// memory and returns).
//
// Each line's output is rescaled to 256 times its input's squared norm
// (Parseval): the tensor memory's FP32 accumulation loses a little of every
// product, always in the same direction.
//
// This is the measurement form of the tcgen05 engine (sn_test_line_fft_engines);
// the fused passes keep the FP32 and mma.sync engines.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sn_internal.h"
#include "tma_ops.cuh"

namespace sn {
namespace {

constexpr int kN = 256;
constexpr int kLines = 8;                    // lines per tile: 8 x 16 vectors = M
constexpr int kThreads = 128;                // one thread per vector (tensor-memory lane)
constexpr int kM = 128, kNr = 32, kK = 32;   // the MMA in reals
constexpr unsigned kOpBytes = kM * kK * 2;   // one FP16 A operand (8 KB)
constexpr unsigned kBBytes = kNr * kK * 2;   // one FP16 B operand (2 KB)
constexpr unsigned kTmemCols = 32;           // FP32 accumulator columns
constexpr long long kWaitCycles = 4000000000LL;
constexpr size_t kSmemBytes = 2 * kOpBytes + 2 * kBBytes;

// Byte offset of element (row, k) of an operand in the K-major layout without
// swizzle: core matrices of 8 rows x 8 halves (16 bytes a row, 128 bytes
// each), the K-neighbouring core matrix 128 bytes on, the next 8-row group
// 512 bytes on (K = 32 halves: 4 core matrices per row group).
__host__ __device__ constexpr unsigned op_off(int row, int k) {
  return (unsigned)(((row >> 3) * 4 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}
constexpr unsigned kLbo = 128, kSbo = 512;

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (K-neighbouring core matrices), stride byte offset (row groups), all
// >> 4; bits 46-47 the descriptor version 1; base offset 0; no swizzle.
__device__ __forceinline__ uint64_t sdesc(unsigned saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((kLbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((kSbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), FP16 A
// and B (bits 7-9, 10-12 = 0), both K-major (bits 15, 16 = 0), N >> 3 at bit
// 17, M >> 4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kNr >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);

__device__ __forceinline__ void umma_f16(unsigned tmem, uint64_t a, uint64_t b, int accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %3, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %4, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(accumulate), "r"(kIdesc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                   tma::smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
// whole warp: allocate ncols tensor-memory columns, address to *dst
__device__ __forceinline__ void tmem_alloc(unsigned* dst, unsigned ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                   tma::smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols)
               : "memory");
}
// whole warp: this thread's lane (row) of 32 consecutive FP32 columns
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// x -> (hi, lo) in FP16 at (row, k) and (row, k + 1) of the two operands
__device__ __forceinline__ void put_split(unsigned char* hi, unsigned char* lo, int row, int k,
                                          float re, float im) {
  const __half hr = __float2half_rn(re), hm = __float2half_rn(im);
  const __half lr = __float2half_rn(re - __half2float(hr)), lm = __float2half_rn(im - __half2float(hm));
  *reinterpret_cast<__half2*>(hi + op_off(row, k)) = __halves2half2(hr, hm);
  *reinterpret_cast<__half2*>(lo + op_off(row, k)) = __halves2half2(lr, lm);
}

// 2^-e with max |x| 2^-e in [2^14, 2^15), e = 0 for a zero row
__device__ __forceinline__ int row_exponent(float mx) { return mx > 0.f ? ilogbf(mx) - 14 : 0; }

struct UmmaArgs {
  float2* data;          // nlines contiguous lines of 256 complex64, in place
  long long nlines;
  const float2* tw;      // w256^j = exp(sign 2 pi i j / 256), j < 256
  const uint4* bmat;     // F_hi then F_lo (2 KB each) in the operand layout
  int* status;
  // TIMED: clock cycles of each phase of a tile, summed over tiles and CTAs
  // (as seen by thread 0, which meets every barrier), then the tiles done
  unsigned long long* cycles;
};

// Phases of a tile, as timed by the TIMED form.
enum { PH_STAGE_A_OPERANDS, PH_STAGE_A_MMA, PH_STAGE_B_OPERANDS, PH_STAGE_B_MMA, PH_OUTPUT, PH_COUNT };

template <bool TIMED>
__global__ void __launch_bounds__(kThreads, 4) umma_line_kernel(UmmaArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ unsigned tmem_slot;
  unsigned char* A_hi = sm;
  unsigned char* A_lo = sm + kOpBytes;
  unsigned char* B_hi = sm + 2 * kOpBytes;
  unsigned char* B_lo = B_hi + kBBytes;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < (int)(2 * kBBytes / 16); i += kThreads) reinterpret_cast<uint4*>(B_hi)[i] = a.bmat[i];
  if (tid == 0) {
    tma::mbar_init(&bar, 1);
    tma::mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(&tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = tmem_slot;
  const unsigned my_rows = tmem + ((unsigned)(warp * 32) << 16);  // this warp's 32 lanes
  const uint64_t dAhi = sdesc(tma::smem_u32(A_hi)), dAlo = sdesc(tma::smem_u32(A_lo));
  const uint64_t dBhi = sdesc(tma::smem_u32(B_hi)), dBlo = sdesc(tma::smem_u32(B_lo));
  constexpr uint64_t kStepK = 256 >> 4;  // K = 16..31: two core matrices on

  // the six products of one stage, the small ones first, then the commit
  auto issue_stage = [&]() {
    tc_fence_after();
    umma_f16(tmem, dAhi, dBlo, 0);
    umma_f16(tmem, dAhi + kStepK, dBlo + kStepK, 1);
    umma_f16(tmem, dAlo, dBhi, 1);
    umma_f16(tmem, dAlo + kStepK, dBhi + kStepK, 1);
    umma_f16(tmem, dAhi, dBhi, 1);
    umma_f16(tmem, dAhi + kStepK, dBhi + kStepK, 1);
    umma_commit(&bar);
  };

  const int li = tid >> 4, c = tid & 15;  // my line within the tile, my column (t, then k1)
  const long long tiles = (a.nlines + kLines - 1) / kLines;
  unsigned phase = 0;
  bool failed = false;
  unsigned long long spent[PH_COUNT] = {};
  unsigned long long done = 0;
  long long mark_t = 0;
  auto mark = [&](int ph) {
    if constexpr (TIMED) {
      if (tid == 0) {
        const long long now = clock64();
        spent[ph] += (unsigned long long)(now - mark_t);
        mark_t = now;
      }
    }
  };
  for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    if constexpr (TIMED) {
      if (tid == 0) mark_t = clock64();
    }
    const long long line = tile * kLines + li;
    const bool valid = line < a.nlines;
    float2* row = a.data + (valid ? line : 0) * kN;
    // ---- stage A: vector (li, t = c) of x[16 r + t]
    float xr[16], xi[16], mx = 0.f;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const float2 z = valid ? row[16 * r + c] : make_float2(0.f, 0.f);
      xr[r] = z.x;
      xi[r] = z.y;
      mx = fmaxf(mx, fmaxf(fabsf(z.x), fabsf(z.y)));
    }
    // the line's squared norm (its 16 threads are one half-warp): the output
    // must carry 256 times it (Parseval)
    float n_in = 0.f;
#pragma unroll
    for (int r = 0; r < 16; ++r) n_in = fmaf(xr[r], xr[r], fmaf(xi[r], xi[r], n_in));
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) n_in += __shfl_xor_sync(0xffffffffu, n_in, o);
    const int ea = row_exponent(mx);
    const float sa = ldexpf(1.f, -ea);
#pragma unroll
    for (int r = 0; r < 16; ++r) put_split(A_hi, A_lo, tid, 2 * r, xr[r] * sa, xi[r] * sa);
    tma::fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    mark(PH_STAGE_A_OPERANDS);
    if (tid == 0) issue_stage();
    bool ok = tma::mbar_wait_bounded(&bar, phase, kWaitCycles);
    phase ^= 1u;
    if (!__syncthreads_and(ok)) {
      failed = true;
      break;
    }
    mark(PH_STAGE_A_MMA);
    tc_fence_after();
    float d[32];
    tmem_ld32(my_rows, d);
    // Y[k1] of column t = c, unscaled, times w256^(t k1)
    const float ua = ldexpf(1.f, ea);
    float yr[16], yi[16], my = 0.f;
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) {
      const float2 w = a.tw[(c * k1) & 255];
      const float re = d[2 * k1] * ua, im = d[2 * k1 + 1] * ua;
      yr[k1] = fmaf(re, w.x, -im * w.y);
      yi[k1] = fmaf(re, w.y, im * w.x);
      my = fmaxf(my, fmaxf(fabsf(yr[k1]), fabsf(yi[k1])));
    }
    // ---- stage B: vector (li, k1) over t; the scale of the line's 16 threads
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, o));
    const int eb = row_exponent(my);
    const float sb = ldexpf(1.f, -eb);
    tc_fence_before();
    __syncthreads();  // every lane read stage A's accumulators; the operands are free
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) put_split(A_hi, A_lo, li * 16 + k1, 2 * c, yr[k1] * sb, yi[k1] * sb);
    tma::fence_proxy_async();
    __syncthreads();
    mark(PH_STAGE_B_OPERANDS);
    if (tid == 0) issue_stage();
    ok = tma::mbar_wait_bounded(&bar, phase, kWaitCycles);
    phase ^= 1u;
    if (!__syncthreads_and(ok)) {
      failed = true;
      break;
    }
    mark(PH_STAGE_B_MMA);
    tc_fence_after();
    tmem_ld32(my_rows, d);
    // X[k1 + 16 k2] with k1 = c, rescaled so that the line keeps 256 times
    // its input norm: the products' accumulation loses a little of it, always
    // in the same direction, and a per-line factor above half an FP32 ulp
    // takes the loss back on average
    float n_out = 0.f;
#pragma unroll
    for (int k = 0; k < 32; ++k) n_out = fmaf(d[k], d[k], n_out);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) n_out += __shfl_xor_sync(0xffffffffu, n_out, o);
    const float ub = ldexpf(1.f, eb);
    const float want = 256.f * n_in, have = n_out * ub * ub;
    const float fix = (have > 0.f && want > 0.f) ? sqrtf(want / have) : 1.f;
    const float ubf = ub * fix;
    if (valid) {
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) row[c + 16 * k2] = make_float2(d[2 * k2] * ubf, d[2 * k2 + 1] * ubf);
    }
    tc_fence_before();
    __syncthreads();  // the accumulators are read before the next tile's products
    mark(PH_OUTPUT);
    ++done;
  }
  if constexpr (TIMED) {
    if (tid == 0 && a.cycles) {
      for (int ph = 0; ph < PH_COUNT; ++ph) atomicAdd(a.cycles + ph, spent[ph]);
      atomicAdd(a.cycles + PH_COUNT, done);
    }
  }
  if (failed) {
    if (tid == 0) atomicExch(a.status, 1);
    // the products in flight still write the accumulators: wait for them (bounded)
    (void)tma::mbar_wait_bounded(&bar, phase ^ 1u, kWaitCycles / 8);
    tc_fence_before();
    __syncthreads();
  }
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace

// F16 in its real 32 x 32 form (row n = 2 k1 + c_out, column k = 2 r + c_in,
// w = exp(sign 2 pi i r k1 / 16)), split into FP16 hi and lo images in the
// operand layout (2 KB each, hi first).
void umma_line_tables(int sign, std::vector<uint16_t>& bmat, std::vector<float2>& tw) {
  constexpr double kTwoPi = 6.28318530717958647692;
  bmat.assign(2 * kBBytes / 2, 0);
  for (int k1 = 0; k1 < 16; ++k1)
    for (int r = 0; r < 16; ++r) {
      const double ph = sign * kTwoPi * (double)((r * k1) % 16) / 16.0;
      const double wr = std::cos(ph), wi = std::sin(ph);
      const double ent[2][2] = {{wr, -wi}, {wi, wr}};  // [c_out][c_in]
      for (int co = 0; co < 2; ++co)
        for (int ci = 0; ci < 2; ++ci) {
          const double x = ent[co][ci];
          const __half hi = __float2half_rn((float)x);
          const __half lo = __float2half_rn((float)(x - (double)__half2float(hi)));
          const unsigned off = op_off(2 * k1 + co, 2 * r + ci) / 2;
          uint16_t hb, lb;
          std::memcpy(&hb, &hi, 2);
          std::memcpy(&lb, &lo, 2);
          bmat[off] = hb;
          bmat[kBBytes / 2 + off] = lb;
        }
    }
  tw.resize(kN);
  for (int j = 0; j < kN; ++j) {
    const double ph = sign * kTwoPi * (double)j / kN;
    tw[j] = make_float2((float)std::cos(ph), (float)std::sin(ph));
  }
}

cudaError_t launch_umma_line(float2* data, long long nlines, const float2* tw, const void* bmat,
                             int* status, unsigned long long* cycles, cudaStream_t s) {
  static bool attr_of[kDeviceSlots] = {};
  bool& attr = attr_of[device_slot()];
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(umma_line_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(umma_line_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kSmemBytes);
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
  const long long tiles = (nlines + kLines - 1) / kLines;
  const long long grid = std::min<long long>(tiles, 4LL * sms);
  UmmaArgs a{data, nlines, tw, static_cast<const uint4*>(bmat), status, cycles};
  if (cycles) umma_line_kernel<true><<<(unsigned)grid, kThreads, kSmemBytes, s>>>(a);
  else umma_line_kernel<false><<<(unsigned)grid, kThreads, kSmemBytes, s>>>(a);
  return cudaGetLastError();
}

}  // namespace sn

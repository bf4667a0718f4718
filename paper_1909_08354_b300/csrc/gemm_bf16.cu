// Strided batched GEMM on the tensor cores: C = alpha * A B + beta * C with A,
// B read as FP32 from global memory, rounded to BF16 when they are staged in
// shared memory, multiplied by mma.sync m16n8k16 with FP32 accumulation.
//
// Every operand has element strides, so transposes, planar/interleaved complex
// parts and gathered mode matrices are plain stride choices.  Optional split-K:
// block (z, sp) sums k in [sp*kchunk, (sp+1)*kchunk) and writes its partial
// product to C + z*sCz + sp*sCsp (beta must be 0); reduce_sum adds partials.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "sn_internal.h"

namespace sn {
namespace {

constexpr int BM = 64, BN = 64, BK = 32, PADK = 8, THREADS = 128;

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  const __nv_bfloat16 a = __float2bfloat16_rn(lo), b = __float2bfloat16_rn(hi);
  return (unsigned)__bfloat16_as_ushort(a) | ((unsigned)__bfloat16_as_ushort(b) << 16);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(THREADS) gemm_kernel(GemmArgs g, int nsplit) {
  __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PADK];  // [m][k]
  __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PADK];  // [n][k]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;  // 2 x 2 warps, 32 x 32 each
  const int gid = lane >> 2, tig = lane & 3;
  const long long z = blockIdx.z / nsplit;
  const int sp = blockIdx.z % nsplit;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kbeg = nsplit > 1 ? sp * g.kchunk : 0;
  const int kend = nsplit > 1 ? min(g.K, kbeg + g.kchunk) : g.K;
  const float* A = g.A + z * g.sAz;
  const float* B = g.B + z * g.sBz;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
  const bool a_kfast = g.sAk == 1;
  const bool b_nfast = g.sBn == 1;

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    // stage A (BM x BK) and B (BK x BN) as BF16, zero outside the matrix
#pragma unroll 4
    for (int e = tid; e < BM * BK; e += THREADS) {
      const int m = a_kfast ? e / BK : e % BM;
      const int k = a_kfast ? e % BK : e / BM;
      const int gm = m0 + m, gk = k0 + k;
      float x = 0.f;
      if (gm < g.M && gk < kend) x = A[(long long)gm * g.sAm + (long long)gk * g.sAk];
      As[m][k] = __float2bfloat16_rn(x);
    }
#pragma unroll 4
    for (int e = tid; e < BN * BK; e += THREADS) {
      const int n = b_nfast ? e % BN : e / BK;
      const int k = b_nfast ? e / BN : e % BK;
      const int gn = n0 + n, gk = k0 + k;
      float x = 0.f;
      if (gn < g.N && gk < kend) x = B[(long long)gk * g.sBk + (long long)gn * g.sBn];
      Bs[n][k] = __float2bfloat16_rn(x);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      unsigned af[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm * 32 + i * 16 + gid;
        af[i][0] = *reinterpret_cast<const unsigned*>(&As[r][kk + 2 * tig]);
        af[i][1] = *reinterpret_cast<const unsigned*>(&As[r + 8][kk + 2 * tig]);
        af[i][2] = *reinterpret_cast<const unsigned*>(&As[r][kk + 2 * tig + 8]);
        af[i][3] = *reinterpret_cast<const unsigned*>(&As[r + 8][kk + 2 * tig + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn * 32 + j * 8 + gid;
        const unsigned b0 = *reinterpret_cast<const unsigned*>(&Bs[c][kk + 2 * tig]);
        const unsigned b1 = *reinterpret_cast<const unsigned*>(&Bs[c][kk + 2 * tig + 8]);
#pragma unroll
        for (int i = 0; i < 2; ++i) mma_bf16(acc[i][j], af[i], b0, b1);
      }
    }
    __syncthreads();
  }
  float* C = g.C + z * g.sCz + (long long)sp * g.sCsp;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + wm * 32 + i * 16 + gid + (r >= 2 ? 8 : 0);
        const int n = n0 + wn * 32 + j * 8 + 2 * tig + (r & 1);
        if (m < g.M && n < g.N) {
          float* p = C + (long long)m * g.sCm + (long long)n * g.sCn;
          const float v = g.alpha * acc[i][j][r];
          *p = (g.beta != 0.f) ? v + g.beta * *p : v;
        }
      }
}

__global__ void reduce_sum_kernel(const float* part, long long count, long long stride, long long n,
                                  float* out, float beta) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (long long j = 0; j < count; ++j) s += part[j * stride + i];
    out[i] = (beta != 0.f) ? s + beta * out[i] : s;
  }
}

}  // namespace

cudaError_t gemm_bf16(const GemmArgs& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.Z <= 0) return cudaSuccess;
  int nsplit = 1;
  if (g.kchunk > 0 && g.kchunk < g.K) nsplit = (g.K + g.kchunk - 1) / g.kchunk;
  const long long zs = (long long)g.Z * nsplit;
  if (zs > 65535) return cudaErrorInvalidValue;
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, (unsigned)zs);
  gemm_kernel<<<grid, THREADS, 0, s>>>(g, nsplit);
  return cudaGetLastError();
}

cudaError_t reduce_sum(const float* part, long long count, long long stride, long long n, float* out,
                       float beta, cudaStream_t s) {
  const long long blocks = (n + 255) / 256;
  reduce_sum_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(part, count, stride,
                                                                                n, out, beta);
  return cudaGetLastError();
}

}  // namespace sn

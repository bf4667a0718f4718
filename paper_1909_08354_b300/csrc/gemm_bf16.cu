// Strided batched GEMM on the tensor cores: C = alpha * A B + beta * C with A,
// B read as FP32 from global memory, rounded to BF16 when they are staged in
// shared memory, multiplied by mma.sync m16n8k16 with FP32 accumulation.
//
// Every operand has element strides, so transposes, planar/interleaved complex
// parts and gathered mode matrices are plain stride choices.  Optional split-K:
// block (z, sp) sums k in [sp*kchunk, (sp+1)*kchunk) and writes its partial
// product to C + z*sCz + sp*sCsp (beta must be 0); reduce_sum adds partials.
//
// The operands of the next k-tile are loaded into registers while the current
// tile is multiplied.  Where an operand's fast dimension is contiguous and
// 16-byte aligned it moves as float4; where C's rows are contiguous and
// aligned, the tile is staged in shared memory and written as float4 rows.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "sn_internal.h"

namespace sn {
namespace {

constexpr int BM = 64, BN = 64, BK = 32, PADK = 8, THREADS = 128;

// the epilogue's activation: x Phi(x) with the error function
__device__ __forceinline__ float gelu_erf(float x) {
  return 0.5f * x * (1.f + erff(x * 0.70710678118654752f));
}
constexpr int TILE = BM * BK;          // elements of one operand tile (BN * BK too)
constexpr int PER = TILE / THREADS;    // elements per thread per operand tile
constexpr int CST = BN + 4;            // row stride of the staged C tile (floats)

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Operand view: element (r, k) of the tile at base + r * sr + k * sk, with
// r < R (rows of A or columns of B) and k < kend.  KFAST: k is the contiguous
// dimension (sk == 1).  VEC: float4 moves along the contiguous dimension.
struct Operand {
  const float* base;
  long long sr, sk;
  int R, kend;
};

// Load tile elements (r0.., k0..) into registers in a fixed per-thread order.
template <bool KFAST, bool VEC>
__device__ __forceinline__ void load_tile(const Operand& o, int r0, int k0, float (&v)[PER],
                                          int tid) {
  if constexpr (VEC) {
#pragma unroll
    for (int i = 0; i < PER / 4; ++i) {
      const int q = tid + THREADS * i;  // float4 index within the tile
      int r, k;
      if constexpr (KFAST) { r = q / (BK / 4); k = (q % (BK / 4)) * 4; }
      else { k = q / (BM / 4); r = (q % (BM / 4)) * 4; }
      const int gr = r0 + r, gk = k0 + k;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if constexpr (KFAST) {
        if (gr < o.R) {
          const float* p = o.base + (long long)gr * o.sr + gk;
          if (gk + 3 < o.kend) {
            x = *reinterpret_cast<const float4*>(p);
          } else {
            if (gk < o.kend) x.x = p[0];
            if (gk + 1 < o.kend) x.y = p[1];
            if (gk + 2 < o.kend) x.z = p[2];
          }
        }
      } else {
        if (gk < o.kend) {
          const float* p = o.base + (long long)gk * o.sk + gr;
          if (gr + 3 < o.R) {
            x = *reinterpret_cast<const float4*>(p);
          } else {
            if (gr < o.R) x.x = p[0];
            if (gr + 1 < o.R) x.y = p[1];
            if (gr + 2 < o.R) x.z = p[2];
          }
        }
      }
      v[4 * i] = x.x; v[4 * i + 1] = x.y; v[4 * i + 2] = x.z; v[4 * i + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = tid + THREADS * i;
      const int r = KFAST ? e / BK : e % BM;
      const int k = KFAST ? e % BK : e / BM;
      const int gr = r0 + r, gk = k0 + k;
      v[i] = (gr < o.R && gk < o.kend) ? o.base[(long long)gr * o.sr + (long long)gk * o.sk] : 0.f;
    }
  }
}

// Registers of load_tile -> BF16 tile S[r][k] in shared memory.
template <bool KFAST, bool VEC>
__device__ __forceinline__ void store_tile(__nv_bfloat16 (*S)[BK + PADK], const float (&v)[PER],
                                           int tid) {
  if constexpr (VEC) {
#pragma unroll
    for (int i = 0; i < PER / 4; ++i) {
      const int q = tid + THREADS * i;
      if constexpr (KFAST) {
        const int r = q / (BK / 4), k = (q % (BK / 4)) * 4;
        const __nv_bfloat162 lo = __floats2bfloat162_rn(v[4 * i], v[4 * i + 1]);
        const __nv_bfloat162 hi = __floats2bfloat162_rn(v[4 * i + 2], v[4 * i + 3]);
        uint2 u;
        u.x = *reinterpret_cast<const unsigned*>(&lo);
        u.y = *reinterpret_cast<const unsigned*>(&hi);
        *reinterpret_cast<uint2*>(&S[r][k]) = u;
      } else {
        const int k = q / (BM / 4), r = (q % (BM / 4)) * 4;
#pragma unroll
        for (int j = 0; j < 4; ++j) S[r + j][k] = __float2bfloat16_rn(v[4 * i + j]);
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = tid + THREADS * i;
      const int r = KFAST ? e / BK : e % BM;
      const int k = KFAST ? e % BK : e / BM;
      S[r][k] = __float2bfloat16_rn(v[i]);
    }
  }
}

// 0: scalar, k-fast; 1: scalar, r-fast; 2: float4, k-fast; 3: float4, r-fast
template <int MA, int MB, bool CVEC>
__global__ void __launch_bounds__(THREADS) gemm_kernel(GemmArgs g, int nsplit) {
  constexpr bool AK = (MA == 0 || MA == 2), AV = MA >= 2;
  constexpr bool BK_ = (MB == 0 || MB == 2), BV = MB >= 2;
  __shared__ __align__(16) unsigned char smem[BM * CST * sizeof(float)];
  auto As = reinterpret_cast<__nv_bfloat16 (*)[BK + PADK]>(smem);  // [m][k]
  auto Bs = reinterpret_cast<__nv_bfloat16 (*)[BK + PADK]>(smem + BM * (BK + PADK) * 2);  // [n][k]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;  // 2 x 2 warps, 32 x 32 each
  const int gid = lane >> 2, tig = lane & 3;
  const long long z = blockIdx.z / nsplit;
  const int sp = blockIdx.z % nsplit;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kbeg = nsplit > 1 ? sp * g.kchunk : 0;
  const int kend = nsplit > 1 ? min(g.K, kbeg + g.kchunk) : g.K;
  const Operand oa{g.A + z * g.sAz, g.sAm, g.sAk, g.M, kend};
  const Operand ob{g.B + z * g.sBz, g.sBn, g.sBk, g.N, kend};
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

  float va[PER], vb[PER];
  if (kbeg < kend) {
    load_tile<AK, AV>(oa, m0, kbeg, va, tid);
    load_tile<BK_, BV>(ob, n0, kbeg, vb, tid);
  }
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    store_tile<AK, AV>(As, va, tid);
    store_tile<BK_, BV>(Bs, vb, tid);
    __syncthreads();
    if (k0 + BK < kend) {  // the next tile is in flight while this one is multiplied
      load_tile<AK, AV>(oa, m0, k0 + BK, va, tid);
      load_tile<BK_, BV>(ob, n0, k0 + BK, vb, tid);
    }
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
  float* C2 = g.C2 != nullptr ? g.C2 + z * g.sCz : nullptr;
  if constexpr (CVEC) {
    // stage the tile, then float4 rows (n contiguous, sCm a multiple of 4, C aligned)
    float* Cs = reinterpret_cast<float*>(smem);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int m = wm * 32 + i * 16 + gid + (r >= 2 ? 8 : 0);
          const int n = wn * 32 + j * 8 + 2 * tig + (r & 1);
          Cs[m * CST + n] = acc[i][j][r];
        }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < BM * BN / 4 / THREADS; ++i) {
      const int q = tid + THREADS * i;
      const int m = q / (BN / 4), n = (q % (BN / 4)) * 4;
      const int gm = m0 + m, gn = n0 + n;
      if (gm >= g.M) continue;
      float* p = C + (long long)gm * g.sCm + gn;
      float* p2 = C2 != nullptr ? C2 + (long long)gm * g.sCm + gn : nullptr;
      const float bm = g.bias != nullptr ? g.bias[gm] : 0.f;
      const float4 a = *reinterpret_cast<const float4*>(&Cs[m * CST + n]);
      if (gn + 3 < g.N) {
        float4 v = make_float4(g.alpha * a.x, g.alpha * a.y, g.alpha * a.z, g.alpha * a.w);
        if (g.beta != 0.f) {
          const float4 c = *reinterpret_cast<const float4*>(p);
          v.x += g.beta * c.x; v.y += g.beta * c.y; v.z += g.beta * c.z; v.w += g.beta * c.w;
        }
        if (g.bias != nullptr) { v.x += bm; v.y += bm; v.z += bm; v.w += bm; }
        *reinterpret_cast<float4*>(p) = v;
        if (p2 != nullptr) {
          if (g.act) v = make_float4(gelu_erf(v.x), gelu_erf(v.y), gelu_erf(v.z), gelu_erf(v.w));
          *reinterpret_cast<float4*>(p2) = v;
        }
      } else {
        const float av[4] = {a.x, a.y, a.z, a.w};
        for (int j = 0; j < 4 && gn + j < g.N; ++j) {
          float v = (g.beta != 0.f) ? g.alpha * av[j] + g.beta * p[j] : g.alpha * av[j];
          if (g.bias != nullptr) v += bm;
          p[j] = v;
          if (p2 != nullptr) p2[j] = g.act ? gelu_erf(v) : v;
        }
      }
    }
  } else {
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
}

// out[i] = sum_j part[j stride + i] (+ beta out[i]).  A block takes 32
// consecutive outputs (one per lane, coalesced) and splits j over its
// kReduceSlices warps, slice w summing j = w, w + kReduceSlices, ... in eight
// interleaved partial sums (eight loads in flight); the partial sums and then
// the slices are added in a fixed order, so the result is the same on every
// run.
constexpr int kReduceSlices = 8;

__global__ void __launch_bounds__(32 * kReduceSlices)
reduce_sum_kernel(const float* part, long long count, long long stride, long long n, float* out,
                  float beta) {
  __shared__ float red[kReduceSlices][32];
  const int lane = threadIdx.x & 31, sl = threadIdx.x >> 5;
  constexpr int S = kReduceSlices;
  for (long long i0 = blockIdx.x * 32LL; i0 < n; i0 += gridDim.x * 32LL) {
    const long long i = i0 + lane;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (i < n) {
      long long j = sl;
      for (; j + 7 * S < count; j += 8 * S) {
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] += part[(j + u * S) * stride + i];
      }
      for (; j < count; j += S) acc[0] += part[j * stride + i];
    }
    red[sl][lane] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
    __syncthreads();
    if (sl == 0 && i < n) {
      float s = 0.f;
#pragma unroll
      for (int w = 0; w < S; ++w) s += red[w][lane];
      out[i] = (beta != 0.f) ? s + beta * out[i] : s;
    }
    __syncthreads();
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// operand mode: float4 moves need the fast stride 1, an aligned base and the
// other strides multiples of 4 elements
int mode_of(const float* base, long long s_fast_k, long long s_fast_r, long long s_other,
            long long s_z) {
  const bool kfast = s_fast_k == 1;
  const bool rfast = !kfast && s_fast_r == 1;
  const bool vec = (kfast || rfast) && aligned16(base) && s_other % 4 == 0 && s_z % 4 == 0;
  if (kfast) return vec ? 2 : 0;
  if (rfast) return vec ? 3 : 1;
  return 0;
}

template <int MA, int MB>
cudaError_t launch3(const GemmArgs& g, int nsplit, bool cvec, dim3 grid, cudaStream_t s) {
  if (cvec) gemm_kernel<MA, MB, true><<<grid, THREADS, 0, s>>>(g, nsplit);
  else gemm_kernel<MA, MB, false><<<grid, THREADS, 0, s>>>(g, nsplit);
  return cudaGetLastError();
}

template <int MA>
cudaError_t launch2(const GemmArgs& g, int mb, int nsplit, bool cvec, dim3 grid, cudaStream_t s) {
  switch (mb) {
    case 0: return launch3<MA, 0>(g, nsplit, cvec, grid, s);
    case 1: return launch3<MA, 1>(g, nsplit, cvec, grid, s);
    case 2: return launch3<MA, 2>(g, nsplit, cvec, grid, s);
    default: return launch3<MA, 3>(g, nsplit, cvec, grid, s);
  }
}

}  // namespace

cudaError_t gemm_bf16(const GemmArgs& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.Z <= 0) return cudaSuccess;
  int nsplit = 1;
  if (g.kchunk > 0 && g.kchunk < g.K) nsplit = (g.K + g.kchunk - 1) / g.kchunk;
  const long long zs = (long long)g.Z * nsplit;
  if (zs > 65535) return cudaErrorInvalidValue;
  // split-K chunks must start on a float4 boundary for the vector loads
  const bool chunk4 = nsplit == 1 || g.kchunk % 4 == 0;
  int ma = mode_of(g.A, g.sAk, g.sAm, g.sAk == 1 ? g.sAm : g.sAk, g.sAz);
  int mb = mode_of(g.B, g.sBk, g.sBn, g.sBk == 1 ? g.sBn : g.sBk, g.sBz);
  if (!chunk4) { ma &= 1; mb &= 1; }
  const bool cvec = g.sCn == 1 && aligned16(g.C) && g.sCm % 4 == 0 && g.sCz % 4 == 0 &&
                    g.sCsp % 4 == 0;
  // the epilogue runs in the staged-C path of a GEMM without split-K
  if ((g.bias != nullptr || g.C2 != nullptr) &&
      (!cvec || nsplit != 1 || (g.C2 != nullptr && !aligned16(g.C2))))
    return cudaErrorInvalidValue;
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, (unsigned)zs);
  switch (ma) {
    case 0: return launch2<0>(g, mb, nsplit, cvec, grid, s);
    case 1: return launch2<1>(g, mb, nsplit, cvec, grid, s);
    case 2: return launch2<2>(g, mb, nsplit, cvec, grid, s);
    default: return launch2<3>(g, mb, nsplit, cvec, grid, s);
  }
}

cudaError_t reduce_sum(const float* part, long long count, long long stride, long long n, float* out,
                       float beta, cudaStream_t s) {
  const long long blocks = (n + 31) / 32;
  reduce_sum_kernel<<<(unsigned)(blocks < 8192 ? blocks : 8192), 32 * kReduceSlices, 0, s>>>(
      part, count, stride, n, out, beta);
  return cudaGetLastError();
}

}  // namespace sn

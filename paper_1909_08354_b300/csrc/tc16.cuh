// Tensor-core engine for 256-point lines: every 16-point DFT stage of the
// line transforms of the split-step method (Sec. III) runs as real 32 x 32
// matrix blocks on mma.sync m16n8k16 (FP16 operands, FP32 accumulation).
//
// A 256-point DFT is 16 x 16 (n = t + 16 r, k = k1 + 16 k2):
//   stage A: for each column t, a 16-point DFT over r       -> Y[k1][t]
//   twiddle: Y[k1][t] * w256^(s t k1)           (FP32, hi/lo table)
//   stage B: for each column k1, a 16-point DFT over t       -> X[k1 + 16 k2]
// A complex 16-point DFT of a column is one real 32 x 32 product with the
// column's (re, im) pairs interleaved along K.  FP16 holds 11 significant
// bits, so operands are split, x = x_hi + x_lo and F = F_hi + F_lo, and each
// block is F_hi x_hi + F_hi x_lo + F_lo x_hi accumulated in FP32 (the dropped
// F_lo x_lo is below 2^-22 of the product).  Before the split every line is
// scaled by a power of two chosen from its largest component (a warp max), so
// no value overflows FP16 and small values stay clear of its subnormals; the
// scale is exact and is removed at the end.
//
// The tensor cores' FP32 accumulation truncates, which shrinks every stage's
// result by a few 1e-8 on average, and F_hi + F_lo is unitary only to ~2e-8;
// both would drain the mass of psi step after step.  Each 256-point transform
// and every 16-point stage are unitary up to a known factor (Parseval), so the
// shrink is measured per line (squared norms summed in FP32 on the scaled
// values) and taken back where it can be: a factor 1 + c with c below an ulp
// does nothing to a value already rounded to FP32, so it is folded into the lo
// part of the next FP16 split, lo = fp16(fma(y, c, y - hi)).  Stage A's
// measured shrink is taken back at stage B's input together with the same
// amount predicted for stage B; the forward transform's measured remainder is
// taken back at the inverse transform's input.  What is left is a random
// per-line factor of order 1e-7 instead of a bias.
//
// Two operand roles are used.  "F-as-A": the DFT matrix is the A operand and
// the data the B operand (columns along N); "data-as-A": the data is the A
// operand (columns along M) and the transposed DFT matrix the B operand.  With
// the fragment layouts of m16n8k16, the accumulators of an F-as-A stage are
// exactly the A fragments of a following data-as-A stage once the K order of
// that stage is permuted by pi(p) = 8 (p / 8) + 2 (p % 4) + (p / 4) % 2, and
// a data-as-A result feeds an F-as-A stage unpermuted.  So FFT . m . IFFT of
// a line runs in registers: only the entry (pattern P -> fragments) and the
// exit cross shared memory.  One warp transforms one line at a time.
#pragma once

#include <cuda_fp16.h>

#include "sn_fft.cuh"

namespace sn {
namespace tc16 {

using snfft::cmul_hl;
using snfft::cx;

constexpr int N = 256;
constexpr int E = 16, T = 16;  // pattern P of a 256-point line
constexpr int LS = 321;        // padded line stride (complex values), odd
constexpr int TWS = 18;        // row stride of the 16 x 16 twiddle tables
constexpr int FRAG_WORDS = 2 * 2 * 4 * 32 * 4 * 2;  // u32 words of the fa + fb tables

// padded position of element n of a line: 4 pad slots after every 16 values,
// which makes both the pattern-P accesses and the fragment accesses
// conflict-free in shared memory
__host__ __device__ constexpr int pt(int n) { return n + 4 * (n >> 4); }
constexpr int MT = pt(N - 1) + 1;  // entries of a padded per-k table

// Shared-memory tables.  fa: A fragments of F (F-as-A stages), fb: B fragments
// of F^T with the pi-permuted K order (data-as-A stages); [dir][hi/lo][q][lane]
// with dir 0 = forward exp(-i ...), 1 = inverse exp(+i ...).  tw: twiddles
// w256^(s a b) / 16 at [dir][hi/lo][a * TWS + b].
struct Tabs {
  uint4 fa[2][2][4][32];
  uint4 fb[2][2][4][32];
  float2 tw[2][2][16 * TWS];
};

__device__ __forceinline__ void mma(float (&d)[4], const uint4& a, unsigned b0, unsigned b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned h2u(__half2 h) {
  unsigned u;
  memcpy(&u, &h, sizeof(u));
  return u;
}

// (re, im) -> FP16 pairs hi = fp16(x), lo = fp16(x - hi), re in the low half
__device__ __forceinline__ void split(float re, float im, unsigned& hi, unsigned& lo) {
  const __half2 h = __floats2half2_rn(re, im);
  const float2 hf = __half22float2(h);
  hi = h2u(h);
  lo = h2u(__floats2half2_rn(re - hf.x, im - hf.y));
}

// the same split of x (1 + c) for a small c: the correction goes into the lo
// part before any rounding of x (1 + c) itself, so it survives even when it
// is far below an ulp of x
__device__ __forceinline__ void split_c(float re, float im, float c, unsigned& hi, unsigned& lo) {
  const __half2 h = __floats2half2_rn(re, im);
  const float2 hf = __half22float2(h);
  hi = h2u(h);
  lo = h2u(__floats2half2_rn(fmaf(re, c, re - hf.x), fmaf(im, c, im - hf.y)));
}

// power-of-two scale s with (largest component) * s < 2^14, and 1 / s, from
// the bit pattern of the warp's largest |component|
__device__ __forceinline__ void line_scale(float mx, float& s, float& inv) {
  unsigned e = __reduce_max_sync(0xffffffffu, __float_as_uint(mx)) >> 23;
  e = e < 14u ? 14u : (e > 254u ? 254u : e);
  s = __uint_as_float((267u - e) << 23);
  inv = __uint_as_float((e - 13u) << 23);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// eps = sqrt(target / got) - 1 of two squared norms, formed without the
// cancellation of 1 + eps, so that fma(y, eps, y) applies it exactly before
// the single rounding of the result (a factor 1 + eps with |eps| below an ulp
// would round back to 1 and leave the value unchanged)
__device__ __forceinline__ float parseval_eps(float target, float got) {
  if (!(got > 0.f)) return 0.f;
  return __fdiv_rn(target - got, got + __fsqrt_rn(target * got));
}

// squared norm of F-as-A accumulators (all lanes: the warp total)
__device__ __forceinline__ float norm_fa(const float (&acc)[2][2][4]) {
  float n = 0.f;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int r = 0; r < 4; ++r) n = fmaf(acc[mt][nt][r], acc[mt][nt][r], n);
  return warp_sum(n);
}
__device__ __forceinline__ float norm_da(const float (&acc)[4][4]) {
  float n = 0.f;
#pragma unroll
  for (int nt = 0; nt < 4; ++nt)
#pragma unroll
    for (int r = 0; r < 4; ++r) n = fmaf(acc[nt][r], acc[nt][r], n);
  return warp_sum(n);
}

__device__ __forceinline__ float amax(float m, cx<float> z) {
  return fmaxf(m, fmaxf(fabsf(z.re), fabsf(z.im)));
}

// F-as-A stage.  b[nt][ks][e]: column 8 nt + gid, K position 8 ks + tig + 4 e.
// acc[mt][nt][r]: mt 0 real / 1 imaginary part of output gid + 8 (r >> 1) for
// column 8 nt + 2 tig + (r & 1).
__device__ __forceinline__ void stage_fa(const uint4 (*fh)[32], const uint4 (*fl)[32],
                                         const unsigned (&bh)[2][2][2],
                                         const unsigned (&bl)[2][2][2], float (&acc)[2][2][4],
                                         int lane) {
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[mt][nt][r] = 0.f;
  // the small hi x lo terms first, then the two hi x hi blocks: only those two
  // additions to a full-size accumulator are truncated at FP32 precision
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const uint4 ah = fh[mt * 2 + ks][lane], al = fl[mt * 2 + ks][lane];
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        mma(acc[mt][nt], al, bh[nt][ks][0], bh[nt][ks][1]);
        mma(acc[mt][nt], ah, bl[nt][ks][0], bl[nt][ks][1]);
      }
    }
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const uint4 ah = fh[mt * 2 + ks][lane];
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) mma(acc[mt][nt], ah, bh[nt][ks][0], bh[nt][ks][1]);
    }
  }
}

// data-as-A stage.  a[ks] = {a0, a1, a2, a3}: column gid / gid + 8, K position
// 8 ks + tig / + 4 (pi-permuted).  acc[nt]: (re, im) of output 4 nt + tig for
// column gid (acc[nt][0..1]) and gid + 8 (acc[nt][2..3]).
__device__ __forceinline__ void stage_da(const uint4* fh, const uint4* fl, const uint4 (&ah)[2],
                                         const uint4 (&al)[2], float (&acc)[4][4], int lane) {
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[nt][r] = 0.f;
    const uint4 bh = fh[nt * 32 + lane], bl = fl[nt * 32 + lane];
    mma(acc[nt], al[0], bh.x, bh.y);
    mma(acc[nt], ah[0], bl.x, bl.y);
    mma(acc[nt], al[1], bh.z, bh.w);
    mma(acc[nt], ah[1], bl.z, bl.w);
    mma(acc[nt], ah[0], bh.x, bh.y);
    mma(acc[nt], ah[1], bh.z, bh.w);
  }
}

// twiddle the F-as-A accumulators and repack them as data-as-A fragments,
// scaled by 1 + c.
// Element (row gid + 8 (r >> 1), column 8 ks + 2 tig + (r & 1)) is multiplied
// by tw[column * TWS + row] (the table is symmetric in its two indices).
__device__ __forceinline__ void twiddle_pack(const float (&acc)[2][2][4], const float2* twh,
                                             const float2* twl, float c, uint4 (&ah)[2],
                                             uint4 (&al)[2], int gid, int tig) {
#pragma unroll
  for (int ks = 0; ks < 2; ++ks) {
    unsigned h[4], l[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int row = gid + 8 * (r >> 1), col = 8 * ks + 2 * tig + (r & 1);
      const float2 wh = twh[col * TWS + row], wl = twl[col * TWS + row];
      const cx<float> y = cmul_hl({acc[0][ks][r], acc[1][ks][r]}, {wh.x, wh.y}, {wl.x, wl.y});
      // fragment register: r 0 -> a0, 2 -> a1, 1 -> a2, 3 -> a3
      const int q = (r >> 1) | ((r & 1) << 1);
      split_c(y.re, y.im, c, h[q], l[q]);
    }
    ah[ks] = make_uint4(h[0], h[1], h[2], h[3]);
    al[ks] = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

// one 256-point DFT (dir 0: exp(-i), 1: exp(+i), unnormalised) of a line held
// in a padded shared buffer, in place, by one warp
template <int DIR>
__device__ __forceinline__ void line_fft(cx<float>* line, const Tabs& tb, int lane) {
  const int gid = lane >> 2, tig = lane & 3;
  cx<float> x[2][4];
  float mx = 0.f;
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 v = reinterpret_cast<const float2*>(line)[pt(gid + 8 * nt + 16 * (tig + 4 * i))];
      x[nt][i] = {v.x, v.y};
      mx = amax(mx, x[nt][i]);
    }
  float s, inv;
  line_scale(mx, s, inv);
  unsigned bh[2][2][2], bl[2][2][2];
  float nin = 0.f;
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int ks = 0; ks < 2; ++ks)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const float re = x[nt][2 * ks + e].re * s, im = x[nt][2 * ks + e].im * s;
        nin = fmaf(re, re, fmaf(im, im, nin));
        split(re, im, bh[nt][ks][e], bl[nt][ks][e]);
      }
  float acc[2][2][4];
  stage_fa(tb.fa[DIR][0], tb.fa[DIR][1], bh, bl, acc, lane);
  // stage A's shrink from Parseval (16 |x s|^2), taken back at stage B's
  // input together with the same amount predicted for stage B
  const float ea = parseval_eps(16.f * warp_sum(nin), norm_fa(acc));
  uint4 ah[2], al[2];
  twiddle_pack(acc, tb.tw[DIR][0], tb.tw[DIR][1], 2.f * ea, ah, al, gid, tig);
  float acc2[4][4];
  stage_da(tb.fb[DIR][0][0], tb.fb[DIR][1][0], ah, al, acc2, lane);
  __syncwarp();
  const float o = 16.f * inv;  // undo the scale and the 1/16 folded into the twiddles (exact)
#pragma unroll
  for (int nt = 0; nt < 4; ++nt)
#pragma unroll
    for (int h = 0; h < 2; ++h)
      reinterpret_cast<float2*>(line)[pt(gid + 8 * h + 16 * (4 * nt + tig))] =
          make_float2(acc2[nt][2 * h] * o, acc2[nt][2 * h + 1] * o);
}

// Spectral multiplier of the fused FFT . M . IFFT: a hi/lo table (kinetic
// factors) or Green's function K(k) computed from k^2.
struct MultTable {
  const float2* hi;  // padded [MT]
  const float2* lo;
  __device__ __forceinline__ cx<float> operator()(cx<float> z, int k) const {
    const float2 h = hi[pt(k)], l = lo[pt(k)];
    return cmul_hl(z, {h.x, h.y}, {l.x, l.y});
  }
};
struct GreenMult {
  const float* k2l;  // padded [MT]
  float k2pm, cN, cY, mu2, cL;  // cL: constant added at every k
  __device__ __forceinline__ cx<float> operator()(cx<float> z, int k) const {
    const float k2 = k2pm + k2l[pt(k)];
    const float den = k2 * (k2 + mu2);
    const float K = ((k2 > 0.f) ? __fdividef(fmaf(cN, k2 + mu2, cY * k2), den) : 0.f) + cL;
    return {z.re * K, z.im * K};
  }
};

// IFFT(M . FFT(line)) of one line in a padded shared buffer, by one warp
template <class Mult>
__device__ __forceinline__ void line_fmi(cx<float>* line, const Tabs& tb, const Mult& mult,
                                         int lane) {
  const int gid = lane >> 2, tig = lane & 3;
  unsigned bh[2][2][2], bl[2][2][2];
  float s1, inv1, nin1 = 0.f;
  {
    cx<float> x[2][4];
    float mx = 0.f;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float2 v =
            reinterpret_cast<const float2*>(line)[pt(gid + 8 * nt + 16 * (tig + 4 * i))];
        x[nt][i] = {v.x, v.y};
        mx = amax(mx, x[nt][i]);
      }
    line_scale(mx, s1, inv1);
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int ks = 0; ks < 2; ++ks)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const float re = x[nt][2 * ks + e].re * s1, im = x[nt][2 * ks + e].im * s1;
          nin1 = fmaf(re, re, fmaf(im, im, nin1));
          split(re, im, bh[nt][ks][e], bl[nt][ks][e]);
        }
    nin1 = warp_sum(nin1);
  }
  float acc[2][2][4];
  uint4 ah[2], al[2];
  float acc2[4][4];
  stage_fa(tb.fa[0][0], tb.fa[0][1], bh, bl, acc, lane);
  float ea = parseval_eps(16.f * nin1, norm_fa(acc));
  twiddle_pack(acc, tb.tw[0][0], tb.tw[0][1], 2.f * ea, ah, al, gid, tig);
  stage_da(tb.fb[0][0][0], tb.fb[0][1][0], ah, al, acc2, lane);
  // what is left of the forward transform's shrink (Parseval: |DFT(x s)/16|^2 =
  // |x s|^2) is taken back at the inverse's input split
  const float ez = parseval_eps(nin1, norm_da(acc2));
  // spectrum entry k1 + 16 k2 with k1 = gid + 8 h, k2 = 4 nt + tig
  float s2, inv2, nin2 = 0.f;
  {
    cx<float> z[4][2];
    float mx = 0.f;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        z[nt][h] = mult({acc2[nt][2 * h], acc2[nt][2 * h + 1]}, gid + 8 * h + 16 * (4 * nt + tig));
        mx = amax(mx, z[nt][h]);
      }
    line_scale(mx, s2, inv2);
    // inverse first stage: column k1 = 8 h + gid, K position k2 = 8 ks + tig + 4 e
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int ks = 0; ks < 2; ++ks)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const float re = z[2 * ks + e][h].re * s2, im = z[2 * ks + e][h].im * s2;
          nin2 = fmaf(re, re, fmaf(im, im, nin2));
          split_c(re, im, ez, bh[h][ks][e], bl[h][ks][e]);
        }
    nin2 = warp_sum(nin2) * (1.f + 2.f * ez);
  }
  stage_fa(tb.fa[1][0], tb.fa[1][1], bh, bl, acc, lane);
  ea = parseval_eps(16.f * nin2, norm_fa(acc));
  twiddle_pack(acc, tb.tw[1][0], tb.tw[1][1], 2.f * ea, ah, al, gid, tig);
  stage_da(tb.fb[1][0][0], tb.fb[1][1][0], ah, al, acc2, lane);
  __syncwarp();
  const float o = 256.f * inv1 * inv2;  // exact power of two
#pragma unroll
  for (int nt = 0; nt < 4; ++nt)
#pragma unroll
    for (int h = 0; h < 2; ++h)
      reinterpret_cast<float2*>(line)[pt(gid + 8 * h + 16 * (4 * nt + tig))] =
          make_float2(acc2[nt][2 * h] * o, acc2[nt][2 * h + 1] * o);
}

// ---- CTA-wide entry points: pattern P registers in and out ------------------
// Every thread of the CTA calls them (they contain barriers).  The CTA holds
// LPB = 16 lines and 8 warps; warp w transforms lines 2w and 2w + 1.  `buf` is
// 16 padded lines of LS values.

__device__ __forceinline__ void put_p(const cx<float> (&v)[E], cx<float>* buf, int l, int t) {
#pragma unroll
  for (int m = 0; m < E; ++m)
    reinterpret_cast<float2*>(buf)[l * LS + pt(t + T * m)] = make_float2(v[m].re, v[m].im);
}
__device__ __forceinline__ void get_p(cx<float> (&v)[E], const cx<float>* buf, int l, int t) {
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const float2 z = reinterpret_cast<const float2*>(buf)[l * LS + pt(t + T * m)];
    v[m] = {z.x, z.y};
  }
}

// In-place DFT of the lines l < nact (a warp-uniform count); threads of other
// lines keep their registers.
template <int DIR>
__device__ __forceinline__ void transform(cx<float> (&v)[E], cx<float>* buf, const Tabs& tb, int l,
                                          int t, int nact) {
  const bool active = l < nact;
  __syncthreads();
  if (active) put_p(v, buf, l, t);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < 2; ++j)
    if (2 * warp + j < nact) line_fft<DIR>(buf + (2 * warp + j) * LS, tb, lane);
  __syncthreads();
  if (active) get_p(v, buf, l, t);
}

// IFFT(M . FFT(line)) of every line; mult_of(L) gives line L's multiplier.
template <class MultOf>
__device__ __forceinline__ void fmi(cx<float> (&v)[E], cx<float>* buf, const Tabs& tb, int l,
                                    int t, const MultOf& mult_of) {
  __syncthreads();
  put_p(v, buf, l, t);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < 2; ++j) line_fmi(buf + (2 * warp + j) * LS, tb, mult_of(2 * warp + j), lane);
  __syncthreads();
  get_p(v, buf, l, t);
}

// Load the tables into shared memory: fragments from `frag` (FRAG_WORDS
// words), twiddles from the FP32 hi/lo table of the 16 x 16 plan (entry
// [r * 16 + j] forward, [N + r * 16 + j] inverse, lo parts after 2N entries),
// scaled by 1/16 (exact).
__device__ __forceinline__ void load_tabs(Tabs* tb, const uint4* frag, const float2* tw, int tid,
                                          int nt) {
  uint4* f = &tb->fa[0][0][0][0];
  for (int i = tid; i < FRAG_WORDS / 4; i += nt) f[i] = frag[i];
  for (int i = tid; i < 2 * 2 * 256; i += nt) {
    const int dir = i >> 9, hl = (i >> 8) & 1, a = (i >> 4) & 15, b = i & 15;
    const float2 w = tw[hl * 2 * N + dir * N + a * 16 + b];
    tb->tw[dir][hl][a * TWS + b] = make_float2(w.x * 0.0625f, w.y * 0.0625f);
  }
}

}  // namespace tc16
}  // namespace sn

// Building blocks of the fused FP32 passes, applied to one tile of LPB lines.
//
// Every function is called by all threads of the CTA (they contain barriers).
// A tile's lines are numbered l = 0..LPB-1; the T threads of line l hold its
// elements in pattern P (see sn_fft.cuh).  `lines` is LPB padded line buffers
// of Plan<N>::LS complex values; `tw` and `mult` point at hi/lo FP32 tables in
// shared or global memory.  CONTIG says that line l is held by the
// consecutive threads [l T, (l + 1) T) (contiguous mapping), so that its
// exchanges need only the barrier of a warp or warp pair (snfft::line_sync).
#pragma once

#include "sn_fft.cuh"
#include "tc16.cuh"

namespace sn {
namespace tile {

using snfft::cconj;
using snfft::cmul_hl;
using snfft::cnorm2;
using snfft::cscale;
using snfft::cx;
using snfft::line_transform;
using snfft::pidx;
using snfft::Plan;

// One DFT of the lines l < nact of the tile (pattern P in and out): the
// FP32 Stockham engine, or the tensor-core engine for 256-point lines (TC).
template <int N, int SIGN, bool CONTIG, bool TC>
__device__ __forceinline__ void xform(cx<float> (&v)[Plan<N>::E], cx<float>* lines,
                                      const cx<float>* tw, const tc16::Tabs* tb, int l, int t,
                                      int nact) {
  if constexpr (TC) {
    static_assert(N == tc16::N, "the tensor-core engine handles 256-point lines");
    tc16::transform<SIGN < 0 ? 0 : 1>(v, lines, *tb, l, t, nact);
  } else {
    line_transform<float, N, SIGN, CONTIG>(v, lines + l * Plan<N>::LS, tw, t, l < nact);
  }
}

template <int N, int LPB>
struct Cfg {
  static constexpr int E = Plan<N>::E;
  static constexpr int T = Plan<N>::T;
  static constexpr int NT = LPB * T;  // threads per CTA
  static constexpr int LS = Plan<N>::LS;
  static constexpr int H = N / 2 + 1;  // half-spectrum length
  static constexpr int TSTR = LPB + 1;  // padded row of a [k][line] staging tile
};

// Tiles of LPB lines: contiguous lines (stride 1) are LPB consecutive `outer`
// indices; strided lines are LPB consecutive `inner` indices of one `outer`.
template <int LPB, bool STRIDED>
struct Tiles {
  long long outer, inner, tiles_i, count;
  __host__ __device__ Tiles(long long o, long long i) : outer(o), inner(i) {
    tiles_i = STRIDED ? (i + LPB - 1) / LPB : 1;
    count = STRIDED ? o * tiles_i : (o + LPB - 1) / LPB;
  }
  // first line id, valid lines, element offset of line l and its (o, i)
  __device__ void at(long long tau, int l, int N, long long& line0, int& nvalid, size_t& base,
                     long long& o, long long& i) const {
    if (STRIDED) {
      o = tau / tiles_i;
      const long long i0 = (tau - o * tiles_i) * LPB;
      nvalid = (int)min((long long)LPB, inner - i0);
      line0 = o * inner + i0;
      i = i0 + l;
      base = (size_t)o * N * inner + i;
    } else {
      const long long o0 = tau * LPB;
      nvalid = (int)min((long long)LPB, outer - o0);
      line0 = o0;
      o = o0 + l;
      i = 0;
      base = (size_t)o * N;
    }
  }
};

// Global loads: L1-cached, or L2 only (CG) for data that other CTAs of the
// same launch have written.
template <bool CG>
__device__ __forceinline__ cx<float> ldg_c(const float2* p) {
  const float2 v = CG ? __ldcg(p) : *p;
  return {v.x, v.y};
}
__device__ __forceinline__ void stg_c(float2* p, cx<float> v) { *p = make_float2(v.re, v.im); }

template <int E, int T, bool CG = false>
__device__ __forceinline__ void load_line(cx<float> (&v)[E], const float2* p, unsigned ustride,
                                          int t, bool valid) {
#pragma unroll
  for (int m = 0; m < E; ++m) {
    cx<float> z = {0.f, 0.f};
    if (valid) z = ldg_c<CG>(p + (unsigned)(t + T * m) * ustride);
    v[m] = z;
  }
}

template <int E, int T>
__device__ __forceinline__ void store_line(const cx<float> (&v)[E], float2* p, unsigned ustride,
                                           int t, bool valid) {
  asm volatile("" : "+l"(p));  // recompute the store addresses instead of keeping them live
  if (valid) {
#pragma unroll
    for (int m = 0; m < E; ++m) stg_c(p + (unsigned)(t + T * m) * ustride, v[m]);
  }
}

// V h of the tile's lines from a staged [k][line] half-spectrum tile: C2R
// inverse FFT of lines (l, l + LPB/2) packed as A + iB.  On entry the tile is
// visible to all threads and the line buffers are free.  Returns the row that
// holds V h of my line, element t + T m at [t + T m], in line l's buffer
// (read before the buffer's next use, which starts with a barrier).
// TILE_IN_LINES: the staged tile occupies the line buffers themselves, so
// every read of it completes before the transform writes them.
// REMAP (strided passes): the thread of (l, t) in the pass's own mapping holds
// line l at position t spread over all warps, so half of every warp would idle
// through the packed transform; the transform then runs in the contiguous
// mapping (line tid / T, position tid % T: whole warps busy, warp-local
// exchanges) and V reaches the owners through shared memory.
template <int N, int LPB, bool CONTIG, bool TC = false, bool REMAP = false,
          bool TILE_IN_LINES = false>
__device__ __forceinline__ const float* potential_c2r(const cx<float>* rtile, cx<float>* lines,
                                                      const cx<float>* tw, int l, int t,
                                                      const tc16::Tabs* tb = nullptr) {
  using C = Cfg<N, LPB>;
  constexpr int E = C::E, T = C::T, LS = C::LS, TSTR = C::TSTR, HALF = LPB / 2;
  constexpr bool CC = REMAP || CONTIG;  // the mapping of the packed transform
  const int lc = REMAP ? (int)threadIdx.x / T : l;
  const int tc = REMAP ? (int)threadIdx.x % T : t;
  cx<float> v[E];
  const bool pa = lc < HALF;
  if (pa) {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int k = tc + T * m;
      cx<float> A, B;
      if (k <= N / 2) {
        A = rtile[k * TSTR + lc];
        B = rtile[k * TSTR + lc + HALF];
        if (k == 0 || k == N / 2) { A.im = 0.f; B.im = 0.f; }
      } else {
        A = cconj(rtile[(N - k) * TSTR + lc]);
        B = cconj(rtile[(N - k) * TSTR + lc + HALF]);
      }
      v[m] = {A.re - B.im, A.im + B.re};  // A + i B
    }
  }
  if constexpr (TILE_IN_LINES) __syncthreads();
  xform<N, +1, CC, TC>(v, lines, tw, tb, lc, tc, HALF);
  if constexpr (REMAP) {
    // the line buffer of lc is read by the threads of line lc only (FP32
    // engine); the tensor-core engine shares all buffers across the CTA
    if constexpr (TC) __syncthreads(); else snfft::line_sync<N, true>();
    if (pa) {
      float* a = reinterpret_cast<float*>(lines + lc * LS);
      float* b = reinterpret_cast<float*>(lines + (lc + HALF) * LS);
#pragma unroll
      for (int m = 0; m < E; ++m) {
        a[tc + T * m] = v[m].re;
        b[tc + T * m] = v[m].im;
      }
    }
  } else {
    // my line's buffer was last read by its own transform (line_sync); line
    // l + HALF sat out the transform, so its buffer is free (FP32 engine)
    if constexpr (TC) __syncthreads(); else snfft::line_sync<N, CONTIG>();
    if (pa) {
      float* a = reinterpret_cast<float*>(lines + l * LS);
      float* b = reinterpret_cast<float*>(lines + (l + HALF) * LS);
#pragma unroll
      for (int m = 0; m < E; ++m) {
        a[t + T * m] = v[m].re;
        b[t + T * m] = v[m].im;
      }
    }
  }
  __syncthreads();
  return reinterpret_cast<const float*>(lines + l * LS);
}

// psi <- exp(-i (V h + V_ext h + g h |psi|^2)) psi.  The angle is reduced to
// [-pi, pi] with a two-part 2 pi and the SFU sine and cosine are taken there.
// The pair is then pulled towards unit modulus by one Newton step,
// (c, s) <- (c, s)(1 - eta/2) with eta = c^2 + s^2 - 1, applied as c + c e so
// that a correction below an ulp of c is not rounded away against 1 + e.
// eta is formed without cancellation: the larger of |c|, |s| (call it b)
// enters as (b - 1)(b + 1), exact up to one rounding, since one factor is
// exact.  Computed as fma(c, c, fma(s, s, -1)) instead, eta carried the
// rounding of s^2 - 1 to the grid near -1, and the corrected pair was biased
// low by ~3e-8 at angles below 0.03: a mass drift of -1.6e-8 per step under a
// strong nonlocal potential (Eq. 4).  The bias is now ~1e-10 (+3e-9 below
// 1e-3 rad, where c itself rounds one-sidedly to the grid at 1).
// vat(m): V at position t + T m of the line.
template <int E, int T, class VAt>
__device__ __forceinline__ void nonlinear_phase_at(cx<float> (&v)[E], VAt vat, float gh,
                                                   const float* vx, float h, unsigned ustride,
                                                   int t, bool valid) {
#pragma unroll
  for (int m = 0; m < E; ++m) {
    // products and sums as explicit fmaf / rounded multiplies: every kernel
    // that inlines this rounds alike
    float th = fmaf(gh, cnorm2(v[m]), vat(m));
    if (vx != nullptr && valid) th = fmaf(vx[(unsigned)(t + T * m) * ustride], h, th);
    const float kq = rintf(th * 0.159154943091895336f);
    float r = fmaf(-kq, 6.28318548202514648f, th);
    r = fmaf(-kq, -1.74845553e-7f, r);
    float sn, cs;
    __sincosf(r, &sn, &cs);
    const bool cbig = fabsf(cs) >= fabsf(sn);
    const float b = cbig ? cs : sn, a = cbig ? sn : cs;
    const float e = -0.5f * fmaf(a, a, (b - 1.f) * (b + 1.f));
    cs = fmaf(cs, e, cs);
    sn = fmaf(sn, e, sn);
    v[m] = {fmaf(v[m].re, cs, __fmul_rn(v[m].im, sn)),
            fmaf(v[m].im, cs, __fmul_rn(-v[m].re, sn))};  // v * exp(-i th)
  }
}
// V from the line's row in shared memory
template <int E, int T>
__device__ __forceinline__ void nonlinear_phase(cx<float> (&v)[E], const float* vrow,
                                                float gh, const float* vx, float h,
                                                unsigned ustride, int t, bool valid) {
  nonlinear_phase_at<E, T>(v, [&](int m) { return vrow[t + T * m]; }, gh, vx, h, ustride, t, valid);
}
// V held in registers, vr[m] at position t + T m
template <int E, int T>
__device__ __forceinline__ void nonlinear_phase(cx<float> (&v)[E], const float (&vr)[E],
                                                float gh, const float* vx, float h,
                                                unsigned ustride, int t, bool valid) {
  nonlinear_phase_at<E, T>(v, [&](int m) { return vr[m]; }, gh, vx, h, ustride, t, valid);
}

// FFT . m . IFFT along my line, m = exp(i A k^2 tau) / N given per k as a
// rotation by three shears, (x, y) -> x1 = x - t y, y1 = y + s x1,
// x2 = x1 - t y1 with t = tan(phi/2), s = sin(phi), then the scale +-1/N.
// Each shear is one FMA and the shear matrices have determinant 1, so the
// rounded coefficients change the angle by ~1e-8 but not the norm: no mass
// drift on average, where the product with a hi + lo factor (two roundings)
// drifts by ~1e-8 per application on the structured spectra of lumps.
template <int N, bool CONTIG>
__device__ __forceinline__ void kinetic(cx<float> (&v)[Plan<N>::E], cx<float>* line_buf,
                                        const cx<float>* tw, const float4* lift, int t) {
  constexpr int E = Plan<N>::E, T = Plan<N>::T;
  line_transform<float, N, -1, CONTIG>(v, line_buf, tw, t, true);
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const float4 q = lift[t + T * m];
    const float x1 = fmaf(-q.x, v[m].im, v[m].re);
    const float y1 = fmaf(q.y, x1, v[m].im);
    const float x2 = fmaf(-q.x, y1, x1);
    v[m] = {x2 * q.z, y1 * q.z};
  }
  line_transform<float, N, +1, CONTIG>(v, line_buf, tw, t, true);
}

// rho = |psi|^2 of the tile and its R2C FFT along the line (two real lines per
// complex FFT).  put(k, ll, value) receives half-spectrum entry k of line ll
// for the valid lines; the calls are spread over all threads with ll fastest.
// REMAP: as in potential_c2r, the packed transform runs in the contiguous
// mapping, fed with |psi|^2 through shared memory.
// density_r2c_rho: the same from the density itself (rho[m] at position
// t + T m of line l; 0 on invalid lines), e.g. a sum over several fields.
template <int N, int LPB, bool CONTIG, class Put, bool TC = false, bool REMAP = false>
__device__ __forceinline__ void density_r2c_rho(const float (&rho)[Plan<N>::E], cx<float>* lines,
                                                const cx<float>* tw, int l, int t, int tid,
                                                int nvalid, Put put,
                                                const tc16::Tabs* tb = nullptr);

template <int N, int LPB, bool CONTIG, class Put, bool TC = false, bool REMAP = false>
__device__ __forceinline__ void density_r2c(const cx<float> (&psi)[Plan<N>::E], bool valid,
                                            cx<float>* lines, const cx<float>* tw, int l, int t,
                                            int tid, int nvalid, Put put,
                                            const tc16::Tabs* tb = nullptr) {
  float rho[Plan<N>::E];
#pragma unroll
  for (int m = 0; m < Plan<N>::E; ++m) rho[m] = valid ? cnorm2(psi[m]) : 0.f;
  density_r2c_rho<N, LPB, CONTIG, Put, TC, REMAP>(rho, lines, tw, l, t, tid, nvalid, put, tb);
}

template <int N, int LPB, bool CONTIG, class Put, bool TC, bool REMAP>
__device__ __forceinline__ void density_r2c_rho(const float (&rho)[Plan<N>::E], cx<float>* lines,
                                                const cx<float>* tw, int l, int t, int tid,
                                                int nvalid, Put put, const tc16::Tabs* tb) {
  using C = Cfg<N, LPB>;
  constexpr int E = C::E, T = C::T, NT = C::NT, LS = C::LS, H = C::H, TSTR = C::TSTR;
  constexpr int HALF = LPB / 2;
  cx<float> v[E];
  constexpr bool CC = REMAP || CONTIG;
  const int lc = REMAP ? tid / T : l;
  const int tc = REMAP ? tid % T : t;
  const bool pc = lc < HALF;  // this thread transforms packed line lc
  const bool pa = l < HALF;   // my own line l is the real part of packed line l % HALF
  __syncthreads();
  if (REMAP || !pa) {
    float* b = reinterpret_cast<float*>(lines + l * LS);
#pragma unroll
    for (int m = 0; m < E; ++m) b[t + T * m] = rho[m];
  }
  __syncthreads();
  if (pc) {
    const float* bb = reinterpret_cast<const float*>(lines + (lc + HALF) * LS);
    if constexpr (REMAP) {
      const float* ba = reinterpret_cast<const float*>(lines + lc * LS);
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = {ba[tc + T * m], bb[tc + T * m]};
    } else {
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = {rho[m], bb[tc + T * m]};
    }
  }
  xform<N, -1, CC, TC>(v, lines, tw, tb, lc, tc, HALF);
  __syncthreads();
  if (pc) {
#pragma unroll
    for (int q = 0; q < E; ++q) lines[lc * LS + pidx<N>(tc + T * q)] = v[q];
  }
  __syncthreads();
  constexpr int NH = (H + T - 1) / T;
  cx<float> hs[NH];
  const cx<float>* zb = lines + (l % HALF) * LS;
#pragma unroll
  for (int q = 0; q < NH; ++q) {
    const int k = t + T * q;
    hs[q] = {0.f, 0.f};
    if (k < H) {
      const cx<float> zk = zb[pidx<N>(k)];
      const cx<float> zn = cconj(zb[pidx<N>((N - k) & (N - 1))]);
      if (pa) {
        hs[q] = cscale(zk + zn, 0.5f);
      } else {
        const cx<float> d = zk - zn;
        hs[q] = {0.5f * d.im, -0.5f * d.re};  // (zk - conj z_{N-k}) / (2i)
      }
    }
  }
  __syncthreads();
  cx<float>* stage = lines;
#pragma unroll
  for (int q = 0; q < NH; ++q) {
    const int k = t + T * q;
    if (k < H) stage[k * TSTR + l] = hs[q];
  }
  __syncthreads();
  for (int idx = tid; idx < H * LPB; idx += NT) {
    const int ll = idx % LPB, k = idx / LPB;
    if (ll < nvalid) put(k, ll, stage[k * TSTR + ll]);
  }
}

// FFT . K(k) . IFFT along my line of the half spectrum, K = cN/k2 + cY/(k2 + mu2)
// with K(0) = 0, plus the constant cL at every k; k2 = k2pm (the two other
// axes) + k2l[k] (this axis).
template <int N, bool CONTIG>
__device__ __forceinline__ void green(cx<float> (&v)[Plan<N>::E], cx<float>* line_buf,
                                      const cx<float>* tw, const float* k2l, float k2pm, float cN,
                                      float cY, float mu2, float cL, int t) {
  constexpr int E = Plan<N>::E, T = Plan<N>::T;
  line_transform<float, N, -1, CONTIG>(v, line_buf, tw, t, true);
#pragma unroll
  for (int m = 0; m < E; ++m) {
    // one division; K's relative error of a few ulp moves the phase V h by far
    // less than the FP32 rounding of psi
    const float k2 = k2pm + k2l[t + T * m];
    const float den = k2 * (k2 + mu2);
    const float K = ((k2 > 0.f) ? __fdividef(fmaf(cN, k2 + mu2, cY * k2), den) : 0.f) + cL;
    v[m] = cscale(v[m], K);
  }
  line_transform<float, N, +1, CONTIG>(v, line_buf, tw, t, true);
}

}  // namespace tile
}  // namespace sn

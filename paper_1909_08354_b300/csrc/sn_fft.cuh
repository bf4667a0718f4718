// Line-FFT engine shared by every pass kernel of the split-step solver.
//
// The symmetric split-step Fourier method (Sec. III) spends its time in DFTs
// along one grid axis at a time: the kinetic propagator of Eq. 1 factors
// exactly into one 1D multiplier per axis, and the spectral solve of Eq. 2 is
// a DFT along every axis.  This header holds the in-register Stockham
// transform that every pass kernel runs on a batch of lines.
//
// Layout contract ("pattern P"): a line of N complex values is owned by
// T = N / E threads; thread t keeps elements t + T*m (m = 0..E-1) in
// registers v[m].  Every transform reads pattern P and leaves its result in
// pattern P with the natural frequency / space index, so a forward transform,
// a pointwise multiplier and an inverse transform chain without reordering.
// N = R0 * R1 (* R2): two or three Stockham stages (fft_plan.h); the data
// crosses shared memory between consecutive stages.  Stage twiddles come from
// a host-built FP64 table rounded once to the working precision.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_plan.h"

namespace snfft {

template <typename R>
struct cx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }

// FP32 complex addition and subtraction as one packed FP32x2 instruction each
// (sm_100 and later): the butterflies are mostly additions, and the passes
// are bound by instruction issue.  a - b is fma(b, -1, a), rounded once like
// a subtraction.
__device__ __forceinline__ cx<float> operator+(cx<float> a, cx<float> b) {
  const float2 r = __fadd2_rn(make_float2(a.re, a.im), make_float2(b.re, b.im));
  return {r.x, r.y};
}
__device__ __forceinline__ cx<float> operator-(cx<float> a, cx<float> b) {
  const float2 r =
      __ffma2_rn(make_float2(b.re, b.im), make_float2(-1.f, -1.f), make_float2(a.re, a.im));
  return {r.x, r.y};
}
template <typename R>
__device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ cx<R> cscale(cx<R> a, R s) { return {a.re * s, a.im * s}; }
template <typename R>
__device__ __forceinline__ cx<R> cconj(cx<R> a) { return {a.re, -a.im}; }
template <typename R>
__device__ __forceinline__ R cnorm2(cx<R> a) { return a.re * a.re + a.im * a.im; }
// FP32: the contraction written out (re^2 + fl(im^2) with one rounding of the
// sum), so that every kernel rounds it alike whatever the compiler would fuse
__device__ __forceinline__ float cnorm2(cx<float> a) {
  return fmaf(a.re, a.re, __fmul_rn(a.im, a.im));
}

// a * (SIGN * i)
template <typename R, int SIGN>
__device__ __forceinline__ cx<R> mul_si(cx<R> a) {
  if constexpr (SIGN < 0) return {a.im, -a.re};
  else return {-a.im, a.re};
}

// a * exp(SIGN * i * theta) with (c, s) = (cos theta, sin theta): the FP64
// engine's constant rotations (the FP32 engine uses rot8 and rot16).
template <typename R, int SIGN>
__device__ __forceinline__ cx<R> rot(cx<R> a, double c, double s) {
  const R cc = (R)c;
  const R ss = (R)(SIGN < 0 ? -s : s);
  return {a.re * cc - a.im * ss, a.re * ss + a.im * cc};
}

// a * exp(SIGN i pi/4) (Q = 1) or a * exp(SIGN i 3pi/4) (Q = 3).  The factor is
// (+-1 + SIGN i) sqrt(1/2): in FP32 the sum and difference of the two parts
// are formed first and then scaled by sqrt(1/2) as a hi + lo pair, two
// additions and two packed FP32x2 instructions instead of eight.
template <typename R, int SIGN, int Q>
__device__ __forceinline__ cx<R> rot8(cx<R> a);

// a * (wh + wl): product with a factor stored as a hi + lo pair (FP32 path).
// Every product and sum is an explicit fmaf or rounded multiply, so all
// kernels that inline it round alike.
__device__ __forceinline__ cx<float> cmul_hl(cx<float> a, cx<float> wh, cx<float> wl) {
  const float ur = fmaf(a.re, wl.re, __fmul_rn(-a.im, wl.im));
  const float ui = fmaf(a.re, wl.im, __fmul_rn(a.im, wl.re));
  return {fmaf(a.re, wh.re, fmaf(-a.im, wh.im, ur)), fmaf(a.re, wh.im, fmaf(a.im, wh.re, ui))};
}

// Multiply by table entry idx: FP32 tables hold hi parts at [0, n) and lo parts
// at [n, 2n); FP64 tables hold the value only.
template <typename R>
__device__ __forceinline__ cx<R> tmul(cx<R> a, const cx<R>* tab, int idx, int n) {
  if constexpr (sizeof(R) == sizeof(float)) {
    return cmul_hl(a, tab[idx], tab[n + idx]);
  } else {
    (void)n;
    return cmul(a, tab[idx]);
  }
}

// a * w (SIGN < 0) or a * conj(w) (SIGN > 0), w = table entry idx
template <typename R, int SIGN>
__device__ __forceinline__ cx<R> tmul_dir(cx<R> a, const cx<R>* tab, int idx, int n) {
  if constexpr (SIGN < 0) {
    return tmul(a, tab, idx, n);
  } else if constexpr (sizeof(R) == sizeof(float)) {
    return cmul_hl(a, cconj(tab[idx]), cconj(tab[n + idx]));
  } else {
    (void)n;
    return cmul(a, cconj(tab[idx]));
  }
}

// ---------------------------------------------------------------------------
// Small DFTs in registers:  X[q] = sum_r x[r] exp(SIGN 2 pi i r q / RAD)
// ---------------------------------------------------------------------------

template <typename R, int SIGN>
__device__ __forceinline__ void dft2(cx<R>* a) {
  cx<R> t = a[0];
  a[0] = t + a[1];
  a[1] = t - a[1];
}

template <typename R, int SIGN>
__device__ __forceinline__ void dft4(cx<R>& x0, cx<R>& x1, cx<R>& x2, cx<R>& x3) {
  const cx<R> t0 = x0 + x2, t1 = x0 - x2, t2 = x1 + x3;
  const cx<R> t3 = mul_si<R, SIGN>(x1 - x3);
  x0 = t0 + t2;
  x2 = t0 - t2;
  x1 = t1 + t3;
  x3 = t1 - t3;
}

constexpr double kC8 = 0.70710678118654752440;   // cos(pi/4)

template <typename R, int SIGN, int Q>
__device__ __forceinline__ cx<R> rot8(cx<R> a) {
  static_assert(Q == 1 || Q == 3, "rot8 turns by pi/4 or 3pi/4");
  if constexpr (sizeof(R) == sizeof(float)) {
    constexpr float h = (float)kC8;
    constexpr float l = (float)(kC8 - (double)(float)kC8);
    constexpr float sg = SIGN < 0 ? -1.f : 1.f;
    const float p = Q == 1 ? a.re - sg * a.im : -a.re - sg * a.im;
    const float q = Q == 1 ? a.im + sg * a.re : -a.im + sg * a.re;
    const float2 r = __ffma2_rn(make_float2(p, q), make_float2(h, h),
                                __fmul2_rn(make_float2(p, q), make_float2(l, l)));
    return {r.x, r.y};
  } else {
    return rot<R, SIGN>(a, Q == 1 ? kC8 : -kC8, kC8);
  }
}

// tan(k pi / 32) and sin(k pi / 16), k = 0..8: the three-shear form of the
// rotations by k pi / 16 inside the radix-16 kernel
constexpr double kTan32[9] = {0.0, 0.0984914033571642530772, 0.198912367379658006912,
                              0.303346683607342391676, 0.414213562373095048802,
                              0.534511135950791641090, 0.668178637919298919998,
                              0.820678790828660330972, 1.0};
constexpr double kSin16[9] = {0.0, 0.195090322016128267848, 0.382683432365089771728,
                              0.555570233019602224743, 0.707106781186547524401,
                              0.831469612302545237079, 0.923879532511286756128,
                              0.980785280403230449126, 1.0};

// a * exp(SIGN i k pi / 16), 0 < k < 16.  In FP32 the rotation is three shears,
// x1 = x - t y, y1 = y + s x1, x2 = x1 - t y1 with t = tan(phi/2), s = sin(phi):
// three FMAs, and each shear has determinant 1, so the rounded t and s move
// the angle by ~1e-8 but leave the norm alone (no mass drift), where a
// product with a rounded cosine and sine pair would not.  Angles past pi/2 are
// turned by phi - pi and negated (the negation folds into the FMA operands).
template <typename R, int SIGN, int K>
__device__ __forceinline__ cx<R> rot16(cx<R> a) {
  static_assert(K > 0 && K < 16, "rot16 turns by k pi / 16, 0 < k < 16");
  if constexpr (sizeof(R) == sizeof(float)) {
    constexpr bool flip = K > 8;
    constexpr int k = flip ? 16 - K : K;                  // |phi| = k pi / 16 after the flip
    constexpr float sg = (SIGN < 0) != flip ? -1.f : 1.f;  // sign of phi
    constexpr float t = sg * (float)kTan32[k], s = sg * (float)kSin16[k];
    const float x1 = fmaf(-t, a.im, a.re);
    const float y1 = fmaf(s, x1, a.im);
    const float x2 = fmaf(-t, y1, x1);
    if constexpr (flip) return {-x2, -y1};
    else return {x2, y1};
  } else {
    constexpr double c = K <= 8 ? kSin16[8 - K] : -kSin16[K - 8];  // cos(K pi / 16)
    constexpr double s = K <= 8 ? kSin16[K] : kSin16[16 - K];       // sin(K pi / 16)
    return rot<R, SIGN>(a, c, s);
  }
}

template <typename R, int SIGN>
__device__ __forceinline__ void dft8(cx<R>* a) {
  // radix-2 decimation in time over two 4-point DFTs
  cx<R> e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  cx<R> o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
  dft4<R, SIGN>(e0, e1, e2, e3);
  dft4<R, SIGN>(o0, o1, o2, o3);
  o1 = rot8<R, SIGN, 1>(o1);
  o2 = mul_si<R, SIGN>(o2);
  o3 = rot8<R, SIGN, 3>(o3);
  a[0] = e0 + o0; a[4] = e0 - o0;
  a[1] = e1 + o1; a[5] = e1 - o1;
  a[2] = e2 + o2; a[6] = e2 - o2;
  a[3] = e3 + o3; a[7] = e3 - o3;
}

template <typename R, int SIGN>
__device__ __forceinline__ void dft16(cx<R>* a) {
  // 16 = 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2
  cx<R> b[16];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    cx<R> x0 = a[n2], x1 = a[n2 + 4], x2 = a[n2 + 8], x3 = a[n2 + 12];
    dft4<R, SIGN>(x0, x1, x2, x3);
    b[4 * n2 + 0] = x0; b[4 * n2 + 1] = x1; b[4 * n2 + 2] = x2; b[4 * n2 + 3] = x3;
  }
  // twiddles W16^(n2 k1)
  b[5] = rot16<R, SIGN, 2>(b[5]);            // n2=1,k1=1 -> 1
  b[6] = rot8<R, SIGN, 1>(b[6]);             // 1,2 -> 2
  b[7] = rot16<R, SIGN, 6>(b[7]);            // 1,3 -> 3
  b[9] = rot8<R, SIGN, 1>(b[9]);             // 2,1 -> 2
  b[10] = mul_si<R, SIGN>(b[10]);            // 2,2 -> 4
  b[11] = rot8<R, SIGN, 3>(b[11]);           // 2,3 -> 6
  b[13] = rot16<R, SIGN, 6>(b[13]);          // 3,1 -> 3
  b[14] = rot8<R, SIGN, 3>(b[14]);           // 3,2 -> 6
  b[15] = rot16<R, -SIGN, 14>(b[15]);        // 3,3 -> 9 (18 pi/16 = -14 pi/16 mod 2 pi)
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    cx<R> x0 = b[k1], x1 = b[4 + k1], x2 = b[8 + k1], x3 = b[12 + k1];
    dft4<R, SIGN>(x0, x1, x2, x3);
    a[k1] = x0; a[k1 + 4] = x1; a[k1 + 8] = x2; a[k1 + 12] = x3;
  }
}

template <typename R, int SIGN, int RAD>
__device__ __forceinline__ void dft(cx<R>* a) {
  if constexpr (RAD == 1) {
  } else if constexpr (RAD == 2) {
    dft2<R, SIGN>(a);
  } else if constexpr (RAD == 4) {
    dft4<R, SIGN>(a[0], a[1], a[2], a[3]);
  } else if constexpr (RAD == 8) {
    dft8<R, SIGN>(a);
  } else {
    static_assert(RAD == 16, "unsupported radix");
    dft16<R, SIGN>(a);
  }
}

// ---------------------------------------------------------------------------
// Per-length plan: E elements per thread, T threads per line, radices R0, R1
// ---------------------------------------------------------------------------

template <int N>
struct Plan {
  static_assert(N >= 8 && N <= 1024 && (N & (N - 1)) == 0, "N must be a power of two in [8,1024]");
  static constexpr int E = plan_e(N);
  static constexpr int T = N / E;
  static constexpr int R0 = plan_r0(N), R1 = plan_r1(N), R2 = plan_r2(N);
  static constexpr int STAGES = plan_stages(N);
  // padded shared-memory line: one pad slot per 16 elements, so that the
  // runs a thread writes start at odd strides; the line stride is odd for
  // two stages and 2 or 4 modulo 16 for three, which keeps the exchanges of
  // the strided passes (lanes spread over 4 to 16 lines) conflict-free
  static constexpr int PAD_SHIFT = 4;
  static constexpr int LS = N + (N >> PAD_SHIFT) + (STAGES < 3 ? 1 : (N == 1024 ? 4 : 2));
  // twiddle table entries (fft_plan.h)
  static constexpr int TWN = plan_twn(N);
  // entries held per table in shared memory: FP32 keeps hi and lo parts
  template <typename R>
  static constexpr int tw_words() { return sizeof(R) == sizeof(float) ? 2 * TWN : TWN; }
};

template <int N>
__device__ __forceinline__ int pidx(int i) { return i + (i >> Plan<N>::PAD_SHIFT); }

// Twiddle tables: fft_plan.h.  The FP32 table appends the lo parts of all TWN
// entries.

// Barrier among the threads that share one line buffer.  CONTIG: line l is
// held by the consecutive threads [l T, (l + 1) T); a line of T <= 32
// threads then sits in one warp (warp barrier) and one of 64 threads in a
// warp pair (named barrier 1 + tid / 64, at most 15 pairs per CTA).  Lines
// spread over the CTA (strided mapping) take the CTA barrier.
template <int N, bool CONTIG>
__device__ __forceinline__ void line_sync() {
  constexpr int T = Plan<N>::T;
  if constexpr (CONTIG && T <= 32) {
    __syncwarp();
  } else if constexpr (CONTIG && T == 64) {
    asm volatile("bar.sync %0, 64;\n" ::"r"(1 + (int)(threadIdx.x >> 6)) : "memory");
  } else {
    __syncthreads();
  }
}

// In-place transform of one line held in pattern P.  Every thread of the CTA
// must call it (it contains barriers: line_sync); `active` masks the
// arithmetic and shared-memory traffic of threads whose line is idle in this
// transform.  CONTIG: the line mapping of line_sync.
template <typename R, int N, int SIGN, bool CONTIG = false>
__device__ __forceinline__ void line_transform(cx<R> (&v)[Plan<N>::E], cx<R>* line_buf,
                                               const cx<R>* tw_sm, int t, bool active) {
  using P = Plan<N>;
  constexpr int E = P::E, T = P::T;
  if constexpr (P::STAGES == 1) {
    if (active) dft<R, SIGN, E>(v);
    return;
  } else if constexpr (P::STAGES == 2) {
    constexpr int RA = SIGN < 0 ? P::R0 : P::R1;  // first stage radix (Ns = 1)
    constexpr int RB = SIGN < 0 ? P::R1 : P::R0;  // second stage radix (Ns = RA)
    constexpr int UA = E / RA, UB = E / RB;
    line_sync<N, CONTIG>();  // previous readers of line_buf are done
    if (active) {
#pragma unroll
      for (int u = 0; u < UA; ++u) {
        cx<R> a[RA];
#pragma unroll
        for (int r = 0; r < RA; ++r) a[r] = v[u + r * UA];
        dft<R, SIGN, RA>(a);
        const int j = t + T * u;
#pragma unroll
        for (int q = 0; q < RA; ++q) line_buf[pidx<N>(j * RA + q)] = a[q];
      }
    }
    line_sync<N, CONTIG>();
    if (active) {
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = line_buf[pidx<N>(t + T * m)];
      const cx<R>* tw = tw_sm + (SIGN < 0 ? 0 : N);
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        const int j = t + T * u;
        const int jm = j & (RA - 1);
        cx<R> a[RB];
        a[0] = v[u];
#pragma unroll
        for (int r = 1; r < RB; ++r) a[r] = tmul(v[u + r * UB], tw, r * RA + jm, P::TWN);
        dft<R, SIGN, RB>(a);
#pragma unroll
        for (int q = 0; q < RB; ++q) v[u + q * UB] = a[q];
      }
    }
  } else {
    // three stages R0, R1, R2 in both directions; the inverse multiplies by
    // the conjugate twiddles.  Stage s (span Ns, radix R) maps input j + r N/R
    // (j < N/R) to output (j / Ns) Ns R + j % Ns + q Ns after the twiddle
    // exp(SIGN 2 pi i (j % Ns) r / (Ns R)).
    constexpr int RA = P::R0, RB = P::R1, RC = P::R2, NB = RA * RB;
    constexpr int UA = E / RA, UB = E / RB, UC = E / RC;
    line_sync<N, CONTIG>();  // previous readers of line_buf are done
    if (active) {
#pragma unroll
      for (int u = 0; u < UA; ++u) {
        cx<R> a[RA];
#pragma unroll
        for (int r = 0; r < RA; ++r) a[r] = v[u + r * UA];
        dft<R, SIGN, RA>(a);
        const int j = t + T * u;
#pragma unroll
        for (int q = 0; q < RA; ++q) line_buf[pidx<N>(j * RA + q)] = a[q];
      }
    }
    line_sync<N, CONTIG>();
    if (active) {
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = line_buf[pidx<N>(t + T * m)];
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        const int jm = (t + T * u) & (RA - 1);
        cx<R> a[RB];
        a[0] = v[u];
#pragma unroll
        for (int r = 1; r < RB; ++r) a[r] = tmul_dir<R, SIGN>(v[u + r * UB], tw_sm, r * RA + jm, P::TWN);
        dft<R, SIGN, RB>(a);
#pragma unroll
        for (int q = 0; q < RB; ++q) v[u + q * UB] = a[q];
      }
    }
    line_sync<N, CONTIG>();  // every read of line_buf is done
    if (active) {
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        const int j = t + T * u;
        const int o = (j / RA) * NB + (j & (RA - 1));
#pragma unroll
        for (int q = 0; q < RB; ++q) line_buf[pidx<N>(o + q * RA)] = v[u + q * UB];
      }
    }
    line_sync<N, CONTIG>();
    if (active) {
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = line_buf[pidx<N>(t + T * m)];
#pragma unroll
      for (int u = 0; u < UC; ++u) {
        const int j = t + T * u;  // < NB
        cx<R> a[RC];
        a[0] = v[u];
#pragma unroll
        for (int r = 1; r < RC; ++r) a[r] = tmul_dir<R, SIGN>(v[u + r * UC], tw_sm, NB + r * NB + j, P::TWN);
        dft<R, SIGN, RC>(a);
#pragma unroll
        for (int q = 0; q < RC; ++q) v[u + q * UC] = a[q];
      }
    }
  }
}

}  // namespace snfft

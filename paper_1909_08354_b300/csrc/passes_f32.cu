// Fused FP32 pass kernels of the merged Strang split step (Sec. III; Eqs. 1-2).
//
// One merged step is six passes over HBM in 3D (two and one in 2D):
//   P1  psi along axis c:  V = C2R IFFT_c of the potential half spectrum,
//       psi <- exp(-i (V + V_ext + g |psi|^2) h) psi, then FFT_c . m_c . IFFT_c
//   P2  psi along axis b:  FFT_b . m_b . IFFT_b
//   P3  psi along axis a:  FFT_a . m_a . IFFT_a, then rho = |psi|^2 and its
//       R2C FFT_a (two real lines packed into one complex line) -> half spectrum
//   P4  half spectrum along b: FFT_b
//   P5  half spectrum along c: FFT_c . K(k) . IFFT_c  (Green's multiplier of Eq. 2 / Eq. 9)
//   P6  half spectrum along b: IFFT_b
// The axis order flips every step so that the half-spectrum axis of P3 is the
// C2R axis of the next P1.  The half spectrum is stored with the half axis
// slowest, [k_h][line], so both the R2C store of P3 and the C2R load of P1 are
// coalesced over 16 neighbouring lines.
#include "sn_fft.cuh"
#include "sn_internal.h"

using namespace snfft;

namespace sn {
namespace {

constexpr int LPB = kLinesPerCta;
constexpr int TSTR = LPB + 1;  // padded row of the [k][line] staging tile

// CTAs per SM the register allocation must allow: 1024 resident threads for
// lines up to 256 points (memory-level parallelism for the HBM stream).
template <int N>
constexpr int min_ctas() {
  constexpr int threads = LPB * Plan<N>::T;
  constexpr int want = 1024 / threads;
  return want < 1 ? 1 : (want > 16 ? 16 : want);
}

__device__ __forceinline__ cx<float> ldc(const float2* p) {
  const float2 v = *p;
  return {v.x, v.y};
}
__device__ __forceinline__ void stc(float2* p, cx<float> v) { *p = make_float2(v.re, v.im); }

// shared memory: twiddles (hi, lo), kinetic factors (hi, lo), line buffers
template <int N>
constexpr size_t psi_smem_bytes() {
  return (size_t)(2 * Plan<N>::TWN + 2 * N + LPB * Plan<N>::LS) * sizeof(cx<float>);
}
template <int N>
constexpr size_t rho_smem_bytes() {
  return (size_t)(2 * Plan<N>::TWN + LPB * Plan<N>::LS) * sizeof(cx<float>);
}

template <int N, bool STRIDED, int VARIANT>
__global__ void __launch_bounds__(LPB * Plan<N>::T, min_ctas<N>())
psi_pass_kernel(PsiPassArgs a) {
  using P = Plan<N>;
  constexpr int E = P::E, T = P::T, NT = LPB * T, LS = P::LS, H = N / 2 + 1;
  constexpr bool NPHASE = VARIANT == PSI_NPHASE;
  constexpr bool DENSITY = VARIANT == PSI_DENSITY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* tw_sm = reinterpret_cast<cx<float>*>(smem_raw);
  cx<float>* mult_sm = tw_sm + 2 * P::TWN;
  cx<float>* lines = mult_sm + 2 * N;

  const int tid = threadIdx.x;
  const int l = STRIDED ? (tid % LPB) : (tid / T);
  const int t = STRIDED ? (tid / LPB) : (tid % T);

  long long line0;  // line id of CTA line 0 (lines are numbered o * inner + i)
  int nvalid;
  size_t base, stride;
  if constexpr (STRIDED) {
    const long long o = blockIdx.y, i0 = (long long)blockIdx.x * LPB;
    nvalid = (int)min((long long)LPB, a.inner - i0);
    line0 = o * a.inner + i0;
    base = (size_t)o * N * a.inner + i0 + l;
    stride = a.inner;
  } else {
    const long long o0 = (long long)blockIdx.x * LPB;
    nvalid = (int)min((long long)LPB, a.outer - o0);
    line0 = o0;
    base = (size_t)(o0 + l) * N;
    stride = 1;
  }
  const bool valid = l < nvalid;
  const size_t nlines = (size_t)(a.outer * a.inner);
  // element m of my line sits at pl + (t + T m) * stride; offsets fit in 32 bits
  // (a grid holds at most 2^30 cells)
  float2* pl = a.psi + base;
  const unsigned ustride = (unsigned)stride;

  for (int k = tid; k < 2 * P::TWN; k += NT) tw_sm[k] = ldc(a.tw + k);
  for (int k = tid; k < 2 * N; k += NT) mult_sm[k] = ldc(a.mult + k);

  cx<float> v[E];
  float vph[E];
  (void)vph;

  if constexpr (NPHASE) {
    // ---- potential: C2R inverse FFT of the half spectrum of lines (l, l + 8)
    cx<float>* tile = lines;
    for (int idx = tid; idx < H * LPB; idx += NT) {
      const int ll = idx % LPB, k = idx / LPB;
      cx<float> z = {0.f, 0.f};
      if (ll < nvalid) z = ldc(a.rh_in + (size_t)k * nlines + line0 + ll);
      tile[k * TSTR + ll] = z;
    }
    __syncthreads();
    const bool pa = l < LPB / 2;
    if (pa) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int k = t + T * m;
        cx<float> A, B;
        if (k <= N / 2) {
          A = tile[k * TSTR + l];
          B = tile[k * TSTR + l + LPB / 2];
          if (k == 0 || k == N / 2) { A.im = 0.f; B.im = 0.f; }
        } else {
          A = cconj(tile[(N - k) * TSTR + l]);
          B = cconj(tile[(N - k) * TSTR + l + LPB / 2]);
        }
        v[m] = {A.re - B.im, A.im + B.re};  // A + i B
      }
    }
    __syncthreads();  // tile consumed before the line buffers are reused
    line_transform<float, N, +1>(v, lines + l * LS, tw_sm, t, pa);
    __syncthreads();
    if (pa) {
      float* up = reinterpret_cast<float*>(lines + (l + LPB / 2) * LS);
#pragma unroll
      for (int m = 0; m < E; ++m) {
        vph[m] = v[m].re;
        up[t + T * m] = v[m].im;
      }
    }
    __syncthreads();
    if (!pa) {
      const float* up = reinterpret_cast<const float*>(lines + l * LS);
#pragma unroll
      for (int m = 0; m < E; ++m) vph[m] = up[t + T * m];
    }
  }
  __syncthreads();  // tables visible; V exchange buffers read

  // ---- load psi (pattern P), nonlinear phase
#pragma unroll
  for (int m = 0; m < E; ++m) {
    cx<float> z = {0.f, 0.f};
    if (valid) z = ldc(pl + (unsigned)(t + T * m) * ustride);
    v[m] = z;
  }
  if constexpr (NPHASE) {
    const float* vx = a.vext != nullptr ? a.vext + base : nullptr;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      float th = vph[m] + a.gh * cnorm2(v[m]);
      if (vx != nullptr && valid) th += vx[(unsigned)(t + T * m) * ustride] * a.h;
      float s, c;
      sincosf(th, &s, &c);
      // one Newton step towards |(c, s)| = 1 removes the modulus error of the pair
      const float f = fmaf(-0.5f, fmaf(c, c, fmaf(s, s, -1.f)), 1.f);
      c *= f;
      s *= f;
      v[m] = {v[m].re * c + v[m].im * s, v[m].im * c - v[m].re * s};  // v * exp(-i th)
    }
  }

  // ---- kinetic factor along this axis
  line_transform<float, N, -1>(v, lines + l * LS, tw_sm, t, true);
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = cmul_hl(v[m], mult_sm[t + T * m], mult_sm[N + t + T * m]);
  line_transform<float, N, +1>(v, lines + l * LS, tw_sm, t, true);

  asm volatile("" : "+l"(pl));  // recompute store addresses instead of keeping 16 live
  if (valid) {
#pragma unroll
    for (int m = 0; m < E; ++m) stc(pl + (unsigned)(t + T * m) * ustride, v[m]);
  }

  if constexpr (DENSITY) {
    // ---- rho = |psi|^2, R2C along this axis, two real lines per complex FFT
    float rho[E];
#pragma unroll
    for (int m = 0; m < E; ++m) rho[m] = valid ? cnorm2(v[m]) : 0.f;
    const bool pa = l < LPB / 2;
    __syncthreads();
    if (!pa) {
      float* b = reinterpret_cast<float*>(lines + l * LS);
#pragma unroll
      for (int m = 0; m < E; ++m) b[t + T * m] = rho[m];
    }
    __syncthreads();
    if (pa) {
      const float* b = reinterpret_cast<const float*>(lines + (l + LPB / 2) * LS);
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = {rho[m], b[t + T * m]};
    }
    line_transform<float, N, -1>(v, lines + l * LS, tw_sm, t, pa);
    __syncthreads();
    if (pa) {
#pragma unroll
      for (int q = 0; q < E; ++q) lines[l * LS + pidx(t + T * q)] = v[q];
    }
    __syncthreads();
    constexpr int NH = (H + T - 1) / T;
    cx<float> hs[NH];
    const cx<float>* zb = lines + (l % (LPB / 2)) * LS;
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      const int k = t + T * i;
      hs[i] = {0.f, 0.f};
      if (k < H) {
        const cx<float> zk = zb[pidx(k)];
        const cx<float> zn = cconj(zb[pidx((N - k) & (N - 1))]);
        if (pa) {
          hs[i] = cscale(zk + zn, 0.5f);
        } else {
          const cx<float> d = zk - zn;
          hs[i] = {0.5f * d.im, -0.5f * d.re};  // (zk - conj z_{N-k}) / (2i)
        }
      }
    }
    __syncthreads();
    cx<float>* tile = lines;
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      const int k = t + T * i;
      if (k < H) tile[k * TSTR + l] = hs[i];
    }
    __syncthreads();
    for (int idx = tid; idx < H * LPB; idx += NT) {
      const int ll = idx % LPB, k = idx / LPB;
      if (ll < nvalid) stc(a.rh_out + (size_t)k * nlines + line0 + ll, tile[k * TSTR + ll]);
    }
  }
}

template <int N, bool STRIDED, int OP>
__global__ void __launch_bounds__(LPB * Plan<N>::T, min_ctas<N>())
rho_pass_kernel(RhoPassArgs a) {
  using P = Plan<N>;
  constexpr int E = P::E, T = P::T, NT = LPB * T, LS = P::LS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* tw_sm = reinterpret_cast<cx<float>*>(smem_raw);
  cx<float>* lines = tw_sm + 2 * P::TWN;

  const int tid = threadIdx.x;
  const int l = STRIDED ? (tid % LPB) : (tid / T);
  const int t = STRIDED ? (tid / LPB) : (tid % T);
  long long o, i;
  int nvalid;
  size_t base, stride;
  if constexpr (STRIDED) {
    o = blockIdx.y;
    const long long i0 = (long long)blockIdx.x * LPB;
    i = i0 + l;
    nvalid = (int)min((long long)LPB, a.inner - i0);
    base = (size_t)o * N * a.inner + i;
    stride = a.inner;
  } else {
    const long long o0 = (long long)blockIdx.x * LPB;
    o = o0 + l;
    i = 0;
    nvalid = (int)min((long long)LPB, a.outer - o0);
    base = (size_t)o * N;
    stride = 1;
  }
  const bool valid = l < nvalid;
  float2* pl = a.data + base;
  const unsigned ustride = (unsigned)stride;
  for (int k = tid; k < 2 * P::TWN; k += NT) tw_sm[k] = ldc(a.tw + k);
  __syncthreads();

  cx<float> v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    cx<float> z = {0.f, 0.f};
    if (valid) z = ldc(pl + (unsigned)(t + T * m) * ustride);
    v[m] = z;
  }
  if constexpr (OP == RHO_INV) {
    line_transform<float, N, +1>(v, lines + l * LS, tw_sm, t, true);
  } else {
    line_transform<float, N, -1>(v, lines + l * LS, tw_sm, t, true);
  }
  if constexpr (OP == RHO_GREEN) {
    long long plane, mid;
    if constexpr (STRIDED) {
      plane = o;
      mid = i;
    } else {
      plane = o / a.mid_n;
      mid = o - plane * a.mid_n;
    }
    float k2pm = 0.f;
    if (valid) k2pm = a.k2p[plane] + a.k2m[mid];
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const float k2 = k2pm + a.k2l[t + T * m];
      const float K = (k2 > 0.f) ? (a.cN / k2 + a.cY / (k2 + a.mu2)) : 0.f;
      v[m] = cscale(v[m], K);
    }
    line_transform<float, N, +1>(v, lines + l * LS, tw_sm, t, true);
  }
  asm volatile("" : "+l"(pl));
  if (valid) {
#pragma unroll
    for (int m = 0; m < E; ++m) stc(pl + (unsigned)(t + T * m) * ustride, v[m]);
  }
}

template <int N, bool STRIDED, int VARIANT>
cudaError_t launch_psi_t(const PsiPassArgs& a, cudaStream_t s) {
  constexpr size_t smem = psi_smem_bytes<N>();
  auto kern = psi_pass_kernel<N, STRIDED, VARIANT>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 block(LPB * Plan<N>::T);
  dim3 grid;
  if (STRIDED) grid = dim3((unsigned)((a.inner + LPB - 1) / LPB), (unsigned)a.outer);
  else grid = dim3((unsigned)((a.outer + LPB - 1) / LPB));
  kern<<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

template <int N, bool STRIDED, int OP>
cudaError_t launch_rho_t(const RhoPassArgs& a, cudaStream_t s) {
  constexpr size_t smem = rho_smem_bytes<N>();
  auto kern = rho_pass_kernel<N, STRIDED, OP>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 block(LPB * Plan<N>::T);
  dim3 grid;
  if (STRIDED) grid = dim3((unsigned)((a.inner + LPB - 1) / LPB), (unsigned)a.outer);
  else grid = dim3((unsigned)((a.outer + LPB - 1) / LPB));
  kern<<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

template <int N>
cudaError_t psi_dispatch(bool strided, int variant, const PsiPassArgs& a, cudaStream_t s) {
  if (strided) {
    switch (variant) {
      case PSI_PLAIN: return launch_psi_t<N, true, PSI_PLAIN>(a, s);
      case PSI_NPHASE: return launch_psi_t<N, true, PSI_NPHASE>(a, s);
      default: return launch_psi_t<N, true, PSI_DENSITY>(a, s);
    }
  }
  switch (variant) {
    case PSI_PLAIN: return launch_psi_t<N, false, PSI_PLAIN>(a, s);
    case PSI_NPHASE: return launch_psi_t<N, false, PSI_NPHASE>(a, s);
    default: return launch_psi_t<N, false, PSI_DENSITY>(a, s);
  }
}

template <int N>
cudaError_t rho_dispatch(bool strided, int op, const RhoPassArgs& a, cudaStream_t s) {
  if (strided) {
    switch (op) {
      case RHO_FWD: return launch_rho_t<N, true, RHO_FWD>(a, s);
      case RHO_GREEN: return launch_rho_t<N, true, RHO_GREEN>(a, s);
      default: return launch_rho_t<N, true, RHO_INV>(a, s);
    }
  }
  switch (op) {
    case RHO_FWD: return launch_rho_t<N, false, RHO_FWD>(a, s);
    case RHO_GREEN: return launch_rho_t<N, false, RHO_GREEN>(a, s);
    default: return launch_rho_t<N, false, RHO_INV>(a, s);
  }
}

}  // namespace

cudaError_t launch_psi_pass_f32(int N, bool strided, int variant, const PsiPassArgs& a,
                                cudaStream_t s) {
  switch (N) {
    case 8: return psi_dispatch<8>(strided, variant, a, s);
    case 16: return psi_dispatch<16>(strided, variant, a, s);
    case 32: return psi_dispatch<32>(strided, variant, a, s);
    case 64: return psi_dispatch<64>(strided, variant, a, s);
    case 128: return psi_dispatch<128>(strided, variant, a, s);
    case 256: return psi_dispatch<256>(strided, variant, a, s);
    case 512: return psi_dispatch<512>(strided, variant, a, s);
    case 1024: return psi_dispatch<1024>(strided, variant, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_rho_pass_f32(int N, bool strided, int op, const RhoPassArgs& a,
                                cudaStream_t s) {
  switch (N) {
    case 8: return rho_dispatch<8>(strided, op, a, s);
    case 16: return rho_dispatch<16>(strided, op, a, s);
    case 32: return rho_dispatch<32>(strided, op, a, s);
    case 64: return rho_dispatch<64>(strided, op, a, s);
    case 128: return rho_dispatch<128>(strided, op, a, s);
    case 256: return rho_dispatch<256>(strided, op, a, s);
    case 512: return rho_dispatch<512>(strided, op, a, s);
    case 1024: return rho_dispatch<1024>(strided, op, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sn

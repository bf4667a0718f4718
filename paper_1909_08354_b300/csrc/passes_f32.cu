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
//
// The kernels are persistent: a CTA loads its tables once and walks tiles of
// 16 lines with a stride of gridDim.x.  While it transforms one tile, the next
// tile's psi is already in flight into registers and (P1) the next tile's half
// spectrum into shared memory through cp.async, so the HBM stream does not
// wait for the arithmetic.
#include <cmath>

#include "sn_fft.cuh"
#include "sn_internal.h"
#include "tile_ops.cuh"

using namespace snfft;

namespace sn {
namespace {

using tile::load_line;
using tile::store_line;

// Lines per CTA: 16 (a 128-byte row of 16 neighbouring lines for the strided
// passes); 8 for 1024-point lines, whose tables, line buffers and staging
// tiles would not fit in shared memory at 16.
template <int N>
__host__ __device__ constexpr int lpb() {
  return N >= 1024 ? kLinesPerCta / 2 : kLinesPerCta;
}

template <int N>
constexpr int cta_threads() {
  return lpb<N>() * Plan<N>::T;
}

// Resident CTAs per SM the register allocation is sized for: 512 threads per
// SM, i.e. up to 128 registers, room for the prefetched tile.
template <int N>
constexpr int min_ctas() {
  constexpr int want = 512 / cta_threads<N>();
  return want < 1 ? 1 : (want > 16 ? 16 : want);
}

// Programmatic dependent launch: the pass kernels of a step follow one
// another on one stream, each reading what the previous one wrote.  Each
// kernel lets the next one launch at once (its CTAs take SMs as this one's
// CTAs retire and stage their constant tables), and waits for the previous
// grid to complete, with its writes visible, before it touches psi or the
// half spectrum.  Without a programmatic predecessor the wait returns at once.
__device__ __forceinline__ void pdl_allow_next() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
__device__ __forceinline__ void pdl_wait_prev() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

__device__ __forceinline__ cx<float> ldc(const float2* p) {
  const float2 v = *p;
  return {v.x, v.y};
}

// 8-byte asynchronous global->shared copy; src_bytes = 0 writes zeros without reading.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool pred) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int n = pred ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(n)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int K>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory");
}

// shared memory: twiddles (hi, lo), kinetic factors (shears), line buffers,
// and for P1 two staging tiles of the half spectrum.  The tensor-core engine
// (TC, 256-point lines) keeps its fragment and twiddle tables, a padded copy
// of the kinetic factors and padded line buffers instead.
template <int N, int VARIANT, bool TC, bool FIELDS = false>
constexpr size_t psi_smem_bytes() {
  // P1: two half-spectrum staging tiles; fused-fields P3: the density sum
  constexpr size_t stage =
      VARIANT == PSI_NPHASE ? 2 * (N / 2 + 1) * (lpb<N>() + 1) * sizeof(cx<float>)
      : (VARIANT == PSI_DENSITY && FIELDS) ? (size_t)N * (lpb<N>() + 1) * sizeof(float)
                                           : 0;
  if constexpr (TC) {
    return sizeof(tc16::Tabs) + 2 * tc16::MT * sizeof(float2) +
           (size_t)lpb<N>() * tc16::LS * sizeof(float2) + stage;
  } else {
    return (size_t)(2 * Plan<N>::TWN + 2 * N + lpb<N>() * Plan<N>::LS) * sizeof(cx<float>) + stage;
  }
}
template <int N, bool TC>
constexpr size_t rho_smem_bytes() {
  if constexpr (TC) {
    return sizeof(tc16::Tabs) + tc16::MT * sizeof(float) + 16 * sizeof(float) +
           (size_t)lpb<N>() * tc16::LS * sizeof(float2);
  } else {
    return (size_t)(2 * Plan<N>::TWN + lpb<N>() * Plan<N>::LS) * sizeof(cx<float>);
  }
}

// FIELDS: a.nfields coupled fields, a.fstride elements apart, in one launch
// (NPHASE, DENSITY; FP32 engine).  Each tile's potential C2R (NPHASE) or
// density R2C (DENSITY) runs once for all fields: the fields' lines of a tile
// follow one another through the kinetic transform, with the potential row
// kept across them in the tile's staging buffer (free once the C2R has read
// it), or their densities summed in registers.
template <int N, bool STRIDED, int VARIANT, bool TC, bool FIELDS = false>
__global__ void __launch_bounds__(cta_threads<N>(), min_ctas<N>())
psi_pass_kernel(PsiPassArgs a) {
  static_assert(!TC || N == tc16::N, "the tensor-core engine handles 256-point lines");
  static_assert(!FIELDS || (!TC && VARIANT != PSI_PLAIN), "fused fields: FP32 NPHASE, DENSITY");
  using P = Plan<N>;
  constexpr int LPB = lpb<N>(), TSTR = LPB + 1;
  constexpr int E = P::E, T = P::T, NT = LPB * T, LS = P::LS, H = N / 2 + 1;
  constexpr bool NPHASE = VARIANT == PSI_NPHASE;
  constexpr bool DENSITY = VARIANT == PSI_DENSITY;
  constexpr bool PF = E <= 16;  // register prefetch of the next tile
  constexpr bool CONTIG = !STRIDED;  // line l held by threads [l T, (l + 1) T)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* tw_sm = reinterpret_cast<cx<float>*>(smem_raw);
  cx<float>* mult_sm = tw_sm + 2 * P::TWN;
  cx<float>* lines = mult_sm + 2 * N;
  tc16::Tabs* tabs = reinterpret_cast<tc16::Tabs*>(smem_raw);
  float2* mult_tc = reinterpret_cast<float2*>(smem_raw + sizeof(tc16::Tabs));
  if constexpr (TC) lines = reinterpret_cast<cx<float>*>(mult_tc + 2 * tc16::MT);
  cx<float>* rstage = lines + LPB * (TC ? tc16::LS : LS);  // P1: two [H][TSTR] tiles

  const int tid = threadIdx.x;
  const int l = STRIDED ? (tid % LPB) : (tid / T);
  const int t = STRIDED ? (tid / LPB) : (tid % T);
  const tile::Tiles<LPB, STRIDED> tiles(a.outer, a.inner);
  const size_t nlines = (size_t)(a.outer * a.inner);
  // element m of a line sits at base + (t + T m) * stride; offsets fit in 32
  // bits (a grid holds at most 2^30 cells)
  const unsigned ustride = STRIDED ? (unsigned)a.inner : 1u;

  pdl_allow_next();
  if constexpr (TC) {
    tc16::load_tabs(tabs, a.tc, a.tw, tid, NT);
    for (int k = tid; k < 2 * N; k += NT) mult_tc[(k / N) * tc16::MT + tc16::pt(k % N)] = a.mult[k];
  } else {
    for (int k = tid; k < 2 * P::TWN; k += NT) tw_sm[k] = ldc(a.tw + k);
    for (int k = tid; k < N; k += NT) reinterpret_cast<float4*>(mult_sm)[k] = a.lift[k];
  }
  pdl_wait_prev();  // psi and the half spectrum come from the previous pass

  // P1: stage the [k][line] half-spectrum tile of tile tau into shared memory
  auto stage_rho = [&](cx<float>* dst, long long tau) {
    long long line0, o, i;
    int nvalid;
    size_t base;
    tiles.at(tau, 0, N, line0, nvalid, base, o, i);
    for (int idx = tid; idx < H * LPB; idx += NT) {
      const int ll = idx % LPB, k = idx / LPB;
      const bool ok = ll < nvalid;
      cp_async8(dst + k * TSTR + ll, a.rh_in + (ok ? (size_t)k * nlines + line0 + ll : 0), ok);
    }
  };

  cx<float> vn[E];
  long long tau = blockIdx.x;
  if (tau < tiles.count) {
    long long line0, o, i;
    int nvalid;
    size_t base;
    tiles.at(tau, l, N, line0, nvalid, base, o, i);
    if constexpr (PF) load_line<E, T>(vn, a.psi + base, ustride, t, l < nvalid);
    if constexpr (NPHASE) stage_rho(rstage, tau);
  }
  if constexpr (NPHASE) cp_async_commit();
  __syncthreads();  // tables

  if constexpr (FIELDS) {
    static_assert(PF, "the fields loop prefetches the next line");
    const int nf = a.nfields;
    const size_t fs = (size_t)a.fstride;
    for (int it = 0; tau < tiles.count; ++it, tau += gridDim.x) {
      long long line0, o, i;
      int nvalid;
      size_t base;
      tiles.at(tau, l, N, line0, nvalid, base, o, i);
      const bool valid = l < nvalid;
      const long long taun = tau + gridDim.x;
      // NPHASE: this tile's potential row, for every field; DENSITY: the sum of
      // the fields' |psi|^2.  Both at [position][line] with an odd row pitch
      // (conflict-free in both mappings; a staging tile's (N + 2)(LPB + 1)
      // floats fit N (LPB + 1)); each thread reads back only what it wrote.
      float* keep = reinterpret_cast<float*>(rstage + (NPHASE ? (it & 1) * (H * TSTR) : 0));
      if constexpr (NPHASE) {
        if (taun < tiles.count) stage_rho(rstage + ((it + 1) & 1) * (H * TSTR), taun);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const float* vrow = tile::potential_c2r<N, LPB, CONTIG, false, STRIDED>(
            rstage + (it & 1) * (H * TSTR), lines, tw_sm, l, t, tabs);
        // the C2R ended with a CTA barrier after its last read of the staging tile
#pragma unroll
        for (int m = 0; m < E; ++m) keep[(t + T * m) * TSTR + l] = vrow[t + T * m];
      }
      for (int j = 0; j < nf; ++j) {
        cx<float> v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = vn[m];
        // start the load of the next (tile, field)
        if (j + 1 < nf) {
          load_line<E, T>(vn, a.psi + base + (size_t)(j + 1) * fs, ustride, t, valid);
        } else if (taun < tiles.count) {
          long long line0n, on, in;
          int nvalidn;
          size_t basen;
          tiles.at(taun, l, N, line0n, nvalidn, basen, on, in);
          load_line<E, T>(vn, a.psi + basen, ustride, t, l < nvalidn);
        }
        if constexpr (NPHASE) {
          tile::nonlinear_phase_at<E, T>(
              v, [&](int m) { return keep[(t + T * m) * TSTR + l]; }, a.gh,
              a.vext != nullptr ? a.vext + base : nullptr, a.h, ustride, t, valid);
        }
        tile::kinetic<N, CONTIG>(v, lines + l * LS, tw_sm, reinterpret_cast<const float4*>(mult_sm),
                                 t);
        store_line<E, T>(v, a.psi + base + (size_t)j * fs, ustride, t, valid);
        if constexpr (DENSITY) {
#pragma unroll
          for (int m = 0; m < E; ++m) {
            float& r = keep[(t + T * m) * TSTR + l];
            r = (j > 0 ? r : 0.f) + (valid ? cnorm2(v[m]) : 0.f);
          }
        }
      }
      if constexpr (DENSITY) {
        float rho[E];
#pragma unroll
        for (int m = 0; m < E; ++m) rho[m] = keep[(t + T * m) * TSTR + l];
        float2* rh = a.rh_out;
        auto put = [&](int k, int ll, cx<float> z) {
          tile::stg_c(rh + (size_t)k * nlines + line0 + ll, z);
        };
        tile::density_r2c_rho<N, LPB, CONTIG, decltype(put), false, STRIDED>(rho, lines, tw_sm, l, t,
                                                                          tid, nvalid, put);
      }
      __syncthreads();  // line buffers and the staging tile are reused next iteration
    }
    if constexpr (NPHASE) cp_async_wait<0>();
    return;
  }

  for (int it = 0; tau < tiles.count; ++it, tau += gridDim.x) {
    long long line0, o, i;
    int nvalid;
    size_t base;
    tiles.at(tau, l, N, line0, nvalid, base, o, i);
    const bool valid = l < nvalid;
    const long long taun = tau + gridDim.x;
    cx<float> v[E];
    const float* vrow = nullptr;
    (void)vrow;

    if constexpr (NPHASE) {
      if (taun < tiles.count) stage_rho(rstage + ((it + 1) & 1) * (H * TSTR), taun);
      cp_async_commit();
      cp_async_wait<1>();
      __syncthreads();
      vrow = tile::potential_c2r<N, LPB, CONTIG, TC, STRIDED>(rstage + (it & 1) * (H * TSTR), lines,
                                                          tw_sm, l, t, tabs);
    }

    // ---- this tile's psi (loaded one iteration ago); start the next tile's load
    if constexpr (PF) {
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = vn[m];
      if (taun < tiles.count) {
        long long line0n, on, in;
        int nvalidn;
        size_t basen;
        tiles.at(taun, l, N, line0n, nvalidn, basen, on, in);
        load_line<E, T>(vn, a.psi + basen, ustride, t, l < nvalidn);
      }
    } else {
      load_line<E, T>(v, a.psi + base, ustride, t, valid);
    }

    if constexpr (NPHASE) {
      tile::nonlinear_phase<E, T>(v, vrow, a.gh, a.vext != nullptr ? a.vext + base : nullptr, a.h,
                                  ustride, t, valid);
    }
    if constexpr (TC) {
      const tc16::MultTable mt{mult_tc, mult_tc + tc16::MT};
      tc16::fmi(v, lines, *tabs, l, t, [&](int) { return mt; });
    } else {
      tile::kinetic<N, CONTIG>(v, lines + l * LS, tw_sm, reinterpret_cast<const float4*>(mult_sm), t);
    }
    store_line<E, T>(v, a.psi + base, ustride, t, valid);

    if constexpr (DENSITY) {
      float2* rh = a.rh_out;
      const bool accum = a.rh_accum != 0;
      auto put = [&](int k, int ll, cx<float> z) {
        float2* p = rh + (size_t)k * nlines + line0 + ll;
        if (accum) z = z + tile::ldg_c<true>(p);  // each element has one writer per launch
        tile::stg_c(p, z);
      };
      tile::density_r2c<N, LPB, CONTIG, decltype(put), TC, STRIDED>(v, valid, lines, tw_sm, l, t, tid,
                                                                nvalid, put, tabs);
    }
    __syncthreads();  // line buffers and the staging tile are reused next iteration
  }
  if constexpr (NPHASE) cp_async_wait<0>();
}

template <int N, bool STRIDED, int OP, bool TC>
__global__ void __launch_bounds__(cta_threads<N>(), min_ctas<N>())
rho_pass_kernel(RhoPassArgs a) {
  static_assert(!TC || N == tc16::N, "the tensor-core engine handles 256-point lines");
  using P = Plan<N>;
  constexpr int LPB = lpb<N>();
  constexpr int E = P::E, T = P::T, NT = LPB * T, LS = P::LS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* tw_sm = reinterpret_cast<cx<float>*>(smem_raw);
  cx<float>* lines = tw_sm + 2 * P::TWN;
  tc16::Tabs* tabs = reinterpret_cast<tc16::Tabs*>(smem_raw);
  float* k2l_tc = reinterpret_cast<float*>(smem_raw + sizeof(tc16::Tabs));  // padded k^2 of the line axis
  float* k2pm_sm = k2l_tc + tc16::MT;                                     // per-line k^2 of the others
  if constexpr (TC) lines = reinterpret_cast<cx<float>*>(k2pm_sm + 16);

  const int tid = threadIdx.x;
  const int l = STRIDED ? (tid % LPB) : (tid / T);
  const int t = STRIDED ? (tid / LPB) : (tid % T);
  const tile::Tiles<LPB, STRIDED> tiles(a.outer, a.inner);
  const unsigned ustride = STRIDED ? (unsigned)a.inner : 1u;
  constexpr bool PF = E <= 16;  // register prefetch of the next tile
  constexpr bool CONTIG = !STRIDED;  // line l held by threads [l T, (l + 1) T)
  pdl_allow_next();
  if constexpr (TC) {
    tc16::load_tabs(tabs, a.tc, a.tw, tid, NT);
    if constexpr (OP == RHO_GREEN)
      for (int k = tid; k < N; k += NT) k2l_tc[tc16::pt(k)] = a.k2l[k];
  } else {
    for (int k = tid; k < 2 * P::TWN; k += NT) tw_sm[k] = ldc(a.tw + k);
  }
  pdl_wait_prev();  // the half spectrum comes from the previous pass

  cx<float> vn[E];
  long long tau = blockIdx.x;
  if (PF && tau < tiles.count) {
    long long line0, o, i;
    int nvalid;
    size_t base;
    tiles.at(tau, l, N, line0, nvalid, base, o, i);
    load_line<E, T>(vn, a.data + base, ustride, t, l < nvalid);
  }
  __syncthreads();

  for (; tau < tiles.count; tau += gridDim.x) {
    long long line0, o, i;
    int nvalid;
    size_t base;
    tiles.at(tau, l, N, line0, nvalid, base, o, i);
    const bool valid = l < nvalid;
    cx<float> v[E];
    if constexpr (PF) {
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = vn[m];
      const long long taun = tau + gridDim.x;
      if (taun < tiles.count) {
        long long line0n, on, in;
        int nvalidn;
        size_t basen;
        tiles.at(taun, l, N, line0n, nvalidn, basen, on, in);
        load_line<E, T>(vn, a.data + basen, ustride, t, l < nvalidn);
      }
    } else {
      load_line<E, T>(v, a.data + base, ustride, t, valid);
    }
    if constexpr (OP == RHO_INV) {
      tile::xform<N, +1, CONTIG, TC>(v, lines, tw_sm, tabs, l, t, LPB);
    } else if constexpr (OP == RHO_FWD) {
      tile::xform<N, -1, CONTIG, TC>(v, lines, tw_sm, tabs, l, t, LPB);
    } else {
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
      if constexpr (TC) {
        if (t == 0) k2pm_sm[l] = k2pm;  // read after the entry barriers of fmi
        tc16::fmi(v, lines, *tabs, l, t, [&](int L) {
          return tc16::GreenMult{k2l_tc, k2pm_sm[L], a.cN, a.cY, a.mu2, a.cL};
        });
      } else {
        tile::green<N, CONTIG>(v, lines + l * LS, tw_sm, a.k2l, k2pm, a.cN, a.cY, a.mu2, a.cL, t);
      }
    }
    store_line<E, T>(v, a.data + base, ustride, t, valid);
  }
}

// Persistent grid: as many CTAs as fit on the device at once (cps = 0), at
// most cps per SM (cps > 0), or one CTA per tile (cps = -1); never more CTAs
// than tiles.  The kernels walk their tiles with a stride of gridDim.x, so
// every choice computes the same values.
template <typename K>
unsigned persistent_ctas(K kern, int threads, size_t smem, long long ntiles, int cps) {
  if (cps < 0) return (unsigned)(ntiles < 0x7fffffffLL ? ntiles : 0x7fffffffLL);
  static int sms_of[kDeviceSlots] = {};
  const int slot = device_slot();
  int& sms = sms_of[slot];
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  if (cps > 0 && cps < per_sm) per_sm = cps;
  const long long cap = (long long)per_sm * sms;
  return (unsigned)(ntiles < cap ? ntiles : cap);
}

// Launch with programmatic stream serialisation (see pdl_allow_next).
template <typename K, typename A>
cudaError_t launch_pdl(K kern, unsigned grid, int threads, size_t smem, cudaStream_t s, const A& a) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int LPB, bool STRIDED>
long long host_tiles(long long outer, long long inner) {
  return STRIDED ? outer * ((inner + LPB - 1) / LPB) : (outer + LPB - 1) / LPB;
}

template <int N, bool STRIDED, int VARIANT, bool TC = false, bool FIELDS = false>
cudaError_t launch_psi_t(const PsiPassArgs& a, cudaStream_t s) {
  constexpr size_t smem = psi_smem_bytes<N, VARIANT, TC, FIELDS>();
  constexpr int threads = cta_threads<N>();
  auto kern = psi_pass_kernel<N, STRIDED, VARIANT, TC, FIELDS>;
  static bool attr_of[kDeviceSlots] = {};
  bool& attr = attr_of[device_slot()];
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const long long ntiles = host_tiles<lpb<N>(), STRIDED>(a.outer, a.inner);
  return launch_pdl(kern, persistent_ctas(kern, threads, smem, ntiles, a.ctas_per_sm), threads, smem,
                    s, a);
}

template <int N, bool STRIDED, int OP, bool TC = false>
cudaError_t launch_rho_t(const RhoPassArgs& a, cudaStream_t s) {
  constexpr size_t smem = rho_smem_bytes<N, TC>();
  constexpr int threads = cta_threads<N>();
  auto kern = rho_pass_kernel<N, STRIDED, OP, TC>;
  static bool attr_of[kDeviceSlots] = {};
  bool& attr = attr_of[device_slot()];
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const long long ntiles = host_tiles<lpb<N>(), STRIDED>(a.outer, a.inner);
  return launch_pdl(kern, persistent_ctas(kern, threads, smem, ntiles, a.ctas_per_sm), threads, smem,
                    s, a);
}

// tensor-core engine: 256-point lines when the caller passes the fragment table
cudaError_t psi_dispatch_tc(bool strided, int variant, const PsiPassArgs& a, cudaStream_t s) {
  if (strided) {
    switch (variant) {
      case PSI_PLAIN: return launch_psi_t<256, true, PSI_PLAIN, true>(a, s);
      case PSI_NPHASE: return launch_psi_t<256, true, PSI_NPHASE, true>(a, s);
      default: return launch_psi_t<256, true, PSI_DENSITY, true>(a, s);
    }
  }
  switch (variant) {
    case PSI_PLAIN: return launch_psi_t<256, false, PSI_PLAIN, true>(a, s);
    case PSI_NPHASE: return launch_psi_t<256, false, PSI_NPHASE, true>(a, s);
    default: return launch_psi_t<256, false, PSI_DENSITY, true>(a, s);
  }
}

cudaError_t rho_dispatch_tc(bool strided, int op, const RhoPassArgs& a, cudaStream_t s) {
  if (strided) {
    switch (op) {
      case RHO_FWD: return launch_rho_t<256, true, RHO_FWD, true>(a, s);
      case RHO_GREEN: return launch_rho_t<256, true, RHO_GREEN, true>(a, s);
      default: return launch_rho_t<256, true, RHO_INV, true>(a, s);
    }
  }
  switch (op) {
    case RHO_FWD: return launch_rho_t<256, false, RHO_FWD, true>(a, s);
    case RHO_GREEN: return launch_rho_t<256, false, RHO_GREEN, true>(a, s);
    default: return launch_rho_t<256, false, RHO_INV, true>(a, s);
  }
}

template <int N>
cudaError_t psi_dispatch(bool strided, int variant, const PsiPassArgs& a, cudaStream_t s) {
  if (a.nfields > 1 && variant != PSI_PLAIN) {
    if (strided)
      return variant == PSI_NPHASE ? launch_psi_t<N, true, PSI_NPHASE, false, true>(a, s)
                                   : launch_psi_t<N, true, PSI_DENSITY, false, true>(a, s);
    return variant == PSI_NPHASE ? launch_psi_t<N, false, PSI_NPHASE, false, true>(a, s)
                                 : launch_psi_t<N, false, PSI_DENSITY, false, true>(a, s);
  }
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
  if (a.tc != nullptr && N == tc16::N) {
    if (a.nfields > 1 && variant != PSI_PLAIN) return cudaErrorInvalidValue;  // one field per launch
    return psi_dispatch_tc(strided, variant, a, s);
  }
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
  if (a.tc != nullptr && N == tc16::N) return rho_dispatch_tc(strided, op, a, s);
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

// ---- tensor-core engine: fragment tables ------------------------------------
// F[j][p] = exp(s 2 pi i j q / 16) with q = p (F-as-A stages) or q = pi(p)
// (data-as-A stages), expanded to the real 32 x 32 block of a complex product
// with (re, im) interleaved along K, split into FP16 hi = fp16(F) and
// lo = fp16(F - hi), and laid out per lane in the m16n8k16 fragment order.
namespace {
int tc_perm(int p) { return 8 * (p >> 3) + 2 * (p & 3) + ((p >> 2) & 1); }
void tc_f(int dir, int j, int q, double& re, double& im) {
  const double a = (dir == 0 ? -2.0 : 2.0) * 3.14159265358979323846 * (double)((j * q) % 16) / 16.0;
  re = std::cos(a);
  im = std::sin(a);
}
unsigned short tc_half(double v, int term) {
  const __half h = __float2half_rn((float)v);
  if (term == 0) return __half_as_ushort(h);
  return __half_as_ushort(__float2half_rn((float)(v - (double)__half2float(h))));
}
unsigned tc_pack(double lo_k, double hi_k, int term) {
  return (unsigned)tc_half(lo_k, term) | ((unsigned)tc_half(hi_k, term) << 16);
}
}  // namespace

void tc16_fragment_table(std::vector<unsigned>& w) {
  w.assign(tc16::FRAG_WORDS, 0u);
  unsigned* fa = w.data();                        // [dir][term][q = mt*2+ks][lane][4]
  unsigned* fb = w.data() + tc16::FRAG_WORDS / 2; // [dir][term][nt][lane][4]
  for (int dir = 0; dir < 2; ++dir)
    for (int term = 0; term < 2; ++term)
      for (int lane = 0; lane < 32; ++lane) {
        const int gid = lane >> 2, tig = lane & 3;
        for (int mt = 0; mt < 2; ++mt)
          for (int ks = 0; ks < 2; ++ks) {
            unsigned* o = fa + ((((dir * 2 + term) * 4 + mt * 2 + ks) * 32 + lane) * 4);
            for (int reg = 0; reg < 4; ++reg) {
              const int j = gid + 8 * (reg & 1);
              const int p = 8 * ks + tig + 4 * (reg >> 1);
              double fr, fi;
              tc_f(dir, j, p, fr, fi);
              o[reg] = mt == 0 ? tc_pack(fr, -fi, term) : tc_pack(fi, fr, term);
            }
          }
        for (int nt = 0; nt < 4; ++nt) {
          unsigned* o = fb + ((((dir * 2 + term) * 4 + nt) * 32 + lane) * 4);
          const int col = 8 * nt + gid, j = col >> 1, part = col & 1;
          for (int ks = 0; ks < 2; ++ks)
            for (int e = 0; e < 2; ++e) {
              const int p = 8 * ks + tig + 4 * e;
              double fr, fi;
              tc_f(dir, j, tc_perm(p), fr, fi);
              o[2 * ks + e] = part == 0 ? tc_pack(fr, -fi, term) : tc_pack(fi, fr, term);
            }
        }
      }
}

}  // namespace sn

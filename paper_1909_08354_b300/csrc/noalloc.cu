// sn_step_2d_noalloc: the fused FP32 split step for 2D complex64 grids that
// allocates no device memory.
//
// Some callers cannot call cudaMalloc: code whose device memory is owned in
// full by another allocator (a framework's caching pool, a fixed arena handed
// out at start-up), or code running where an allocation's latency or its
// possible failure is not acceptable (a real-time loop, a plugin or callback
// that must not grow the process's footprint).  This entry point serves them:
// the caller passes psi in device memory, and every piece of working memory
// the step needs (the potential's half spectrum and the FP64-built tables) lives
// in one file-scope static __device__ array of fixed size.  Every GPU that
// loads the library holds that array until the process exits.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <string>

#include "fft_plan.h"
#include "sn.h"
#include "sn_internal.h"

using namespace sn;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxN = SN_NOALLOC_MAX_N;  // per axis

// Carving of the scratch array, in float2 units, each region 256-byte aligned.
constexpr size_t align32(size_t words) { return (words + 31) / 32 * 32; }
constexpr size_t kRhoWords = align32((size_t)(kMaxN / 2 + 1) * kMaxN);  // half spectrum
constexpr size_t kTwWords = align32(4 * (size_t)kMaxN);    // twiddles (hi, lo) of one axis
constexpr size_t kMultWords = align32(2 * (size_t)kMaxN);  // one kinetic table (a float4 of shears per k)
constexpr size_t kK2Words = align32((size_t)kMaxN / 2 + 1);  // k^2 floats of one axis
constexpr size_t kOffTw = kRhoWords;
constexpr size_t kOffMult = kOffTw + 2 * kTwWords;
constexpr size_t kOffK2 = kOffMult + 4 * kMultWords;
constexpr size_t kOffZero = kOffK2 + 2 * kK2Words;
constexpr size_t kScratchWords = kOffZero + 32;

static __device__ __align__(256) float2 sn_noalloc_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
// device address of the array, per device; atomic because two host threads may
// make the first call on one device at the same time (both store the same value)
std::atomic<float2*> g_scratch_ptr[kMaxDevices] = {};

sn_status fail(sn_status st, const char* m) {
  set_thread_error(m);
  return st;
}

sn_status cuda_fail(cudaError_t e, const char* what) {
  char m[256];
  std::snprintf(m, sizeof(m), "sn_step_2d_noalloc: %s: %s", what, cudaGetErrorString(e));
  return fail(SN_ECUDA, m);
}

double wavenumber(int j, int n, double L) { return 2.0 * kPi / L * (double)(j < n / 2 ? j : j - n); }

// hi = fl(x), lo = fl(x - hi) for n complex values: hi parts to out[0, n), lo parts to out[n, 2n)
void split_hilo(const double2* v, int n, float2* out) {
  for (int i = 0; i < n; ++i) {
    const float hr = (float)v[i].x, hi = (float)v[i].y;
    out[i] = make_float2(hr, hi);
    out[n + i] = make_float2((float)(v[i].x - (double)hr), (float)(v[i].y - (double)hi));
  }
}

// Once per device, with that device current: the device address of the array.
sn_status scratch_for_current_device(float2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(SN_ENOTSUP, "sn_step_2d_noalloc: device index too large");
  float2* ptr = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!ptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, sn_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    ptr = reinterpret_cast<float2*>(p);
    g_scratch_ptr[dev].store(ptr, std::memory_order_release);
  }
  *out = ptr;
  return SN_OK;
}

}  // namespace

extern "C" sn_status sn_step_2d_noalloc(float* psi, int ny, int nx, double Ly, double Lx,
                                        const sn_kernel* k, double dt, int nsteps,
                                        void* cuda_stream) {
  if (!psi) return fail(SN_EINVAL, "sn_step_2d_noalloc: psi is NULL");
  if (!k) return fail(SN_EINVAL, "sn_step_2d_noalloc: kernel is NULL");
  const int n[2] = {ny, nx};
  const double L[2] = {Ly, Lx};
  for (int a = 0; a < 2; ++a) {
    if (n[a] < 8 || (n[a] & (n[a] - 1)) != 0)
      return fail(SN_EINVAL, "sn_step_2d_noalloc: ny and nx must be powers of two >= 8");
    if (n[a] > kMaxN)
      return fail(SN_ENOTSUP,
                  "sn_step_2d_noalloc: ny and nx must be <= SN_NOALLOC_MAX_N (the static scratch "
                  "array holds the half spectrum of a 512 x 512 grid)");
    if (!(L[a] > 0.0) || !std::isfinite(L[a]))
      return fail(SN_EINVAL, "sn_step_2d_noalloc: Ly and Lx must be finite and > 0");
  }
  if (!std::isfinite(dt)) return fail(SN_EINVAL, "sn_step_2d_noalloc: dt must be finite");
  if (nsteps < 0) return fail(SN_EINVAL, "sn_step_2d_noalloc: nsteps must be >= 0");
  if (const char* why = kernel_invalid(*k))
    return fail(SN_EINVAL, (std::string("sn_step_2d_noalloc: ") + why).c_str());
  if (k->v_ext) return fail(SN_ENOTSUP, "sn_step_2d_noalloc: v_ext is not supported");
  if (nsteps == 0) return SN_OK;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  // The tables below are copied from host (stack) memory, which a captured
  // graph would read again, long after this call returned: refused while the
  // stream is being captured.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t ce = cudaStreamIsCapturing(stream, &cap);
  if (ce != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    if (ce != cudaSuccess) (void)cudaGetLastError();
    return fail(SN_ENOTSUP,
                "sn_step_2d_noalloc: the stream is being captured; the call uploads its tables "
                "from host memory and cannot run inside a stream capture");
  }

  float2* s = nullptr;
  sn_status st = scratch_for_current_device(&s);
  if (st != SN_OK) return st;
  float2* rhohat = s;
  float2* tw[2] = {s + kOffTw, s + kOffTw + kTwWords};
  float2* mult[2][2] = {{s + kOffMult, s + kOffMult + kMultWords},
                        {s + kOffMult + 2 * kMultWords, s + kOffMult + 3 * kMultWords}};
  float* k2[2] = {reinterpret_cast<float*>(s + kOffK2),
                  reinterpret_cast<float*>(s + kOffK2 + kK2Words)};
  float* zero = reinterpret_cast<float*>(s + kOffZero);

  // Tables for this call (the array keeps whatever an earlier call left).  They
  // are built on the stack, one buffer per upload (about 76 KB in all); a copy
  // from pageable host memory is staged before cudaMemcpyAsync returns, so the
  // buffers may go out of scope when the call returns.
  cudaError_t e = cudaSuccess;
  double2 t64[2 * kMaxN];
  float2 tw32[2][4 * kMaxN];
  float lift32[2][2][4 * kMaxN];
  float kf[2][kMaxN];
  for (int a = 0; a < 2 && e == cudaSuccess; ++a) {
    const int ntw = snfft::plan_twiddles(n[a], t64);  // at most 2 n[a] entries
    if (ntw > 0) {
      split_hilo(t64, ntw, tw32[a]);
      e = cudaMemcpyAsync(tw[a], tw32[a], 2 * ntw * sizeof(float2), cudaMemcpyHostToDevice,
                          stream);
    }
    for (int f = 0; f < 2 && e == cudaSuccess; ++f) {
      sn::kinetic_lift_table(n[a], L[a], k->coeff_lap, f ? dt : 0.5 * dt, lift32[a][f]);
      e = cudaMemcpyAsync(mult[a][f], lift32[a][f], 4 * n[a] * sizeof(float),
                          cudaMemcpyHostToDevice, stream);
    }
    if (e == cudaSuccess) {
      for (int j = 0; j < n[a]; ++j) {
        const double kk = wavenumber(j, n[a], L[a]);
        kf[a][j] = (float)(kk * kk);
      }
      e = cudaMemcpyAsync(k2[a], kf[a], n[a] * sizeof(float), cudaMemcpyHostToDevice, stream);
    }
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(zero, 0, sizeof(float), stream);
  if (e != cudaSuccess) return cuda_fail(e, "table upload");

  const long long cells = (long long)ny * nx;
  const GreenCoeffs gc = green_coeffs(*k);
  const double mu2 = gc.mu2, cN = gc.cN * dt / (double)cells, cY = gc.cY * dt / (double)cells;
  float2* p = reinterpret_cast<float2*>(psi);
  // Merged Strang steps: round r applies the kinetic factor along both axes
  // (half step in the first and last round), with the nonlinear phase in the
  // first pass of every round after the first and the density in the last
  // pass of every round before the last; the axis order flips every round.
  for (int r = 0; r <= nsteps; ++r) {
    const bool odd = (r & 1) != 0;
    const int full = (r == 0 || r == nsteps) ? 0 : 1;
    const int order[2] = {odd ? 1 : 0, odd ? 0 : 1};
    for (int i = 0; i < 2; ++i) {
      const int a = order[i];
      int variant = PSI_PLAIN;
      if (i == 0 && r > 0) variant = PSI_NPHASE;
      if (i == 1 && r < nsteps) variant = PSI_DENSITY;
      PsiPassArgs pa{};
      pa.psi = p;
      pa.outer = a == 0 ? 1 : ny;
      pa.inner = a == 0 ? nx : 1;
      pa.lift = reinterpret_cast<const float4*>(mult[a][full]);
      pa.tw = tw[a];
      pa.rh_in = rhohat;
      pa.vext = nullptr;
      pa.h = (float)dt;
      pa.gh = (float)(k->g_local * dt);
      pa.rh_out = rhohat;
      e = launch_psi_pass_f32(n[a], a == 0, variant, pa, stream);
      if (e != cudaSuccess) return cuda_fail(e, "psi pass launch");
    }
    if (r < nsteps) {
      const int h = order[1], c = order[0];
      RhoPassArgs ra{};
      ra.data = rhohat;
      ra.outer = n[h] / 2 + 1;
      ra.inner = 1;
      ra.tw = tw[c];
      ra.k2p = k2[h];
      ra.k2m = zero;
      ra.k2l = k2[c];
      ra.mid_n = 1;
      ra.cN = (float)cN;
      ra.cY = (float)cY;
      ra.mu2 = (float)mu2;
      e = launch_rho_pass_f32(n[c], false, RHO_GREEN, ra, stream);
      if (e != cudaSuccess) return cuda_fail(e, "green pass launch");
    }
  }
  return SN_OK;
}

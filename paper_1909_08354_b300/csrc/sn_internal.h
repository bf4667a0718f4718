// Host-side internals of libsn: pass argument blocks, launchers, grid state.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sn.h"

namespace sn {

constexpr int kLinesPerCta = 16;  // lines per CTA in the fused FP32 passes

// Kinds of kernel launch, for per-kind timing and launch counts.
enum PassKind {
  K_PSI = 0,        // psi pass: FFT . m . IFFT along one axis
  K_PSI_NPHASE,     // psi pass with the C2R potential + nonlinear phase prologue
  K_PSI_DENSITY,    // psi pass with the |psi|^2 R2C epilogue
  K_RHO_FWD,        // half-spectrum forward FFT along one axis
  K_RHO_GREEN,      // half-spectrum FFT . K(k) . IFFT along one axis
  K_RHO_INV,        // half-spectrum inverse FFT along one axis
  K_F64_FFT,        // plain FP64 step: one axis FFT
  K_F64_EW,         // plain FP64 step: one elementwise kernel
  K_OBS,            // observables kernels
  K_RESIDENT,       // plane-resident 2D steps (all rounds of a call in one launch)
  K_NUM_KINDS
};

struct PsiPassArgs {
  float2* psi;
  long long outer, inner;  // lines = outer * inner; element stride inner (strided) or 1
  const float2* mult;      // 2N entries: hi then lo parts of exp(i A k^2 tau) / N (TC engine)
  const float4* lift;      // N entries: the same factor as three shears (FP32 engine)
  const float2* tw;        // twiddle table of this N (hi parts, then lo parts)
  const float2* rh_in;     // NPHASE: half spectrum [N/2+1][lines]
  const float* vext;       // NPHASE: optional V_ext in psi layout (NULL for none)
  float h;                 // NPHASE: step h (multiplies V_ext)
  float gh;                // NPHASE: g * h
  float2* rh_out;          // DENSITY: half spectrum [N/2+1][lines]
  int rh_accum;            // DENSITY: add to rh_out (the density of a further field)
  int nfields;             // NPHASE, DENSITY (FP32 engine): fields in this launch (0, 1: one)
  long long fstride;       // elements from one field to the next
  int ctas_per_sm;         // schedule: 0 = as many as fit, k > 0 = at most k, -1 = one per tile
  const uint4* tc;         // tensor-core fragment table (256-point lines), or NULL
  long long rh_lines;      // TMA edge passes: lines of a half-spectrum row (its stride;
                           // 0 = outer * inner), more when the launch covers a slab of them
};

struct RhoPassArgs {
  float2* data;
  long long outer, inner;
  const float2* tw;
  const float* k2p;  // GREEN: k^2 of the half axis, indexed by plane
  const float* k2m;  // GREEN: k^2 of the middle axis (or a single 0)
  const float* k2l;  // GREEN: k^2 of the line axis
  long long mid_n;   // GREEN, contiguous lines: outer = plane * mid_n + mid
  float cN, cY, mu2; // GREEN: K = cN/k2 + cY/(k2 + mu2), zero at k2 = 0
  float cL;          // GREEN: constant added to K at every k (a local term)
  int ctas_per_sm;   // schedule, as in PsiPassArgs
  const uint4* tc;   // tensor-core fragment table (256-point lines), or NULL
};

// Message returned by sn_last_error(NULL) on this thread.
void set_thread_error(const char* msg);

// The kernel of sn_kernel as K(k) = cN / k^2 + cY / (k^2 + mu2) for k != 0
// (K(0) = 0), before any step or normalisation factor:
//   NMC:     cN = -4 pi G, cY = -4 pi G alpha_Y, mu2 = 1/lambda_Y^2 (1 if alpha_Y = 0);
//   POISSON: B D / (C - k^2) = cY / (k^2 + mu2) with cY = -B D, mu2 = -C (C < 0),
//            or cN = -B D (C = 0).
struct GreenCoeffs {
  double cN, cY, mu2;
};
GreenCoeffs green_coeffs(const sn_kernel& k);
// NULL if k is a valid kernel, else the reason (for an SN_EINVAL message).
const char* kernel_invalid(const sn_kernel& k);

// Per-device once-only settings (kernel attributes, SM counts) are kept in
// arrays indexed by the current device, clamped to [0, kDeviceSlots).
constexpr int kDeviceSlots = 64;
int device_slot();

enum PsiVariant { PSI_PLAIN = 0, PSI_NPHASE = 1, PSI_DENSITY = 2 };
enum RhoOp { RHO_FWD = 0, RHO_GREEN = 1, RHO_INV = 2 };

cudaError_t launch_psi_pass_f32(int N, bool strided, int variant, const PsiPassArgs& a,
                                cudaStream_t s);

// ---- TMA-staged line passes (passes_tma.cu) ------------------------------------
// The plain kinetic pass and the three half-spectrum passes with their tiles
// moved by the tensor-memory accelerator; same arithmetic as the
// register-staged kernels above, bit for bit.
enum LineOp { LINE_KINETIC = 0, LINE_FWD = 1, LINE_GREEN = 2, LINE_INV = 3 };
struct LinePassArgs {
  void* data;              // complex64 lines, in place
  long long outer, inner;  // as in PsiPassArgs
  const float2* tw;        // twiddles of N
  const float4* lift;      // LINE_KINETIC: kinetic shears
  const float* k2p;        // LINE_GREEN: as in RhoPassArgs
  const float* k2m;
  const float* k2l;
  long long mid_n;
  float cN, cY, mu2, cL;
  int* status;             // device word set to 1 if a bounded tile wait expired
  int ctas_per_sm;         // schedule, as in PsiPassArgs
};
// Whether the TMA passes take lines of length N in this geometry (N = 128 or
// 256, a driver that exports the tensor-map encoder).
bool line_pass_tma_supported(int N, bool strided, long long outer, long long inner);
// cudaErrorNotSupported if !line_pass_tma_supported.
cudaError_t launch_line_pass_tma(int N, bool strided, int op, const LinePassArgs& a,
                                 cudaStream_t s);
// ---- plane-resident 2D steps (resident_2d.cu) -----------------------------------
// Rounds of merged split steps of an N x N complex64 grid held in one CTA's
// shared memory; the same arithmetic as the tiled passes, bit for bit.
struct Resident2dArgs {
  float2* psi;             // N x N state, read at the start and written at the end
  float2* rh;              // half spectrum [N/2 + 1][N], likewise (the open merge's potential)
  const float2* tw;        // twiddles of N (hi parts, then lo parts)
  const float4* lift[4];   // kinetic shears [2 axis + full] (half step, full step)
  const float* k2[2];      // k^2 per axis
  float cN, cY, mu2;       // Green's multiplier (h / N folded in), as RhoPassArgs
  float gh;                // g h
  int rounds;              // rounds of this launch
  int nphase, full, odd;   // the first round: nonlinear phase, full kinetic step, axis order
};
bool resident_2d_supported(int ny, int nx);

// ---- the tcgen05 line engine (umma_line.cu), a measurement form ---------------
// In-place 256-point DFTs (sign as in sn_test_line_fft_f32) of nlines
// contiguous complex64 lines, both radix-16 stages on tcgen05.mma; tw and bmat
// from umma_line_tables (device copies); status set to 1 on an expired wait.
// cycles (NULL: untimed): 6 device counters that receive the clock cycles of
// each phase of a tile summed over tiles (stage A operands, stage A products,
// stage B operands, stage B products, output), then the tiles done.
void umma_line_tables(int sign, std::vector<uint16_t>& bmat, std::vector<float2>& tw);
cudaError_t launch_umma_line(float2* data, long long nlines, const float2* tw, const void* bmat,
                             int* status, unsigned long long* cycles, cudaStream_t s);

// ---- the fused FNO layer (fno_layer_umma.cu) --------------------------------------
// Forward (back = 0): z = WxI^T B1 + W v + bias and vout = act ? GELU(z) : z
// for every (b, o, y, x) of a spectral layer (layouts as in fno.cu).  Backward
// (back = 1, v the gradient dz): vout = (WxI^T B1 + W^T dz) GELU'(zp), or
// without the factor when zp is NULL; z and bias unused.  tcgen05.mma with
// BF16 operands.
bool fno_layer_umma_supported(int C, int Q, int s);
cudaError_t launch_fno_layer_umma(const float* v, const float* B1, const float* WxI, const float* W,
                                  const float* bias, float* z, float* vout, const float* zp, int B,
                                  int C, int s, int Q, int act, int back, int* status, cudaStream_t st);

// ---- distributed shared memory rates (dsmem_rate.cu) ---------------------------
// Aggregate GB/s over the GPU for clusters of csize CTAs: remote float4 reads
// of a peer's shared memory, the same reads of a CTA's own, and bulk copies
// pushed into a peer's shared memory.  cudaErrorLaunchTimeout if a bounded
// copy wait expired.
cudaError_t measure_dsmem(int csize, double* read_remote, double* read_local, double* push);

// ---- a batch instance stepped as a grid (the scan's graph schedule) -----------
// g is a 2D complex64 grid of one field on the FP32 engine without V_ext.
// prepare: its kernel and the kinetic tables of dt, before any capture
// (blocks while old tables may still be read).  round: round r of an n-step
// call on its stream, the Strang merge closed at both ends (r = 0: Kin(h/2)
// and the density; 0 < r < n: Nl(h), Kin(h), density; r = n: Nl(h), Kin(h/2));
// *launches receives the kernels it launched.  status: its pass status word
// (SN_ETIMEOUT after an expired tile wait).
sn_status batch_grid_prepare(sn_grid g, const sn_kernel& k, double dt);
sn_status batch_grid_round(sn_grid g, int r, int nsteps, double dt, long long* launches);
sn_status batch_grid_status(sn_grid g);
void* batch_grid_psi(sn_grid g);
cudaError_t launch_resident_2d(int n, const Resident2dArgs& a, cudaStream_t s);

// The potential pass (PSI_NPHASE) and the density pass (PSI_DENSITY) of one
// field on the FP32 engine, TMA-staged; cudaErrorNotSupported for geometries
// or options it does not take (several fields, an accumulated density, the
// tensor-core engine).  status as in LinePassArgs.
cudaError_t launch_edge_pass_tma(int N, bool strided, int variant, const PsiPassArgs& a,
                                 int* status, cudaStream_t s);
cudaError_t launch_rho_pass_f32(int N, bool strided, int op, const RhoPassArgs& a,
                                cudaStream_t s);
// Kinetic factor exp(i A k_j^2 tau) / n of the FP32 passes, j < n, as a rotation
// by three shears: out[4j .. 4j+3] = (tan(phi/2), sin(phi), +-1/n, 0), phi the
// angle reduced to [-pi/2, pi/2] (the sign of the scale carries the rest).
void kinetic_lift_table(int n, double L, double A, double tau, float* out4);
// FP16 fragment tables of the tensor-core engine (tc16.cuh), tc16::FRAG_WORDS words
void tc16_fragment_table(std::vector<unsigned>& words);

// ---- plain FP64 path -------------------------------------------------------
cudaError_t launch_fft_f64(int N, bool strided, int sign, double2* data, long long outer,
                           long long inner, const double2* tw, cudaStream_t s);
cudaError_t launch_mult_kinetic_f64(double2* psi, const int* n, int ndim, const double2* const* m,
                                    cudaStream_t s);
// w = |psi|^2, or w += |psi|^2 with accumulate
cudaError_t launch_density_f64(const double2* psi, double2* w, long long cells, cudaStream_t s,
                               bool accumulate = false);
// w *= K(k) + cL, K as in GreenCoeffs (zero at k = 0)
cudaError_t launch_green_f64(double2* w, const int* n, int ndim, const double* const* k2,
                             double cN, double cY, double mu2, cudaStream_t s, double cL = 0.0);
cudaError_t launch_phase_f64(double2* psi, const double2* w, const double* vext, double h,
                             double gh, long long cells, cudaStream_t s);
cudaError_t launch_widen_f32_to_f64(const float2* in, double2* out, long long cells,
                                    cudaStream_t s);
// out = (sqrt(sum_j |psi_j|^2), 0) over count fields psi_j = psi + j cells
// (complex64 if f32, else complex128): a state whose density is the total one
cudaError_t launch_total_amplitude(const void* psi, bool f32, int count, long long cells,
                                   double2* out, cudaStream_t s);

// ---- self-gravitating fluid, Eq. 16 (FP64, fluid_f64.cu) -------------------
struct FluidPhase {
  double nu, h_over_nu;  // psi <- psi exp(-i U h / nu)
  double w, n_poly, cp;  // V_p = w ln rho (n = 1) or cp rho^(n-1), cp = n w / (n - 1)
  double rho_floor;      // floor of rho under sqrt and ln
  int floor_mode;        // SN_FLOOR_MAX: max(rho, floor); SN_FLOOR_SMOOTH: rho + floor
};
cudaError_t launch_fluid_prep_f64(const double2* psi, double2* wa, double floor, int floor_mode,
                                  long long cells, cudaStream_t s);
cudaError_t launch_lap_mult_f64(double2* w, const int* n, int ndim, const double* const* k2,
                                double scale, cudaStream_t s);
cudaError_t launch_fluid_source_f64(const double2* psi, const double2* wlap, double2* w,
                                    const double* gamma, const double* beta, long long cells,
                                    cudaStream_t s);
// wphi: phi_N (real part); wlap: lap sqrt rho (imaginary part)
cudaError_t launch_fluid_phase_f64(double2* psi, const double2* wphi, const double2* wlap,
                                   const double* phi_c, const FluidPhase& p, long long cells,
                                   cudaStream_t s);

// ---- observables (FP64) ----------------------------------------------------
enum ObsQ {
  Q_MASS = 0, Q_RHO2, Q_VEXT, Q_CX0, Q_SX0, Q_CX1, Q_SX1, Q_CX2, Q_SX2,
  Q_EKIN0, Q_P0, Q_EKIN1, Q_P1, Q_EKIN2, Q_P2, Q_EPOT, Q_NUM
};
constexpr int kObsBlocks = 592;  // 4 x 148 SMs
// The observables kernels add their per-block sums to partials (zeroed first),
// so that several fields accumulate into one set.
// cs[a][j] = (cos, sin)(2 pi x_j / L_a) for the ndim axes; cs_one = {(1, 0)}
cudaError_t launch_obs_space(const double2* psi, const double* vext, const int* n, int ndim,
                             const double2* const* cs, const double2* cs_one, double* partials,
                             cudaStream_t s);
cudaError_t launch_obs_kaxis(const double2* fa, const int* n, int ndim, int axis,
                             const double* kax, double* partials, cudaStream_t s);
cudaError_t launch_obs_green(const double2* rhohat, const int* n, int ndim,
                             const double* const* k2, double cN, double cY, double mu2,
                             double* partials, cudaStream_t s);
cudaError_t launch_obs_finish(const double* partials, int nq, double* out, cudaStream_t s);
// FP32-transform observables of complex64 states (obs_f32.cu), into the same
// partial slots: spectral sums along `axis` (lines (outer, inner) of N
// points, L the axis length) into Q_EKIN0 + 2 axis and Q_P0 + 2 axis; the
// density pass along the last axis (contiguous lines of N points; n0, n1 the
// padded 3D sizes of the axes before it) into Q_MASS .. Q_SX2, writing the
// half spectrum of rho [N/2 + 1][cells / N] to rh; the Green's sum over the
// half spectrum's lines of N points (geometry and k^2 tables as the step's
// Green's pass, nh the half axis' length) into Q_EPOT.
cudaError_t launch_obs32_spec(int N, const float2* psi, long long outer, long long inner,
                              const float2* tw, double L, int axis, double* partials,
                              cudaStream_t s);
cudaError_t launch_obs32_density(int N, const float2* psi, int nfields, long long cells,
                                 const float* vext, float2* rh, int n0, int n1, const float2* tw,
                                 double* partials, cudaStream_t s);
cudaError_t launch_obs32_green(int N, const float2* rh, long long outer, long long inner,
                               long long mid_n, const float* k2p, const float* k2m,
                               const float* k2l, int nh, double cN, double cY, double mu2,
                               const float2* tw, double* partials, cudaStream_t s);
// Fluid energy sums (Eq. 16) into partials [kObsBlocks][Q_NUM] at q = 0..3 (zeroed
// first): rho phi_N (Re wphi), rho phi_C (phi_c may be NULL), eps(rho), a lap(a)
// (Im wlap = lap a, a = sqrt(max(rho, floor)))
cudaError_t launch_obs_fluid(const double2* psi, const double2* wphi, const double2* wlap,
                             const double* phi_c, double w, double n_poly, double floor,
                             int floor_mode, long long cells, double* partials, cudaStream_t s);

// ---- BF16 tensor-core GEMM (FNO surrogate) -------------------------------
// C[z] = alpha * A[z] B[z] + beta * C[z]; element (m,k) of A[z] at
// A + z sAz + m sAm + k sAk, (k,n) of B at B + z sBz + k sBk + n sBn, (m,n) of C
// at C + z sCz + m sCm + n sCn.  kchunk > 0 splits K: partial sums of chunk sp
// go to C + z sCz + sp sCsp (beta must be 0).
struct GemmArgs {
  const float* A;
  long long sAz, sAm, sAk;
  const float* B;
  long long sBz, sBk, sBn;
  float* C;
  long long sCz, sCm, sCn, sCsp;
  int M, N, K, Z, kchunk;
  float alpha, beta;
  // optional epilogue (no split-K; rows of C contiguous and 16-byte aligned):
  // C = alpha A B + beta C + bias[m], and C2 (the strides of C) = GELU of
  // that (act) or a copy; NULL bias and C2 for none
  const float* bias;
  float* C2;
  int act;
};
cudaError_t gemm_bf16(const GemmArgs& g, cudaStream_t s);
// out[i] = sum_{j<count} part[j*stride + i] (+ beta * out[i]) for i < n
cudaError_t reduce_sum(const float* part, long long count, long long stride, long long n, float* out,
                       float beta, cudaStream_t s);

}  // namespace sn

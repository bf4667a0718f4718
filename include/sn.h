/*
 * libsn -- B300 (sm_103a) split-step solver of the generalized
 * Schroedinger-Newton system.
 *
 * The system (Sec. II, Eqs. 1-2) is
 *     i dpsi/dt = A lap(psi) + B phi psi + G(|psi|^2) psi,
 *     lap(phi) + C phi = D |psi|^2,
 * and the local nonlinearity G(|psi|^2) = g |psi|^2.  The potential is solved
 * spectrally (Sec. III): B phi_k = K(k) rho_k with K(0) = 0 (the mean density
 * is removed) and one of two kernels (sn_kernel.kind):
 *   SN_KERNEL_NMC: the Newton + Yukawa multiplier that the modified Poisson
 *     equation of the non-minimal matter-curvature coupling gives for constant
 *     coefficients (Eq. 9; Eq. 14 is its alpha -> 0 limit), B = 1:
 *       K(k) = -4 pi G [1/k^2 + alpha_Y / (k^2 + 1/lambda_Y^2)];
 *   SN_KERNEL_POISSON: Eq. 2 itself with constants B, C <= 0, D, the form of
 *     the optical media of Sec. II A -- thermo-optical (Eq. 4: phi = dn,
 *     C = -1/sigma^2, D = -zeta mu / kappa) and nematic liquid crystals
 *     (Eq. 5: phi = theta, C = -2q/nu, D = -2/nu):
 *       K(k) = B D / (C - k^2).
 * Time stepping is the symmetric split-step Fourier method (Sec. III):
 *     S(h) = Kin(h/2) Nl(h) Kin(h/2),
 *     Kin(tau) = F^-1 exp(i A k^2 tau) F,
 *     Nl(h) psi = exp(-i (phi + V_ext + g |psi|^2) h) psi.
 *
 * Conventions for every call:
 *   - ndim is 2 or 3; arrays are C-ordered with the slowest axis first
 *     ((ny, nx) or (nz, ny, nx)); n[] and L[] are given in that order.
 *   - each n[a] is a power of two in [8, 1024]; L[a] > 0 is the box length.
 *   - psi is interleaved (re, im): complex64 (two floats) for SN_C64 grids,
 *     complex128 (two doubles) for SN_C128 grids.  Node-centred coordinates
 *     x_j = -L/2 + j L / n.
 *   - the library owns all device memory of a grid; callers own every host
 *     buffer and every device buffer they pass in.  set/get calls copy.
 *   - every call returns an sn_status; no exception crosses the boundary.
 *     Work is queued on the grid's CUDA stream; a failure inside a kernel
 *     surfaces at the next call that synchronises (sn_get_state,
 *     sn_observables, or sn_sync).
 *   - a grid may be used by one host thread at a time.
 */
#ifndef SN_H_
#define SN_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sn_grid_s* sn_grid; /* opaque handle */

typedef enum {
  SN_OK = 0,
  SN_EINVAL = -1,      /* invalid argument; nothing was queued */
  SN_ENOMEM = -2,      /* device allocation failed */
  SN_ECUDA = -3,       /* a CUDA call or kernel failed; see sn_last_error */
  SN_ETIMEOUT = -4,    /* a bounded device wait expired */
  SN_ENONFINITE = -5,  /* the state holds NaN or Inf */
  SN_ENOTSUP = -6      /* valid request this build does not support */
} sn_status;

typedef enum {
  SN_C64 = 0,  /* complex64 state; fused FP32 passes */
  SN_C128 = 1  /* complex128 state; plain FP64 step */
} sn_dtype;

/* Kernel of the potential (see the top of this file). */
typedef enum {
  SN_KERNEL_NMC = 0,     /* Newton + Yukawa of Eq. 9 / Eq. 14: G, alpha_Y, lambda_Y */
  SN_KERNEL_POISSON = 1  /* Eq. 2 with constants B, C, D (Eqs. 4 and 5)             */
} sn_kernel_kind;

/* Parameters of Eqs. 1-2 as used by the step (Sec. II; Eq. 9 / Eq. 14).
 * Zero-initialise it and set what is needed: kind 0 is SN_KERNEL_NMC. */
typedef struct {
  double coeff_lap;  /* A of Eq. 1; -0.5 for i psi_t = -(1/2) lap psi + ...   */
  double G;          /* NMC: K(k) = -4 pi G (1/k^2 + alpha_Y / (k^2 + 1/lambda_Y^2)) */
  double alpha_Y;    /* NMC: Yukawa strength; 0 gives the pure Newton kernel    */
  double lambda_Y;   /* NMC: Yukawa range (> 0 when alpha_Y != 0)               */
  double g_local;    /* local term g |psi|^2                                     */
  int zero_k0;       /* must be 1: the whole multiplier is zero at k = 0         */
  const double* v_ext; /* optional real external potential (C order, ncells
                          doubles), NULL for none; copied by sn_set_kernel       */
  int v_ext_on_device; /* 1 if v_ext is a device pointer, 0 if host             */
  int kind;          /* sn_kernel_kind                                           */
  double B, C, D;    /* POISSON: B of Eq. 1 and C (<= 0), D of Eq. 2;
                        K(k) = B D / (C - k^2); ignored for NMC                  */
} sn_kernel;

/* Observables at the current integer step (FP64, computed on the device).
 *   mass = dV sum |psi|^2
 *   e_kin = -A (dV/N) sum_k k^2 |F psi|^2
 *   e_pot = (1/2) dV sum phi rho + dV sum V_ext rho
 *   e_nl = (g/2) dV sum rho^2,  e_total = e_kin + e_pot + e_nl
 *   centroid[a] = (L_a / 2 pi) arg(sum rho exp(2 pi i x_a / L_a))
 *   momentum[a] = (dV/N) sum_k k_a |F psi|^2 (Nyquist k_a counted as 0)
 * Axis entries are in array order; entries beyond ndim are 0. */
typedef struct {
  double mass, e_kin, e_pot, e_nl, e_total;
  double centroid[3], momentum[3];
  long long step;
} sn_obs;

/* Create a grid (Sec. II: psi on a periodic box of ndim dimensions).
 * out: receives the handle.  n, L: ndim entries each, slowest axis first.
 * dtype: SN_C64 or SN_C128.  cuda_stream: a cudaStream_t the caller keeps
 * alive for the grid's lifetime, or NULL for a library-created stream.
 * psi starts at zero and the kernel at {A=-0.5, G=1, alpha_Y=0, g=0}.
 * Errors: SN_EINVAL for bad arguments, SN_ENOMEM, SN_ECUDA. */
sn_status sn_create_grid(sn_grid* out, int ndim, const int* n, const double* L, int dtype,
                         void* cuda_stream);

/* Set the parameters of Eqs. 1-2 (see sn_kernel).  Copies v_ext.  Errors:
 * SN_EINVAL for non-finite values, an unknown kind, lambda_Y <= 0 with
 * alpha_Y != 0 (NMC), C > 0 (POISSON), or zero_k0 != 1. */
sn_status sn_set_kernel(sn_grid g, const sn_kernel* k);

/* Self-gravitating fluid of Sec. II B: the Madelung form of the continuity
 * and Euler equations of a polytropic fluid (P = w rho^n) with gravity from
 * General Relativity's Newtonian limit or from the pure non-minimal
 * matter-curvature coupling (alpha = 0), Eq. 16:
 *     i nu psi_t = -(nu^2/2) lap psi + [nu^2 V_B + phi_N + phi_C + V_p] psi,
 *   V_B = lap(sqrt rho) / (2 sqrt rho)                       (Bohm potential),
 *   lap phi_N = beta(r) lap rho + gamma(r) rho, k = 0 removed      (Eq. 15),
 *   phi_C = ln[1 - (r0/(r + r0))^lambda]                           (Eq. 13),
 *   V_p = w ln rho (n = 1) or n w/(n - 1) rho^(n - 1)              (Eq. 17),
 *   GR:  gamma = 1/2, beta = 0, phi_C = 0;
 *   NMC: gamma = (1 - q)/2, beta = lambda q/(r + r0), q = (r0/(r + r0))^lambda
 *        (Eqs. 11-12), r0 = M / (4 pi),
 * rho = |psi|^2, r the distance from the box centre (the node x = 0), taken
 * as at least half the smallest grid spacing (phi_C is -infinite at r = 0);
 * sqrt rho and ln rho use max(rho, rho_floor), or with floor_mode =
 * SN_FLOOR_SMOOTH rho + rho_floor: the kink of sqrt(max(rho, floor)) where
 * the density crosses the floor makes the Bohm term spike there, by an
 * amount that grows as the grid refines, and the spike radiates
 * high-wavenumber waves (group speed ~ nu k) across the box. */
typedef enum { SN_GRAVITY_GR = 0, SN_GRAVITY_NMC = 1 } sn_gravity;
typedef struct {
  double nu;        /* > 0: the analogue of hbar, psi = sqrt(rho) exp(i Phi / nu) */
  double w;         /* polytropic coefficient                                    */
  double n_poly;    /* polytropic exponent (any finite value)                    */
  int model;        /* sn_gravity                                                */
  double lambda;    /* NMC: coupling strength (> 0)                              */
  double M;         /* NMC: mass setting r0 = M / (4 pi) (> 0)                   */
  double rho_floor; /* > 0                                                       */
  int floor_mode;   /* SN_FLOOR_MAX: sqrt rho and ln rho of max(rho, rho_floor);
                       SN_FLOOR_SMOOTH: of rho + rho_floor (no kink where rho
                       crosses the floor)                                        */
} sn_fluid;
enum { SN_FLOOR_MAX = 0, SN_FLOOR_SMOOTH = 1 };

/* Switch an SN_C128 grid to the fluid model of Eq. 16 (f != NULL) or back
 * to Eqs. 1-2 (f == NULL; sn_set_kernel also switches back).  sn_step then
 * takes symmetric split steps of Eq. 16: Kin(h/2) with A = -nu/2, the exact
 * potential sub-step psi exp(-i U h / nu) (U depends on rho only), Kin(h/2).
 * The profiles gamma, beta, phi_C are built once here, in FP64 on the host.
 * In this mode sn_observables reports mass, centroids, momenta and the
 * energies of the solver's form i psi_t = -(nu/2) lap psi + (U/nu) psi:
 * e_kin = (nu/2) int |grad psi|^2, e_pot = (1/2 int phi_N rho + int phi_C
 * rho) / nu, e_nl = (-(nu^2/2) int |grad sqrt rho|^2 + int eps(rho)) / nu with
 * eps the polytropic internal energy (d eps / d rho = V_p); under GR their sum
 * is the conserved Hamiltonian.  Errors: SN_ENOTSUP on SN_C64
 * grids (this build steps Eq. 16 in FP64 only) and on grids of several fields
 * (sn_set_fields), SN_EINVAL for bad values, SN_ENOMEM, SN_ECUDA. */
sn_status sn_set_fluid(sn_grid g, const sn_fluid* f);

/* Several coupled wave functions (Sec. II: Eqs. 1-2 generalize to multiple
 * wave functions coupled through the nonlinearities).  The grid holds count
 * fields psi_0 .. psi_{count-1}; each obeys Eq. 1 with the same A, and all
 * see one index change: phi of Eq. 2 (or the Newton + Yukawa kernel) sourced
 * by the total density rho = sum_j |psi_j|^2, the local term g_local rho of
 * that same total density, and v_ext.  With count = 1 this is Eqs. 1-2.
 * Each field's mass is conserved.  sn_observables then reports mass, e_kin
 * and momenta summed over the fields, and the centroids, e_pot and e_nl of
 * the total density (e_total is the Hamiltonian of the coupled system).
 * The call synchronises the grid's stream, sets the state to zero and the
 * step counter to 0.  Errors: SN_EINVAL (count outside [1, SN_MAX_FIELDS]),
 * SN_ENOTSUP (count > 1 in the fluid mode of sn_set_fluid), SN_ENOMEM,
 * SN_ECUDA.  sn_get_fields returns the count (0 for a NULL grid). */
#define SN_MAX_FIELDS 16
sn_status sn_set_fields(sn_grid g, int count);
int sn_get_fields(sn_grid g);

/* Copy a state in: psi holds fields x ncells complex values of the grid's
 * dtype, field j at offset j ncells (fields = 1 unless sn_set_fields set
 * more), host memory (on_device = 0; the call returns after the copy) or
 * device memory (on_device = 1; ordered on the grid's stream).  Resets the
 * step counter to 0. */
sn_status sn_set_state(sn_grid g, const void* psi, int on_device);

/* Copy the state out (same layout as sn_set_state).  Host copies block until
 * done.  The state is always at an integer step: on a complex64 grid whose
 * merge is open (see sn_step) the closing Nl(h) Kin(h/2) is applied to a copy
 * (three psi passes), and the grid's own state stays open. */
sn_status sn_get_state(sn_grid g, void* psi_out, int on_device);

/* Advance nsteps symmetric split steps of size dt (Sec. III).  Consecutive
 * steps are merged (Kin(h/2) Kin(h/2) = Kin(h)).  On complex64 grids the
 * merge stays open across calls: the grid keeps Kin(h/2) psi and the
 * potential of its density, and a following sn_step with the same dt
 * continues the merge, so n steps cost n rounds of passes however the calls
 * split them.  Every call that reads the state (sn_get_state, sn_observables)
 * sees it at the integer step; a change of dt, of the kernel (sn_set_kernel),
 * of the engine or an sn_autotune first closes the merge in place.  Complex128
 * grids close the merge within each step.  nsteps = 0 is a no-op.  dt may be
 * negative (time reversal).  Asynchronous on the grid's stream.
 * Errors: SN_EINVAL (non-finite dt, nsteps < 0), SN_ECUDA. */
sn_status sn_step(sn_grid g, double dt, int nsteps);

/* Compute the observables of the current state (blocks until done).
 * Errors: SN_ENONFINITE if any sum is NaN or Inf, SN_ECUDA. */
sn_status sn_observables(sn_grid g, sn_obs* out);

/* Wait for the grid's queued work; returns SN_ECUDA if a kernel failed. */
sn_status sn_sync(sn_grid g);

/* Number of kernels this grid has launched since creation. */
long long sn_launch_count(sn_grid g);

/* Run sn_step(g, dt, nsteps) with a CUDA event pair around every kernel and
 * report, per kernel kind k (0 <= k < nkinds, kinds as listed by
 * sn_kind_name), the summed device time in ms, the launch count and the
 * algorithmic HBM bytes those launches move.  Blocks until done.  The step
 * itself is identical to sn_step. */
sn_status sn_profile_step(sn_grid g, double dt, int nsteps, double* ms, long long* launches,
                          double* bytes, int nkinds);

/* Name of kernel kind k, or NULL past the last kind. */
const char* sn_kind_name(int k);

/* Schedule of the fused complex64 passes: for each pass kind k < SN_SCHED_KINDS
 * (the first kinds of sn_kind_name: psi_pass, psi_pass_nphase,
 * psi_pass_density, rho_fwd, rho_green, rho_inv) and axis a < 3 (psi passes:
 * the axis of the transformed lines; half-spectrum passes: the half axis), the
 * CTAs per SM of its persistent grid: 0 = as many as fit (the default),
 * 1 .. SN_SCHED_MAX_CTAS = at most that many, -1 = one CTA per tile of lines.
 * Every schedule computes bit-identical results; only the speed differs.
 * Layout of the 3 SN_SCHED_KINDS values: [3 k + a].  A full schedule
 * (SN_SCHED_VALUES values) appends, at [3 SN_SCHED_KINDS + 3 k + a], the tile
 * staging of each kind and axis: SN_STAGING_TMA, SN_STAGING_REGISTERS (see
 * sn_set_staging), or -1 for the grid's own staging.
 * sn_get_schedule: out holds at least 3 SN_SCHED_KINDS values (the staging
 * part is written when it holds SN_SCHED_VALUES).  sn_set_schedule: exactly
 * 3 SN_SCHED_KINDS values (the CTAs; staging entries unchanged) or
 * SN_SCHED_VALUES values, CTAs in [-1, SN_SCHED_MAX_CTAS] and staging in
 * [-1, SN_STAGING_REGISTERS], else SN_EINVAL.
 * sn_autotune: pick the schedule by the device time of whole steps (CUDA
 * events around sn_step(g, dt, steps) only, so the overlap of consecutive
 * passes counts).  For each pass kind and axis the step uses, one after
 * another, first the other staging is timed and kept if it is more than 1%
 * faster, then the CTA candidates 0, -1, 1, 2, 3, 4, 6, 8 are timed and the
 * fastest kept if it is more than 1% faster; the result is kept only if it
 * beats the default schedule by at least 0.5% over 3 x steps.  An open merge
 * (sn_step) is closed first.  The state and the step
 * counter are restored; blocks until done.  Errors: SN_ENOTSUP on SN_C128
 * grids, SN_EINVAL (non-finite dt, steps < 1), SN_ENOMEM, SN_ECUDA. */
#define SN_SCHED_KINDS 6
#define SN_SCHED_MAX_CTAS 64
#define SN_SCHED_VALUES (6 * SN_SCHED_KINDS)
sn_status sn_get_schedule(sn_grid g, int* out, int n);
sn_status sn_set_schedule(sn_grid g, const int* in, int n);
sn_status sn_autotune(sn_grid g, double dt, int steps);

/* Line-transform engine of a complex64 grid's fused step.  Every pass of
 * sn_step is a batch of 1D DFTs along one axis (the split-step Fourier method
 * of Sec. III: the kinetic factor of Eq. 1 per axis, and the spectral solve of
 * Eq. 2 / the Eq. 9 kernel); the engine decides how they are computed.
 *   SN_ENGINE_FP32 (default): FP32 radix-16/32 Stockham stages on CUDA cores.
 *   SN_ENGINE_TC16: on axes of length 256, each 16-point DFT stage runs on
 *     the tensor cores as real 32 x 32 blocks of FP16 operands split into
 *     hi + lo parts (F_hi x_hi + F_hi x_lo + F_lo x_hi, FP32 accumulation,
 *     per-line power-of-two scaling); twiddles and the spectral multipliers
 *     stay FP32.  Axes of other lengths keep the FP32 engine.
 * Both engines give the same step to FP32 rounding.  The paper's own solver
 * has no counterpart of this switch (its FFTs are library calls).
 * Errors: SN_EINVAL (NULL grid, unknown engine), SN_ENOTSUP (TC16 on a
 * complex128 grid), SN_ENOMEM / SN_ECUDA (table upload). */
typedef enum { SN_ENGINE_FP32 = 0, SN_ENGINE_TC16 = 1, SN_ENGINE_UMMA = 2 } sn_engine;
sn_status sn_set_engine(sn_grid g, int engine);

/* How the fused complex64 passes move their tiles of lines between HBM and
 * shared memory; the arithmetic, and so every result, is the same bit for bit.
 *   SN_STAGING_TMA: each tile travels as one bulk tensor copy of the
 *     tensor-memory accelerator into a shared-memory slot, and back out, while
 *     the CTA transforms the tile in its other slot.  Taken by the passes of
 *     128- and 256-point lines on the FP32 engine: the plain kinetic, the
 *     potential, the density and the half-spectrum passes of one field, the
 *     plain and half-spectrum passes of several; the other passes keep
 *     register staging.  A tile wait
 *     that does not end within about 2 s makes the next synchronising call
 *     (sn_sync, sn_get_state to host, sn_observables) return SN_ETIMEOUT.
 *   SN_STAGING_REGISTERS: every thread loads its elements of the next tile
 *     into registers while it transforms the current one.
 *   SN_STAGING_RESIDENT: on a square 2D grid of 64^2 or 128^2 cells (one
 *     field, FP32 engine, no V_ext) the whole state stays in one CTA's shared
 *     memory for all steps of an sn_step call: one launch per call, no HBM
 *     traffic between the passes (one SM; pays off where the tiled passes are
 *     launch-bound).  Other grids take SN_STAGING_TMA.  Same bits.
 * Without a call, a grid of one field takes SN_STAGING_TMA and a grid of
 * several fields (sn_set_fields) SN_STAGING_REGISTERS, whose plain passes keep
 * the overlap with the fused-fields potential and density passes.
 * Errors: SN_EINVAL (NULL grid, unknown mode). */
typedef enum { SN_STAGING_TMA = 0, SN_STAGING_REGISTERS = 1, SN_STAGING_RESIDENT = 2 } sn_staging;
sn_status sn_set_staging(sn_grid g, int mode);

/* Slab blocking of the 3D FP32 step (Sec. III; the merged Strang round of
 * Eqs. 1-2).  Of the three psi passes of a round, the ones along y and x
 * (array axes 1 and 2) stay within the planes of fixed z.  With planes > 0 the
 * pair runs slab by slab over z, `planes` planes per slab: the second pass of
 * the pair reads the slab the first one has just written while it is still
 * in L2, instead of the whole state from HBM.  It applies to grids of one
 * field on the FP32 engine whose pair of passes both take the TMA-staged
 * kernels (128- or 256-point lines), with planes < n[0]; other grids ignore it.
 * The arithmetic and the results are the same bit for bit; only the launches
 * change (two per slab instead of two per round).  0 (the default) turns it
 * off.  Errors: SN_EINVAL (NULL grid, planes < 0). */
sn_status sn_set_blocking(sn_grid g, int planes);

/* How sn_observables computes (the quantities of sn_obs, Sec. III):
 *   SN_OBS_FP64 (default): the state widened to FP64, FP64 FFTs and sums;
 *   SN_OBS_FP32 (complex64 grids): the FP32 line transforms of the step with
 *     FP64 sums -- e_kin and the momenta from one read-only pass per axis (1D
 *     Parseval per line), the density's half spectrum along the last axis
 *     (mass, rho^2, V_ext and centroid sums in the same pass), e_pot from
 *     sum K(k) |F rho|^2 over it.  About 1e-7 relative to the FP64 values,
 *     at a small fraction of their cost (FP64 arithmetic is slow on B300).
 * The Eq. 16 fluid's observables always take the FP64 path.
 * Errors: SN_EINVAL (NULL grid, unknown mode), SN_ENOTSUP (SN_OBS_FP32 on a
 * complex128 grid). */
typedef enum { SN_OBS_FP64 = 0, SN_OBS_FP32 = 1 } sn_obs_mode;
sn_status sn_set_obs_mode(sn_grid g, int mode);

/* Test hook: in-place unnormalised DFTs, sign -1 (exp(-i ...)) or +1, of
 * nlines contiguous complex64 lines of length n (power of two, 8..1024) in
 * device memory, computed by the fused passes' line engine (engine as in
 * sn_set_engine; TC16 applies to n = 256).  Synchronous on cuda_stream (NULL:
 * the legacy default stream).  Errors: SN_EINVAL, SN_ECUDA (message in
 * sn_last_error(NULL)). */
sn_status sn_test_line_fft_f32(void* data, long long nlines, int n, int sign, int engine,
                               void* cuda_stream);

/* Test and measurement hook: reps launches of in-place unnormalised DFTs of
 * nlines contiguous complex64 lines of length n in device memory (the data
 * is transformed reps times), on one of three line engines:
 *   SN_ENGINE_FP32, SN_ENGINE_TC16: the fused passes' engines, as
 *     sn_test_line_fft_f32;
 *   SN_ENGINE_UMMA (n = 256 only; not an engine of sn_set_engine): both
 *     radix-16 stages of each line on tcgen05.mma, split-FP16 operands in
 *     shared memory and FP32 accumulators in tensor memory (Sec. III's FFT in
 *     the tensor-core form of the split step).
 * *ms_per_launch (if not NULL) receives the CUDA-event time of one launch.
 * Synchronous on cuda_stream.  Errors: SN_EINVAL, SN_ECUDA, SN_ETIMEOUT (a
 * bounded wait of the UMMA kernel expired; the data is incomplete). */
sn_status sn_test_line_fft_engines(void* data, long long nlines, int n, int sign, int engine,
                                   int reps, double* ms_per_launch, void* cuda_stream);
/* Where the tcgen05 line engine's time goes: one launch of SN_ENGINE_UMMA on
 * nlines (>= 1) contiguous 256-point complex64 lines in device memory (in
 * place, as sn_test_line_fft_engines), in a form whose thread 0 of each CTA
 * reads the SM clock at the phase boundaries of every tile of 8 lines (the
 * arithmetic is the same).  cycles_per_tile[5] receives the clock cycles of
 * each phase per tile, averaged over all tiles: [0] stage A's operands (load,
 * norm, scale, FP16 split into shared memory), [1] stage A's six products
 * (issue to completion), [2] stage B's operands (tensor-memory read, twiddle,
 * scale, split), [3] stage B's products, [4] the output (tensor-memory read,
 * Parseval rescale, store).  *tiles receives the tiles done.  Synchronous on
 * cuda_stream.  Errors: SN_EINVAL, SN_ECUDA, SN_ETIMEOUT. */
sn_status sn_test_umma_phases(void* data, long long nlines, int sign, double* cycles_per_tile,
                              long long* tiles, void* cuda_stream);

/* Measurement hook: the distributed-shared-memory rates of thread-block
 * clusters of cluster_size CTAs (2, 4 or 8), as many clusters as are
 * resident, one CTA per SM.  rates[0]: float4 reads of a peer's 128 KB of
 * shared memory (map_shared_rank), rates[1]: the same reads of the CTA's own,
 * rates[2]: bulk copies (cp.async.bulk.shared::cluster) pushed into a peer's
 * shared memory; aggregate GB/s over the GPU.  These are the exchange rates
 * of a plane held across a cluster (Sec. III's transposes between the axis
 * passes of one plane).  Blocks.  Errors: SN_EINVAL, SN_ECUDA, SN_ETIMEOUT (a
 * bounded copy wait expired). */
sn_status sn_test_dsmem_rates(int cluster_size, double* rates);

/* ---------------------------------------------------------------------------
 * Batched scan: many independent 2D complex64 problems of uneven size
 * advanced together (Sec. III step applied to each; e.g. a scan over the
 * coupling strength and range of the Eq. 9 kernel and over initial
 * conditions).  Instance i is an n[i] x n[i] periodic grid of box length L[i]
 * in both axes with its own kernel parameters and time step.  Three schedules
 * (sn_set_batch_schedule):
 *
 * SN_BATCH_PERSISTENT (the default): one sn_step_batch call runs all merged
 * steps of all instances in a single persistent cooperative launch, captured
 * once into a CUDA graph and replayed while nsteps is unchanged.
 *
 * SN_BATCH_CLASSES: the same persistent kernel launched once per size class
 * (the instances of one n, largest n first), each launch running all steps
 * of its class; the launches are captured together.  The same bits as
 * SN_BATCH_PERSISTENT.
 *
 * SN_BATCH_GRAPH: each round of merged steps (the psi passes along both axes
 * and the Green's pass on the half spectrum) is a CUDA graph in which every
 * instance is a branch of its own, running the fused pass kernels of the
 * single-grid step (sn_step) on a grid of the instance's shape; the branches
 * run concurrently and the graph is launched once per round.  Instance i then
 * gives what sn_step gives for it, bit for bit.  Each call copies the states
 * into those grids and back (16 bytes a cell per call).
 *
 * Inside the launch, work items (round, pass, instance, tile) are taken in a
 * fixed order (within a pass, larger instances first), and an item waits for
 * the previous pass of its instance.  Each
 * wait has a clock-cycle limit (sn_set_batch_wait_limit; about 2 s by default);
 * when a wait expires the kernel records it and returns, and the next
 * synchronising call returns SN_ETIMEOUT and leaves the batch state
 * incomplete.  Batch calls report messages through sn_last_error(NULL).
 * ------------------------------------------------------------------------- */
typedef struct sn_batch_s* sn_batch;

enum sn_batch_schedule {
  SN_BATCH_PERSISTENT = 0, /* one persistent cooperative launch per call */
  SN_BATCH_GRAPH = 1,      /* a graph per round, an instance per branch */
  SN_BATCH_CLASSES = 2     /* one persistent launch per size class */
};

/* n[i]: power of two in [8, 1024]; L[i] > 0.  cuda_stream as for sn_create_grid.
 * States start at zero, kernels at {A=-0.5, G=1, alpha_Y=0, g=0}. */
sn_status sn_create_batch(sn_batch* out, int count, const int* n, const double* L,
                          void* cuda_stream);
/* k[count]: per-instance parameters (v_ext must be NULL: SN_ENOTSUP). */
sn_status sn_set_kernel_batch(sn_batch b, const sn_kernel* k);
/* Copy instance `index` in or out (n[index]^2 complex64, host or device). */
sn_status sn_set_state_batch(sn_batch b, int index, const void* psi, int on_device);
sn_status sn_get_state_batch(sn_batch b, int index, void* psi_out, int on_device);
/* nsteps merged steps of every instance, instance i with step dt[i]; async. */
sn_status sn_step_batch(sn_batch b, const double* dt, int nsteps);
/* Observables of instance `index` (blocks). */
sn_status sn_observables_batch(sn_batch b, int index, sn_obs* out);
/* Wait for the batch's work; SN_ETIMEOUT if a dependency wait (persistent
 * schedule) or a pass kernel's tile wait (graph schedule) expired. */
sn_status sn_batch_sync(sn_batch b);
/* Clock cycles one dependency wait may spin before it gives up (>= 0). */
sn_status sn_set_batch_wait_limit(sn_batch b, long long cycles);
/* Register budget of the batch's launch: per_sm = 3 (80 registers a thread,
 * three resident CTAs per SM; the default), 2 (128) or 1 (255).  The launch
 * stays cooperative with as many CTAs as are resident, so the dependency
 * waits end whatever the choice; the results are the same bit for bit.
 * Errors: SN_EINVAL (NULL batch, per_sm outside 1..3). */
sn_status sn_set_batch_ctas(sn_batch b, int per_sm);
/* The batch's schedule: SN_BATCH_PERSISTENT, SN_BATCH_CLASSES or
 * SN_BATCH_GRAPH (see above);
 * it takes effect at the next sn_step_batch.  The graph schedule's first call
 * makes a grid and a stream per instance, and its round graphs are captured
 * again when a dt or a kernel changes.  Errors: SN_EINVAL (NULL batch, another
 * value).  sn_get_batch_schedule returns the schedule, -1 for NULL. */
sn_status sn_set_batch_schedule(sn_batch b, int schedule);
int sn_get_batch_schedule(sn_batch b);
/* Time `steps` merged steps of the batch (steps dt[i]) on the persistent
 * and per-class schedules at each register budget (3, 2, 1 CTAs per SM) and
 * on the graph schedule, keep the fastest (another candidate must beat the
 * current one by 2 %), and restore every instance's state.  The schedule kept
 * is read with sn_get_batch_schedule; *chosen (if not NULL) receives the
 * register budget kept (the graph schedule leaves it as it was).  Blocks.
 * Errors: SN_EINVAL (NULL batch or dt, steps < 1), SN_ECUDA, SN_ETIMEOUT as
 * sn_batch_sync. */
sn_status sn_autotune_batch(sn_batch b, const double* dt, int steps, int* chosen);
/* Kernel launches of this batch: one per sn_step_batch call on the persistent
 * schedule, one per size class on the per-class schedule; on the graph
 * schedule the pass kernels of every round of every instance. */
long long sn_batch_launch_count(sn_batch b);
void sn_destroy_batch(sn_batch b);

/* ---------------------------------------------------------------------------
 * Fourier-neural-operator surrogate of the solver: predicts the 2D state 50
 * steps ahead from the state and the kernel parameters given as constant
 * input channels; the plain split step is its fallback and its reference.
 *   v0 = P a + pb;  z_l = Spec_l(v_l) + W_l v_l + b_l,  v_{l+1} = gelu(z_l)
 *   (no gelu after the last layer);  Spec(v) keeps the modes
 *   ky in {0..m-1} u {s-m..s-1}, kx in {0..m-1}:
 *   Spec(v) = (1/s^2) sum w_kx Re(U e^{+i th}), U = R V per mode, V = sum v e^{-i th}
 *   (phi, dr, di) = Q2 gelu(Q1 v_L + q1b) + q2b;  out = psi e^{-i phi} + (dr + i di)
 *   with psi = a[0] + i a[1] (the head turns the input state by a learned phase
 *   field, the dominant effect of the nonlinear sub-step over 50 steps)
 * Parameters are one flat FP32 vector in the order P, pb, then per layer R
 * ([2m][m][C][C][re,im]), W, b, then Q1, q1b, Q2, q2b.  Every contraction runs
 * on the tensor cores with BF16 operands and FP32 accumulation.  All array
 * arguments are device pointers, planar [B][channels][s][s] FP32.
 * ------------------------------------------------------------------------- */
typedef struct sn_fno_s* sn_fno;
sn_status sn_fno_create(sn_fno* out, int s, int c_in, int width, int modes, int layers, int proj,
                        int batch_max, void* cuda_stream);
long long sn_fno_param_count(sn_fno f);
/* Copy parameters in (resets the Adam moments) or out; host or device. */
sn_status sn_fno_set_params(sn_fno f, const float* p, int on_device);
sn_status sn_fno_get_params(sn_fno f, float* p, int on_device);
/* Gradients of the last sn_fno_backward (same layout as the parameters). */
sn_status sn_fno_get_grads(sn_fno f, float* g, int on_device);
/* Replace the gradients that sn_fno_adam will apply (same layout), e.g. by
 * their average over data-parallel ranks.  Blocks until copied.  Errors:
 * SN_EINVAL (NULL argument), SN_ECUDA. */
sn_status sn_fno_set_grads(sn_fno f, const float* g, int on_device);
/* out[B][2][s][s] from in[B][c_in][s][s]; keeps the activations for backward. */
sn_status sn_fno_forward(sn_fno f, const float* in, float* out, int B);
/* loss = mean_b ||out_b - target_b|| / ||target_b|| of the last forward (host
 * double); stores dloss/dout for sn_fno_backward.  Blocks. */
sn_status sn_fno_loss(sn_fno f, const float* target, int B, double* loss);
/* Gradients of that loss with respect to every parameter (overwritten). */
sn_status sn_fno_backward(sn_fno f);
/* One Adam step with step count t >= 1 (bias-corrected moments). */
sn_status sn_fno_adam(sn_fno f, double lr, double beta1, double beta2, double eps, int t);
/* Wait for the network's work.  SN_ETIMEOUT if a bounded wait of the fused
 * layer kernel (SN_FNO_LAYER_UMMA) expired; the outputs are then incomplete. */
sn_status sn_fno_sync(sn_fno f);
/* How the second half of each spectral layer runs: the inverse truncated DFT
 * along x, the 1x1 convolution, the bias and the activation.
 *   SN_FNO_LAYER_GEMMS: two strided BF16 GEMMs (mma.sync) and an
 *     elementwise bias/activation pass;
 *   SN_FNO_LAYER_UMMA (the default where it applies): one tcgen05 kernel
 *     (and its backward form, W^T and GELU' of the layer below), both products
 *     as one accumulation
 *     in tensor memory (BF16 operands, FP32 accumulation) with the bias and
 *     the activation in its epilogue, three passes over the activations
 *     instead of six.  Width <= 64, 2 x modes <= 64, s <= 256.
 * The backward and every other contraction are the same in both forms.
 * Errors: SN_EINVAL (NULL, unknown form), SN_ENOTSUP (a network the fused
 * form does not take). */
typedef enum { SN_FNO_LAYER_GEMMS = 0, SN_FNO_LAYER_UMMA = 1 } sn_fno_layer_form;
sn_status sn_fno_set_layer_form(sn_fno f, int form);
void sn_fno_destroy(sn_fno f);
/* Surrogate input/output marshalling on the device: X[b] = (re psi, im psi,
 * feats[b][0..nfeat-1] as constant planes), planar [B][2+nfeat][cells];
 * psi[b] (interleaved complex64) from Y[b] = (re, im) planes. */
sn_status sn_fno_pack(const float* psi, const float* feats, int nfeat, float* X, int B,
                      long long cells, void* cuda_stream);
sn_status sn_fno_unpack(const float* Y, float* psi, int B, long long cells, void* cuda_stream);
/* Input of the corrector form of the surrogate: X[b] = (re a, im a, re c,
 * im c, feats[b][0..nfeat-1] as constant planes), planar [B][4+nfeat][cells],
 * from two interleaved complex64 states per sample (a: the state the head
 * turns, e.g. a coarse solve of the same horizon; c: the starting state). */
sn_status sn_fno_pack2(const float* psi_a, const float* psi_c, const float* feats, int nfeat,
                       float* X, int B, long long cells, void* cuda_stream);
/* out[b] = sum |psi_b|^2 (FP64, device output) for B complex64 states of `cells` values. */
sn_status sn_mass_c64(const float* psi, int B, long long cells, double* out, void* cuda_stream);
/* Test hook: the BF16 tensor-core GEMM C[z] = alpha A[z] B[z] + beta C[z] on
 * device pointers with element strides (see the FNO), synchronous. */
sn_status sn_test_gemm_bf16(const float* A, long long sAz, long long sAm, long long sAk,
                            const float* B, long long sBz, long long sBk, long long sBn, float* C,
                            long long sCz, long long sCm, long long sCn, int M, int N, int K, int Z,
                            float alpha, float beta);

/* Largest ny and nx accepted by sn_step_2d_noalloc. */
#define SN_NOALLOC_MAX_N 512

/* Allocation-free variant of the fused FP32 step for 2D complex64 grids.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc -- code whose device memory is owned in full by
 * another allocator (a framework's caching pool, a fixed arena), or code that
 * runs where an allocation's latency or possible failure is not acceptable.
 *
 * psi: device pointer to ny*nx complex64 values (interleaved re, im, C order,
 * x fastest), advanced in place by nsteps merged split steps of size dt with
 * the same passes and tables as sn_step on an SN_C64 grid (the results agree
 * to FP32 rounding).  Ly, Lx: box lengths.  k: as for sn_set_kernel, with
 * v_ext == NULL.  cuda_stream: the stream to queue on (NULL: legacy default).
 *
 * No device memory is allocated or freed: the working memory (the potential's
 * half spectrum and the per-call tables, about 1.1 MB) is one file-scope
 * static device array of fixed size, which every GPU that loads the library
 * holds until the process exits.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress) with the device current.
 * All calls share the array, so calls whose work overlaps on the GPU (e.g. on
 * two streams) race and give wrong results; serialise them.  Each call
 * rewrites the tables it uses, and the half spectrum is always written before
 * it is read.  The table upload copies from host (stack) memory on
 * cuda_stream; the steps themselves are queued asynchronously.  Because a
 * captured graph would replay those copies from host memory that no longer
 * holds the tables, the call is refused (SN_ENOTSUP) while cuda_stream is
 * being captured.
 *
 * Errors (message in sn_last_error(NULL)): SN_ENOTSUP if ny or nx exceeds
 * SN_NOALLOC_MAX_N, v_ext is given, or cuda_stream is being captured;
 * SN_EINVAL for other bad arguments; SN_ECUDA if a CUDA call fails. */
sn_status sn_step_2d_noalloc(float* psi, int ny, int nx, double Ly, double Lx,
                             const sn_kernel* k, double dt, int nsteps, void* cuda_stream);

/* Free the grid and its device memory (waits for its queued work). */
void sn_destroy_grid(sn_grid g);

/* Last error message of this grid, or of the calling thread's last failed
 * sn_create_grid when g is NULL.  Never NULL. */
const char* sn_last_error(sn_grid g);

#ifdef __cplusplus
}
#endif

#endif /* SN_H_ */

// Batched split steps of many independent 2D complex64 instances of uneven
// size in one persistent launch (a parameter scan over the kernel of Eq. 2 /
// Eq. 9 and over initial conditions; each instance is its own Sec. III
// problem).
//
// Work is a queue of items (round r, slot s, instance i, tile j), in that
// order, with the instances of a slot ordered by decreasing n.  A 2D merged step has three slots per round: the psi pass along the
// first axis (with the potential and nonlinear phase after round 0), the psi
// pass along the second axis (with the density before the last round), and
// the Green's-multiply pass on the half spectrum.  CTA c takes items
// c, c + G, c + 2G, ... in increasing order.  An item waits until all items
// of the previous slot of its instance are done (a per-instance counter):
// every dependency has a smaller queue index, each CTA works in increasing
// order and all CTAs are co-resident (cooperative launch), so the waits always
// end.  Each wait is still bounded by a clock limit; on expiry the kernel
// records an error word and every CTA returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "scan_kernel.cuh"
#include "sn.h"
#include "sn_internal.h"

using namespace sn;
using snfft::cx;
using snfft::Plan;

using namespace sn_scan;

// ============================================================================

struct sn_batch_s {
  int count = 0;
  std::vector<int> n;
  std::vector<double> L;
  std::vector<sn_kernel> kp;
  std::vector<double> dt;  // dt the kinetic tables were built for (NaN: none)
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<Inst> host_inst;
  // queue position -> instance: largest n first, so that neighbouring work
  // items (taken by CTAs at the same time) run the same item function and
  // share the instruction cache
  std::vector<int> order;
  Inst* dev_inst = nullptr;
  float2* tw[kMaxLog2 + 1] = {};
  std::vector<float2*> mult;
  std::vector<float*> k2;
  int4* items = nullptr;  // one round's work items in queue order
  unsigned long long per_round = 0, last = 0;  // items of a full round; of the last (psi passes only)
  // SN_BATCH_CLASSES: the same items class by class (instances of one n, in
  // queue order), class c's round at class_items + class_off[c]
  int4* class_items = nullptr;
  std::vector<unsigned long long> class_off, class_per_round, class_last;
  unsigned* done = nullptr;
  int* err = nullptr;
  long long wait_limit = 4000000000LL;  // about 2 s at the B300's 2 GHz
  int grid = 0;               // CTAs of the launch: resident CTAs per SM x SMs
  int cps = kDefaultCtasPerSm;  // the register budget's CTAs per SM (1 .. 3)
  int grid_of[4] = {};        // grid per budget
  long long launches = 0;
  // a captured launch (memsets + kernel), keyed by nsteps
  cudaGraphExec_t graph = nullptr;
  int graph_steps = -1;
  long long graph_limit = -1;
  int graph_cps = -1;
  int graph_sched = -1;
  // observables of one instance go through a grid of the same shape
  std::vector<sn_grid> obs_grid;
  // the graph schedule (SN_BATCH_GRAPH): a grid per instance on a stream of
  // its own, only for capture; the captured rounds [first, middle even, middle
  // odd, last even, last odd], with the kernels each launches, for the dt and
  // kernels in graph_dt and graph_kp
  int schedule = SN_BATCH_PERSISTENT;
  std::vector<sn_grid> step_grid;
  std::vector<cudaStream_t> step_stream;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  cudaGraphExec_t round_graph[5] = {};
  long long round_launches[5] = {};
  std::vector<double> graph_dt;
  std::vector<sn_kernel> graph_kp;
  std::vector<void*> allocs;
};

namespace {

sn_status bfail(sn_status st, const std::string& m) {
  set_thread_error(m.c_str());
  return st;
}
sn_status bcuda(cudaError_t e, const char* what) {
  return bfail(e == cudaErrorMemoryAllocation ? SN_ENOMEM : SN_ECUDA,
               std::string("batch: ") + what + ": " + cudaGetErrorString(e));
}

template <typename T>
cudaError_t balloc(sn_batch b, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) return e;
  b->allocs.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return cudaSuccess;
}

void split_hilo(const std::vector<double2>& v, float2* out) {
  const size_t n = v.size();
  for (size_t i = 0; i < n; ++i) {
    const float hr = (float)v[i].x, hi = (float)v[i].y;
    out[i] = make_float2(hr, hi);
    out[n + i] = make_float2((float)(v[i].x - (double)hr), (float)(v[i].y - (double)hi));
  }
}

double wavenumber(int j, int n, double L) { return 2.0 * kPi / L * (double)(j < n / 2 ? j : j - n); }

}  // namespace

extern "C" {

namespace {
ScanKern scan_kernel_of(int cps) {
  return cps == 1 ? scan_kernel_1() : cps == 2 ? scan_kernel_2() : scan_kernel_3();
}
// Kernel attributes of register budget cps and its cooperative grid: the
// shared memory of the resident CTAs (1 KB reserved each), the rest of the
// SM's 256 KB left to L1 for the twiddle and kinetic tables and spills; at
// most cps CTAs per SM.
cudaError_t prep_scan_kernel(int cps, int smem_sm, int sms, int* grid) {
  ScanKern k = scan_kernel_of(cps);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  if (e != cudaSuccess) return e;
  if (smem_sm > 0) {
    const double need = (double)cps * (double)(kSmemBytes + 1024 + 64);
    const int pct = std::min(100, (int)std::ceil(100.0 * need / smem_sm));
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct)) != cudaSuccess)
      return e;
  }
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, kSmemBytes)) != cudaSuccess)
    return e;
  *grid = std::min(per_sm, cps) * sms;
  return cudaSuccess;
}
}  // namespace

sn_status sn_create_batch(sn_batch* out, int count, const int* n, const double* L,
                          void* cuda_stream) {
  if (!out) return bfail(SN_EINVAL, "sn_create_batch: out is NULL");
  *out = nullptr;
  if (count < 1 || !n || !L) return bfail(SN_EINVAL, "sn_create_batch: count >= 1, n and L required");
  for (int i = 0; i < count; ++i) {
    if (n[i] < 8 || n[i] > 1024 || (n[i] & (n[i] - 1)))
      return bfail(SN_EINVAL, "sn_create_batch: each n must be a power of two in [8, 1024]");
    if (!(L[i] > 0.0) || !std::isfinite(L[i]))
      return bfail(SN_EINVAL, "sn_create_batch: each L must be finite and > 0");
  }
  sn_batch b = new sn_batch_s();
  b->count = count;
  b->n.assign(n, n + count);
  b->L.assign(L, L + count);
  sn_kernel k0{};
  k0.coeff_lap = -0.5;
  k0.G = 1.0;
  k0.lambda_Y = 1.0;
  k0.zero_k0 = 1;
  b->kp.assign(count, k0);
  b->dt.assign(count, std::nan(""));
  b->host_inst.resize(count);
  b->mult.assign(count, nullptr);
  b->k2.assign(count, nullptr);
  b->obs_grid.assign(count, nullptr);
  auto bail = [&](sn_status st) {
    sn_destroy_batch(b);
    return st;
  };
  cudaError_t e;
  if (cuda_stream) {
    b->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  } else {
    if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess)
      return bail(bcuda(e, "cudaStreamCreate"));
    b->own_stream = true;
  }
  b->order.resize(count);
  for (int i = 0; i < count; ++i) b->order[i] = i;
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return n[x] > n[y]; });
  for (int i = 0; i < count; ++i) {
    Inst& d = b->host_inst[i];
    const int N = n[i];
    const int lpb = lines_per_tile(N);
    d.n = N;
    d.t_psi = (unsigned)((N + lpb - 1) / lpb);
    d.t_rho = (unsigned)((N / 2 + 1 + lpb - 1) / lpb);
    const size_t cells = (size_t)N * N;
    if ((e = balloc(b, &d.psi, cells)) != cudaSuccess) return bail(bcuda(e, "cudaMalloc(psi)"));
    if ((e = cudaMemset(d.psi, 0, cells * sizeof(float2))) != cudaSuccess)
      return bail(bcuda(e, "cudaMemset(psi)"));
    if ((e = balloc(b, &d.rho, (size_t)(N / 2 + 1) * N)) != cudaSuccess)
      return bail(bcuda(e, "cudaMalloc(rho)"));
    const int l2 = log2i(N);
    if (!b->tw[l2]) {
      std::vector<double2> t64((size_t)snfft::plan_twn(N));
      snfft::plan_twiddles(N, t64.data());
      std::vector<float2> t32(std::max<size_t>(2 * t64.size(), 2));
      if (!t64.empty()) split_hilo(t64, t32.data());
      if ((e = balloc(b, &b->tw[l2], t32.size())) != cudaSuccess) return bail(bcuda(e, "cudaMalloc(tw)"));
      if ((e = cudaMemcpy(b->tw[l2], t32.data(), t32.size() * sizeof(float2), cudaMemcpyHostToDevice)) !=
          cudaSuccess)
        return bail(bcuda(e, "cudaMemcpy(tw)"));
    }
    d.tw = b->tw[l2];
    if ((e = balloc(b, &b->mult[i], (size_t)4 * N)) != cudaSuccess) return bail(bcuda(e, "cudaMalloc(mult)"));
    d.mult = b->mult[i];
    std::vector<float> k2(N);
    for (int j = 0; j < N; ++j) {
      const double k = wavenumber(j, N, L[i]);
      k2[j] = (float)(k * k);
    }
    if ((e = balloc(b, &b->k2[i], (size_t)N)) != cudaSuccess) return bail(bcuda(e, "cudaMalloc(k2)"));
    if ((e = cudaMemcpy(b->k2[i], k2.data(), N * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
      return bail(bcuda(e, "cudaMemcpy(k2)"));
    d.k2 = b->k2[i];
  }
  // one round: slot 0 of every instance (in queue order), then slot 1, then slot 2
  std::vector<int4> items;
  for (int s = 0; s < 3; ++s)
    for (int p = 0; p < count; ++p) {
      const Inst& d = b->host_inst[b->order[p]];
      const unsigned tiles = s == 2 ? d.t_rho : d.t_psi;
      const int before = (s >= 1 ? (int)d.t_psi : 0) + (s >= 2 ? (int)d.t_psi : 0);
      for (unsigned j = 0; j < tiles; ++j)
        items.push_back(make_int4(p, s | (before << 2), (int)j, (int)(2 * d.t_psi + d.t_rho)));
    }
  b->per_round = items.size();
  for (int i = 0; i < count; ++i) b->last += 2ull * b->host_inst[i].t_psi;
  // class by class: the queue positions [p0, p1) of one n
  std::vector<int4> citems;
  for (int p0 = 0; p0 < count;) {
    int p1 = p0;
    while (p1 < count && n[b->order[p1]] == n[b->order[p0]]) ++p1;
    b->class_off.push_back(citems.size());
    unsigned long long last = 0;
    for (const int4& it : items)
      if (it.x >= p0 && it.x < p1) citems.push_back(it);
    for (int p = p0; p < p1; ++p) last += 2ull * b->host_inst[b->order[p]].t_psi;
    b->class_per_round.push_back(citems.size() - b->class_off.back());
    b->class_last.push_back(last);
    p0 = p1;
  }
  if ((e = balloc(b, &b->items, items.size())) != cudaSuccess) return bail(bcuda(e, "cudaMalloc(items)"));
  if ((e = cudaMemcpy(b->items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return bail(bcuda(e, "cudaMemcpy(items)"));
  if ((e = balloc(b, &b->class_items, citems.size())) != cudaSuccess)
    return bail(bcuda(e, "cudaMalloc(class items)"));
  if ((e = cudaMemcpy(b->class_items, citems.data(), citems.size() * sizeof(int4),
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(bcuda(e, "cudaMemcpy(class items)"));
  if ((e = balloc(b, &b->dev_inst, (size_t)count)) != cudaSuccess) return bail(bcuda(e, "cudaMalloc(inst)"));
  if ((e = balloc(b, &b->done, (size_t)count)) != cudaSuccess) return bail(bcuda(e, "cudaMalloc(done)"));
  if ((e = balloc(b, &b->err, (size_t)2)) != cudaSuccess) return bail(bcuda(e, "cudaMalloc(err)"));
  if ((e = cudaMemset(b->err, 0, 2 * sizeof(int))) != cudaSuccess) return bail(bcuda(e, "cudaMemset(err)"));
  int dev = 0, sms = 0, smem_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  for (int c = 1; c <= 3; ++c) {
    if ((e = prep_scan_kernel(c, smem_sm, sms, &b->grid_of[c])) != cudaSuccess)
      return bail(bcuda(e, "scan kernel attributes"));
    if (b->grid_of[c] < 1) return bail(bfail(SN_ENOTSUP, "sn_create_batch: scan kernel does not fit on an SM"));
  }
  b->grid = b->grid_of[b->cps];
  *out = b;
  return SN_OK;
}

sn_status sn_set_kernel_batch(sn_batch b, const sn_kernel* k) {
  if (!b || !k) return bfail(SN_EINVAL, "sn_set_kernel_batch: NULL argument");
  for (int i = 0; i < b->count; ++i) {
    const sn_kernel& x = k[i];
    if (const char* why = kernel_invalid(x))
      return bfail(SN_EINVAL, std::string("sn_set_kernel_batch: ") + why);
    if (x.v_ext) return bfail(SN_ENOTSUP, "sn_set_kernel_batch: v_ext is not supported in a batch");
  }
  for (int i = 0; i < b->count; ++i) {
    if (k[i].coeff_lap != b->kp[i].coeff_lap) b->dt[i] = std::nan("");
    b->kp[i] = k[i];
  }
  return SN_OK;
}

sn_status sn_set_state_batch(sn_batch b, int index, const void* psi, int on_device) {
  if (!b || !psi || index < 0 || index >= b->count)
    return bfail(SN_EINVAL, "sn_set_state_batch: bad argument");
  const size_t bytes = (size_t)b->n[index] * b->n[index] * sizeof(float2);
  cudaError_t e = cudaMemcpyAsync(b->host_inst[index].psi, psi, bytes,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  b->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? SN_OK : bcuda(e, "sn_set_state_batch copy");
}

sn_status sn_get_state_batch(sn_batch b, int index, void* psi_out, int on_device) {
  if (!b || !psi_out || index < 0 || index >= b->count)
    return bfail(SN_EINVAL, "sn_get_state_batch: bad argument");
  sn_status st = sn_batch_sync(b);
  if (st != SN_OK) return st;
  const size_t bytes = (size_t)b->n[index] * b->n[index] * sizeof(float2);
  cudaError_t e = cudaMemcpyAsync(psi_out, b->host_inst[index].psi, bytes,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  b->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? SN_OK : bcuda(e, "sn_get_state_batch copy");
}

sn_status sn_set_batch_wait_limit(sn_batch b, long long cycles) {
  if (!b || cycles < 0) return bfail(SN_EINVAL, "sn_set_batch_wait_limit: bad argument");
  b->wait_limit = cycles;
  return SN_OK;
}

namespace {

void drop_round_graphs(sn_batch b) {
  for (cudaGraphExec_t& x : b->round_graph) {
    if (x) cudaGraphExecDestroy(x);
    x = nullptr;
  }
}

// The graph schedule's grids, streams and events (released together).
void drop_step_grids(sn_batch b) {
  drop_round_graphs(b);
  for (sn_grid g : b->step_grid) sn_destroy_grid(g);
  for (cudaStream_t s : b->step_stream)
    if (s) cudaStreamDestroy(s);
  b->step_grid.clear();
  b->step_stream.clear();
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  if (b->join_ev) cudaEventDestroy(b->join_ev);
  b->fork_ev = b->join_ev = nullptr;
  b->graph_dt.clear();
}

// ... made at the schedule's first use; a failure leaves none of them.
sn_status ensure_step_grids(sn_batch b) {
  if (!b->step_grid.empty()) return SN_OK;
  cudaError_t e;
  if ((e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->join_ev, cudaEventDisableTiming)) != cudaSuccess) {
    drop_step_grids(b);
    return bcuda(e, "cudaEventCreate");
  }
  b->step_grid.assign(b->count, nullptr);
  b->step_stream.assign(b->count, nullptr);
  for (int i = 0; i < b->count; ++i) {
    if ((e = cudaStreamCreateWithFlags(&b->step_stream[i], cudaStreamNonBlocking)) != cudaSuccess) {
      drop_step_grids(b);
      return bcuda(e, "cudaStreamCreate");
    }
    const int n2[2] = {b->n[i], b->n[i]};
    const double L2[2] = {b->L[i], b->L[i]};
    sn_status st = sn_create_grid(&b->step_grid[i], 2, n2, L2, SN_C64, b->step_stream[i]);
    if (st != SN_OK) {
      drop_step_grids(b);
      return st;
    }
  }
  return SN_OK;
}

// Round graph t (0: the first round; 1, 2: a middle round of even, odd index;
// 3, 4: the last round of even, odd index): every instance's round on its own
// branch, the largest instances first.
sn_status capture_round(sn_batch b, int t, const double* dt) {
  static const int rr[5] = {0, 2, 1, 2, 1}, nn[5] = {2, 4, 4, 2, 1};
  cudaGraph_t gr = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return bcuda(e, "cudaStreamBeginCapture");
  sn_status st = SN_OK;
  long long total = 0;
  e = cudaEventRecord(b->fork_ev, b->stream);
  for (int p = 0; p < b->count && e == cudaSuccess && st == SN_OK; ++p) {
    const int i = b->order[p];
    if ((e = cudaStreamWaitEvent(b->step_stream[i], b->fork_ev, 0)) != cudaSuccess) break;
    long long k = 0;
    st = batch_grid_round(b->step_grid[i], rr[t], nn[t], dt[i], &k);
    total += k;
    if (st != SN_OK) break;
    if ((e = cudaEventRecord(b->join_ev, b->step_stream[i])) != cudaSuccess) break;
    e = cudaStreamWaitEvent(b->stream, b->join_ev, 0);
  }
  const cudaError_t e_end = cudaStreamEndCapture(b->stream, &gr);
  if (st == SN_OK && e == cudaSuccess) e = e_end;
  if (st == SN_OK && e == cudaSuccess) e = cudaGraphInstantiate(&b->round_graph[t], gr, 0);
  if (gr) cudaGraphDestroy(gr);
  if (st != SN_OK) return st;
  if (e != cudaSuccess) return bcuda(e, "round graph capture");
  b->round_launches[t] = total;
  return SN_OK;
}

// nsteps merged steps on the graph schedule: the states into the instance
// grids, rounds 0 .. nsteps as graph launches, the states back.
sn_status step_graph(sn_batch b, const double* dt, int nsteps) {
  sn_status st = ensure_step_grids(b);
  if (st != SN_OK) return st;
  cudaError_t e;
  bool same = b->graph_dt.size() == (size_t)b->count;
  for (int i = 0; same && i < b->count; ++i)
    same = b->graph_dt[i] == dt[i] &&
           std::memcmp(&b->graph_kp[i], &b->kp[i], sizeof(sn_kernel)) == 0;
  if (!same) {
    // the captured launches carry the kernels' coefficients of dt; the
    // tables they read may still be in use by queued rounds
    if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return bcuda(e, "sync");
    drop_round_graphs(b);
    for (int i = 0; i < b->count; ++i)
      if ((st = batch_grid_prepare(b->step_grid[i], b->kp[i], dt[i])) != SN_OK) return st;
    b->graph_dt.assign(dt, dt + b->count);
    b->graph_kp = b->kp;
  }
  for (int i = 0; i < b->count; ++i) {
    const size_t bytes = (size_t)b->n[i] * b->n[i] * sizeof(float2);
    if ((e = cudaMemcpyAsync(batch_grid_psi(b->step_grid[i]), b->host_inst[i].psi, bytes,
                             cudaMemcpyDeviceToDevice, b->stream)) != cudaSuccess)
      return bcuda(e, "state copy");
  }
  for (int r = 0; r <= nsteps; ++r) {
    const int t = r == 0 ? 0 : r < nsteps ? 1 + (r & 1) : 3 + (r & 1);
    if (!b->round_graph[t] && (st = capture_round(b, t, dt)) != SN_OK) return st;
    if ((e = cudaGraphLaunch(b->round_graph[t], b->stream)) != cudaSuccess)
      return bcuda(e, "cudaGraphLaunch");
    b->launches += b->round_launches[t];
  }
  for (int i = 0; i < b->count; ++i) {
    const size_t bytes = (size_t)b->n[i] * b->n[i] * sizeof(float2);
    if ((e = cudaMemcpyAsync(b->host_inst[i].psi, batch_grid_psi(b->step_grid[i]), bytes,
                             cudaMemcpyDeviceToDevice, b->stream)) != cudaSuccess)
      return bcuda(e, "state copy");
  }
  return SN_OK;
}

}  // namespace

sn_status sn_step_batch(sn_batch b, const double* dt, int nsteps) {
  if (!b || !dt) return bfail(SN_EINVAL, "sn_step_batch: NULL argument");
  if (nsteps < 0) return bfail(SN_EINVAL, "sn_step_batch: nsteps must be >= 0");
  for (int i = 0; i < b->count; ++i)
    if (!std::isfinite(dt[i])) return bfail(SN_EINVAL, "sn_step_batch: dt must be finite");
  if (nsteps == 0) return SN_OK;
  if (b->schedule == SN_BATCH_GRAPH) return step_graph(b, dt, nsteps);
  cudaError_t e;
  bool changed = false;
  for (int i = 0; i < b->count; ++i) {
    Inst& d = b->host_inst[i];
    const sn_kernel& k = b->kp[i];
    const int N = b->n[i];
    const double h = dt[i];
    const double cells = (double)N * N;
    const GreenCoeffs gc = green_coeffs(k);
    const Inst before = d;
    d.cN = (float)(gc.cN * h / cells);
    d.cY = (float)(gc.cY * h / cells);
    d.mu2 = (float)gc.mu2;
    d.gh = (float)(k.g_local * h);
    if (std::memcmp(&before, &d, sizeof(Inst)) != 0) changed = true;
    if (!(h == b->dt[i])) {
      if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return bcuda(e, "sync");
      std::vector<float> m32(8 * (size_t)N);
      for (int f = 0; f < 2; ++f)
        kinetic_lift_table(N, b->L[i], k.coeff_lap, f ? h : 0.5 * h, m32.data() + 4 * N * f);
      if ((e = cudaMemcpy(b->mult[i], m32.data(), m32.size() * sizeof(float), cudaMemcpyHostToDevice)) !=
          cudaSuccess)
        return bcuda(e, "cudaMemcpy(mult)");
      b->dt[i] = h;
    }
  }
  if (changed || b->launches == 0) {
    if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return bcuda(e, "sync");
    std::vector<Inst> queued(b->count);
    for (int p = 0; p < b->count; ++p) queued[p] = b->host_inst[b->order[p]];
    if ((e = cudaMemcpy(b->dev_inst, queued.data(), sizeof(Inst) * b->count,
                        cudaMemcpyHostToDevice)) != cudaSuccess)
      return bcuda(e, "cudaMemcpy(inst)");
  }
  ScanArgs a{};
  a.inst = b->dev_inst;
  a.count = b->count;
  a.nsteps = nsteps;
  a.items = b->items;
  a.per_round = b->per_round;
  a.total = b->per_round * (unsigned long long)nsteps + b->last;
  a.done = b->done;
  a.err = b->err;
  a.wait_limit = b->wait_limit;

  if (b->graph && (b->graph_steps != nsteps || b->graph_limit != b->wait_limit ||
                   b->graph_cps != b->cps || b->graph_sched != b->schedule)) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  if (!b->graph) {
    // capture: zero the counters, then one cooperative launch of the whole
    // scan, or (SN_BATCH_CLASSES) one per class, largest n first
    cudaGraph_t gr = nullptr;
    if ((e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return bcuda(e, "cudaStreamBeginCapture");
    cudaError_t e1 = cudaMemsetAsync(b->done, 0, sizeof(unsigned) * b->count, b->stream);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)b->grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kSmemBytes;
    cfg.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e2 = e1;
    if (b->schedule == SN_BATCH_CLASSES) {
      for (size_t c = 0; c < b->class_off.size() && e2 == cudaSuccess; ++c) {
        ScanArgs ac = a;
        ac.items = b->class_items + b->class_off[c];
        ac.per_round = b->class_per_round[c];
        ac.total = ac.per_round * (unsigned long long)nsteps + b->class_last[c];
        e2 = cudaLaunchKernelEx(&cfg, scan_kernel_of(b->cps), ac);
      }
    } else if (e2 == cudaSuccess) {
      e2 = cudaLaunchKernelEx(&cfg, scan_kernel_of(b->cps), a);
    }
    e = cudaStreamEndCapture(b->stream, &gr);
    if (e2 != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      return bcuda(e2, "scan launch capture");
    }
    if (e != cudaSuccess) return bcuda(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->graph, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return bcuda(e, "cudaGraphInstantiate");
    b->graph_steps = nsteps;
    b->graph_limit = b->wait_limit;
    b->graph_cps = b->cps;
    b->graph_sched = b->schedule;
  }
  if ((e = cudaGraphLaunch(b->graph, b->stream)) != cudaSuccess) return bcuda(e, "cudaGraphLaunch");
  b->launches += b->schedule == SN_BATCH_CLASSES ? (long long)b->class_off.size() : 1;
  return SN_OK;
}

sn_status sn_set_batch_ctas(sn_batch b, int per_sm) {
  if (!b) return bfail(SN_EINVAL, "sn_set_batch_ctas: batch is NULL");
  if (per_sm < 1 || per_sm > 3) return bfail(SN_EINVAL, "sn_set_batch_ctas: per_sm must be 1, 2 or 3");
  b->cps = per_sm;
  b->grid = b->grid_of[per_sm];
  return SN_OK;
}

sn_status sn_autotune_batch(sn_batch b, const double* dt, int steps, int* chosen) {
  if (!b || !dt) return bfail(SN_EINVAL, "sn_autotune_batch: NULL argument");
  if (steps < 1) return bfail(SN_EINVAL, "sn_autotune_batch: steps must be >= 1");
  cudaError_t e;
  // the instances' states, restored after the timed launches
  size_t total = 0;
  for (int i = 0; i < b->count; ++i) total += (size_t)b->host_inst[i].n * b->host_inst[i].n;
  float2* saved = nullptr;
  if ((e = cudaMalloc(&saved, total * sizeof(float2))) != cudaSuccess)
    return bcuda(e, "cudaMalloc(autotune copy)");
  auto copy_all = [&](bool save) {
    size_t off = 0;
    for (int i = 0; i < b->count && e == cudaSuccess; ++i) {
      const size_t cells = (size_t)b->host_inst[i].n * b->host_inst[i].n;
      float2* p = b->host_inst[i].psi;
      e = cudaMemcpyAsync(save ? saved + off : p, save ? p : saved + off, cells * sizeof(float2),
                          cudaMemcpyDeviceToDevice, b->stream);
      off += cells;
    }
  };
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  copy_all(true);
  // candidates: the persistent kernel in one launch and one launch per class,
  // each at 3, 2 and 1 CTAs per SM, and the graph schedule
  struct Cand {
    int schedule, cps;
  };
  std::vector<Cand> cands;
  for (int sch : {SN_BATCH_PERSISTENT, SN_BATCH_CLASSES})
    for (int c = 3; c >= 1; --c) cands.push_back({sch, c});
  cands.push_back({SN_BATCH_GRAPH, b->cps});
  const Cand keep{b->schedule, b->cps};
  auto same = [](const Cand& x, const Cand& y) {
    return x.schedule == y.schedule && (x.schedule == SN_BATCH_GRAPH || x.cps == y.cps);
  };
  Cand best = keep;
  float best_ms = 0.f, keep_ms = 0.f;
  sn_status st = SN_OK;
  for (const Cand& cand : cands) {
    if (e != cudaSuccess || st != SN_OK) break;
    b->schedule = cand.schedule;
    b->cps = cand.cps;
    b->grid = b->grid_of[cand.cps];
    // the first call captures this candidate's graphs; the second is timed
    if ((st = sn_step_batch(b, dt, steps)) != SN_OK) break;
    if ((e = cudaEventRecord(t0, b->stream)) != cudaSuccess) break;
    if ((st = sn_step_batch(b, dt, steps)) != SN_OK) break;
    if ((e = cudaEventRecord(t1, b->stream)) != cudaSuccess) break;
    if ((st = sn_batch_sync(b)) != SN_OK) break;
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, t0, t1)) != cudaSuccess) break;
    if (same(cand, keep)) keep_ms = ms;
    if (best_ms == 0.f || ms < best_ms) {
      best_ms = ms;
      best = cand;
    }
  }
  // a candidate other than the current one must be at least 2% faster
  if (keep_ms > 0.f && !same(best, keep) && best_ms > 0.98f * keep_ms) best = keep;
  copy_all(false);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaFree(saved);
  // the graph schedule keeps the budget as it was
  b->schedule = best.schedule;
  b->cps = best.schedule == SN_BATCH_GRAPH ? keep.cps : best.cps;
  b->grid = b->grid_of[b->cps];
  if (st != SN_OK) return st;
  if (e != cudaSuccess) return bcuda(e, "sn_autotune_batch");
  if (chosen) *chosen = b->cps;
  return SN_OK;
}

sn_status sn_batch_sync(sn_batch b) {
  if (!b) return bfail(SN_EINVAL, "sn_batch_sync: batch is NULL");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "sn_batch_sync");
  int err[2] = {0, 0};
  if ((e = cudaMemcpy(err, b->err, sizeof(err), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return bcuda(e, "sn_batch_sync error word");
  if (err[0] != 0) {
    cudaMemset(b->err, 0, sizeof(err));
    return bfail(SN_ETIMEOUT, "sn_batch_sync: a dependency wait expired at work item " +
                                  std::to_string(err[1]) + "; the batch state is incomplete");
  }
  // the graph schedule's pass kernels report through their grids' status words
  for (sn_grid g : b->step_grid) {
    if (!g) continue;
    sn_status st = batch_grid_status(g);
    if (st != SN_OK) return bfail(st, std::string("sn_batch_sync: ") + sn_last_error(g));
  }
  return SN_OK;
}

sn_status sn_set_batch_schedule(sn_batch b, int schedule) {
  if (!b) return bfail(SN_EINVAL, "sn_set_batch_schedule: batch is NULL");
  if (schedule != SN_BATCH_PERSISTENT && schedule != SN_BATCH_GRAPH && schedule != SN_BATCH_CLASSES)
    return bfail(SN_EINVAL, "sn_set_batch_schedule: unknown schedule");
  b->schedule = schedule;
  return SN_OK;
}

int sn_get_batch_schedule(sn_batch b) { return b ? b->schedule : -1; }

long long sn_batch_launch_count(sn_batch b) { return b ? b->launches : 0; }

sn_status sn_observables_batch(sn_batch b, int index, sn_obs* out) {
  if (!b || !out || index < 0 || index >= b->count)
    return bfail(SN_EINVAL, "sn_observables_batch: bad argument");
  sn_status st = sn_batch_sync(b);
  if (st != SN_OK) return st;
  if (!b->obs_grid[index]) {
    const int n2[2] = {b->n[index], b->n[index]};
    const double L2[2] = {b->L[index], b->L[index]};
    st = sn_create_grid(&b->obs_grid[index], 2, n2, L2, SN_C64, b->stream);
    if (st != SN_OK) return st;
  }
  sn_grid g = b->obs_grid[index];
  if ((st = sn_set_kernel(g, &b->kp[index])) != SN_OK) return st;
  if ((st = sn_set_state(g, b->host_inst[index].psi, 1)) != SN_OK) return st;
  return sn_observables(g, out);
}

void sn_destroy_batch(sn_batch b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (sn_grid g : b->obs_grid) sn_destroy_grid(g);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  drop_step_grids(b);
  for (void* p : b->allocs) cudaFree(p);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // extern "C"

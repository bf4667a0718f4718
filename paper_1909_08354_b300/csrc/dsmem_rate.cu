// Distributed-shared-memory rates of a thread-block cluster, the measurement
// behind the plane-resident cluster schedule's design (a 256^2 plane split
// over a cluster needs three quarters of it from the other CTAs in every
// column pass): how fast a CTA reads its peers' shared memory, against its
// own, and how fast bulk copies push data into a peer's shared memory.
//
//   read kernel: each CTA of a cluster fills its 128 KB of shared memory,
//     then reads it back `iters` times as float4 loads, from a peer
//     (map_shared_rank, the peer changing every pass) or from itself;
//   push kernel: each CTA copies 96 KB of its shared memory into the next
//     CTA's receive buffer with cp.async.bulk.shared::cluster.shared::cta,
//     completing on the receiver's mbarrier, once per pass.
// Every access stays inside the allocations; every wait is bounded (an
// expired wait sets the status word and the kernel finishes its passes
// without waiting).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "sn_internal.h"
#include "tma_ops.cuh"

namespace cg = cooperative_groups;

namespace sn {
namespace {

constexpr int kReadBytes = 128 * 1024, kReadThreads = 512;
constexpr int kPushHalf = 96 * 1024, kPushThreads = 128, kPushChunk = 16384;
constexpr long long kWait = 2000000000LL;

__global__ void dsmem_read_kernel(float4* out, int iters, int remote) {
  extern __shared__ float4 smr[];
  cg::cluster_group cl = cg::this_cluster();
  const int tid = threadIdx.x, nt = blockDim.x, words = kReadBytes / 16;
  for (int i = tid; i < words; i += nt) smr[i] = make_float4((float)i, 1.f, 2.f, 3.f);
  cl.sync();
  const unsigned C = cl.num_blocks(), r = cl.block_rank();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int it = 0; it < iters; ++it) {
    unsigned peer = r;
    if (remote && C > 1) peer = (r + 1 + (unsigned)it % (C - 1)) % C;
    const float4* rp = cl.map_shared_rank(smr, peer);
#pragma unroll 4
    for (int i = tid; i < words; i += nt) {
      const float4 v = rp[i];
      acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
  }
  cl.sync();  // no CTA leaves while a peer may still read its shared memory
  out[blockIdx.x * nt + tid] = acc;
}

__global__ void dsmem_push_kernel(int* status, int iters) {
  extern __shared__ __align__(128) unsigned char smp[];
  __shared__ __align__(8) uint64_t bar;
  cg::cluster_group cl = cg::this_cluster();
  unsigned char* send = smp;
  unsigned char* recv = smp + kPushHalf;
  const int tid = threadIdx.x;
  for (int i = tid; i < kPushHalf / 4; i += blockDim.x) reinterpret_cast<int*>(send)[i] = i;
  if (tid == 0) {
    tma::mbar_init(&bar, 1);
    tma::mbar_fence_init();
  }
  __syncthreads();
  const unsigned C = cl.num_blocks(), r = cl.block_rank(), peer = (r + 1) % C;
  bool bad = false;
  for (int it = 0; it < iters; ++it) {
    if (tid == 0) tma::mbar_expect_tx(&bar, kPushHalf);
    cl.sync();  // every receiver is armed and has consumed the previous copy
    if (tid == 0) {
      unsigned rb, pb;
      asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(rb) : "r"(tma::smem_u32(recv)), "r"(peer));
      asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(pb) : "r"(tma::smem_u32(&bar)), "r"(peer));
      for (int off = 0; off < kPushHalf; off += kPushChunk)
        asm volatile(
            "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                rb + off),
            "r"(tma::smem_u32(send) + off), "r"(kPushChunk), "r"(pb)
            : "memory");
      if (!bad && !tma::mbar_wait_bounded(&bar, (unsigned)(it & 1), kWait)) bad = true;
    }
    __syncthreads();
  }
  if (tid == 0 && bad) {
    atomicExch(status, 1);
    // copies of the last pass may still be landing: wait for them, bounded
    (void)tma::mbar_wait_bounded(&bar, (unsigned)((iters - 1) & 1), kWait / 8);
  }
  cl.sync();
}

cudaError_t launch_cluster(const void* kern, int csize, int threads, size_t smem, void** args,
                           int* clusters_out) {
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)csize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3((unsigned)csize);
  int ncl = 0;
  cudaError_t e = cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg);
  if (e != cudaSuccess) return e;
  if (ncl < 1) return cudaErrorNotSupported;
  ncl = std::min(ncl, 148 * 16 / csize);
  cfg.gridDim = dim3((unsigned)(ncl * csize));
  *clusters_out = ncl;
  return cudaLaunchKernelExC(&cfg, kern, args);
}

}  // namespace

cudaError_t measure_dsmem(int csize, double* read_remote, double* read_local, double* push) {
  static bool attr_of[kDeviceSlots] = {};
  bool& attr = attr_of[device_slot()];
  cudaError_t e = cudaSuccess;
  if (!attr) {
    e = cudaFuncSetAttribute(dsmem_read_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kReadBytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(dsmem_read_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(dsmem_push_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * kPushHalf);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(dsmem_push_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  float4* out = nullptr;
  int* status = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaMalloc(&out, sizeof(float4) * 148 * 16 * kReadThreads);
  if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  auto timed = [&](const void* kern, int threads, size_t smem, void** args, double bytes_per_cta,
                   double* gbs) -> cudaError_t {
    int ncl = 0;
    cudaError_t r = launch_cluster(kern, csize, threads, smem, args, &ncl);  // warm-up
    if (r == cudaSuccess) r = cudaEventRecord(t0);
    if (r == cudaSuccess) r = launch_cluster(kern, csize, threads, smem, args, &ncl);
    if (r == cudaSuccess) r = cudaEventRecord(t1);
    if (r == cudaSuccess) r = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (r == cudaSuccess) r = cudaEventElapsedTime(&ms, t0, t1);
    if (r == cudaSuccess) *gbs = bytes_per_cta * ncl * csize / (ms * 1e-3) / 1e9;
    return r;
  };
  int iters = 100, remote = 1;
  void* rargs[3] = {&out, &iters, &remote};
  if (e == cudaSuccess)
    e = timed((const void*)dsmem_read_kernel, kReadThreads, kReadBytes, rargs, (double)iters * kReadBytes,
              read_remote);
  remote = 0;
  if (e == cudaSuccess)
    e = timed((const void*)dsmem_read_kernel, kReadThreads, kReadBytes, rargs, (double)iters * kReadBytes,
              read_local);
  int piters = 200;
  void* pargs[2] = {&status, &piters};
  if (e == cudaSuccess)
    e = timed((const void*)dsmem_push_kernel, kPushThreads, 2 * kPushHalf, pargs,
              (double)piters * kPushHalf, push);
  int st = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaFree(out);
  cudaFree(status);
  if (e == cudaSuccess && st != 0) e = cudaErrorLaunchTimeout;
  return e;
}

}  // namespace sn

sn_status sn_test_dsmem_rates(int cluster_size, double* rates) {
  if (!rates || cluster_size < 2 || cluster_size > 8 || (cluster_size & (cluster_size - 1)) != 0) {
    sn::set_thread_error("sn_test_dsmem_rates: bad argument");
    return SN_EINVAL;
  }
  const cudaError_t e = sn::measure_dsmem(cluster_size, &rates[0], &rates[1], &rates[2]);
  if (e == cudaErrorLaunchTimeout) {
    sn::set_thread_error("sn_test_dsmem_rates: a bounded copy wait expired");
    return SN_ETIMEOUT;
  }
  if (e != cudaSuccess) {
    sn::set_thread_error((std::string("sn_test_dsmem_rates: ") + cudaGetErrorString(e)).c_str());
    return SN_ECUDA;
  }
  return SN_OK;
}

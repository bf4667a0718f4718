// Programmatic dependent launch for the FP64 step's and the fluid model's
// kernels, which follow one another on one stream, each reading what the
// previous one wrote.  A kernel lets the next one launch at once
// (pdl_allow_next) and waits for the previous grid to complete, with its
// writes visible, before it reads anything that grid may have written
// (pdl_wait_prev); without a programmatic predecessor the wait returns at
// once.  Every kernel launched through launch_pdl calls pdl_wait_prev before
// its first read of such data.
#pragma once

#include <cuda_runtime.h>

namespace sn {

__device__ __forceinline__ void pdl_allow_next() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
__device__ __forceinline__ void pdl_wait_prev() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// Whether launch_pdl asks for programmatic serialisation on this host thread
// (a plain stream-ordered launch otherwise; the kernels' wait then returns at
// once).  A step whose launches are replayed from a captured graph turns it
// off while it runs (PdlOff): there the programmatic edges between the small
// FP64 kernels made the replayed fluid step slower, 0.23 -> 0.44 ms at 256^2.
inline thread_local bool g_pdl_launches = true;
struct PdlOff {
  bool saved;
  PdlOff() : saved(g_pdl_launches) { g_pdl_launches = false; }
  ~PdlOff() { g_pdl_launches = saved; }
};

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = g_pdl_launches ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

}  // namespace sn

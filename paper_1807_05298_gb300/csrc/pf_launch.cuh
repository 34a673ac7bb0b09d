// Kernel launches with programmatic dependent launch (PDL, sm_90 and later).
//
// A kernel launched through launch() may be scheduled while the kernel before
// it in the stream is still finishing, which hides most of the launch gap
// between the many short kernels of a Krylov iteration.  Every kernel
// launched this way starts with PF_PDL_ENTRY(): it first lets its own
// dependent start launching, then waits until the preceding grid has
// completed and its memory is visible (griddepcontrol.wait), before it reads
// anything.  The dependent grid cannot launch before every block of this one
// has started, so the early trigger never starves this grid of SMs.
// Without the launch attribute both instructions are no-ops.
#pragma once

#include <cuda_runtime.h>

#define PF_PDL_ENTRY()                                                  \
  do {                                                                  \
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");     \
    asm volatile("griddepcontrol.wait;" ::: "memory");                  \
  } while (0)

namespace pf {

// process-wide switch (pf_set_programmatic_launch); off by default
bool pdl_enabled();

template <typename... KArgs, typename... Args>
inline void launch(void (*kern)(KArgs...), unsigned int grid, unsigned int block, size_t smem, cudaStream_t st,
                   Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// One thread-block cluster of `cluster` blocks (<= 16; above 8 the kernel must
// allow non-portable cluster sizes, which this sets once per kernel).
template <typename... KArgs, typename... Args>
inline void launch_cluster(void (*kern)(KArgs...), unsigned int cluster, unsigned int block, cudaStream_t st,
                           Args... args) {
  if (cluster > 8) {
    static bool set = false;  // per kernel instantiation
    if (!set) {
      cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      set = true;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 2 : 1;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

}  // namespace pf

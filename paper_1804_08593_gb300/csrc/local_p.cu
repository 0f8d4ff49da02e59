// Instantiations of the persistent local-solve kernel for one storage precision (compiled
// once per precision: -DDWF_LOCAL_P=<precision id>), with its cooperative launch.
#include "dwf_internal.h"
#include "local_kernel.cuh"

#ifndef DWF_LOCAL_P
#error "local_p.cu is compiled once per storage precision: DWF_LOCAL_P"
#endif

namespace dwf {

template <int P, int LS, int V>
static cudaError_t launch_v(const SimdArgs& a, int* grid_cap, int nsm, cudaStream_t st,
                            bool query) {
  auto k = simd_local_kernel<P, LS, V>;
  const size_t smem = simd_smem_bytes<P>(LS, simd_rs(V));
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  if (query) {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * LS / simd_nsl<P>(), smem);
    if (e != cudaSuccess) return e;
    *grid_cap = per_sm * nsm;
    return cudaSuccess;
  }
  // a cooperative launch through the extensible API (capturable in a CUDA graph)
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(a.nslots * a.C));
  cfg.blockDim = dim3(32, LS / simd_nsl<P>());
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, a);
}

template <int P, int LS>
static cudaError_t launch_ls(const SimdArgs& a, int v, int* grid_cap, int nsm, cudaStream_t st,
                             bool query) {
  if constexpr (P == P64) {   // one variant: direct loads, one slice per thread
    return launch_v<P, LS, 0>(a, grid_cap, nsm, st, query);
  } else {
    switch (v) {
      case 1: return launch_v<P, LS, 1>(a, grid_cap, nsm, st, query);
      case 2: return launch_v<P, LS, 2>(a, grid_cap, nsm, st, query);
      default: return launch_v<P, LS, 0>(a, grid_cap, nsm, st, query);
    }
  }
}

template <>
cudaError_t simd_launch_p<DWF_LOCAL_P>(const SimdArgs& a, int Ls, int v, int* grid_cap, int nsm,
                                       cudaStream_t st, bool query) {
  switch (Ls) {
    case 4: return launch_ls<DWF_LOCAL_P, 4>(a, v, grid_cap, nsm, st, query);
    case 6: return launch_ls<DWF_LOCAL_P, 6>(a, v, grid_cap, nsm, st, query);
    case 8: return launch_ls<DWF_LOCAL_P, 8>(a, v, grid_cap, nsm, st, query);
    case 10: return launch_ls<DWF_LOCAL_P, 10>(a, v, grid_cap, nsm, st, query);
    case 12: return launch_ls<DWF_LOCAL_P, 12>(a, v, grid_cap, nsm, st, query);
    case 16: return launch_ls<DWF_LOCAL_P, 16>(a, v, grid_cap, nsm, st, query);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dwf

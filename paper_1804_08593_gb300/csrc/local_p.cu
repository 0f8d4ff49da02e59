// Instantiations of the persistent local-solve kernel for one storage precision (compiled
// once per precision: -DDWF_LOCAL_P=<precision id>), with its cooperative launch.
#include "dwf_internal.h"
#include "local_kernel.cuh"

#ifndef DWF_LOCAL_P
#error "local_p.cu is compiled once per storage precision: DWF_LOCAL_P"
#endif

namespace dwf {

template <int P, int LS>
static cudaError_t launch_ls(const SimdArgs& a, int* grid_cap, int nsm, cudaStream_t st,
                             bool query) {
  auto k = simd_local_kernel<P, LS>;
  const size_t smem = simd_smem_bytes<P>(LS);
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
  SimdArgs b = a;
  void* args[] = {&b};
  return cudaLaunchCooperativeKernel((const void*)k, dim3((unsigned)(a.nslots * a.C)),
                                     dim3(32, LS / simd_nsl<P>()), args, smem, st);
}

template <>
cudaError_t simd_launch_p<DWF_LOCAL_P>(const SimdArgs& a, int Ls, int* grid_cap, int nsm,
                                       cudaStream_t st, bool query) {
  switch (Ls) {
    case 4: return launch_ls<DWF_LOCAL_P, 4>(a, grid_cap, nsm, st, query);
    case 6: return launch_ls<DWF_LOCAL_P, 6>(a, grid_cap, nsm, st, query);
    case 8: return launch_ls<DWF_LOCAL_P, 8>(a, grid_cap, nsm, st, query);
    case 10: return launch_ls<DWF_LOCAL_P, 10>(a, grid_cap, nsm, st, query);
    case 12: return launch_ls<DWF_LOCAL_P, 12>(a, grid_cap, nsm, st, query);
    case 16: return launch_ls<DWF_LOCAL_P, 16>(a, grid_cap, nsm, st, query);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dwf

// Launch/dispatch of the stage kernel for one storage precision (included by stage_f*.cu so
// that the precisions compile in parallel).
#pragma once

#include "dwf_internal.h"

namespace dwf {

template <int P, int LS, bool DAG, bool BLK>
static cudaError_t stage_launch_one(const StageArgs& a, cudaStream_t st) {
  auto k = stage_kernel<P, LS, DAG, BLK>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)stage_smem_bytes<P>(LS, true));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const size_t sm = stage_smem_bytes<P>(LS, a.post != nullptr);
  dim3 grid((unsigned)(a.Vp / 32)), block(32, LS);
  k<<<grid, block, sm, st>>>(a);
  return cudaGetLastError();
}

template <int P, int LS>
static cudaError_t stage_dispatch_ls(const StageArgs& a, bool dag, bool blocked,
                                     cudaStream_t st) {
  if (dag)
    return blocked ? stage_launch_one<P, LS, true, true>(a, st)
                   : stage_launch_one<P, LS, true, false>(a, st);
  return blocked ? stage_launch_one<P, LS, false, true>(a, st)
                 : stage_launch_one<P, LS, false, false>(a, st);
}

template <int P>
cudaError_t launch_stage(const StageArgs& a, int Ls, bool dag, bool blocked, cudaStream_t st) {
  switch (Ls) {
    case 4: return stage_dispatch_ls<P, 4>(a, dag, blocked, st);
    case 6: return stage_dispatch_ls<P, 6>(a, dag, blocked, st);
    case 8: return stage_dispatch_ls<P, 8>(a, dag, blocked, st);
    case 10: return stage_dispatch_ls<P, 10>(a, dag, blocked, st);
    case 12: return stage_dispatch_ls<P, 12>(a, dag, blocked, st);
    case 16: return stage_dispatch_ls<P, 16>(a, dag, blocked, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dwf

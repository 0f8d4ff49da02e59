// Dispatch of the stage kernel on (storage precision, Ls); the instantiations live in the
// per-(precision, Ls) objects built from stage_ls.cu.
#include "dwf_internal.h"
#include "stage.cuh"

namespace dwf {

template <int P, bool DAG>
static cudaError_t launch_stage_pd(const StageArgs& a, int Ls, bool blocked, cudaStream_t st) {
  switch (Ls) {
    case 4: return stage_dispatch_ls<P, 4, DAG>(a, blocked, st);
    case 6: return stage_dispatch_ls<P, 6, DAG>(a, blocked, st);
    case 8: return stage_dispatch_ls<P, 8, DAG>(a, blocked, st);
    case 10: return stage_dispatch_ls<P, 10, DAG>(a, blocked, st);
    case 12: return stage_dispatch_ls<P, 12, DAG>(a, blocked, st);
    case 16: return stage_dispatch_ls<P, 16, DAG>(a, blocked, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int P>
static cudaError_t launch_stage_p(const StageArgs& a, int Ls, bool dag, bool blocked,
                                  cudaStream_t st) {
  return dag ? launch_stage_pd<P, true>(a, Ls, blocked, st)
             : launch_stage_pd<P, false>(a, Ls, blocked, st);
}

cudaError_t launch_stage_prec(int prec, const StageArgs& args, int Ls, bool dag, bool blocked,
                              cudaStream_t st) {
  StageArgs a = args;
  finish_stage_args(a, Ls);
  switch (prec) {
    case P64: return launch_stage_p<P64>(a, Ls, dag, blocked, st);
    case P32: return launch_stage_p<P32>(a, Ls, dag, blocked, st);
    case P16: return launch_stage_p<P16>(a, Ls, dag, blocked, st);
    default: return launch_stage_p<PB16>(a, Ls, dag, blocked, st);
  }
}

}  // namespace dwf

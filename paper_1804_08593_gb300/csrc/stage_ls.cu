// Stage kernel instantiations for one storage precision and one Ls, selected by the build
// (-DDWF_STAGE_P=<precision id> -DDWF_STAGE_LS=<Ls>), so that the many kernel variants
// compile in parallel translation units.
#include "stage_inst.cuh"

#if !defined(DWF_STAGE_P) || !defined(DWF_STAGE_LS)
#error "stage_ls.cu is compiled once per (precision, Ls) with DWF_STAGE_P and DWF_STAGE_LS"
#endif

namespace dwf {
template cudaError_t stage_dispatch_ls<DWF_STAGE_P, DWF_STAGE_LS>(const StageArgs&, bool, bool,
                                                                  cudaStream_t);
}  // namespace dwf

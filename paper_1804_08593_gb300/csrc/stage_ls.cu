// Stage kernel instantiations for one storage precision, one Ls and one of Dh / Dh^dag,
// selected by the build (-DDWF_STAGE_P=<precision id> -DDWF_STAGE_LS=<Ls>
// -DDWF_STAGE_DAG=<0|1>), so that the many kernel variants compile in parallel translation
// units.
#include "stage_inst.cuh"

#if !defined(DWF_STAGE_P) || !defined(DWF_STAGE_LS) || !defined(DWF_STAGE_DAG)
#error "stage_ls.cu is compiled once per (precision, Ls, dag): DWF_STAGE_P, _LS, _DAG"
#endif

namespace dwf {
template cudaError_t stage_dispatch_ls<DWF_STAGE_P, DWF_STAGE_LS, (DWF_STAGE_DAG != 0)>(
    const StageArgs&, bool, cudaStream_t);
}  // namespace dwf

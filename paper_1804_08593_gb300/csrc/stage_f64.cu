// Stage kernel instantiations for P64 storage.
#include "stage_inst.cuh"

namespace dwf {
template cudaError_t launch_stage<P64>(const StageArgs&, int, bool, bool, cudaStream_t);
}  // namespace dwf

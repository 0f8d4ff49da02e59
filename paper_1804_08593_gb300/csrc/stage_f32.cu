// Stage kernel instantiations for P32 storage.
#include "stage_inst.cuh"

namespace dwf {
template cudaError_t launch_stage<P32>(const StageArgs&, int, bool, bool, cudaStream_t);
}  // namespace dwf

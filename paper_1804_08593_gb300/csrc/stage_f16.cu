// Stage kernel instantiations for P16 storage.
#include "stage_inst.cuh"

namespace dwf {
template cudaError_t launch_stage<P16>(const StageArgs&, int, bool, bool, cudaStream_t);
}  // namespace dwf

// das_vu2.cu — tiled DAS instantiations with 2 voxel(s) per thread along u.
#include "das_kernels.cuh"

namespace rcbf {
template int configure_das_vu<2>(int, bool, bool, bool, int*);
template int launch_das_vu<2>(const DasArgs&, int, bool, bool, bool, bool, cudaStream_t);
}  // namespace rcbf

// das_vu1.cu — tiled DAS instantiations with 1 voxel(s) per thread along u.
#include "das_kernels.cuh"

namespace rcbf {
template int configure_das_vu<1>(int, bool, bool, bool, int*);
template int launch_das_vu<1>(const DasArgs&, int, bool, bool, bool, bool, cudaStream_t);
}  // namespace rcbf

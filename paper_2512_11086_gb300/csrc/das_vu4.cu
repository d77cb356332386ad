// das_vu4.cu — tiled DAS instantiations with 4 voxel(s) per thread along u.
#include "das_kernels.cuh"

namespace rcbf {
template int configure_das_vu<4>(int, bool, bool, bool, int*);
template int launch_das_vu<4>(const DasArgs&, int, bool, bool, bool, bool, cudaStream_t);
}  // namespace rcbf

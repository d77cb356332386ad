// das_vu4_real.cu — tiled DAS instantiations with 4 voxel(s) per thread along u, real data.
#include "das_kernels.cuh"

namespace rcbf {
template int configure_das_vu<4, false, false>(int, bool, bool, int*);
template int launch_das_vu<4, false, false>(const DasArgs&, int, bool, bool, bool, int, int,
                                          cudaStream_t);
}  // namespace rcbf

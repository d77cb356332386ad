// das_vu4_cplx.cu — tiled DAS instantiations with 4 voxel(s) per thread along u, complex data.
#include "das_kernels.cuh"

namespace rcbf {
template int configure_das_vu<4, true, false>(int, bool, bool, int*);
template int launch_das_vu<4, true, false>(const DasArgs&, int, bool, bool, bool, int, int,
                                          cudaStream_t);
}  // namespace rcbf

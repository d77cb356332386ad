// das_vu2_cplx.cu — tiled DAS instantiations with 2 voxel(s) per thread along u, complex data.
#include "das_kernels.cuh"

namespace rcbf {
template int configure_das_vu<2, true, false>(int, bool, bool, int*);
template int launch_das_vu<2, true, false>(const DasArgs&, int, bool, bool, bool, int, int,
                                          cudaStream_t);
}  // namespace rcbf

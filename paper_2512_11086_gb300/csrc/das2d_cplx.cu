// das2d_cplx.cu — tiled DAS instantiations for the 2D receive aperture (non-separable
// receive paths), 1 voxel per thread along u, complex data.
#include "das_kernels.cuh"

namespace rcbf {
template int configure_das_vu<1, true, true>(int, bool, bool, int*);
template int launch_das_vu<1, true, true>(const DasArgs&, int, bool, bool, bool, int, int,
                                          cudaStream_t);
}  // namespace rcbf

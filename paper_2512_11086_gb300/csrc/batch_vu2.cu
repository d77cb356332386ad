// batch_vu2.cu — persistent batch kernel instantiations with 2 voxel(s) per thread along u.
#include "batch_kernel.cuh"

namespace rcbf {
template int batch_configure_vu<2>(int, bool, int*, size_t*);
template int batch_launch_vu<2>(int, bool, unsigned, size_t, const int4*, int, const BatchFrame*, int*, int, long long,
                                 int, bool, cudaStream_t);
}  // namespace rcbf

// das_kernels.cuh — the tiled DAS kernel (one tile per CTA) and its host
// launcher / configuration, instantiated per voxels-per-thread class in
// das_vu1.cu, das_vu2.cu and das_vu4.cu so they compile in parallel.
#pragma once

#include "das_tile.cuh"

namespace rcbf {

template <int VU, int WS, bool CPLX, bool APOD>
__global__ void __launch_bounds__(kDasThreads, 2)
das_tiled_kernel(DasArgs a) {
    using C = DasCfg<VU, WS, CPLX>;
    extern __shared__ __align__(128) unsigned char smem[];
    das_pipe_init<C::COPIES>(smem + C::OFF_BAR, reinterpret_cast<volatile int*>(smem + C::OFF_ABORT));
    DasPipe pipe{0u};   // stage counter of this CTA
    if (!das_unit<VU, WS, CPLX, APOD>(a, blockIdx.x, smem, pipe) && threadIdx.x == 0)
        atomicOr(a.status, kStatusWaitExpired);
}

template <int VU, int WS, bool CPLX, bool APOD>
int das_cfg_one(int* per_sm) {
    using C = DasCfg<VU, WS, CPLX>;
    auto k = das_tiled_kernel<VU, WS, CPLX, APOD>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) != cudaSuccess)
        return check_launch("das: set shared memory");
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kDasThreads, C::SMEM) != cudaSuccess)
        return check_launch("das: occupancy");
    if (per_sm) *per_sm = n;
    return RCBF_OK;
}

template <int VU>
int configure_das_vu(int ws, bool cplx, int* per_sm) {
    int rc;
#define RCBF_CFG(WSV, CP)                                                        \
    if ((rc = das_cfg_one<VU, WSV, CP, false>(per_sm)) != RCBF_OK) return rc;   \
    if ((rc = das_cfg_one<VU, WSV, CP, true>(nullptr)) != RCBF_OK) return rc;
    if (ws == 48) { if (cplx) { RCBF_CFG(48, true) } else { RCBF_CFG(48, false) } }
    else if (ws == 64) { if (cplx) { RCBF_CFG(64, true) } else { RCBF_CFG(64, false) } }
    else { if (cplx) { RCBF_CFG(128, true) } else { RCBF_CFG(128, false) } }
#undef RCBF_CFG
    return RCBF_OK;
}

template <int VU>
int launch_das_vu(const DasArgs& a, int ws, bool cplx, bool apod, cudaStream_t s) {
    const unsigned grid = (unsigned)a.tiles_u * a.tiles_v * a.tiles_w * a.n_split;
#define RCBF_LAUNCH(WSV, CP, AP)                                                                   \
    das_tiled_kernel<VU, WSV, CP, AP><<<grid, kDasThreads, DasCfg<VU, WSV, CP>::SMEM, s>>>(a);    \
    return check_launch("das_tiled_kernel");
#define RCBF_WS(WSV)                                                                               \
    if (cplx) { if (apod) { RCBF_LAUNCH(WSV, true, true) } else { RCBF_LAUNCH(WSV, true, false) } } \
    else { if (apod) { RCBF_LAUNCH(WSV, false, true) } else { RCBF_LAUNCH(WSV, false, false) } }
    if (ws == 48) { RCBF_WS(48) }
    else if (ws == 64) { RCBF_WS(64) }
    else { RCBF_WS(128) }
#undef RCBF_WS
#undef RCBF_LAUNCH
}

}  // namespace rcbf

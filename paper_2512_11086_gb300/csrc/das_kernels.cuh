// das_kernels.cuh — the tiled DAS kernel (one tile per CTA) and its host
// launcher / configuration, instantiated per voxels-per-thread class in
// das_vu1.cu, das_vu2.cu and das_vu4.cu so they compile in parallel.
#pragma once

#include "das_tile.cuh"

namespace rcbf {

template <int VU, int WS, bool CPLX, bool APOD, bool CUBIC>
__global__ void __launch_bounds__(kDasThreads, 2)
das_tiled_kernel(DasArgs a) {
    using C = DasCfg<VU, WS, CPLX, CUBIC>;
    extern __shared__ __align__(128) unsigned char smem[];
    das_pipe_init<C::COPIES>(smem + C::OFF_BAR, reinterpret_cast<volatile int*>(smem + C::OFF_ABORT));
    DasPipe pipe{0u};   // stage counter of this CTA
    if (!das_unit<VU, WS, CPLX, APOD, CUBIC>(a, blockIdx.x, smem, pipe) && threadIdx.x == 0)
        atomicOr(a.status, kStatusWaitExpired);
}

template <int VU, int WS, bool CPLX, bool APOD, bool CUBIC>
int das_cfg_one(int* per_sm) {
    using C = DasCfg<VU, WS, CPLX, CUBIC>;
    auto k = das_tiled_kernel<VU, WS, CPLX, APOD, CUBIC>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) != cudaSuccess)
        return check_launch("das: set shared memory");
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kDasThreads, C::SMEM) != cudaSuccess)
        return check_launch("das: occupancy");
    if (per_sm) *per_sm = n;
    return RCBF_OK;
}

// Complex data with cubic pieces has no 128-interval class (it would not fit
// two CTAs per SM); such windows run the plain form.
template <int VU>
int configure_das_vu(int ws, bool cplx, bool cubic, int* per_sm) {
    int rc;
#define RCBF_CFG(WSV, CP, CU)                                                           \
    if ((rc = das_cfg_one<VU, WSV, CP, false, CU>(per_sm)) != RCBF_OK) return rc;      \
    if ((rc = das_cfg_one<VU, WSV, CP, true, CU>(nullptr)) != RCBF_OK) return rc;
#define RCBF_CFG_WS(WSV)                                                                \
    if (cubic) { if (cplx) { RCBF_CFG(WSV, true, true) } else { RCBF_CFG(WSV, false, true) } } \
    else { if (cplx) { RCBF_CFG(WSV, true, false) } else { RCBF_CFG(WSV, false, false) } }
    if (ws == 48) { RCBF_CFG_WS(48) }
    else if (ws == 64) { RCBF_CFG_WS(64) }
    else {
        if (cubic && cplx) return set_error(RCBF_EUNSUPPORTED, "das: no complex cubic 128-interval class");
        if (cubic) { RCBF_CFG(128, false, true) }
        else { if (cplx) { RCBF_CFG(128, true, false) } else { RCBF_CFG(128, false, false) } }
    }
#undef RCBF_CFG_WS
#undef RCBF_CFG
    return RCBF_OK;
}

template <int VU>
int launch_das_vu(const DasArgs& a, int ws, bool cplx, bool apod, bool cubic, cudaStream_t s) {
    const unsigned grid = (unsigned)a.tiles_u * a.tiles_v * a.tiles_w * a.n_split;
#define RCBF_LAUNCH(WSV, CP, AP, CU)                                                                       \
    das_tiled_kernel<VU, WSV, CP, AP, CU><<<grid, kDasThreads, DasCfg<VU, WSV, CP, CU>::SMEM, s>>>(a);    \
    return check_launch("das_tiled_kernel");
#define RCBF_AP(WSV, CP, CU) \
    if (apod) { RCBF_LAUNCH(WSV, CP, true, CU) } else { RCBF_LAUNCH(WSV, CP, false, CU) }
#define RCBF_WS(WSV)                                                                          \
    if (cubic) { if (cplx) { RCBF_AP(WSV, true, true) } else { RCBF_AP(WSV, false, true) } } \
    else { if (cplx) { RCBF_AP(WSV, true, false) } else { RCBF_AP(WSV, false, false) } }
    if (ws == 48) { RCBF_WS(48) }
    else if (ws == 64) { RCBF_WS(64) }
    else {
        if (cubic && cplx) return set_error(RCBF_EUNSUPPORTED, "das: no complex cubic 128-interval class");
        if (cubic) { RCBF_AP(128, false, true) }
        else { if (cplx) { RCBF_AP(128, true, false) } else { RCBF_AP(128, false, false) } }
    }
#undef RCBF_WS
#undef RCBF_AP
#undef RCBF_LAUNCH
}

}  // namespace rcbf

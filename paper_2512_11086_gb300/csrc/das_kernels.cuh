// das_kernels.cuh — the tiled DAS kernel (one tile per CTA) and its host
// launcher / configuration, instantiated per voxels-per-thread class and
// real / complex data in das_vu{1,2,4}_{real,cplx}.cu, and for the 2D receive
// aperture (one voxel per thread along u) in das2d_{real,cplx}.cu, so they
// compile in parallel.
#pragma once

#include "das_tile.cuh"

namespace rcbf {

template <int VU, int WS, bool CPLX, bool APOD, bool CUBIC, bool IQ, bool D2>
__global__ void __launch_bounds__(kDasThreads, 2)
das_tiled_kernel(DasArgs a) {
    using C = DasCfg<VU, WS, CPLX, CUBIC, D2, APOD, IQ>;
    extern __shared__ __align__(128) unsigned char smem[];
    if (a.vls_split) {
        // a tile across a virtual-line-source focal depth is left to the
        // plain kernel (uniform over the CTA: nothing set up yet)
        const int n_tiles = a.tiles_u * a.tiles_v * a.tiles_w;
        const int tile = (int)(blockIdx.x % (unsigned)n_tiles);
        if (tile_across_focus(a, tile % a.tiles_u, (tile / a.tiles_u) % a.tiles_v, tile / (a.tiles_u * a.tiles_v)))
            return;
    }
    das_pipe_init<C::COPIES>(smem + C::OFF_BAR, reinterpret_cast<volatile int*>(smem + C::OFF_ABORT));
    DasPipe pipe{0u};   // stage counter of this CTA
    if (!das_unit<VU, WS, CPLX, APOD, CUBIC, IQ, D2>(a, blockIdx.x, a.n_split, smem, pipe) && threadIdx.x == 0)
        atomicOr(a.status, kStatusWaitExpired);
}

template <int VU, int WS, bool CPLX, bool APOD, bool CUBIC, bool IQ, bool D2>
int das_cfg_one(int* per_sm) {
    using C = DasCfg<VU, WS, CPLX, CUBIC, D2, APOD, IQ>;
    auto k = das_tiled_kernel<VU, WS, CPLX, APOD, CUBIC, IQ, D2>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) != cudaSuccess)
        return check_launch("das: set shared memory");
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kDasThreads, C::SMEM) != cudaSuccess)
        return check_launch("das: occupancy");
    if (per_sm) *per_sm = n;
    return RCBF_OK;
}

// Instantiated forms: window classes of 48, 64, 96 and 128 intervals; real or
// complex data, with or without weights, linear or cubic pieces, and (complex
// only) IQ beamforming. Complex data with cubic
// pieces has no 128-interval class (it would not fit two CTAs per SM); such
// windows run the plain form. The 2D receive aperture (D2) has no 48 class:
// its windows of up to 48 intervals use the 64 class.
template <int VU, bool CPLX_T, bool D2 = false>
int configure_das_vu(int ws, bool cubic, bool iq, int* per_sm) {
    constexpr bool cplx = CPLX_T;
    int rc;
#define RCBF_CFG(WSV, CP, CU, Q)                                                           \
    if ((rc = das_cfg_one<VU, WSV, CP, false, CU, Q, D2>(per_sm)) != RCBF_OK) return rc;  \
    if ((rc = das_cfg_one<VU, WSV, CP, true, CU, Q, D2>(nullptr)) != RCBF_OK) return rc;
#define RCBF_CFG_C(WSV, CU) \
    if (iq) { RCBF_CFG(WSV, true, CU, true) } else { RCBF_CFG(WSV, true, CU, false) }
#define RCBF_CFG_WS(WSV)                                                                   \
    if constexpr (CPLX_T) { if (cubic) { RCBF_CFG_C(WSV, true) } else { RCBF_CFG_C(WSV, false) } } \
    else { if (cubic) { RCBF_CFG(WSV, false, true, false) } else { RCBF_CFG(WSV, false, false, false) } }
    if (ws == 48) {
        if constexpr (D2) return set_error(RCBF_EUNSUPPORTED, "das: the 2D aperture has no 48-interval class");
        else { RCBF_CFG_WS(48) }
    }
    else if (ws == 64) { RCBF_CFG_WS(64) }
    else if (ws == 96) { RCBF_CFG_WS(96) }
    else {
        if (cubic && cplx) return set_error(RCBF_EUNSUPPORTED, "das: no complex cubic 128-interval class");
        if constexpr (CPLX_T) { RCBF_CFG_C(128, false) }
        else { if (cubic) { RCBF_CFG(128, false, true, false) } else { RCBF_CFG(128, false, false, false) } }
    }
#undef RCBF_CFG_WS
#undef RCBF_CFG_C
#undef RCBF_CFG
    return RCBF_OK;
}

template <int VU, bool CPLX_T, bool D2 = false>
int launch_das_vu(const DasArgs& a, int ws, bool apod, bool cubic, bool iq, cudaStream_t s) {
    constexpr bool cplx = CPLX_T;
    const unsigned grid = (unsigned)a.tiles_u * a.tiles_v * a.tiles_w * a.n_split;
#define RCBF_LAUNCH(WSV, CP, AP, CU, Q)                                                                               \
    das_tiled_kernel<VU, WSV, CP, AP, CU, Q, D2><<<grid, kDasThreads, DasCfg<VU, WSV, CP, CU, D2, AP, Q>::SMEM, s>>>(a); \
    return check_launch("das_tiled_kernel");
#define RCBF_AP(WSV, CP, CU, Q) \
    if (apod) { RCBF_LAUNCH(WSV, CP, true, CU, Q) } else { RCBF_LAUNCH(WSV, CP, false, CU, Q) }
#define RCBF_C(WSV, CU) \
    if (iq) { RCBF_AP(WSV, true, CU, true) } else { RCBF_AP(WSV, true, CU, false) }
#define RCBF_WS(WSV)                                                                                  \
    if constexpr (CPLX_T) { if (cubic) { RCBF_C(WSV, true) } else { RCBF_C(WSV, false) } }            \
    else { if (cubic) { RCBF_AP(WSV, false, true, false) } else { RCBF_AP(WSV, false, false, false) } }
    if (ws == 48) {
        if constexpr (D2) return set_error(RCBF_EUNSUPPORTED, "das: the 2D aperture has no 48-interval class");
        else { RCBF_WS(48) }
    }
    else if (ws == 64) { RCBF_WS(64) }
    else if (ws == 96) { RCBF_WS(96) }
    else {
        if (cubic && cplx) return set_error(RCBF_EUNSUPPORTED, "das: no complex cubic 128-interval class");
        if constexpr (CPLX_T) { RCBF_C(128, false) }
        else { if (cubic) { RCBF_AP(128, false, true, false) } else { RCBF_AP(128, false, false, false) } }
    }
#undef RCBF_WS
#undef RCBF_C
#undef RCBF_AP
#undef RCBF_LAUNCH
}

}  // namespace rcbf

// das_kernels.cuh — the tiled DAS kernel (one tile per CTA) and its host
// launcher / configuration, instantiated per voxels-per-thread class and
// real / complex data in das_vu{1,2,4}_{real,cplx}.cu, and for the 2D receive
// aperture (one voxel per thread along u) in das2d_{real,cplx}.cu, so they
// compile in parallel.
#pragma once

#include "das_tile.cuh"

namespace rcbf {

// Block b < tiles * n_split - tail_units: unit b (tile b % tiles, channel
// split b / tiles), written to partial image b / tiles. The last tail_units
// units run as tail_parts blocks each, the blocks scheduled last: part p of
// unit (tile t, split s) takes the p-th part of the split's channel chunks
// and writes partial image s (p = 0) or n_split + s (tail_parts - 1) + p - 1,
// images that the launcher clears for the tiles without such parts. With one
// split and no tail the unit writes the image itself.
template <int VU, int WS, bool CPLX, bool APOD, bool CUBIC, bool IQ, bool D2>
__global__ void __launch_bounds__(kDasThreads, 2)
das_tiled_kernel(DasArgs a, int tail_units, int tail_parts) {
    using C = DasCfg<VU, WS, CPLX, CUBIC, D2, APOD, IQ>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int n_tiles = a.tiles_u * a.tiles_v * a.tiles_w;
    const int n_bulk = n_tiles * a.n_split - tail_units;
    const int b = (int)blockIdx.x;
    int unit = b, n_split = a.n_split, slice = a.n_split > 1 || tail_units > 0 ? b / n_tiles : -1;
    if (b >= n_bulk) {
        const int u = n_bulk + (b - n_bulk) / tail_parts, p = (b - n_bulk) % tail_parts;
        const int s = u / n_tiles;
        unit = (s * tail_parts + p) * n_tiles + u % n_tiles;
        n_split = a.n_split * tail_parts;
        slice = p == 0 ? s : a.n_split + s * (tail_parts - 1) + p - 1;
    }
    if (a.vls_split) {
        // a tile across a virtual-line-source focal depth is left to the
        // plain kernel (uniform over the CTA: nothing set up yet)
        const int tile = unit % n_tiles;
        if (tile_across_focus(a, tile % a.tiles_u, (tile / a.tiles_u) % a.tiles_v, tile / (a.tiles_u * a.tiles_v)))
            return;
    }
    das_pipe_init<C::COPIES>(smem + C::OFF_BAR, reinterpret_cast<volatile int*>(smem + C::OFF_ABORT));
    DasPipe pipe{0u};   // stage counter of this CTA
    if (!das_unit<VU, WS, CPLX, APOD, CUBIC, IQ, D2>(a, unit, n_split, smem, pipe, slice) && threadIdx.x == 0)
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
int launch_das_vu(const DasArgs& a, int ws, bool apod, bool cubic, bool iq, int tail_units, int tail_parts,
                  cudaStream_t s) {
    constexpr bool cplx = CPLX_T;
    const unsigned grid = (unsigned)a.tiles_u * a.tiles_v * a.tiles_w * a.n_split + tail_units * (tail_parts - 1);
#define RCBF_LAUNCH(WSV, CP, AP, CU, Q)                                                                               \
    das_tiled_kernel<VU, WSV, CP, AP, CU, Q, D2><<<grid, kDasThreads, DasCfg<VU, WSV, CP, CU, D2, AP, Q>::SMEM, s>>>( \
        a, tail_units, tail_parts);                                                                                   \
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

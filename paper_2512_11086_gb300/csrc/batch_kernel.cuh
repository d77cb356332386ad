// batch_kernel.cuh — many frames of uneven size in one persistent launch
// (§METHODS "Data Processing": several pre-uploaded parameter sets;
// §OPTIMIZATIONS "Data Transfer": frames kept in flight).
//
// Work items are decode tiles (128 columns of one frame) and DAS units (one
// voxel tile of one frame, or at a phase's tail one ordered channel part of
// a tile). Resident CTAs take items in list order through an
// atomic ticket. The host orders the list so that the decode of frame f+1
// precedes the DAS of frame f, and a DAS item waits (bounded by a time limit)
// until every decode item of its frame has completed. Every item it waits for
// holds a smaller ticket and never waits itself, so the waits always end
// unless a frame's completion count is made unreachable on purpose (the
// host-side test hook of rcbf_batch_set_wait), in which case the wait expires
// and the status word records it.
//
// Frames are grouped into phases by DAS window class and tile extent (one
// kernel instance each); every phase is one persistent launch with its own
// ticket and its own item list (a frame's decode items sit in its phase).
// Phases after the first are launched as programmatic dependents: every CTA
// allows the next phase to launch as soon as it starts, so the next phase's
// CTAs take the SM slots that this phase's CTAs free at its tail, and every
// CTA waits for the previous phase's completion before it exits, so the
// completion of the last phase implies that of all.
#pragma once

#include "das_tile.cuh"
#include "decode_tile.cuh"

namespace rcbf {

struct alignas(16) BatchFrame {
    DasArgs das;        // DAS of the frame (rf = its decoded buffer, image = its image)
    DecodeArgs dec;     // decode of the frame (valid when n_decode > 0)
    int n_decode;       // decode items of the frame (0: the frame is not encoded)
    int decode_f16;     // 1: split-byte FP16 form, 0: split-byte int8 form
    int order;          // Hadamard order
    int out_dtype;      // RCBF_F16 or RCBF_F32
};

static_assert(sizeof(DasArgs) % 8 == 0, "DasArgs is copied in 8-byte words");
static_assert(alignof(BatchFrame) >= 16 && sizeof(BatchFrame) % 16 == 0, "frame descriptors stay 16-byte aligned");

enum : int { kItemDecode = 0, kItemDas = 1 };
// counter slots: the status word, one completion count per frame, then one
// ticket per phase
enum : int { kBatchStatus = 0, kBatchDone = 1 };

template <int VU, int WS, bool DEC>
struct BatchCfg {
    using D = DasCfg<VU, WS, false>;
    static constexpr int OFF_ARGS = ((D::SMEM + 15) / 16) * 16;
    static constexpr int SMEM_DAS = OFF_ARGS + (int)((sizeof(DasArgs) + 15) / 16) * 16;
    static constexpr int SMEM_DEC = DecodeCfg<256>::STAGE_BYTES;     // one staged tile of the largest order
    static constexpr int SMEM = (DEC && SMEM_DEC > SMEM_DAS) ? SMEM_DEC : SMEM_DAS;
    static_assert(SMEM_DEC <= D::OFF_BAR, "a decode tile must not overlap the DAS mbarriers");
};

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int N, int DT>
__device__ __forceinline__ void batch_decode_n(const BatchFrame& f, long long tile, unsigned char* smem) {
    if (f.decode_f16) decode_one_tile<N, DT, true>(f.dec, tile, smem);
    else decode_one_tile<N, DT, false>(f.dec, tile, smem);
}

template <int DT>
__device__ __forceinline__ void batch_decode_dt(const BatchFrame& f, long long tile, unsigned char* smem) {
    switch (f.order) {
        case 32: batch_decode_n<32, DT>(f, tile, smem); break;
        case 64: batch_decode_n<64, DT>(f, tile, smem); break;
        case 128: batch_decode_n<128, DT>(f, tile, smem); break;
        default: batch_decode_n<256, DT>(f, tile, smem); break;
    }
}

// DEC: the item list may hold decode items (a phase without them runs an
// instance without the decode code)
template <int VU, int WS, bool DEC>
__global__ void __launch_bounds__(kDasThreads, 2)
batch_kernel(const int4* __restrict__ items, int n_items, const BatchFrame* __restrict__ frames,
             int* counters, int ticket_slot, long long wait_ns, int withhold) {
    using C = BatchCfg<VU, WS, DEC>;
    using D = typename C::D;
    extern __shared__ __align__(128) unsigned char smem[];
    DasArgs* s_args = reinterpret_cast<DasArgs*>(smem + C::OFF_ARGS);
    __shared__ int s_item, s_ok;
    // the next phase (independent frames) may launch now; its CTAs start as
    // this phase's CTAs exit (no effect on a launch without dependents)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    das_pipe_init<D::COPIES>(smem + D::OFF_BAR, reinterpret_cast<volatile int*>(smem + D::OFF_ABORT));
    DasPipe pipe{0u};
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counters + ticket_slot, 1);
        __syncthreads();
        const int t = s_item;
        if (t >= n_items) break;
        const int4 it = items[t];
        const BatchFrame& fr = frames[it.y];
        if (DEC && it.x == kItemDecode) {
            if (fr.out_dtype == RCBF_F16) batch_decode_dt<RCBF_F16>(fr, it.z, smem);
            else batch_decode_dt<RCBF_F32>(fr, it.z, smem);
            if (threadIdx.x == 0) {
                __threadfence();                                   // release the decoded tile
                atomicAdd(counters + kBatchDone + it.y, 1);
            }
        } else {
            if (threadIdx.x == 0) {
                int ok = 1;
                const int need = fr.n_decode + (it.y == withhold ? 1 : 0);
                if (need > 0) {
                    const unsigned long long t0 = global_ns();
                    while (ld_acquire(counters + kBatchDone + it.y) < need) {
                        if (global_ns() - t0 > (unsigned long long)wait_ns) {
                            ok = 0;
                            atomicOr(counters + kBatchStatus, kStatusWaitExpired);
                            break;
                        }
                        __nanosleep(200);
                    }
                }
                s_ok = ok;
            }
            __syncthreads();
            if (s_ok) {
                // the frame's DAS arguments, then order the acquired decode
                // output before the TMA (async proxy) reads of it
                const long long* src = reinterpret_cast<const long long*>(&fr.das);
                long long* dst = reinterpret_cast<long long*>(s_args);
                for (int q = threadIdx.x; q < (int)(sizeof(DasArgs) / 8); q += kDasThreads) dst[q] = src[q];
                asm volatile("fence.proxy.async.global;" ::: "memory");
                __syncthreads();
                const bool ok = das_unit<VU, WS, false, false>(*s_args, it.z, it.w, smem, pipe);
                if (__syncthreads_or(!ok)) {
                    if (threadIdx.x == 0) atomicOr(counters + kBatchStatus, kStatusWaitExpired);
                    break;
                }
            }
        }
        __syncthreads();   // s_item, s_args and the staging buffers are reused
    }
    // completion of this phase implies completion of the previous one (a
    // no-op for a launch that is not a programmatic dependent)
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <int VU, int WS, bool DEC>
int batch_configure(int* per_sm, size_t* smem) {
    using C = BatchCfg<VU, WS, DEC>;
    auto k = batch_kernel<VU, WS, DEC>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) != cudaSuccess)
        return check_launch("batch: set shared memory");
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kDasThreads, C::SMEM) != cudaSuccess)
        return check_launch("batch: occupancy");
    *per_sm = n < 1 ? 1 : n;
    *smem = C::SMEM;
    return RCBF_OK;
}

template <int VU, int WS>
int batch_configure_ws(bool dec, int* per_sm, size_t* smem) {
    return dec ? batch_configure<VU, WS, true>(per_sm, smem) : batch_configure<VU, WS, false>(per_sm, smem);
}

template <int VU>
int batch_configure_vu(int ws, bool dec, int* per_sm, size_t* smem) {
    if (ws == 48) return batch_configure_ws<VU, 48>(dec, per_sm, smem);
    if (ws == 64) return batch_configure_ws<VU, 64>(dec, per_sm, smem);
    if (ws == 96) return batch_configure_ws<VU, 96>(dec, per_sm, smem);
    return batch_configure_ws<VU, 128>(dec, per_sm, smem);
}

template <int VU, int WS, bool DEC>
int batch_launch(unsigned grid, size_t smem, const int4* items, int n_items, const BatchFrame* frames, int* counters,
                 int ticket_slot, long long wait_ns, int withhold, bool dependent, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kDasThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = dependent ? 1 : 0;
    if (cudaLaunchKernelEx(&cfg, batch_kernel<VU, WS, DEC>, items, n_items, frames, counters, ticket_slot, wait_ns,
                           withhold) != cudaSuccess)
        return check_launch("batch_kernel launch");
    return check_launch("batch_kernel");
}

template <int VU, int WS>
int batch_launch_ws(bool dec, unsigned grid, size_t smem, const int4* items, int n_items, const BatchFrame* frames,
                    int* counters, int ticket_slot, long long wait_ns, int withhold, bool dependent, cudaStream_t s) {
    return dec ? batch_launch<VU, WS, true>(grid, smem, items, n_items, frames, counters, ticket_slot, wait_ns,
                                            withhold, dependent, s)
               : batch_launch<VU, WS, false>(grid, smem, items, n_items, frames, counters, ticket_slot, wait_ns,
                                             withhold, dependent, s);
}

template <int VU>
int batch_launch_vu(int ws, bool dec, unsigned grid, size_t smem, const int4* items, int n_items,
                    const BatchFrame* frames, int* counters, int ticket_slot, long long wait_ns, int withhold,
                    bool dependent, cudaStream_t s) {
    if (ws == 48)
        return batch_launch_ws<VU, 48>(dec, grid, smem, items, n_items, frames, counters, ticket_slot, wait_ns,
                                       withhold, dependent, s);
    if (ws == 64)
        return batch_launch_ws<VU, 64>(dec, grid, smem, items, n_items, frames, counters, ticket_slot, wait_ns,
                                       withhold, dependent, s);
    if (ws == 96)
        return batch_launch_ws<VU, 96>(dec, grid, smem, items, n_items, frames, counters, ticket_slot, wait_ns,
                                       withhold, dependent, s);
    return batch_launch_ws<VU, 128>(dec, grid, smem, items, n_items, frames, counters, ticket_slot, wait_ns,
                                    withhold, dependent, s);
}

}  // namespace rcbf

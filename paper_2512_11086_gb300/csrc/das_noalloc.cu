// das_noalloc.cu — delay-and-sum for callers that cannot allocate device
// memory.
//
// Who needs this: code that runs where cudaMalloc / cudaFree are off limits —
// for example under a host framework that owns every device allocation
// through its own pool, or in a real-time acquisition loop that forbids
// allocation after start-up.
// rcbf_plan allocates (decode tables, the status word and the partial images
// of the channel-split DAS), so such callers cannot use it. rcbf_das_noalloc
// takes the parameter block directly and runs the same DAS kernels; the one
// piece of scratch they need, the partial images of the channel split (plus
// the kernels' status word), lives in a file-scope __device__ array of fixed
// size that the module loader places on every device that loads the library
// and that stays there until the process exits.
#include <algorithm>
#include <mutex>
#include <string>

#include "internal.cuh"

namespace rcbf {
namespace {

// 16 MiB of scratch: 64 floats for the status word, the rest for partial
// images (channel splits x planes x voxels).
constexpr size_t kNoAllocScratchFloats = size_t(4) << 20;
constexpr size_t kNoAllocHeaderFloats = 64;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

std::mutex g_noalloc_mutex;
float* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device. In host code the
// array's name is only a stand-in, so its address must come from
// cudaGetSymbolAddress, once per device, with that device current.
int noalloc_scratch(float** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return check_launch("rcbf_das_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(RCBF_EUNSUPPORTED, "rcbf_das_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return set_error(RCBF_ECUDA, std::string("rcbf_das_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_noalloc_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return RCBF_OK;
}

}  // namespace
}  // namespace rcbf

using namespace rcbf;

extern "C" int rcbf_das_noalloc(const rcbf_params* params, const void* decoded, const float* apod, float c,
                                float* image, void* stream) {
    int rc = plan_validate(params);
    if (rc != RCBF_OK) return rc;
    if (params->tx_wave == RCBF_TX_PLANE)
        return set_error(RCBF_EUNSUPPORTED, "rcbf_das_noalloc: plane-wave directions need a plan (device table)");
    if (!decoded || !image) return set_error(RCBF_EINVAL, "rcbf_das_noalloc: NULL buffer");
    if ((reinterpret_cast<uintptr_t>(decoded) & 15u) || (reinterpret_cast<uintptr_t>(image) & 3u) ||
        (apod && (reinterpret_cast<uintptr_t>(apod) & 3u)))
        return set_error(RCBF_EINVAL, "rcbf_das_noalloc: decoded must be 16-byte aligned, image and apod 4-byte aligned");

    PlanHost h{};
    h.p = *params;
    h.p.decode_matrix = nullptr;
    h.p.demod_taps = nullptr;
    h.p.demod_taps_imag = nullptr;
    h.p.tx_angles = nullptr;
    plan_geometry(h);
    if (h.p.das_variant == RCBF_DAS_TILED && !h.tiled_ok)
        return set_error(RCBF_EUNSUPPORTED, "rcbf_das_noalloc: the tiled form needs n_ch % 8 == 0, n_tx % 8 == 0 "
                                            "(4 for complex) and an image axis parallel to the transmit elements");
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&h.n_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return check_launch("rcbf_das_noalloc: device attribute");

    const double cc = c > 0.f ? (double)c : h.p.c;
    DasArgs a;
    std::string why;
    const bool fits = das_prepare(h, cc, &a, &why) == RCBF_OK;
    const bool tiled = h.p.das_variant == RCBF_DAS_TILED && fits;
    if (tiled) {
        if ((rc = configure_das(h)) != RCBF_OK) return rc;
        const int cls = das_class_index(a.W, h.p.acq_kind == RCBF_HERCULES_2D);
        const size_t planes = h.p.decoded_dtype == RCBF_CF32 ? 2 : 1;
        // the tail parts' extra partial images only where the scratch holds them
        if ((size_t)das_slices(h, cls) * planes * (size_t)a.image_plane > kNoAllocScratchFloats - kNoAllocHeaderFloats) {
            h.tail_parts[cls] = 1;
            h.tail_units[cls] = 0;
        }
        const int split = das_slices(h, cls);
        const size_t need = split > 1 ? (size_t)split * planes * (size_t)a.image_plane : 0;
        if (need > kNoAllocScratchFloats - kNoAllocHeaderFloats)
            return set_error(RCBF_EINVAL, "rcbf_das_noalloc: the channel-split partial images need " +
                                              std::to_string(need * 4) + " bytes, more than the " +
                                              std::to_string((kNoAllocScratchFloats - kNoAllocHeaderFloats) * 4) +
                                              "-byte static scratch; use rcbf_plan / rcbf_das");
    }

    float* scratch = nullptr;
    if ((rc = noalloc_scratch(&scratch)) != RCBF_OK) return rc;
    int* status = reinterpret_cast<int*>(scratch);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    a.rf = decoded;
    a.apod = apod;
    a.image = image;
    a.status = status;
    // the status word must start at zero; the partial images are fully
    // rewritten by every call before they are read
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess)
        return check_launch("rcbf_das_noalloc: clear status");
    if (!tiled) return launch_das_plain(h, a, s);
    h.d_partial = scratch + kNoAllocHeaderFloats;
    if (!h.vls_split) return launch_das(h, a, s);
    a.vls_split = 1;                 // tiles across a VLS focal depth: the plain form
    rc = launch_das(h, a, s);
    return rc != RCBF_OK ? rc : launch_das_plain(h, a, s);
}

extern "C" int rcbf_das_noalloc_status(void* stream) {
    float* scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc != RCBF_OK) return rc;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return check_launch("rcbf_das_noalloc_status: synchronize");
    int st = 0;
    if (cudaMemcpy(&st, scratch, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return check_launch("rcbf_das_noalloc_status: read status");
    if (st) return set_error(RCBF_ETIMEOUT, "rcbf_das_noalloc_status: a bounded device wait of the last "
                                            "rcbf_das_noalloc call on this device expired; its image is incomplete");
    return RCBF_OK;
}

// batch.cu — host side of the batched stream (rcbf_batch_*): one persistent
// launch decodes and beamforms many frames of uneven size (§METHODS "Data
// Processing": several pre-uploaded parameter sets, each frame with its own
// acquisition and image description).
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "batch_kernel.cuh"

namespace rcbf {
template <int VU> int batch_configure_vu(int ws, bool dec, int* per_sm, size_t* smem);
template <int VU> int batch_launch_vu(int ws, bool dec, unsigned grid, size_t smem, const int4* items, int n_items,
                                      const BatchFrame* frames, int* counters, int ticket_slot, long long wait_ns,
                                      int withhold, bool dependent, cudaStream_t s);

// one persistent launch: the frames of one (window class, tile extent) group
struct BatchPhase {
    int vu = 2;
    int ws = 48;
    bool dec = false;        // the phase holds decode items
    int item0 = 0;           // first item of the phase in the batch's item list
    int n_items = 0;
    unsigned grid = 1;
    size_t smem = 0;
};
}  // namespace rcbf

struct rcbf_batch_s {
    int n_frames = 0;
    int n_items = 0;
    std::vector<rcbf::BatchPhase> phases;
    long long n_counters = 0;            // status, per-frame decode counts, per-phase tickets, tile flags
    long long wait_ns = 1000000000LL;   // bounded wait of a DAS item on its frame's decode
    int withhold = -1;                  // test hook: a frame whose decode never completes
    int4* d_items = nullptr;
    rcbf::BatchFrame* d_frames = nullptr;
    int* d_counters = nullptr;
    std::vector<rcbf::TcJob> tc_jobs;   // frames decoded by the tcgen05 kernel ahead of the persistent launch
};

using namespace rcbf;

namespace {

int batch_fail(rcbf_batch_s* b, int code, const std::string& msg) {
    rcbf_batch_destroy(b);
    return set_error(code, msg);
}

int class_of(int W) { return W <= 48 ? 48 : W <= 64 ? 64 : W <= 96 ? 96 : 128; }

// tail of a phase: the last kTailQuarters / 4 waves of the grid (tiles in
// ticket order) are split into up to kTailParts ordered channel parts.
// Measured on four B-scan frames (2048 tiles, 6.7 waves of 304 CTAs): every
// tile in halves 8.65 ms per step, whole tiles 8.92 ms; whole tiles with a
// tail of 1/2, 3/4, 1, 3/2 or 2 waves in halves 8.534, 8.534, 8.546, 8.551,
// 8.583 ms; 1/2 or 3/4 of a wave in quarters 8.590, 8.598 ms.
constexpr long long kTailQuarters = 3;
constexpr int kTailParts = 2;

}  // namespace

namespace rcbf {
int* batch_status_word(rcbf_batch_t batch) { return batch ? batch->d_counters + kBatchStatus : nullptr; }
}  // namespace rcbf

extern "C" {

int rcbf_batch_create(const rcbf_plan_t* plans, uint32_t n_frames, const int16_t* const* rf,
                      void* const* decoded, float* const* images, rcbf_batch_t* out_batch) {
    if (!out_batch) return set_error(RCBF_EINVAL, "rcbf_batch_create: out_batch is NULL");
    *out_batch = nullptr;
    if (!plans || !decoded || !images || n_frames == 0)
        return set_error(RCBF_EINVAL, "rcbf_batch_create: NULL array or zero frames");
    std::vector<BatchFrame> frames(n_frames);
    std::vector<TcJob> tc_jobs;
    std::vector<int> frame_ws(n_frames), frame_vu(n_frames);
    for (uint32_t f = 0; f < n_frames; ++f) {
        const rcbf_plan_t p = plans[f];
        const std::string at = "rcbf_batch_create: frame " + std::to_string(f) + ": ";
        if (!p) return set_error(RCBF_EINVAL, at + "NULL plan");
        const PlanHost& h = p->h;
        if (h.p.decoded_dtype != RCBF_F16 && h.p.decoded_dtype != RCBF_F32)
            return set_error(RCBF_EUNSUPPORTED, at + "decoded_dtype must be RCBF_F16 or RCBF_F32");
        if (h.p.das_variant != RCBF_DAS_TILED || !h.tiled_ok)
            return set_error(RCBF_EUNSUPPORTED, at + "the plan must use the tiled DAS");
        if (h.p.f_number > 0.0) return set_error(RCBF_EUNSUPPORTED, at + "batch frames use no F# window");
        if (h.p.interp != RCBF_LINEAR) return set_error(RCBF_EUNSUPPORTED, at + "batch frames use linear interpolation");
        if (h.p.iq_freq > 0.0 || h.p.demod_decimation)
            return set_error(RCBF_EUNSUPPORTED, at + "batch frames are RF frames without demodulation");
        if (h.p.acq_kind == RCBF_HERCULES_2D)
            return set_error(RCBF_EUNSUPPORTED, at + "batch frames use separable (row-column) delays");
        if (h.vls_split)
            return set_error(RCBF_EUNSUPPORTED, at + "a virtual-line-source focal plane inside the image needs "
                                                     "the plain form for the tiles across it");
        if (!decoded[f] || !images[f] || (h.p.hadamard_order && (!rf || !rf[f])))
            return set_error(RCBF_EINVAL, at + "NULL buffer");
        if ((reinterpret_cast<uintptr_t>(decoded[f]) & 15u) || (reinterpret_cast<uintptr_t>(images[f]) & 3u) ||
            (h.p.hadamard_order && (reinterpret_cast<uintptr_t>(rf[f]) & 15u)))
            return set_error(RCBF_EINVAL, at + "misaligned buffer");
        BatchFrame& fr = frames[f];
        std::memset(&fr, 0, sizeof(fr));
        std::string why;
        if (das_prepare(h, h.p.c, &fr.das, &why) != RCBF_OK) return set_error(RCBF_EUNSUPPORTED, at + why);
        fr.das.rf = decoded[f];
        fr.das.image = images[f];
        fr.das.apod = nullptr;
        fr.das.n_split = 1;
        fr.das.partial = nullptr;
        fr.das.withhold = 0;            // the plan's DAS test hook does not apply to a batch
        fr.das.wait_ns = kWaitNs;
        frame_ws[f] = class_of(fr.das.W);
        frame_vu[f] = h.das.bu / 32;
        fr.out_dtype = (int)h.p.decoded_dtype;
        fr.order = (int)h.p.n_tx;
        if (h.p.hadamard_order && h.p.decode_variant == RCBF_DECODE_TC) {
            // decoded by its own tcgen05 launch ahead of the persistent kernel
            // (stream order makes its output visible to the frame's DAS items)
            TcJob job;
            if (decode_tc_prepare(h, (int)h.p.decoded_dtype, rf[f], decoded[f], &job) != RCBF_OK)
                return set_error(RCBF_EUNSUPPORTED, at + rcbf_last_error());
            tc_jobs.push_back(job);
        } else if (h.p.hadamard_order) {
            fr.n_decode = (int)(((long long)h.p.n_ch * h.p.n_samples + kDecodeCols - 1) / kDecodeCols);
            fr.decode_f16 = h.p.decode_variant == RCBF_DECODE_MMA_F16 ? 1 : 0;
            DecodeArgs& d = fr.dec;
            d.rf = rf[f];
            d.out = decoded[f];
            d.afrag = h.d_afrag;
            d.afrag16 = h.d_afrag16;
            d.hsum = h.d_hsum;
            d.hmat = h.d_hmat;
            d.n_cols = (long long)h.p.n_ch * h.p.n_samples;
            d.n = (int)h.p.n_tx;
            d.dtype = (int)h.p.decoded_dtype;
            d.inv_n = 1.0f / (float)h.p.n_tx;
            if (!h.d_afrag) return set_error(RCBF_EUNSUPPORTED, at + "the tensor-core decode needs n_tx in {32, 64, 128, 256}");
        }
    }
    // phases: frames grouped by (window class, tile extent along u), in order
    // of first appearance; within a phase the frames keep their order and the
    // decode of frame f+1 precedes the DAS of frame f
    std::vector<std::pair<int, int>> keys;
    std::vector<std::vector<int>> members;
    for (uint32_t f = 0; f < n_frames; ++f) {
        const std::pair<int, int> key(frame_ws[f], frame_vu[f]);
        size_t p = 0;
        while (p < keys.size() && keys[p] != key) ++p;
        if (p == keys.size()) {
            keys.push_back(key);
            members.emplace_back();
        }
        members[p].push_back((int)f);
    }
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    std::vector<int4> items;
    std::vector<BatchPhase> phases;
    std::vector<long long> flag_off(n_frames, -1);      // tile flags of frames with a channel split
    long long n_flags = 0;
    for (size_t p = 0; p < keys.size(); ++p) {
        BatchPhase ph;
        ph.ws = keys[p].first;
        ph.vu = keys[p].second;
        const std::vector<int>& fs = members[p];
        for (int f : fs) ph.dec = ph.dec || frames[f].n_decode > 0;
        int per_sm = 1, rc;
        switch (ph.vu) {
            case 1: rc = batch_configure_vu<1>(ph.ws, ph.dec, &per_sm, &ph.smem); break;
            case 2: rc = batch_configure_vu<2>(ph.ws, ph.dec, &per_sm, &ph.smem); break;
            default: rc = batch_configure_vu<4>(ph.ws, ph.dec, &per_sm, &ph.smem); break;
        }
        if (rc != RCBF_OK) return rc;
        const int slots = sms * per_sm;
        // channel split of the phase's DAS units. Whole tiles carry the bulk
        // of a phase (every split repeats the tile set-up and the pipeline
        // fill), but a wave of whole tiles leaves part of the grid idle at the
        // end of the phase. So the last tiles in ticket order are split into
        // ordered channel parts (summed into the image in part order): the
        // CTAs that run out of whole tiles first pick up the parts, and the
        // phase ends within about one part's time.
        long long tiles_all = 0;
        for (int f : fs) {
            const DasArgs& a = frames[f].das;
            tiles_all += (long long)a.tiles_u * a.tiles_v * a.tiles_w;
        }
        const long long tail = std::min(tiles_all, kTailQuarters * slots / 4);
        long long tile_seq = 0;               // tiles of the phase before the current one
        ph.item0 = (int)items.size();
        auto push_decode = [&](int f) {
            for (int t = 0; t < frames[f].n_decode; ++t) items.push_back(make_int4(kItemDecode, f, t, 0));
        };
        auto push_das = [&](int f) {
            DasArgs& a = frames[f].das;
            const int tiles = a.tiles_u * a.tiles_v * a.tiles_w;
            const int chunks = a.n_ch / 8;
            int parts = 1;
            while (parts * 2 <= kTailParts && chunks % (parts * 2) == 0) parts *= 2;
            a.n_split = 1;
            for (int t = 0; t < tiles; ++t, ++tile_seq) {
                const int q = tile_seq >= tiles_all - tail ? parts : 1;
                if (q > 1 && flag_off[f] < 0) {
                    flag_off[f] = n_flags;
                    n_flags += tiles;
                }
                // the parts of a tile take consecutive tickets
                for (int sp = 0; sp < q; ++sp) items.push_back(make_int4(kItemDas, f, sp * tiles + t, q));
            }
        };
        push_decode(fs[0]);
        for (size_t k = 0; k < fs.size(); ++k) {
            if (k + 1 < fs.size()) push_decode(fs[k + 1]);
            push_das(fs[k]);
        }
        ph.n_items = (int)items.size() - ph.item0;
        ph.grid = (unsigned)std::min<long long>((long long)slots, (long long)ph.n_items);
        phases.push_back(ph);
    }
    const long long flags0 = kBatchDone + (long long)n_frames + (long long)phases.size();
    const long long n_counters = flags0 + n_flags;

    rcbf_batch_s* b = new rcbf_batch_s();
    b->tc_jobs = tc_jobs;
    b->n_frames = (int)n_frames;
    b->n_items = (int)items.size();
    b->n_counters = n_counters;
    if (cudaMalloc(&b->d_items, items.size() * sizeof(int4)) != cudaSuccess ||
        cudaMalloc(&b->d_frames, frames.size() * sizeof(BatchFrame)) != cudaSuccess ||
        cudaMalloc(&b->d_counters, n_counters * sizeof(int)) != cudaSuccess)
        return batch_fail(b, RCBF_ENOMEM, "rcbf_batch_create: cudaMalloc");
    for (uint32_t f = 0; f < n_frames; ++f) {
        frames[f].das.status = b->d_counters + kBatchStatus;
        frames[f].das.tile_flags = flag_off[f] >= 0 ? b->d_counters + flags0 + flag_off[f] : nullptr;
    }
    if (cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_frames, frames.data(), frames.size() * sizeof(BatchFrame), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->d_counters, 0, n_counters * sizeof(int)) != cudaSuccess)
        return batch_fail(b, RCBF_ECUDA, "rcbf_batch_create: copy work list");
    b->phases = phases;
    *out_batch = b;
    return RCBF_OK;
}

int rcbf_batch_run(rcbf_batch_t batch, void* stream) {
    if (!batch) return set_error(RCBF_EINVAL, "rcbf_batch_run: batch is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(batch->d_counters, 0, batch->n_counters * sizeof(int), s) != cudaSuccess)
        return check_launch("rcbf_batch_run: reset counters");
    for (const TcJob& job : batch->tc_jobs) {
        const int rc = decode_tc_run(job, batch->d_counters + kBatchStatus, batch->wait_ns, s);
        if (rc != RCBF_OK) return rc;
    }
    for (size_t p = 0; p < batch->phases.size(); ++p) {
        const BatchPhase& ph = batch->phases[p];
        const int4* items = batch->d_items + ph.item0;
        const int slot = kBatchDone + batch->n_frames + (int)p;
        const bool dependent = p > 0;
        int rc;
        switch (ph.vu) {
            case 1: rc = batch_launch_vu<1>(ph.ws, ph.dec, ph.grid, ph.smem, items, ph.n_items, batch->d_frames,
                                            batch->d_counters, slot, batch->wait_ns, batch->withhold, dependent, s);
                break;
            case 2: rc = batch_launch_vu<2>(ph.ws, ph.dec, ph.grid, ph.smem, items, ph.n_items, batch->d_frames,
                                            batch->d_counters, slot, batch->wait_ns, batch->withhold, dependent, s);
                break;
            default: rc = batch_launch_vu<4>(ph.ws, ph.dec, ph.grid, ph.smem, items, ph.n_items, batch->d_frames,
                                             batch->d_counters, slot, batch->wait_ns, batch->withhold, dependent, s);
                break;
        }
        if (rc != RCBF_OK) return rc;
    }
    return RCBF_OK;
}

int rcbf_batch_status(rcbf_batch_t batch, void* stream) {
    if (!batch) return set_error(RCBF_EINVAL, "rcbf_batch_status: batch is NULL");
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return check_launch("rcbf_batch_status: synchronize");
    int st = 0;
    if (cudaMemcpy(&st, batch->d_counters + kBatchStatus, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return check_launch("rcbf_batch_status: read status");
    if (st) return set_error(RCBF_ETIMEOUT, "rcbf_batch_status: a bounded device wait expired");
    return RCBF_OK;
}

int rcbf_batch_set_wait(rcbf_batch_t batch, uint64_t wait_ns, int32_t withhold_frame) {
    if (!batch) return set_error(RCBF_EINVAL, "rcbf_batch_set_wait: batch is NULL");
    if (wait_ns == 0 || withhold_frame < -1 || withhold_frame >= batch->n_frames)
        return set_error(RCBF_EINVAL, "rcbf_batch_set_wait: wait_ns must be > 0 and withhold_frame in [-1, n_frames)");
    batch->wait_ns = (long long)std::min<uint64_t>(wait_ns, (uint64_t)10000000000ULL);
    batch->withhold = withhold_frame;
    return RCBF_OK;
}

void rcbf_batch_destroy(rcbf_batch_t batch) {
    if (!batch) return;
    if (batch->d_items) cudaFree(batch->d_items);
    if (batch->d_frames) cudaFree(batch->d_frames);
    if (batch->d_counters) cudaFree(batch->d_counters);
    delete batch;
}

}  // extern "C"

// pipeline.cu — the upload ring (§OPTIMIZATIONS "Data Transfer": frames kept
// in flight so that uploads never stall the GPU).
//
// n_slots sets of device buffers, each bound to its own batch and captured
// once as a CUDA graph. A step through slot k:
//   h2d stream:     wait(slot k done) ; copy inputs ; record copied
//   compute stream: wait(copied) ; graph ; record computed
//   d2h stream:     wait(computed) ; copy images ; record done
// Three streams, so the uploads of step s+1 run while step s computes and the
// read-back of step s-1 drains. The host waits for a slot's previous step only
// when it reuses the slot, and then folds that step's batch status (copied
// to pinned host memory behind the images, so no synchronous copy is needed)
// into the pipeline's sticky status.
#include <string>
#include <vector>

#include "internal.cuh"

using namespace rcbf;

namespace {

struct Slot {
    std::vector<void*> in;          // per frame: encoded RF (int16) or decoded input
    std::vector<void*> dec;         // per frame: decoded buffer
    std::vector<float*> img;        // per frame: image
    rcbf_batch_t batch = nullptr;
    cudaGraphExec_t graph = nullptr;
    cudaEvent_t copied = nullptr, computed = nullptr, done = nullptr;
    int* h_status = nullptr;        // pinned: the batch status word of the slot's last step
    bool busy = false;
};

size_t dtype_bytes(uint32_t dt) { return dt == RCBF_F16 ? 2 : 4; }

}  // namespace

struct rcbf_pipeline_s {
    std::vector<rcbf_plan_t> plans;
    std::vector<size_t> in_bytes, img_bytes;
    std::vector<bool> encoded;
    std::vector<Slot> slots;
    cudaStream_t h2d = nullptr, compute = nullptr, d2h = nullptr;
    int next = 0;
    int status = 0;
};

namespace {

// the slot's done event has completed: its status copy has landed
int fold_status(rcbf_pipeline_s* p, Slot& s) {
    p->status |= *reinterpret_cast<volatile int*>(s.h_status);
    s.busy = false;
    return RCBF_OK;
}

int pipeline_fail(rcbf_pipeline_s* p, int code, const std::string& msg) {
    rcbf_pipeline_destroy(p);
    return set_error(code, msg);
}

}  // namespace

extern "C" {

int rcbf_pipeline_create(const rcbf_plan_t* plans, uint32_t n_frames, uint32_t n_slots,
                         rcbf_pipeline_t* out_pipeline) {
    if (!out_pipeline) return set_error(RCBF_EINVAL, "rcbf_pipeline_create: out_pipeline is NULL");
    *out_pipeline = nullptr;
    if (!plans || n_frames == 0) return set_error(RCBF_EINVAL, "rcbf_pipeline_create: no frames");
    if (n_slots < 2 || n_slots > 8) return set_error(RCBF_EINVAL, "rcbf_pipeline_create: n_slots must be in [2, 8]");
    for (uint32_t f = 0; f < n_frames; ++f)
        if (!plans[f]) return set_error(RCBF_EINVAL, "rcbf_pipeline_create: NULL plan");
    rcbf_pipeline_s* p = new rcbf_pipeline_s();
    p->plans.assign(plans, plans + n_frames);
    for (uint32_t f = 0; f < n_frames; ++f) {
        const rcbf_params& q = plans[f]->h.p;
        const size_t samples = (size_t)q.n_tx * q.n_ch * q.n_samples;
        const bool enc = q.hadamard_order != 0;
        p->encoded.push_back(enc);
        p->in_bytes.push_back(samples * (enc ? sizeof(int16_t) : dtype_bytes(q.decoded_dtype)));
        p->img_bytes.push_back((size_t)q.out_dims[0] * q.out_dims[1] * q.out_dims[2] * sizeof(float));
    }
    if (cudaStreamCreateWithFlags(&p->h2d, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->compute, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->d2h, cudaStreamNonBlocking) != cudaSuccess)
        return pipeline_fail(p, RCBF_ECUDA, "rcbf_pipeline_create: streams");
    p->slots.resize(n_slots);
    for (Slot& s : p->slots) {
        std::vector<const int16_t*> rf(n_frames, nullptr);
        for (uint32_t f = 0; f < n_frames; ++f) {
            const rcbf_params& q = plans[f]->h.p;
            const size_t samples = (size_t)q.n_tx * q.n_ch * q.n_samples;
            void* dec = nullptr;
            float* img = nullptr;
            if (cudaMalloc(&dec, samples * dtype_bytes(q.decoded_dtype)) != cudaSuccess ||
                cudaMalloc(reinterpret_cast<void**>(&img), p->img_bytes[f]) != cudaSuccess) {
                if (dec) cudaFree(dec);
                return pipeline_fail(p, RCBF_ENOMEM, "rcbf_pipeline_create: cudaMalloc slot buffers");
            }
            s.dec.push_back(dec);
            s.img.push_back(img);
            void* in = dec;
            if (p->encoded[f]) {
                in = nullptr;
                if (cudaMalloc(&in, p->in_bytes[f]) != cudaSuccess)
                    return pipeline_fail(p, RCBF_ENOMEM, "rcbf_pipeline_create: cudaMalloc slot RF");
                rf[f] = static_cast<const int16_t*>(in);
            }
            s.in.push_back(in);
        }
        const int rc = rcbf_batch_create(plans, n_frames, rf.data(), s.dec.data(), s.img.data(), &s.batch);
        if (rc != RCBF_OK) {
            const std::string m = rcbf_last_error();
            return pipeline_fail(p, rc, m);
        }
        if (cudaEventCreateWithFlags(&s.copied, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.computed, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess)
            return pipeline_fail(p, RCBF_ECUDA, "rcbf_pipeline_create: events");
        if (cudaHostAlloc(reinterpret_cast<void**>(&s.h_status), sizeof(int), cudaHostAllocDefault) != cudaSuccess)
            return pipeline_fail(p, RCBF_ENOMEM, "rcbf_pipeline_create: pinned status word");
        *s.h_status = 0;
        // capture the batch launch (a counter reset and one persistent kernel)
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(p->compute, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return pipeline_fail(p, RCBF_ECUDA, "rcbf_pipeline_create: begin capture");
        const int rr = rcbf_batch_run(s.batch, p->compute);
        const cudaError_t ec = cudaStreamEndCapture(p->compute, &g);
        if (rr != RCBF_OK || ec != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            return pipeline_fail(p, RCBF_ECUDA, "rcbf_pipeline_create: capture of the batch launch");
        }
        const cudaError_t ei = cudaGraphInstantiate(&s.graph, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) return pipeline_fail(p, RCBF_ECUDA, "rcbf_pipeline_create: instantiate graph");
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return pipeline_fail(p, RCBF_ECUDA, "rcbf_pipeline_create: synchronise");
    *out_pipeline = p;
    return RCBF_OK;
}

int rcbf_pipeline_submit(rcbf_pipeline_t p, const void* const* host_inputs, float* const* host_images) {
    if (!p) return set_error(RCBF_EINVAL, "rcbf_pipeline_submit: pipeline is NULL");
    if (!host_inputs || !host_images) return set_error(RCBF_EINVAL, "rcbf_pipeline_submit: NULL array");
    const size_t n = p->plans.size();
    for (size_t f = 0; f < n; ++f)
        if (!host_inputs[f] || !host_images[f]) return set_error(RCBF_EINVAL, "rcbf_pipeline_submit: NULL host buffer");
    Slot& s = p->slots[p->next];
    if (s.busy) {
        if (cudaEventSynchronize(s.done) != cudaSuccess) return check_launch("rcbf_pipeline_submit: wait for the slot");
        const int rc = fold_status(p, s);
        if (rc != RCBF_OK) return rc;
    }
    for (size_t f = 0; f < n; ++f)
        if (cudaMemcpyAsync(s.in[f], host_inputs[f], p->in_bytes[f], cudaMemcpyHostToDevice, p->h2d) != cudaSuccess)
            return check_launch("rcbf_pipeline_submit: upload");
    if (cudaEventRecord(s.copied, p->h2d) != cudaSuccess ||
        cudaStreamWaitEvent(p->compute, s.copied, 0) != cudaSuccess ||
        cudaGraphLaunch(s.graph, p->compute) != cudaSuccess ||
        cudaEventRecord(s.computed, p->compute) != cudaSuccess ||
        cudaStreamWaitEvent(p->d2h, s.computed, 0) != cudaSuccess)
        return check_launch("rcbf_pipeline_submit: enqueue");
    for (size_t f = 0; f < n; ++f)
        if (cudaMemcpyAsync(host_images[f], s.img[f], p->img_bytes[f], cudaMemcpyDeviceToHost, p->d2h) != cudaSuccess)
            return check_launch("rcbf_pipeline_submit: read-back");
    if (cudaMemcpyAsync(s.h_status, batch_status_word(s.batch), sizeof(int), cudaMemcpyDeviceToHost, p->d2h) !=
            cudaSuccess ||
        cudaEventRecord(s.done, p->d2h) != cudaSuccess)
        return check_launch("rcbf_pipeline_submit: record");
    s.busy = true;
    p->next = (p->next + 1) % (int)p->slots.size();
    return RCBF_OK;
}

int rcbf_pipeline_wait(rcbf_pipeline_t p) {
    if (!p) return set_error(RCBF_EINVAL, "rcbf_pipeline_wait: pipeline is NULL");
    if (cudaStreamSynchronize(p->d2h) != cudaSuccess) return check_launch("rcbf_pipeline_wait: synchronise");
    for (Slot& s : p->slots)
        if (s.busy) {
            const int rc = fold_status(p, s);
            if (rc != RCBF_OK) return rc;
        }
    const int st = p->status;
    p->status = 0;
    if (st) return set_error(RCBF_ETIMEOUT, "rcbf_pipeline_wait: a bounded device wait expired");
    return RCBF_OK;
}

void rcbf_pipeline_destroy(rcbf_pipeline_t p) {
    if (!p) return;
    if (p->d2h) cudaStreamSynchronize(p->d2h);
    if (p->compute) cudaStreamSynchronize(p->compute);
    if (p->h2d) cudaStreamSynchronize(p->h2d);
    for (Slot& s : p->slots) {
        if (s.graph) cudaGraphExecDestroy(s.graph);
        if (s.batch) rcbf_batch_destroy(s.batch);
        for (size_t f = 0; f < s.in.size(); ++f)
            if (s.in[f] && s.in[f] != s.dec[f]) cudaFree(s.in[f]);
        for (void* d : s.dec) if (d) cudaFree(d);
        for (float* i : s.img) if (i) cudaFree(i);
        if (s.copied) cudaEventDestroy(s.copied);
        if (s.computed) cudaEventDestroy(s.computed);
        if (s.done) cudaEventDestroy(s.done);
        if (s.h_status) cudaFreeHost(s.h_status);
    }
    if (p->h2d) cudaStreamDestroy(p->h2d);
    if (p->compute) cudaStreamDestroy(p->compute);
    if (p->d2h) cudaStreamDestroy(p->d2h);
    delete p;
}

}  // extern "C"

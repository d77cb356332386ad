// ceilings.cu — microbenchmarks of the on-chip ceilings that bound the tiled
// DAS: shared-memory 8-byte loads, FP32 FMA issue (scalar and packed f32x2)
// and shared integer reductions. Each kernel runs at the DAS kernel's
// occupancy (256 threads, 100 KB of shared memory per CTA, so two CTAs per SM,
// one CTA per resident slot), with bounded loops and no waits.
#include "internal.cuh"

using namespace rcbf;

namespace {

constexpr int kThreads = 256;
constexpr int kSmem = 100 * 1024;        // two CTAs per SM, as the DAS kernels
constexpr int kLdsIters = 16384;
constexpr int kFmaIters = 65536;
constexpr int kRedIters = 4096;

// Each thread reads 8 B at byte offset 8 * (tid + 256 u), u = 0..7: a warp
// covers 256 contiguous bytes (two wavefronts, no bank conflict). The loads
// are volatile, so none is hoisted out of the loop. Thread 0 of CTA 0 also
// records SM cycles and global-timer nanoseconds over its loop (the clock).
__global__ void __launch_bounds__(kThreads, 2) lds64_kernel(float* sink, long long* clk) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2* s = reinterpret_cast<float2*>(smem);
    for (int q = threadIdx.x; q < 8 * kThreads; q += kThreads) s[q] = make_float2((float)q, 1.0f);
    __syncthreads();
    const uint32_t base = static_cast<uint32_t>(__cvta_generic_to_shared(s + threadIdx.x));
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned long long g0, g1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g0));
    const long long t0 = clock64();
    for (int it = 0; it < kLdsIters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            float x, y;
            asm volatile("ld.volatile.shared.v2.f32 {%0,%1}, [%2];" : "=f"(x), "=f"(y) : "r"(base + 2048u * u));
            acc[u] = fmaf(x, y, acc[u]);
        }
    }
    const long long t1 = clock64();
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g1));
    float t = 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u) t += acc[u];
    if (t == -1.0f) sink[0] = t;             // never true: keeps the loads
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        clk[0] = t1 - t0;
        clk[1] = (long long)(g1 - g0);
    }
}

// Eight independent FMA chains per thread (scalar, or packed pairs).
template <bool PACKED>
__global__ void __launch_bounds__(kThreads, 2) ffma_kernel(float* sink, float b, float c) {
    extern __shared__ __align__(16) unsigned char smem[];
    (void)smem;
    if (PACKED) {
        unsigned long long a[8], bb, cc;
        asm("mov.b64 %0, {%1,%1};" : "=l"(bb) : "f"(b));
        asm("mov.b64 %0, {%1,%1};" : "=l"(cc) : "f"(c));
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float v = (float)(threadIdx.x + k);
            asm("mov.b64 %0, {%1,%1};" : "=l"(a[k]) : "f"(v));
        }
        for (int it = 0; it < kFmaIters; ++it) {
#pragma unroll
            for (int k = 0; k < 8; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(bb), "l"(cc));
        }
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float lo, hi;
            asm("mov.b64 {%0,%1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[k]));
            t += lo + hi;
        }
        if (t == -1.0f) sink[0] = t;
    } else {
        float a[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = (float)(threadIdx.x + k);
        for (int it = 0; it < kFmaIters; ++it) {
#pragma unroll
            for (int k = 0; k < 8; ++k) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[k]) : "f"(b), "f"(c));
        }
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += a[k];
        if (t == -1.0f) sink[0] = t;
    }
}

// Shared integer reductions: lane l of warp w adds to word 32 w + l (distinct
// addresses, one bank per lane), eight per iteration to eight blocks.
__global__ void __launch_bounds__(kThreads, 2) red_kernel(int* sink) {
    extern __shared__ __align__(16) unsigned char smem[];
    int* s = reinterpret_cast<int*>(smem);
    for (int q = threadIdx.x; q < 8 * kThreads; q += kThreads) s[q] = 0;
    __syncthreads();
    const uint32_t base = static_cast<uint32_t>(__cvta_generic_to_shared(s + threadIdx.x));
    for (int it = 0; it < kRedIters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
            asm volatile("red.shared.add.s32 [%0], %1;" :: "r"(base + 1024u * u), "r"(it) : "memory");
    }
    __syncthreads();
    if (s[threadIdx.x] == -7) sink[0] = s[threadIdx.x];
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Timer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

}  // namespace

extern "C" int rcbf_measure_ceilings(rcbf_ceilings* out, void* stream) {
    if (!out) return set_error(RCBF_EINVAL, "rcbf_measure_ceilings: out is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return check_launch("rcbf_measure_ceilings: device");
    if (cudaFuncSetAttribute(lds64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem) != cudaSuccess ||
        cudaFuncSetAttribute(ffma_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem) != cudaSuccess ||
        cudaFuncSetAttribute(ffma_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem) != cudaSuccess ||
        cudaFuncSetAttribute(red_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem) != cudaSuccess)
        return check_launch("rcbf_measure_ceilings: set shared memory");
    const unsigned grid = (unsigned)sms * 2;
    void* scratch = nullptr;
    if (cudaMalloc(&scratch, 64) != cudaSuccess) return set_error(RCBF_ENOMEM, "rcbf_measure_ceilings: cudaMalloc");
    float* fsink = static_cast<float*>(scratch);
    long long* cyc = reinterpret_cast<long long*>(static_cast<char*>(scratch) + 32);
    Timer tm;
    float ms[4] = {0, 0, 0, 0};
    int rc = RCBF_OK;
    if (cudaEventCreate(&tm.a) != cudaSuccess || cudaEventCreate(&tm.b) != cudaSuccess) rc = check_launch("rcbf_measure_ceilings: events");
    for (int k = 0; k < 4 && rc == RCBF_OK; ++k) {
        for (int rep = 0; rep < 2 && rc == RCBF_OK; ++rep) {   // the first pass warms up
            if (cudaEventRecord(tm.a, s) != cudaSuccess) { rc = check_launch("rcbf_measure_ceilings: record"); break; }
            if (k == 0) lds64_kernel<<<grid, kThreads, kSmem, s>>>(fsink, cyc);
            else if (k == 1) ffma_kernel<false><<<grid, kThreads, kSmem, s>>>(fsink, 0.999f, 1e-3f);
            else if (k == 2) ffma_kernel<true><<<grid, kThreads, kSmem, s>>>(fsink, 0.999f, 1e-3f);
            else red_kernel<<<grid, kThreads, kSmem, s>>>(reinterpret_cast<int*>(fsink));
            if (cudaEventRecord(tm.b, s) != cudaSuccess || cudaEventSynchronize(tm.b) != cudaSuccess ||
                cudaEventElapsedTime(&ms[k], tm.a, tm.b) != cudaSuccess)
                rc = check_launch("rcbf_measure_ceilings: kernel");
        }
    }
    long long clk[2] = {0, 0};
    if (rc == RCBF_OK && cudaMemcpy(clk, cyc, sizeof(clk), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = check_launch("rcbf_measure_ceilings: read clock");
    cudaFree(scratch);
    if (rc != RCBF_OK) return rc;
    const double threads = (double)grid * kThreads;
    out->lds64_bytes_per_s = threads * kLdsIters * 8.0 * 8.0 / (ms[0] * 1e-3);
    out->ffma_lane_ops_per_s = threads * kFmaIters * 8.0 / (ms[1] * 1e-3);
    out->ffma2_lane_ops_per_s = threads * kFmaIters * 8.0 * 2.0 / (ms[2] * 1e-3);
    out->red_shared_per_s = threads / 32.0 * kRedIters * 8.0 / (ms[3] * 1e-3);
    out->sm_clock_hz = clk[1] > 0 ? (double)clk[0] / ((double)clk[1] * 1e-9) : 0.0;
    return RCBF_OK;
}

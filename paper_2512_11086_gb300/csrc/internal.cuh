// internal.cuh — plan layout, kernel argument blocks and PTX helpers shared
// by the library's translation units (decode, DAS, adjoint, batch, API).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <string>

#include "rcbf.h"

namespace rcbf {

// ---------------------------------------------------------------- limits
constexpr int kMaxOrder = 256;        // largest Hadamard order / transmit count
constexpr int kMaxChannels = 256;     // receive channels per plan
constexpr int kDasThreads = 256;      // threads of a DAS tile CTA
constexpr int kTileVoxels = 1024;     // voxels of a DAS tile (4 per thread)
constexpr int kCI = 8;                // transmits per staged chunk
constexpr int kCJ = 8;                // channels per staged chunk
constexpr int kDecodeThreads = 256;
constexpr int kDecodeCols = 128;      // columns (channel x sample) per decode tile
constexpr long long kWaitNs = 1000000000LL;   // default bound of a device-side mbarrier wait: one second

// Status bits written by kernels into a plan's device status word.
constexpr int kStatusWaitExpired = 1;

// ------------------------------------------------------ DAS argument block
// Voxel index space is reordered so that u is the fast (lane) axis:
// u = x normally, u = y when the image has nx == 1 and ny > 1.
struct DasArgs {
    double q0[3];          // array-frame position of voxel (0,0,0)
    double Gu[3], Gv[3], Gw[3];   // array-frame step per index along u, v, w
    int n_u, n_v, n_w;
    long long out_su, out_sv, out_sw;   // image strides (floats) along u, v, w
    int tiles_u, tiles_v, tiles_w;
    int bu, bv, bw;        // tile extents (bu = 32*VU, bv*bw = 8*VR)
    int n_tx, n_ch, n_s;
    int tx_axis, rx_axis;  // lateral coordinate of an element: 0 -> q.x, 1 -> q.y
    double tx_e0, tx_pitch, rx_e0, rx_pitch;   // e_i = e0 + i*pitch
    double fs_over_c;      // samples per metre of path
    double t0fs;           // t0 * fs (samples)
    double c;              // speed of sound of this call
    double fs;
    double iq_ratio;       // iq_freq / fs: IQ beamforming phase per sample (0 = RF data)
    double tx_focus;       // virtual line source depth [m]
    const float2* tx_dir;  // plane waves: (sin a_i, cos a_i) per transmit (device)
    int tx_wave;           // rcbf_tx_wave
    int acq_kind;          // rcbf_acq_kind (RCBF_HERCULES_2D: non-separable receive)
    int vls_split;         // 1: the tiled kernel skips tiles across the VLS focal depth and the plain
                           // kernel computes only their voxels (tile_across_focus)
    float f_number;
    int interp;            // rcbf_interp
    int W;                 // pairs per window actually used (<= compiled stride)
    int lo;                // window start offset in samples (<= 0)
    int H;                 // W / 2: centring of the per-window line intercepts
    int raw_samples;       // raw samples staged per window (multiple of 8)
    float reach_a, reach_b;// tile reach of the transmit / receive delays in samples (+ slack)
    int n_split;           // channel split of every tile (units = tiles x n_split)
    float* partial;        // [n_split][planes][voxels] partial images (n_split > 1)
    long long partial_stride;  // floats between splits
    int dtype;             // rcbf_dtype of the decoded RF
    float scale;           // 1/N for RCBF_I32 input, else 1
    long long plane_stride;// elements between real and imaginary planes (complex)
    const void* rf;
    const float* apod;     // per-channel weights or nullptr
    float* image;
    long long image_plane; // floats between image planes (complex)
    int* status;
    long long wait_ns;     // bound of each mbarrier wait of the tiled forms (global-timer ns)
    int withhold;          // test hook: 1 = every tiled DAS unit omits its first window copy, so
                           // its first wait expires (rcbf_plan_set_wait); 0 in normal use
    int reserved_w;
    int* tile_flags;       // batch form of a channel split (n_split > 1): per tile, the number of
                           // splits already added into the image; split s waits (bounded) until
                           // it reads s, adds its sums into the image and publishes s + 1, so
                           // the image is summed in split order with no partial buffers
                           // (nullptr: partial images and a reduce kernel)
    // adjoint outputs (backward only)
    const float* grad_image;
    float* grad_rf;
    float* grad_c;
    float* grad_apod;
};

struct DecodeArgs {
    const int16_t* rf;
    void* out;
    const uint32_t* afrag;  // A = H^T fragments, permuted for the ldmatrix.trans B order
    const int8_t* hmat;     // H[k][i] row-major (plain variant)
    const uint32_t* afrag16;// A = H^T fragments of the FP16 form (natural k order)
    const int* hsum;        // h_i = sum_k H[k][i] (FP16 form correction)
    long long n_cols;       // n_ch * n_samples
    int n;                  // order
    int dtype;              // RCBF_I32 / RCBF_F32 / RCBF_F16
    float inv_n;
};

// ----------------------------------------------------------------- plan
struct PlanHost {
    rcbf_params p;
    DasArgs das;            // geometry part filled at plan time
    double r_alpha_m;       // tile radius in the (lateral_tx, z) plane [m] (2D aperture: the transmit path's largest spread over a tile's box)
    double r_beta_m;        // tile radius in the (lateral_rx, z) plane [m]
    int vu;                 // voxels per thread along u (1, 2, 4)
    bool swap_uv;           // u = y
    bool tiled_ok;          // geometry and sizes admit the tiled DAS
    uint32_t* d_afrag;      // device A fragments
    int8_t* d_hmat;         // device H (plain decode)
    uint32_t* d_afrag16;    // device A fragments, FP16 form
    int* d_hsum;            // device column sums of H
    uint16_t* d_atc;        // device A = H^T operand image of the tcgen05 decode (FP16 +-1, K-major,
                            // 128-byte swizzled, rows >= n zero), copied whole into shared memory
    int* d_status;          // device status word
    int n_sms;              // SMs of the plan's device
    int decode_blocks_per_sm;
    int das_blocks_per_sm[4];   // by window stride class (48, 64, 96, 128)
    int n_split[4];         // channel split by window stride class
    int tail_parts[4];      // parts of each of the last tail_units units (1: none)
    int tail_units[4];      // units at the end of the grid run as tail_parts blocks each
    float* d_partial;       // DAS partial images (channel split), plan-owned
    size_t partial_floats;
    int16_t* d_taps;        // device demodulation FIR taps (demod_decimation > 0)
    int16_t* d_taps_im;     // their imaginary parts (complex taps), else nullptr
    float2* d_tx_dir;       // device plane-wave directions (tx_wave == RCBF_TX_PLANE)
    bool has_tx_angle0;     // tx_angle0 holds the first plane-wave angle (the params' pointer is not kept)
    double tx_angle0;
    bool force_plain;       // the geometry admits no tile windows (2D aperture forms the tiled form lacks)
    bool vls_split;         // a VLS focal plane crosses a DAS tile: the tiles across it run the plain form
    bool vls_split_bwd;     // a VLS focal plane crosses a tile of the adjoint's own tiling
    // adjoint tile with lanes over z: 32 voxels along u by bwd_bv x bwd_bw
    // rows (bwd_bv = 0: no such tile keeps the window within 128 samples)
    int bwd_bv, bwd_bw;
    double bwd_r_alpha_m, bwd_r_beta_m;
};

}  // namespace rcbf

struct rcbf_plan_s {
    rcbf::PlanHost h;
};

namespace rcbf {

// Thread-local error message helpers (api.cu).
int set_error(int code, const std::string& msg);
int check_launch(const char* what);

// Host-side plan pieces (api.cu): argument validation and the geometry /
// tile set-up of a plan, neither of which touches the device.
int plan_validate(const rcbf_params* p);
void plan_geometry(PlanHost& h);

// Window geometry of a DAS call at speed of sound c (host side).
int das_prepare(const PlanHost& h, double c, DasArgs* a, std::string* why);
// das_prepare for another tile (bu, bv, bw) with its radii [m]
int das_prepare_tile(const PlanHost& h, double c, int bu, int bv, int bw, double r_alpha_m, double r_beta_m,
                     DasArgs* a, std::string* why);

// Kernel launchers (one per translation unit).
int launch_decode(const PlanHost& h, const int16_t* rf, void* out, cudaStream_t s);
// The tcgen05 form of the decode (decode_tc.cu): launch, and plan-time set-up.
int launch_decode_tc(const PlanHost& h, int dtype, const int16_t* rf, void* out, cudaStream_t s);
int configure_decode_tc(const PlanHost& h, int dtype);
// A tcgen05 decode bound to fixed buffers (the tensor maps encoded once), for
// the batch: prepared at rcbf_batch_create, launched by every rcbf_batch_run.
struct TcJob {
    CUtensorMap in_map, out_map;
    const uint16_t* atc;
    const int* hsum;
    long long n_cols;
    float inv_n;
    int n, dtype;
    unsigned grid;
};
int decode_tc_prepare(const PlanHost& h, int dtype, const int16_t* rf, void* out, TcJob* job);
// Demodulation fused into the decode (demod_decode.cu).
bool demod_decode_supported(const PlanHost& h, std::string* why);
int configure_demod_decode(const PlanHost& h);
int launch_demod_decode(const PlanHost& h, const int16_t* rf, float* out, cudaStream_t s);
int decode_tc_run(const TcJob& job, int* status, long long wait_ns, cudaStream_t s);
// Device address of a batch's status word (batch.cu).
int* batch_status_word(rcbf_batch_t batch);
int launch_demodulate(const PlanHost& h, const int16_t* rf, int16_t* iq, cudaStream_t s);
int launch_das(const PlanHost& h, const DasArgs& a, cudaStream_t s);
int launch_das_plain(const PlanHost& h, const DasArgs& a, cudaStream_t s);
// mode: 0 plain, 1 tiled with the plan's tile (lanes along u), 2 tiled with
// the adjoint tile (lanes over z; a.bu must be 32)
int launch_das_backward(const PlanHost& h, const DasArgs& a, int mode, cudaStream_t s);
int configure_decode(PlanHost& h);
int das_class_index(int W, bool d2);
int configure_das(PlanHost& h);
int das_slices(const PlanHost& h, int c);   // partial images of window class c (1: none)

// ------------------------------------------------------------ PTX helpers
// ---- transmit waves (line element, plane wave, virtual line source): the
// FP64 reference entry of transmit e at the tile reference point, and the FP32
// offset of a voxel from it. Entry: (x, y, frac, K) with A = K + frac the
// reference transmit delay in samples; x, y per wave:
//   line   (L, d)                   L = lat_ref - e, d = sqrt(L^2 + Z^2)
//   plane  (sin a, cos a)
//   vls    (L, sgn * dv)            dv = sqrt(L^2 + (Z - f)^2), sgn = sign(Z - f)
__device__ __forceinline__ double tx_ref_distance(const DasArgs& a, int e, double lat_ref, double zr, float* x,
                                                  float* y) {
    if (a.tx_wave == RCBF_TX_PLANE) {
        const float2 sc = a.tx_dir[e];
        *x = sc.x;
        *y = sc.y;
        return zr * (double)sc.y + lat_ref * (double)sc.x;
    }
    const double L = lat_ref - (a.tx_e0 + e * a.tx_pitch);
    if (a.tx_wave == RCBF_TX_VLS) {
        const double dz = zr - a.tx_focus;
        const double dv = (dz >= 0.0 ? 1.0 : -1.0) * sqrt(L * L + dz * dz);
        *x = (float)L;
        *y = (float)dv;
        return a.tx_focus + dv;
    }
    const double d = sqrt(L * L + zr * zr);
    *x = (float)L;
    *y = (float)d;
    return d;
}

// Transmit delay of the voxel at offsets (dL, dZ) from the reference, in
// samples relative to the entry's reference (before the window clamp).
// Zf = z of the reference (FP32), Zfoc = reference z minus the focus depth.
__device__ __forceinline__ float tx_offset(int wave, float4 tx, float dL, float dZ, float Zf, float Zfoc, float fsc) {
    if (wave == RCBF_TX_PLANE) return tx.z + fmaf(dZ, tx.y, dL * tx.x) * fsc;
    if (wave == RCBF_TX_VLS) {
        // the tiled form never sees a tile across the focal depth (the plain
        // kernel computes those), so the voxel is on the reference's side:
        // the same cancellation-free difference, signed like the reference
        const float Lv = tx.x + dL, Zv = Zfoc + dZ;
        const float dv = sqrtf(Lv * Lv + Zv * Zv);
        const float num = dL * (2.0f * tx.x + dL) + dZ * (2.0f * Zfoc + dZ);
        const float diff = __fdividef(num, dv + fabsf(tx.y));
        return tx.z + (tx.y >= 0.f ? diff : -diff) * fsc;
    }
    // cancellation-free d(v) - d(ref) = (dL (2L + dL) + dZ (2Z + dZ)) / (d(v) + d(ref))
    const float Lv = tx.x + dL, Zv = Zf + dZ;
    const float d = sqrtf(Lv * Lv + Zv * Zv);
    const float num = dL * (2.0f * tx.x + dL) + dZ * (2.0f * Zf + dZ);
    return tx.z + __fdividef(num, d + tx.y) * fsc;
}

// FP32 transmit path of transmit i to (lat_tx, z) (the plain forms).
// Whether voxel tile (tu, tv, tw) reaches the virtual-line-source focal depth
// (its bounding box in z contains tx_focus, boundary included): off axis the
// VLS delay jumps there, so such a tile has no sample window and runs the
// plain form. The tiled and the plain kernels evaluate the same expression.
__device__ __forceinline__ bool tile_across_focus(const DasArgs& a, int tu, int tv, int tw) {
    const double cu = tu * a.bu + 0.5 * (a.bu - 1), cv = tv * a.bv + 0.5 * (a.bv - 1), cw = tw * a.bw + 0.5 * (a.bw - 1);
    const double zc = a.q0[2] + a.Gu[2] * cu + a.Gv[2] * cv + a.Gw[2] * cw;
    const double hz = 0.5 * (fabs(a.Gu[2]) * (a.bu - 1) + fabs(a.Gv[2]) * (a.bv - 1) + fabs(a.Gw[2]) * (a.bw - 1));
    return fabs(a.tx_focus - zc) <= hz + 1e-9;
}

__device__ __forceinline__ float tx_distance_f32(const DasArgs& a, int i, float lat_tx, float z) {
    if (a.tx_wave == RCBF_TX_PLANE) {
        const float2 sc = a.tx_dir[i];
        return fmaf(z, sc.y, lat_tx * sc.x);
    }
    const float dx = lat_tx - ((float)a.tx_e0 + i * (float)a.tx_pitch);
    if (a.tx_wave == RCBF_TX_VLS) {
        const float f = (float)a.tx_focus, dz = z - f;
        const float dv = sqrtf(dx * dx + dz * dz);
        return f + (dz >= 0.f ? dv : -dv);
    }
    return sqrtf(dx * dx + z * z);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;"
                 :: "r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on an mbarrier phase that also gives up when another thread
// of the CTA has raised the abort flag; raises it itself when its own time
// budget (limit_ns of global-timer time, counted from the first failed poll
// so that a wait that succeeds at once reads no timer) runs out. Returns
// false on abort.
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort,
                                                   long long limit_ns = kWaitNs) {
    unsigned long long t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
        if ((it & 15u) == 15u) {
            if (*abort) return false;
            const unsigned long long now = globaltimer_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > (unsigned long long)limit_ns) break;
        }
    }
    *abort = 1;
    return false;
}

// Bounded wait on an mbarrier phase; returns false after limit_ns.
__device__ __forceinline__ bool mbar_wait_parity(uint32_t bar, uint32_t parity, long long limit_ns = kWaitNs) {
    volatile int never = 0;
    return mbar_wait_or_abort(bar, parity, &never, limit_ns);
}

// 1-D bulk copy global -> shared (TMA engine), completion on an mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

}  // namespace rcbf

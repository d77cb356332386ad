// das.cu — DAS dispatch, the plain FP32 form, and per-call window set-up.
//
// The plain form is the direct reading of Eq. (1)-(3) on the GPU: one thread
// per voxel, FP32 voxel position and distances (the transmit distances of the
// voxel cached per thread), fractional sample s = (d_tx + d_rx) fs / c - t0 fs,
// floor / fraction, and two global loads through the read-only cache for a
// linear interpolation (four for the cubic Hermite spline), zero outside the
// record.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace rcbf {

template <int VU, bool CPLX, bool D2> int configure_das_vu(int ws, bool cubic, bool iq, int* per_sm);
template <int VU, bool CPLX, bool D2>
int launch_das_vu(const DasArgs& a, int ws, bool apod, bool cubic, bool iq, int tail_units, int tail_parts,
                  cudaStream_t s);

namespace {
template <int VU>
int configure_vu(int ws, bool cplx, bool cubic, bool iq, bool d2, int* per_sm) {
    if (d2) {
        if constexpr (VU == 1)
            return cplx ? configure_das_vu<1, true, true>(ws, cubic, iq, per_sm)
                        : configure_das_vu<1, false, true>(ws, cubic, iq, per_sm);
        else
            return set_error(RCBF_EUNSUPPORTED, "das: the 2D aperture tiles hold one voxel per thread along u");
    }
    return cplx ? configure_das_vu<VU, true, false>(ws, cubic, iq, per_sm)
                : configure_das_vu<VU, false, false>(ws, cubic, iq, per_sm);
}
template <int VU>
int launch_vu(const DasArgs& a, int ws, bool cplx, bool apod, bool cubic, bool iq, bool d2, int tu, int tp,
              cudaStream_t s) {
    if (d2) {
        if constexpr (VU == 1)
            return cplx ? launch_das_vu<1, true, true>(a, ws, apod, cubic, iq, tu, tp, s)
                        : launch_das_vu<1, false, true>(a, ws, apod, cubic, iq, tu, tp, s);
        else
            return set_error(RCBF_EUNSUPPORTED, "das: the 2D aperture tiles hold one voxel per thread along u");
    }
    return cplx ? launch_das_vu<VU, true, false>(a, ws, apod, cubic, iq, tu, tp, s)
                : launch_das_vu<VU, false, false>(a, ws, apod, cubic, iq, tu, tp, s);
}
}  // namespace

namespace {

template <int DT>
__device__ __forceinline__ float plain_load(const void* rf, long long idx, float scale) {
    if (DT == RCBF_F16) return __half2float(__ldg(static_cast<const __half*>(rf) + idx));
    if (DT == RCBF_I32) return (float)__ldg(static_cast<const int*>(rf) + idx) * scale;
    return __ldg(static_cast<const float*>(rf) + idx);
}

// Trace sample k (zero outside the record).
template <int DT>
__device__ __forceinline__ float plain_sample(const void* rf, long long base, int k, int n_s, float scale) {
    return (k >= 0 && k < n_s) ? plain_load<DT>(rf, base + k, scale) : 0.f;
}

// Cubic Hermite value at fraction f of interval n: slopes are central
// differences of the four samples k = n-1 .. n+2.
template <int DT>
__device__ __forceinline__ float plain_cubic(const void* rf, long long base, int n, float f, int n_s, float scale) {
    const float p0 = plain_sample<DT>(rf, base, n - 1, n_s, scale), p1 = plain_sample<DT>(rf, base, n, n_s, scale);
    const float p2 = plain_sample<DT>(rf, base, n + 1, n_s, scale), p3 = plain_sample<DT>(rf, base, n + 2, n_s, scale);
    const float m1 = 0.5f * (p2 - p0), m2 = 0.5f * (p3 - p1), d = p2 - p1;
    const float a2 = 3.0f * d - 2.0f * m1 - m2, a3 = -2.0f * d + m1 + m2;
    return fmaf(fmaf(fmaf(a3, f, a2), f, m1), f, p1);
}

// Interpolated sample of trace (i, j) at fractional sample s (linear or cubic).
template <int DT, bool CUBIC>
__device__ __forceinline__ float plain_interp(const void* rf, long long base, float s, int n_s, float scale) {
    const float fl = floorf(s);
    const float f = s - fl;
    const int n = (int)fl;
    if (CUBIC) return plain_cubic<DT>(rf, base, n, f, n_s, scale);
    const float r0 = plain_sample<DT>(rf, base, n, n_s, scale), r1 = plain_sample<DT>(rf, base, n + 1, n_s, scale);
    return (1.0f - f) * r0 + f * r1;
}

// HERCULES with its 2D receive aperture: one transmit wave, a point-element
// receive path per (row i, column j) (not separable), F# window on the radial
// lateral distance (FN). One thread per voxel, FP32; the receive distance is
// x * rsqrt(x) of the squared distance (x > 0 below the array).
template <int DT, bool CPLX, bool CUBIC, bool IQ, bool FN>
__global__ void __launch_bounds__(128)
das_plain_2d_kernel(DasArgs a) {
    const long long n_vox = (long long)a.n_u * a.n_v * a.n_w;
    const long long vox = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (vox >= n_vox) return;
    const int iu = (int)(vox % a.n_u);
    const int iv = (int)((vox / a.n_u) % a.n_v);
    const int iw = (int)(vox / ((long long)a.n_u * a.n_v));
    float q[3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
        q[d] = (float)a.q0[d] + (float)a.Gu[d] * iu + (float)a.Gv[d] * iv + (float)a.Gw[d] * iw;
    const float lat_tx = q[a.tx_axis], lat_rx = q[a.rx_axis], z = q[2];
    const float fsc = (float)a.fs_over_c, t0fs = (float)a.t0fs;
    float d_wave;
    if (a.tx_wave == RCBF_TX_PLANE) {
        const float2 sc = a.tx_dir[0];
        d_wave = fmaf(z, sc.y, lat_tx * sc.x);
    } else {
        const float f = (float)a.tx_focus, dz = z - f;
        d_wave = sqrtf(q[0] * q[0] + q[1] * q[1] + dz * dz) + f;
    }
    const float rk = (float)(a.iq_ratio * a.fs_over_c);
    const double t0c = a.iq_ratio * a.t0fs;
    const float ph_t0 = (float)(t0c - floor(t0c));
    float ph_tx = 0.f;
    if (IQ) {
        const float p = rk * d_wave;
        ph_tx = p - rintf(p) - ph_t0;
    }
    float acc = 0.f, acci = 0.f;
    for (int i = 0; i < a.n_tx; ++i) {
        const float dt = lat_tx - ((float)a.tx_e0 + i * (float)a.tx_pitch);
        const float p2 = dt * dt + z * z;
        for (int j = 0; j < a.n_ch; ++j) {
            const float dr = lat_rx - ((float)a.rx_e0 + j * (float)a.rx_pitch);
            float w = a.apod ? __ldg(a.apod + j) : 1.0f;
            if (FN) {
                const float al = a.f_number * sqrtf(fmaf(dr, dr, dt * dt)), az = fabsf(z);
                if (al < 0.5f * az) { const float cs = cospif(al / az); w *= cs * cs; }
                else w = 0.f;
                if (w == 0.f) continue;
            }
            const float x2 = fmaf(dr, dr, p2);
            const float d_rx = x2 * rsqrtf(x2);
            const float s = (d_wave + d_rx) * fsc - t0fs;
            const long long base = ((long long)i * a.n_ch + j) * a.n_s;
            float vr = plain_interp<DT, CUBIC>(a.rf, base, s, a.n_s, a.scale), vi = 0.f;
            if (CPLX) vi = plain_interp<DT, CUBIC>(a.rf, a.plane_stride + base, s, a.n_s, a.scale);
            if (IQ) {
                const float prx = rk * d_rx;
                float x = ph_tx + (prx - rintf(prx));
                x -= rintf(x);
                float sn, cs;
                __sincosf(6.28318530717958648f * x, &sn, &cs);
                const float r0 = vr * cs - vi * sn;
                vi = fmaf(vr, sn, vi * cs);
                vr = r0;
            }
            acc += w * vr;
            if (CPLX) acci += w * vi;
        }
    }
    const long long o = (long long)iw * a.out_sw + (long long)iv * a.out_sv + (long long)iu * a.out_su;
    a.image[o] = acc;
    if (CPLX) a.image[a.image_plane + o] = acci;
}

template <int DT, bool CPLX, bool CUBIC, bool IQ>
__global__ void __launch_bounds__(128)
das_plain_kernel(DasArgs a) {
    const long long n_vox = (long long)a.n_u * a.n_v * a.n_w;
    const long long vox = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (vox >= n_vox) return;
    const int iu = (int)(vox % a.n_u);
    const int iv = (int)((vox / a.n_u) % a.n_v);
    const int iw = (int)(vox / ((long long)a.n_u * a.n_v));
    // split VLS image: only the voxels of tiles across the focal depth
    if (a.vls_split && !tile_across_focus(a, iu / a.bu, iv / a.bv, iw / a.bw)) return;
    float q[3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
        q[d] = (float)a.q0[d] + (float)a.Gu[d] * iu + (float)a.Gv[d] * iv + (float)a.Gw[d] * iw;
    const float lat_tx = q[a.tx_axis], lat_rx = q[a.rx_axis], z = q[2];
    const float fsc = (float)a.fs_over_c, t0fs = (float)a.t0fs;
    float dtx[kMaxOrder];
    for (int i = 0; i < a.n_tx; ++i) {
        dtx[i] = tx_distance_f32(a, i, lat_tx, z);
    }
    float acc = 0.f, acci = 0.f;
    // IQ phase r s = r fs/c d_tx + r fs/c d_rx - r t0 fs, each term reduced to
    // a fraction of a cycle before the sum (the absolute terms reach ~10^2 cycles)
    const float rk = (float)(a.iq_ratio * a.fs_over_c);
    const double t0c = a.iq_ratio * a.t0fs;
    const float ph_t0 = (float)(t0c - floor(t0c));
    for (int j = 0; j < a.n_ch; ++j) {
        const float dx = lat_rx - ((float)a.rx_e0 + j * (float)a.rx_pitch);
        const float drx = sqrtf(dx * dx + z * z);
        float ph_rx = 0.f;
        if (IQ) {
            const float prx = rk * drx;
            ph_rx = prx - rintf(prx) - ph_t0;
        }
        float w = a.apod ? __ldg(a.apod + j) : 1.0f;
        if (a.f_number > 0.f) {
            const float al = a.f_number * fabsf(dx), az = fabsf(z);
            if (al < 0.5f * az) { const float cs = cospif(al / az); w *= cs * cs; }
            else w = 0.f;
        }
        if (w == 0.f) continue;
        for (int i = 0; i < a.n_tx; ++i) {
            const float s = (dtx[i] + drx) * fsc - t0fs;
            const float fl = floorf(s);
            const float f = s - fl;
            const int n = (int)fl;
            const long long base = ((long long)i * a.n_ch + j) * a.n_s;
            float vr, vi = 0.f;
            if (CUBIC) {
                vr = plain_cubic<DT>(a.rf, base, n, f, a.n_s, a.scale);
                if (CPLX) vi = plain_cubic<DT>(a.rf, a.plane_stride + base, n, f, a.n_s, a.scale);
            } else {
                const bool in0 = n >= 0 && n < a.n_s, in1 = n + 1 >= 0 && n + 1 < a.n_s;
                const float r0 = in0 ? plain_load<DT>(a.rf, base + n, a.scale) : 0.f;
                const float r1 = in1 ? plain_load<DT>(a.rf, base + n + 1, a.scale) : 0.f;
                vr = (1.0f - f) * r0 + f * r1;
                if (CPLX) {
                    const float i0 = in0 ? plain_load<DT>(a.rf, a.plane_stride + base + n, a.scale) : 0.f;
                    const float i1 = in1 ? plain_load<DT>(a.rf, a.plane_stride + base + n + 1, a.scale) : 0.f;
                    vi = (1.0f - f) * i0 + f * i1;
                }
            }
            if (IQ) {
                const float ptx = rk * dtx[i];
                float x = (ptx - rintf(ptx)) + ph_rx;
                x -= rintf(x);
                float sn, cs;
                __sincosf(6.28318530717958648f * x, &sn, &cs);
                const float r0 = vr * cs - vi * sn;
                vi = fmaf(vr, sn, vi * cs);
                vr = r0;
            }
            acc += w * vr;
            if (CPLX) acci += w * vi;
        }
    }
    const long long o = (long long)iw * a.out_sw + (long long)iv * a.out_sv + (long long)iu * a.out_su;
    a.image[o] = acc;
    if (CPLX) a.image[a.image_plane + o] = acci;
}

// Sum of the channel-split partial images in split order (deterministic).
__global__ void __launch_bounds__(256)
das_reduce_kernel(const float* __restrict__ partial, float* __restrict__ image, long long n,
                  long long stride, int n_split) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float acc = partial[i];
        for (int k = 1; k < n_split; ++k) acc += partial[(long long)k * stride + i];
        image[i] = acc;
    }
}

}  // namespace

int launch_das_plain(const PlanHost& h, const DasArgs& a, cudaStream_t s) {
    (void)h;
    const long long n_vox = (long long)a.n_u * a.n_v * a.n_w;
    const unsigned grid = (unsigned)((n_vox + 127) / 128);
#define RCBF_PLAIN(K, CU, ...)                                                                  \
    switch (a.dtype) {                                                                          \
        case RCBF_F32: K<RCBF_F32, false, CU, false __VA_ARGS__><<<grid, 128, 0, s>>>(a); break;  \
        case RCBF_F16: K<RCBF_F16, false, CU, false __VA_ARGS__><<<grid, 128, 0, s>>>(a); break;  \
        case RCBF_I32: K<RCBF_I32, false, CU, false __VA_ARGS__><<<grid, 128, 0, s>>>(a); break;  \
        case RCBF_CF32:                                                                         \
            if (a.iq_ratio > 0.0) K<RCBF_F32, true, CU, true __VA_ARGS__><<<grid, 128, 0, s>>>(a); \
            else K<RCBF_F32, true, CU, false __VA_ARGS__><<<grid, 128, 0, s>>>(a);                 \
            break;                                                                              \
        default: return set_error(RCBF_EUNSUPPORTED, "das: unsupported decoded dtype");         \
    }
#define RCBF_PLAIN_2D(CU)                                                                       \
    if (a.f_number > 0.f) { RCBF_PLAIN(das_plain_2d_kernel, CU, , true) }                       \
    else { RCBF_PLAIN(das_plain_2d_kernel, CU, , false) }
    if (a.acq_kind == RCBF_HERCULES_2D) {
        if (a.interp == RCBF_CUBIC) { RCBF_PLAIN_2D(true) } else { RCBF_PLAIN_2D(false) }
        return check_launch("das_plain_2d_kernel");
    }
    if (a.interp == RCBF_CUBIC) { RCBF_PLAIN(das_plain_kernel, true, ) } else { RCBF_PLAIN(das_plain_kernel, false, ) }
#undef RCBF_PLAIN_2D
#undef RCBF_PLAIN
    return check_launch("das_plain_kernel");
}

// Window geometry of one call. With R the tile radius in samples (transmit
// plus receive plane), every voxel of a tile reads trace (i, j) inside
// [K_i + K_j + lo, K_i + K_j + lo + W]: alpha, beta lie within R_a, R_b of
// their references and the references' fractional parts are in [0, 1).
int das_prepare(const PlanHost& h, double c, DasArgs* a, std::string* why) {
    return das_prepare_tile(h, c, h.das.bu, h.das.bv, h.das.bw, h.r_alpha_m, h.r_beta_m, a, why);
}

int das_prepare_tile(const PlanHost& h, double c, int bu, int bv, int bw, double r_alpha_m, double r_beta_m,
                     DasArgs* a, std::string* why) {
    *a = h.das;
    a->bu = bu;
    a->bv = bv;
    a->bw = bw;
    a->tiles_u = (a->n_u + bu - 1) / bu;
    a->tiles_v = (a->n_v + bv - 1) / bv;
    a->tiles_w = (a->n_w + bw - 1) / bw;
    a->c = c;
    a->fs_over_c = h.p.fs / c;
    a->t0fs = h.p.t0 * h.p.fs;
    if (h.p.acq_kind == RCBF_HERCULES_2D) {
        // 2D receive aperture: the receive path varies over the tile by at
        // most the diagonal D of its bounding box, the transmit wave's path by
        // at most r_alpha (its largest spread over a tile's box, in metres);
        // the kernel places each window from box bounds (no common offset lo)
        double e2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            const double ext = std::fabs(a->Gu[d]) * (bu - 1) + std::fabs(a->Gv[d]) * (bv - 1) + std::fabs(a->Gw[d]) * (bw - 1);
            e2 += ext * ext;
        }
        const double X = (std::sqrt(e2) + r_alpha_m) * a->fs_over_c;
        a->lo = 0;
        a->W = (int)std::floor(4.0 + X + 0.02) + 1;
    } else {
        const double R = (r_alpha_m + r_beta_m) * a->fs_over_c;
        a->lo = (int)std::floor(-R) - 1;
        a->W = (int)std::floor(4.0 + 2.0 * R + 0.01) + 1;
    }
    a->H = a->W / 2;
    a->raw_samples = ((a->W + 8 + 7) / 8) * 8;
    // alpha and beta are clamped to reference +- reach in the kernel; the
    // 0.004-sample slack per side stays inside the 0.01 slack of W, so every
    // interval index lands in [0, W-1] whatever the input (NaN included)
    a->reach_a = (float)(r_alpha_m * a->fs_over_c + 0.004);
    a->reach_b = (float)(r_beta_m * a->fs_over_c + 0.004);
    if (h.p.acq_kind == RCBF_HERCULES_2D) a->reach_a = 0.004f;   // slack of the kernel's box bounds
    if (a->interp == RCBF_CUBIC) {
        // the 4-point stencil of interval n reaches one sample before the
        // window start and two after its interval: copies start one sample
        // early and carry two more
        a->raw_samples = ((a->W + 10 + 7) / 8) * 8;
    }
    if (a->W > 128) {
        if (why) *why = "das: the voxel tile spans more than 128 samples at this speed of sound; choose a smaller tile";
        return RCBF_EUNSUPPORTED;
    }
    if (h.force_plain) {
        if (why) *why = "das: a 2D receive aperture with an F# window or a tile wider than 32 voxels runs the plain form";
        return RCBF_EUNSUPPORTED;
    }
    if (a->interp == RCBF_CUBIC && a->dtype == RCBF_CF32 && a->W > 64) {
        if (why) *why = "das: complex cubic windows above 64 samples run the plain form";
        return RCBF_EUNSUPPORTED;
    }
    return RCBF_OK;
}

// window class of W intervals (the 2D receive aperture starts at 64)
static int stride_class(int W, bool d2) { return W <= 48 && !d2 ? 48 : W <= 64 ? 64 : W <= 96 ? 96 : 128; }
static int class_index(int ws) { return ws == 48 ? 0 : ws == 64 ? 1 : ws == 96 ? 2 : 3; }

int das_class_index(int W, bool d2) { return class_index(stride_class(W, d2)); }

int das_slices(const PlanHost& h, int c) {
    const int sp = std::max(1, h.n_split[c]);
    return h.tail_parts[c] > 1 && h.tail_units[c] > 0 ? sp * h.tail_parts[c] : sp;
}

int launch_das(const PlanHost& h, const DasArgs& a_in, cudaStream_t s) {
    DasArgs a = a_in;
    const bool d2 = a.acq_kind == RCBF_HERCULES_2D;
    const int ws = stride_class(a.W, d2);
    const bool cplx = a.dtype == RCBF_CF32;
    const bool apod = a.apod != nullptr || a.f_number > 0.f;
    const bool cubic = a.interp == RCBF_CUBIC;
    const bool iq = cplx && a.iq_ratio > 0.0;
    const int c = class_index(ws);
    a.n_split = std::max(1, h.n_split[c]);
    const int tp = std::max(1, h.tail_parts[c]), tu = tp > 1 ? h.tail_units[c] : 0;
    const int slices = das_slices(h, c);
    a.partial = h.d_partial;
    a.partial_stride = a.image_plane * (cplx ? 2 : 1);
    // the partial images of tail parts p >= 1 hold only the tail tiles' sums
    if (slices > a.n_split &&
        cudaMemsetAsync(a.partial + (long long)a.n_split * a.partial_stride, 0,
                        (size_t)(slices - a.n_split) * a.partial_stride * sizeof(float), s) != cudaSuccess)
        return check_launch("das: clear the tail partial images");
    int rc;
    switch (h.vu) {
        case 1: rc = launch_vu<1>(a, ws, cplx, apod, cubic, iq, d2, tu, tp, s); break;
        case 2: rc = launch_vu<2>(a, ws, cplx, apod, cubic, iq, d2, tu, tp, s); break;
        default: rc = launch_vu<4>(a, ws, cplx, apod, cubic, iq, d2, tu, tp, s); break;
    }
    if (rc != RCBF_OK || slices == 1) return rc;
    const long long n = a.partial_stride;
    long long blocks = (n + 255) / 256;
    if (blocks > (long long)h.n_sms * 8) blocks = (long long)h.n_sms * 8;
    das_reduce_kernel<<<(unsigned)blocks, 256, 0, s>>>(a.partial, a.image, n, a.partial_stride, slices);
    return check_launch("das_reduce_kernel");
}

int configure_das(PlanHost& h) {
    if (h.p.das_variant == RCBF_DAS_PLAIN || !h.tiled_ok) return RCBF_OK;
    const bool cplx = h.p.decoded_dtype == RCBF_CF32;
    const bool cubic = h.p.interp == RCBF_CUBIC;
    const bool iq = cplx && h.p.iq_freq > 0.0;
    const bool d2 = h.p.acq_kind == RCBF_HERCULES_2D;
    if (d2 && h.force_plain) return RCBF_OK;
    for (int c = 0; c < 4; ++c) {
        const int ws = c == 0 ? 48 : c == 1 ? 64 : c == 2 ? 96 : 128;
        int rc, n = 0;
        if ((cubic && cplx && ws == 128) || (d2 && ws == 48)) {   // plain form / 64 class
            h.das_blocks_per_sm[c] = 0;
            h.n_split[c] = 1;
            h.tail_parts[c] = 1;
            h.tail_units[c] = 0;
            continue;
        }
        switch (h.vu) {
            case 1: rc = configure_vu<1>(ws, cplx, cubic, iq, d2, &n); break;
            case 2: rc = configure_vu<2>(ws, cplx, cubic, iq, d2, &n); break;
            default: rc = configure_vu<4>(ws, cplx, cubic, iq, d2, &n); break;
        }
        if (rc != RCBF_OK) return rc;
        h.das_blocks_per_sm[c] = n;
        // channel split: the smallest power of two (dividing the channel
        // chunks, at most 16) whose units make three waves of the resident
        // CTA slots; then the last 3/4 wave of units in up to four channel
        // parts each (scheduled last), so the grid ends within about one
        // part's time
        const long long tiles = (long long)h.das.tiles_u * h.das.tiles_v * h.das.tiles_w;
        const long long slots = (long long)h.n_sms * (n > 0 ? n : 1);
        const int chunks = (int)h.p.n_ch / kCJ;
        int sp = 1;
        while (tiles * sp < 3 * slots && sp * 2 <= chunks && chunks % (sp * 2) == 0 && sp < 16) sp *= 2;
        int parts = 1;
        while (parts * 2 <= 4 && (chunks / sp) % (parts * 2) == 0) parts *= 2;
        h.n_split[c] = sp;
        h.tail_parts[c] = parts;
        h.tail_units[c] = parts > 1 ? (int)std::min(tiles * sp, 3 * slots / 4) : 0;
    }
    return RCBF_OK;
}

}  // namespace rcbf

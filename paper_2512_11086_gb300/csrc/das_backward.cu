// das_backward.cu — adjoint of the delay-and-sum of Eq. (1) for an upstream
// gradient G = dL/dimage: gradients with respect to the decoded RF samples,
// the speed of sound c and the per-channel apodization weights w_j. The paper
// has no adjoint; it is Eq. (1) differentiated for speed-of-sound autofocus.
//
// With s = s_ij(v), n = floor(s), f = s - n and a_j(v) = w_j W_j(v):
//   dL/dr_ij[n]   += a_j(v) G(v) (1 - f),   dL/dr_ij[n+1] += a_j(v) G(v) f
//   dL/dc         += a_j(v) G(v) (r[n+1] - r[n]) ds/dc,   ds/dc = -(d_tx + d_rx) fs / c^2
//                                                               = -(s + t0 fs) / c
//   dL/dw_j       += W_j(v) G(v) lerp(r_ij, s) = sum_n r_ij[n] (dL/dr_ij[n]) / w_j
// (complex data: the two planes contribute independently).
//
// Tiled form: per-tile FP64 reference delays and TMA windows as in the
// forward. Per stage each (transmit, channel) window gets two shared-memory
// accumulators over the intervals n of the window: G0[n] = sum g and
// G1[n] = sum g f over the voxels v whose delay falls in interval n, with
// g = W_j(v) G(v) and f the fraction within the interval. Everything else is
// exact arithmetic on them once the stage is done:
//   c[n] = G0[n] - G1[n] + G1[n-1]                (lerp weights of sample n)
//   dL/dr_ij[n] = w_j c[n],   dL/dw_j += sum_n r[n] c[n],
//   dL/dc (before -w_j / c) += sum_n (r[n+1] - r[n]) ((n + S0 + t0 fs) G0[n] + G1[n])
// (S0 + n + f is the voxel's absolute sample position). So a voxel costs two
// accumulator updates per plane and nothing else. Windows of neighbouring
// tiles overlap, so dL/dr is added with global atomics. Delays are recomputed
// per tile, never stored. The plain form is one thread per voxel with global
// atomics.
//
// The window accumulators are 32-bit fixed point. Shared-memory float atomics
// retry per conflicting lane, and neighbouring voxels along the lane axis
// often hit the same sample; integer atomics do not retry, and integer sums do
// not depend on order. The scale is 2^e with 1024 * max|G| * 2^e < 2^30 over
// the tile (W_j <= 1 and 0 <= f <= 1): an accumulator collects at most one
// term per voxel of the 1024-voxel tile, so it cannot overflow, and a term is
// rounded to 2^-e <= 2^-19 max|G| (a relative 2e-6 of the largest term of the
// tile). c[n] = G0[n] - G1[n] + G1[n-1] is a sum of at most 1024 such terms
// with weights in [0, 1], so it is formed exactly in 32-bit integers.
#include <algorithm>

#include "das_tile.cuh"

namespace rcbf {

namespace {

constexpr int kBwdCI = 4;          // transmits per backward stage
constexpr int kBwdCJ = 4;          // channels per backward stage

// ZL: lanes on tile rows (the z-major row index), each thread four
// consecutive voxels along u. Along z the delay grows by a sizeable fraction
// of a sample per voxel, so the 32 lanes of a warp rarely meet on one sample
// and the shared atomics rarely serialise; with lanes along u (ZL false) the
// lanes near a receive element's axis share a sample.
// WS: window intervals of the class (every W <= WS). Three accumulator sets
// (stages s-1, s and s+1 in flight: flushed, summed, cleared) and two raw
// window buffers and alpha tables.
template <int VU, bool CPLX, int WS>
struct BwdCfg {
    static constexpr int VR = 4 / VU;
    static constexpr int ROWS = 8 * VR;
    static constexpr int BU = 32 * VU;
    static constexpr int NWIN = kBwdCI * kBwdCJ;
    static constexpr int PLANES = CPLX ? 2 : 1;
    static constexpr int COPIES = NWIN * PLANES;
    static constexpr int RAWS = WS + 8;
    static constexpr int RAW_WIN_BYTES = RAWS * 4 * PLANES;
    static constexpr int GW = WS + 2;                // accumulator intervals per window plane (stride)
    static constexpr int GROUPS = (7 + WS + 1 + 3) / 4;   // 4-sample groups a window's cells can touch
    static constexpr int ACC_INTS = NWIN * PLANES * GW;   // one accumulator (G0 or G1)
    static constexpr int ACC_BUF = 2 * ACC_INTS;          // G0 and G1 of one stage
    static constexpr int OFF_RAW = 0;
    static constexpr int OFF_GRAD = OFF_RAW + 2 * NWIN * RAW_WIN_BYTES;   // int [3][G0, G1]
    static constexpr int OFF_TX = OFF_GRAD + 3 * ACC_BUF * 4;
    static constexpr int OFF_RX = OFF_TX + kMaxOrder * 16;
    static constexpr int OFF_ALPHA = OFF_RX + kMaxChannels * 16;       // float[2][CI][ROWS]
    static constexpr int OFF_WIN = OFF_ALPHA + 2 * kBwdCI * ROWS * 4;  // int S0[2][NWIN], int off[2][NWIN]
    static constexpr int OFF_GW = OFF_WIN + 4 * NWIN * 4;              // float[kMaxChannels]
    static constexpr int OFF_RED = OFF_GW + kMaxChannels * 4;          // float[8]
    static constexpr int OFF_MAX = OFF_RED + 32;                       // float[8]: per-warp max|G|
    static constexpr int OFF_BAR = OFF_MAX + 32;                       // uint64[2]
    static constexpr int SMEM = OFF_BAR + 16;
    static_assert(OFF_RAW % 128 == 0 && OFF_GRAD % 16 == 0 && ACC_INTS % 4 == 0 && OFF_TX % 16 == 0 &&
                  OFF_BAR % 8 == 0 && (ACC_BUF * 4) % 16 == 0, "alignment");
};

// FN: receive F# window active (a per-voxel weight W_j(v)); VEC_RED: dL/dr
// is 16-byte aligned, so window cells go out as four-float reductions.
template <int VU, bool CPLX, bool ZL, bool FN, bool VEC_RED, int WS>
__global__ void __launch_bounds__(kDasThreads, 2)
das_bwd_kernel(DasArgs a, int tail_units, int tail_parts) {
    using C = BwdCfg<VU, CPLX, WS>;
    static_assert(!ZL || VU == 1, "lanes on rows need 32 rows of 32 voxels");
    // tile row -> (v, w): z-fastest when lanes run over rows
    const StageDiv rdiv(ZL ? a.bw : a.bv);
    auto row_v = [&](int row) { return ZL ? rdiv.div(row) : rdiv.mod(row); };
    auto row_w = [&](int row) { return ZL ? rdiv.mod(row) : rdiv.div(row); };
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float4* s_tx = reinterpret_cast<float4*>(smem + C::OFF_TX);
    float4* s_rx = reinterpret_cast<float4*>(smem + C::OFF_RX);
    float* s_alpha = reinterpret_cast<float*>(smem + C::OFF_ALPHA);
    int* s_S0 = reinterpret_cast<int*>(smem + C::OFF_WIN);
    int* s_off = s_S0 + 2 * C::NWIN;
    float* s_gw = reinterpret_cast<float*>(smem + C::OFF_GW);
    float* s_red = reinterpret_cast<float*>(smem + C::OFF_RED);
    int* gwin = reinterpret_cast<int*>(smem + C::OFF_GRAD);
    float* s_max = reinterpret_cast<float*>(smem + C::OFF_MAX);
    unsigned char* raw = smem + C::OFF_RAW;
    const uint32_t bar0 = smem_u32(smem + C::OFF_BAR);

    if (tid == 0) {
        mbar_init(bar0, C::COPIES);
        mbar_init(bar0 + 8, C::COPIES);
        fence_mbar_init();
    }
    for (int q = tid; q < 3 * C::ACC_BUF; q += kDasThreads) gwin[q] = 0;
    for (int q = tid; q < kMaxChannels; q += kDasThreads) s_gw[q] = 0.f;

    // ---- unit -> (tile, channel split). The last tail_units (tile, split)
    // units run as tail_parts blocks of an equal part of the split's channel
    // chunks each, the blocks scheduled last, so the grid's last wave ends
    // within about one part's time (the partial sums go to dL/dr by atomics
    // either way)
    const int n_tiles = a.tiles_u * a.tiles_v * a.tiles_w;
    const int n_bulk = n_tiles * a.n_split - tail_units;
    const int b = (int)blockIdx.x;
    const int unit = b < n_bulk ? b : n_bulk + (b - n_bulk) / tail_parts;
    const int tile = unit % n_tiles;
    const int split = unit / n_tiles;
    const int n_ic = a.n_tx / kBwdCI;
    const StageDiv sdiv(n_ic);               // stage -> (transmit group, channel chunk)
    const int js_full = (a.n_ch / kBwdCJ) / a.n_split;
    const int js = b < n_bulk ? js_full : js_full / tail_parts;
    const int jc0 = split * js_full + (b < n_bulk ? 0 : ((b - n_bulk) % tail_parts) * js);
    const int NS = n_ic * js;

    const int tu = tile % a.tiles_u, tv = (tile / a.tiles_u) % a.tiles_v, tw = tile / (a.tiles_u * a.tiles_v);
    const int u0 = tu * C::BU, v0 = tv * a.bv, w0 = tw * a.bw;
    const double cu = u0 + 0.5 * (C::BU - 1), cv = v0 + 0.5 * (a.bv - 1), cw = w0 + 0.5 * (a.bw - 1);
    const double qx = a.q0[0] + a.Gu[0] * cu + a.Gv[0] * cv + a.Gw[0] * cw;
    const double qy = a.q0[1] + a.Gu[1] * cu + a.Gv[1] * cv + a.Gw[1] * cw;
    const double zr = a.q0[2] + a.Gu[2] * cu + a.Gv[2] * cv + a.Gw[2] * cw;
    const double lat_tx_ref = a.tx_axis ? qy : qx, lat_rx_ref = a.rx_axis ? qy : qx;
    const int j_lo = jc0 * kBwdCJ, n_rx = js * kBwdCJ;
    for (int e = tid; e < a.n_tx + n_rx; e += kDasThreads) {
        if (e < a.n_tx) {
            float tx0, tx1;
            const double d = tx_ref_distance(a, e, lat_tx_ref, zr, &tx0, &tx1);
            const double A = d * a.fs_over_c - a.t0fs;
            const double K = floor(A);
            s_tx[e] = make_float4(tx0, tx1, (float)(A - K - (double)a.lo - 0.5 - (double)a.H),
                                  __int_as_float((int)K));
        } else {
            const int j = j_lo + e - a.n_tx;
            const double L = lat_rx_ref - (a.rx_e0 + j * a.rx_pitch);
            const double d = sqrt(L * L + zr * zr);
            const double B = d * a.fs_over_c;
            const double K = floor(B);
            s_rx[j] = make_float4((float)L, (float)d, (float)(B - K), __int_as_float((int)K));
        }
    }

    // this thread's voxels: offsets, validity and the scaled upstream gradient
    const float Zf = (float)zr, fsc = (float)a.fs_over_c;
    const float Zfoc = (float)(zr - a.tx_focus);   // reference depth below the virtual line sources
    float dlr[4], dz[4], gs_re[4], gs_im[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int uu = ZL ? 4 * warp + k : lane + 32 * (k % VU);
        const int row = ZL ? lane : warp * C::VR + k / VU;
        const int rv = row_v(row), rw = row_w(row);
        const float du = (float)uu - 0.5f * (C::BU - 1);
        const float dv = (float)rv - 0.5f * (a.bv - 1);
        const float dw = (float)rw - 0.5f * (a.bw - 1);
        dlr[k] = (float)(a.rx_axis ? a.Gu[1] : a.Gu[0]) * du + (float)(a.rx_axis ? a.Gv[1] : a.Gv[0]) * dv +
                 (float)(a.rx_axis ? a.Gw[1] : a.Gw[0]) * dw;
        dz[k] = (float)a.Gu[2] * du + (float)a.Gv[2] * dv + (float)a.Gw[2] * dw;
        const int iu = u0 + uu, iv = v0 + rv, iw = w0 + rw;
        const bool in = iu < a.n_u && iv < a.n_v && iw < a.n_w;
        const long long o = (long long)iw * a.out_sw + (long long)iv * a.out_sv + (long long)iu * a.out_su;
        gs_re[k] = in ? a.grad_image[o] : 0.f;       // voxels outside the image carry no gradient
        gs_im[k] = (in && CPLX) ? a.grad_image[a.image_plane + o] : 0.f;
    }
    float g_max = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) g_max = fmaxf(g_max, fmaxf(fabsf(gs_re[k]), fabsf(gs_im[k])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) g_max = fmaxf(g_max, __shfl_xor_sync(0xffffffffu, g_max, o));
    if (lane == 0) s_max[warp] = g_max;
    __syncthreads();
#pragma unroll
    for (int w = 0; w < kDasThreads / 32; ++w) g_max = fmaxf(g_max, s_max[w]);
    // x + 1.5 * 2^23 holds round(x) in its low mantissa bits for |x| < 2^22
    // (every fixed-point term is below 2^20 in magnitude)
    constexpr float kQ = 12582912.0f;
    constexpr uint32_t kQbits = 0x4B400000u;
    float inv_scale;
    int q_re[4], q_im[4];                   // round(scaled G): the G0 term without an F# window
    {
        int ex = 0;
        frexpf(g_max, &ex);                 // max|G| < 2^ex
        const int e = min(max(20 - ex, -120), 120);
        const float scale = ldexpf(1.0f, e);
        inv_scale = ldexpf(1.0f, -e);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            gs_re[k] *= scale;
            gs_im[k] *= scale;
            q_re[k] = (int)(__float_as_uint(gs_re[k] + kQ) - kQbits);
            q_im[k] = (int)(__float_as_uint(gs_im[k] + kQ) - kQbits);
        }
    }
    const f2x gs2_re[2] = {pk(gs_re[0], gs_re[1]), pk(gs_re[2], gs_re[3])};
    const f2x gs2_im[2] = {pk(gs_im[0], gs_im[1]), pk(gs_im[2], gs_im[3])};
    const int qsum_re = q_re[0] + q_re[1] + q_re[2] + q_re[3];
    const int qsum_im = q_im[0] + q_im[1] + q_im[2] + q_im[3];

    const int es = 4;
    // stage s: raw buffer s & 1 (its window starts in s_S0 / s_off), alpha
    // table s & 1, accumulator s % 3
    auto issue = [&](int s) {
        if (tid >= C::COPIES) return;
        const int b = s & 1;
        const int win = CPLX ? (tid >> 1) : tid;
        const int plane = CPLX ? (tid & 1) : 0;
        const int ii = win / kBwdCJ, jj = win % kBwdCJ;
        const int i = sdiv.mod(s) * kBwdCI + ii, j = (jc0 + sdiv.div(s)) * kBwdCJ + jj;
        const int S0 = __float_as_int(s_tx[i].w) + __float_as_int(s_rx[j].w) + a.lo;
        const int A = S0 & ~7;
        if (plane == 0) { s_off[b * C::NWIN + win] = S0 - A; s_S0[b * C::NWIN + win] = S0; }
        const int lo_s = max(A, 0), hi_s = min(A + a.raw_samples, a.n_s);
        unsigned char* dst = raw + (b * C::NWIN + win) * C::RAW_WIN_BYTES + plane * C::RAWS * 4;
        const int pre = (min(lo_s, A + a.raw_samples) - A) * es;
        const int body = hi_s > lo_s ? (hi_s - lo_s) * es : 0;
        const int total = a.raw_samples * es;
        for (int o = 0; o < pre; o += 16) *reinterpret_cast<uint4*>(dst + o) = make_uint4(0, 0, 0, 0);
        for (int o = pre + body; o < total; o += 16) *reinterpret_cast<uint4*>(dst + o) = make_uint4(0, 0, 0, 0);
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar0 + 8 * b, (uint32_t)body);
        if (body > 0) {
            const char* src = static_cast<const char*>(a.rf) +
                ((long long)plane * a.plane_stride + ((long long)i * a.n_ch + j) * a.n_s + lo_s) * es;
            bulk_g2s(smem_u32(dst + pre), src, (uint32_t)body, bar0 + 8 * b);
        }
    };
    // transmit terms of stage s for every tile row
    const float gvt_row = (float)(a.tx_axis ? a.Gv[1] : a.Gv[0]), gwt_row = (float)(a.tx_axis ? a.Gw[1] : a.Gw[0]);
    const float gvz_row = (float)a.Gv[2], gwz_row = (float)a.Gw[2];
    auto make_alpha = [&](int s) {
        // the last warps (warp 0 issues the copies)
        const int at = tid - (kDasThreads - kBwdCI * C::ROWS);
        if (at < 0) return;
        const int ii = at / C::ROWS, row = at % C::ROWS;
        const float dv = (float)row_v(row) - 0.5f * (a.bv - 1);
        const float dw = (float)row_w(row) - 0.5f * (a.bw - 1);
        const float dL = gvt_row * dv + gwt_row * dw;
        const float dzz = gvz_row * dv + gwz_row * dw;
        const float4 tx = s_tx[sdiv.mod(s) * kBwdCI + ii];
        const float al = tx_offset(a.tx_wave, tx, dL, dzz, Zf, Zfoc, fsc);
        s_alpha[(s & 1) * kBwdCI * C::ROWS + ii * C::ROWS + row] = fminf(fmaxf(al, tx.z - a.reach_a), tx.z + a.reach_a);
    };

    make_alpha(0);
    __syncthreads();

    const float hp = 0.5f + (float)a.H;
    // per channel of the chunk: w_j and the dL/dw_j partial; per (voxel,
    // channel): beta + 0.5 + H and (F# window) W_j(v)
    // receive terms of voxel pairs (k, k+1) packed in f32x2 registers
    f2x betah2[2][kBwdCJ];
    uint32_t merge_ok = 0;                  // bit jj: channel jj's receive terms lie within one sample
    float win_w[FN ? 4 : 1][kBwdCJ], wj[kBwdCJ], pw[kBwdCJ];
    float gc = 0.f;                         // dL/dc partial (times -c, scaled)
    bool ok = true;
    uint32_t phase = 0;                     // parity of each raw buffer's next phase
    constexpr uint32_t kG1 = 4u * C::ACC_INTS;                  // G1 after G0
    constexpr uint32_t kIm = 4u * C::NWIN * C::GW;              // plane 1 after plane 0

    // Iteration s: copy the windows of stage s; accumulate stage s (the sums
    // need the window starts only, not the samples); flush stage s-1 (its
    // windows were copied a whole iteration earlier); compute the transmit
    // terms of stage s+1 and clear the accumulator of stage s+1 (last flushed
    // in the previous iteration). One barrier per iteration orders every
    // hand-over: accumulator s is complete before its flush in iteration s+1
    // and cleared in iteration s+2 before stage s+3 uses it. The channel
    // weights and dL/dw partials follow the flushed stage's channel chunk.
    for (int s = 0; s <= NS; ++s) {
        if (s < NS) issue(s);
        if (s < NS) {
            const int ic = sdiv.mod(s), jc = jc0 + sdiv.div(s);
            if (ic == 0) {
#pragma unroll
                for (int jj = 0; jj < kBwdCJ; ++jj) {
                    const float4 rx = s_rx[jc * kBwdCJ + jj];
                    float bt[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float Zv = Zf + dz[k];
                        const float Lv = rx.x + dlr[k];
                        const float d = sqrtf(Lv * Lv + Zv * Zv);
                        const float num = dlr[k] * (2.0f * rx.x + dlr[k]) + dz[k] * (2.0f * Zf + dz[k]);
                        const float b0 = rx.z + __fdividef(num, d + rx.y) * fsc;
                        bt[k] = fminf(fmaxf(b0, rx.z - a.reach_b), rx.z + a.reach_b) + hp;
                        if (FN) win_w[FN ? k : 0][jj] = hann_weight(a.f_number, Lv, Zv);
                    }
                    betah2[0][jj] = pk(bt[0], bt[1]);
                    betah2[1][jj] = pk(bt[2], bt[3]);
                    if (ZL) {
                        // the thread's four voxels differ only in their receive terms:
                        // if these lie within one sample in every lane, so do the
                        // delays of every transmit, and the voxels span at most two
                        // adjacent intervals (no per-window test needed)
                        const float spread = fmaxf(fmaxf(bt[0], bt[1]), fmaxf(bt[2], bt[3])) -
                                             fminf(fminf(bt[0], bt[1]), fminf(bt[2], bt[3]));
                        const uint32_t m = __reduce_max_sync(0xffffffffu, __float_as_uint(spread));
                        merge_ok = (merge_ok & ~(1u << jj)) | (__uint_as_float(m) < 1.0f ? 1u << jj : 0u);
                    }
                }
            }

            // ---- interval sums G0, G1 of every window of stage s. With uh =
            // u + 0.5 + H (u the window-relative delay), the interval is
            // n = round(uh - 0.5) and the fraction f = uh - n: t = uh + 2^23 - 0.5
            // holds n in its low mantissa bits.
            const uint32_t abase = smem_u32(gwin + (s % 3) * C::ACC_BUF) - (0x4B000000u << 2);
            const float* alp = s_alpha + (s & 1) * kBwdCI * C::ROWS;
#pragma unroll 1
            for (int ii = 0; ii < kBwdCI; ++ii) {
                const float al_row = ZL ? alp[ii * C::ROWS + lane] : 0.f;
#pragma unroll
                for (int jj = 0; jj < kBwdCJ; ++jj) {
                    const int win = ii * kBwdCJ + jj;
                    const uint32_t wb0 = abase + 4u * (uint32_t)(win * C::GW);      // G0, plane 0
                    // the four voxels' intervals (t holds the interval in its low
                    // bits) and fractions, voxel pairs in f32x2 registers
                    uint32_t tb[4];
                    float fr[4];
                    f2x fr2[2];
#pragma unroll
                    for (int kp = 0; kp < 2; ++kp) {
                        const float a0 = ZL ? al_row : alp[ii * C::ROWS + warp * C::VR + (2 * kp) / VU];
                        const float a1v = ZL ? al_row : alp[ii * C::ROWS + warp * C::VR + (2 * kp + 1) / VU];
                        const f2x uh2 = add2(pk(a0, a1v), betah2[kp][jj]);
                        const f2x t2 = add2(uh2, pk(8388607.5f, 8388607.5f));
                        fr2[kp] = fma2(add2(t2, pk(-8388608.0f, -8388608.0f)), pk(-1.0f, -1.0f), uh2);
                        float t0, t1;
                        upk(t2, t0, t1);
                        tb[2 * kp] = __float_as_uint(t0);
                        tb[2 * kp + 1] = __float_as_uint(t1);
                        upk(fr2[kp], fr[2 * kp], fr[2 * kp + 1]);
                    }
                    // fixed-point G1 terms round(g f): the float bits of g f + 1.5 * 2^23
                    // (without an F# window g is the voxel's scaled gradient)
                    uint32_t bq[2][4];
                    if constexpr (!FN) {
#pragma unroll
                        for (int p = 0; p < (CPLX ? 2 : 1); ++p) {
#pragma unroll
                            for (int kp = 0; kp < 2; ++kp) {
                                float x0, x1;
                                upk(fma2(p ? gs2_im[kp] : gs2_re[kp], fr2[kp], pk(kQ, kQ)), x0, x1);
                                bq[p][2 * kp] = __float_as_uint(x0);
                                bq[p][2 * kp + 1] = __float_as_uint(x1);
                            }
                        }
                    }
                    // With lanes over z a thread's four voxels are consecutive along
                    // u. Where the delay changes slowly along u they fall into at
                    // most two adjacent intervals in every lane: then per plane the
                    // interval sums go out as two or four reductions, not eight.
                    uint32_t span = 2;
                    uint32_t tmin = 0;
                    if (ZL) {
                        tmin = min(min(tb[0], tb[1]), min(tb[2], tb[3]));
                        span = (merge_ok >> jj) & 1u ? 1u
                             : __reduce_max_sync(0xffffffffu, max(max(tb[0], tb[1]), max(tb[2], tb[3])) - tmin);
                    }
                    if (ZL && span <= 1) {
                        const uint32_t s0 = (tmin << 2) + wb0;
                        uint32_t d[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) d[k] = tb[k] - tmin;             // 0 or 1
                        const uint32_t dsum = d[0] + d[1] + d[2] + d[3];
#pragma unroll
                        for (int p = 0; p < (CPLX ? 2 : 1); ++p) {
                            uint32_t lo0, hi0, lo1, hi1;
                            if constexpr (!FN) {
                                // sums over the voxels of the upper interval (d = 1) and of
                                // all four, in wrapping 32-bit arithmetic (the true values fit)
                                const int* q = p ? q_im : q_re;
                                hi0 = d[0] * (uint32_t)q[0] + d[1] * (uint32_t)q[1] + d[2] * (uint32_t)q[2] +
                                      d[3] * (uint32_t)q[3];
                                lo0 = (uint32_t)(p ? qsum_im : qsum_re) - hi0;
                                const uint32_t hb = d[0] * bq[p][0] + d[1] * bq[p][1] + d[2] * bq[p][2] + d[3] * bq[p][3];
                                const uint32_t sb = bq[p][0] + bq[p][1] + bq[p][2] + bq[p][3];
                                hi1 = hb - dsum * kQbits;
                                lo1 = sb - hb - (4u - dsum) * kQbits;
                            } else {
                                int qs = 0, a1 = 0, g1 = 0, b1 = 0;
#pragma unroll
                                for (int k = 0; k < 4; ++k) {
                                    const float g = (p ? gs_im[k] : gs_re[k]) * win_w[FN ? k : 0][jj];
                                    const int qk = (int)(__float_as_uint(g + kQ) - kQbits);
                                    const int q1 = (int)(__float_as_uint(fmaf(g, fr[k], kQ)) - kQbits);
                                    qs += qk;
                                    a1 += (int)d[k] * qk;
                                    g1 += q1;
                                    b1 += (int)d[k] * q1;
                                }
                                lo0 = (uint32_t)(qs - a1);
                                hi0 = (uint32_t)a1;
                                lo1 = (uint32_t)(g1 - b1);
                                hi1 = (uint32_t)b1;
                            }
                            const uint32_t sp0 = s0 + (p ? kIm : 0u);
                            asm volatile("red.shared.add.s32 [%0], %1;" :: "r"(sp0), "r"(lo0) : "memory");
                            asm volatile("red.shared.add.s32 [%0], %1;" :: "r"(sp0 + kG1), "r"(lo1) : "memory");
                            if (span == 1) {
                                asm volatile("red.shared.add.s32 [%0], %1;" :: "r"(sp0 + 4u), "r"(hi0) : "memory");
                                asm volatile("red.shared.add.s32 [%0], %1;" :: "r"(sp0 + 4u + kG1), "r"(hi1) : "memory");
                            }
                        }
                        continue;
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t g0 = (tb[k] << 2) + wb0;
#pragma unroll
                        for (int p = 0; p < (CPLX ? 2 : 1); ++p) {
                            int qk, q1;
                            if constexpr (!FN) {
                                qk = p ? q_im[k] : q_re[k];
                                q1 = (int)(bq[p][k] - kQbits);
                            } else {
                                const float g = (p ? gs_im[k] : gs_re[k]) * win_w[FN ? k : 0][jj];
                                qk = (int)(__float_as_uint(g + kQ) - kQbits);
                                q1 = (int)(__float_as_uint(fmaf(g, fr[k], kQ)) - kQbits);
                            }
                            const uint32_t gp = g0 + (p ? kIm : 0u);
                            asm volatile("red.shared.add.s32 [%0], %1;" :: "r"(gp), "r"(qk) : "memory");
                            asm volatile("red.shared.add.s32 [%0], %1;" :: "r"(gp + kG1), "r"(q1) : "memory");
                        }
                    }
                }
            }
            if (s + 1 < NS) make_alpha(s + 1);
        }
        if (s > 0) {
            // ---- flush stage t = s - 1: accumulators -> dL/dr = w_j c, dL/dw_j
            // and dL/dc partials. Cells go out in groups of four samples
            // starting at a multiple of 4 (window starts are A + off with A a
            // multiple of 8; traces are multiples of 8 long, so a group lies
            // wholly inside or wholly outside its trace).
            const int t = s - 1, tb = t & 1;
            const int ic = sdiv.mod(t), jc = jc0 + sdiv.div(t);
            ok = mbar_wait_parity(bar0 + 8 * tb, (phase >> tb) & 1u, a.wait_ns) && ok;
            phase ^= 1u << tb;
            const int* acc = gwin + (t % 3) * C::ACC_BUF;
            if (ic == 0) {
#pragma unroll
                for (int jj = 0; jj < kBwdCJ; ++jj) {
                    wj[jj] = a.apod ? __ldg(a.apod + jc * kBwdCJ + jj) : 1.0f;
                    pw[jj] = 0.f;
                }
            }
            // the items beyond a whole number per thread go to warps 1 and 2,
            // which neither issue copies nor compute transmit terms
            const int ft = (tid + kDasThreads - 32) % kDasThreads;
            for (int q = ft; q < C::NWIN * C::PLANES * C::GROUPS; q += kDasThreads) {
                const int g = q % C::GROUPS, wp = q / C::GROUPS;
                const int win = wp % C::NWIN, plane = wp / C::NWIN;
                const int off = s_off[tb * C::NWIN + win];
                const int n0 = 4 * g - off;
                if (n0 > a.W) continue;
                const int* G0 = acc + (plane * C::NWIN + win) * C::GW;
                const int* G1 = G0 + C::ACC_INTS;
                // intervals n0-1 .. n0+3 (valid ones are 0 .. W-1)
                int g0[4], g1[5];
#pragma unroll
                for (int e = 0; e < 5; ++e) {
                    const int n = n0 - 1 + e;
                    const bool in = n >= 0 && n < a.W;
                    g1[e] = in ? G1[n] : 0;
                    if (e > 0) g0[e - 1] = in ? G0[n] : 0;
                }
                if ((g0[0] | g0[1] | g0[2] | g0[3] | g1[0] | g1[1] | g1[2] | g1[3] | g1[4]) == 0) continue;
                // raw sample of cell n is at window index off + n = 4g + e
                const float* rw = reinterpret_cast<const float*>(raw + (tb * C::NWIN + win) * C::RAW_WIN_BYTES +
                                                                 plane * C::RAWS * 4) + 4 * g;
                const float4 r4 = *reinterpret_cast<const float4*>(rw);
                const float r5 = (n0 + 3 < a.W) ? rw[4] : 0.f;     // right end of interval n0+3
                const float rr[5] = {r4.x, r4.y, r4.z, r4.w, r5};
                const float cwin = (float)s_S0[tb * C::NWIN + win] + (float)a.t0fs + (float)n0;
                float c4[4], pr = 0.f, pc = 0.f;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    // exact in wrapping 32-bit arithmetic: |c| < 1024 * 2^20 (every term of
                    // the tile is below 2^20 and weighs at most one)
                    c4[e] = (float)(int)((uint32_t)g0[e] - (uint32_t)g1[e + 1] + (uint32_t)g1[e]);
                    pr = fmaf(rr[e], c4[e], pr);
                    // interval n0+e: slope times position-weighted sum
                    pc = fmaf(rr[e + 1] - rr[e], fmaf((float)e + cwin, (float)g0[e], (float)g1[e + 1]), pc);
                }
                const int jj = win % kBwdCJ;
                float w_sel = 1.f;
#pragma unroll
                for (int u = 0; u < kBwdCJ; ++u) {
                    if (u == jj) {
                        pw[u] += pr;
                        w_sel = wj[u];
                    }
                }
                gc = fmaf(w_sel, pc, gc);
                const int S = s_S0[tb * C::NWIN + win] - off + 4 * g;
                if (S < 0 || S >= a.n_s || !a.grad_rf) continue;
                const int ii = win / kBwdCJ;
                const int i = ic * kBwdCI + ii, j = jc * kBwdCJ + jj;
                float* dst = a.grad_rf + (long long)plane * a.plane_stride + ((long long)i * a.n_ch + j) * a.n_s + S;
                const float m = w_sel * inv_scale;
                if (VEC_RED) {
                    asm volatile("red.global.add.v4.f32 [%0], {%1,%2,%3,%4};"
                                 :: "l"(dst), "f"(c4[0] * m), "f"(c4[1] * m), "f"(c4[2] * m), "f"(c4[3] * m)
                                 : "memory");
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (c4[e] != 0.f) atomicAdd(dst + e, c4[e] * m);
                }
            }
            if (ic == n_ic - 1) {
                // this channel chunk is complete: dL/dw_j partials
#pragma unroll
                for (int jj = 0; jj < kBwdCJ; ++jj) {
                    float v = pw[jj];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0 && v != 0.f) atomicAdd(s_gw + jc * kBwdCJ + jj, v * inv_scale);
                }
            }
        }
        // clear the accumulator of stage s+1 (it held stage s-2, flushed in
        // the previous iteration)
        {
            int4* clr = reinterpret_cast<int4*>(gwin + ((s + 1) % 3) * C::ACC_BUF);
            const int ct = (tid + kDasThreads - 96) % kDasThreads;     // the remainder to warp 3
            for (int q = ct; q < C::ACC_BUF / 4; q += kDasThreads) clr[q] = make_int4(0, 0, 0, 0);
        }
        if (__syncthreads_or(!ok)) {
            // a bounded wait expired: give the copies still in flight (stages
            // s and, if its wait failed, s-1) a bounded chance to land, then stop
            if (s < NS) mbar_wait_parity(bar0 + 8 * (s & 1), (phase >> (s & 1)) & 1u, a.wait_ns);
            if (s > 0) mbar_wait_parity(bar0 + 8 * ((s - 1) & 1), ((phase >> ((s - 1) & 1)) & 1u) ^ 1u, a.wait_ns);
            if (tid == 0) atomicOr(a.status, kStatusWaitExpired);
            return;
        }
    }

    // ---- dL/dc and dL/dw partials of this unit
    if (a.grad_c) {
        float v = gc * inv_scale;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_red[warp] = v;
        __syncthreads();
        if (tid == 0) {
            float t = 0.f;
            for (int w = 0; w < kDasThreads / 32; ++w) t += s_red[w];
            atomicAdd(a.grad_c, -t / (float)a.c);
        }
    }
    if (a.grad_apod) {
        __syncthreads();
        for (int j = j_lo + tid; j < j_lo + n_rx; j += kDasThreads)
            if (s_gw[j] != 0.f) atomicAdd(a.grad_apod + j, s_gw[j]);
    }
}

// Plain form: one thread per voxel, FP32 distances, global atomics.
template <bool CPLX>
__global__ void __launch_bounds__(128)
das_bwd_plain_kernel(DasArgs a) {
    const long long n_vox = (long long)a.n_u * a.n_v * a.n_w;
    const long long vox = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (vox >= n_vox) return;
    const int iu = (int)(vox % a.n_u), iv = (int)((vox / a.n_u) % a.n_v), iw = (int)(vox / ((long long)a.n_u * a.n_v));
    const float qx = (float)a.q0[0] + (float)a.Gu[0] * iu + (float)a.Gv[0] * iv + (float)a.Gw[0] * iw;
    const float qy = (float)a.q0[1] + (float)a.Gu[1] * iu + (float)a.Gv[1] * iv + (float)a.Gw[1] * iw;
    const float z = (float)a.q0[2] + (float)a.Gu[2] * iu + (float)a.Gv[2] * iv + (float)a.Gw[2] * iw;
    const float lat_tx = a.tx_axis ? qy : qx, lat_rx = a.rx_axis ? qy : qx;
    const long long o = (long long)iw * a.out_sw + (long long)iv * a.out_sv + (long long)iu * a.out_su;
    const float gre = a.grad_image[o], gim = CPLX ? a.grad_image[a.image_plane + o] : 0.f;
    const float fsc = (float)a.fs_over_c, t0fs = (float)a.t0fs, inv_c = 1.0f / (float)a.c;
    const float* rf = static_cast<const float*>(a.rf);
    float gc = 0.f;
    for (int j = 0; j < a.n_ch; ++j) {
        const float dxr = lat_rx - ((float)a.rx_e0 + j * (float)a.rx_pitch);
        const float drx = sqrtf(dxr * dxr + z * z);
        const float W = a.f_number > 0.f ? hann_weight(a.f_number, dxr, z) : 1.0f;
        if (W == 0.f) continue;
        const float a_j = (a.apod ? __ldg(a.apod + j) : 1.0f) * W;
        float gw = 0.f;
        for (int i = 0; i < a.n_tx; ++i) {
            const float dtx = tx_distance_f32(a, i, lat_tx, z);
            const float s = (dtx + drx) * fsc - t0fs;
            const float fl = floorf(s);
            const float f = s - fl;
            const int n = (int)fl;
            const long long base = ((long long)i * a.n_ch + j) * a.n_s;
            const bool in0 = n >= 0 && n < a.n_s, in1 = n + 1 >= 0 && n + 1 < a.n_s;
            for (int p = 0; p < (CPLX ? 2 : 1); ++p) {
                const float g = p ? gim : gre;
                const long long pb = p * a.plane_stride + base;
                const float r0 = in0 ? __ldg(rf + pb + n) : 0.f;
                const float r1 = in1 ? __ldg(rf + pb + n + 1) : 0.f;
                if (a.grad_rf && g != 0.f) {
                    if (in0) atomicAdd(a.grad_rf + pb + n, a_j * g * (1.0f - f));
                    if (in1) atomicAdd(a.grad_rf + pb + n + 1, a_j * g * f);
                }
                gc += a_j * g * (r1 - r0) * (s + t0fs);
                gw += g * ((1.0f - f) * r0 + f * r1);
            }
        }
        if (a.grad_apod && gw != 0.f) atomicAdd(a.grad_apod + j, W * gw);
    }
    if (a.grad_c) {
        float v = gc;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0) atomicAdd(a.grad_c, -v * inv_c);
    }
}

// channel split and tail: units of a tile and a power-of-two part of its
// channel chunks, at least kBwdMinWaves waves of them, the last 3/4 wave of
// units split into up to kBwdTailParts blocks each. Measured on the autofocus
// workload (128 tiles, 32 chunks, 304 CTA slots): 16 splits without a tail
// 2.508 ms; 16 splits, the last 3/4 or 1 wave halved 2.447, 2.442 ms; 8
// splits, the last 3/4 wave in quarters 2.436 ms; 8 splits with a halved
// wave 2.506 ms; 4 splits with a wave in quarters 2.495 ms.
constexpr long long kBwdMinWaves = 3;
constexpr int kBwdTailParts = 4;
constexpr long long kBwdTailQuarters = 3;

template <int VU, bool CPLX, bool ZL, bool FN, bool VEC_RED, int WS>
int launch_bwd_tiled_v(const PlanHost& h, DasArgs a, cudaStream_t s) {
    using C = BwdCfg<VU, CPLX, WS>;
    auto k = das_bwd_kernel<VU, CPLX, ZL, FN, VEC_RED, WS>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) != cudaSuccess)
        return check_launch("das_backward: set shared memory");
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kDasThreads, C::SMEM) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const long long tiles = (long long)a.tiles_u * a.tiles_v * a.tiles_w;
    const long long slots = (long long)h.n_sms * per_sm;
    const int chunks = a.n_ch / kBwdCJ;
    int sp = 1;
    while (tiles * sp < kBwdMinWaves * slots && sp * 2 <= chunks && chunks % (sp * 2) == 0 && sp < 32) sp *= 2;
    a.n_split = sp;
    // tail: the last units split into parts (when a unit's chunks divide)
    const long long units = tiles * sp;
    int parts = 1;
    while (parts * 2 <= kBwdTailParts && (chunks / sp) % (parts * 2) == 0) parts *= 2;
    const int tail = parts > 1 ? (int)std::min(units, kBwdTailQuarters * slots / 4) : 0;
    const unsigned grid = (unsigned)(units + (long long)tail * (parts - 1));
    k<<<grid, kDasThreads, C::SMEM, s>>>(a, tail, parts);
    return check_launch("das_bwd_kernel");
}

template <int VU, bool CPLX, bool ZL, int WS>
int launch_bwd_tiled_ws(const PlanHost& h, const DasArgs& a, cudaStream_t s) {
    const bool fn = a.f_number > 0.f;
    const bool vec = (reinterpret_cast<uintptr_t>(a.grad_rf) & 15u) == 0;
    if (fn) return vec ? launch_bwd_tiled_v<VU, CPLX, ZL, true, true, WS>(h, a, s)
                       : launch_bwd_tiled_v<VU, CPLX, ZL, true, false, WS>(h, a, s);
    return vec ? launch_bwd_tiled_v<VU, CPLX, ZL, false, true, WS>(h, a, s)
               : launch_bwd_tiled_v<VU, CPLX, ZL, false, false, WS>(h, a, s);
}

// Windows of up to 96 intervals keep two CTAs per SM (the 96 class, built for
// the lanes-over-z tile of the autofocus path); larger ones use the 128 class.
template <int VU, bool CPLX, bool ZL>
int launch_bwd_tiled(const PlanHost& h, const DasArgs& a, cudaStream_t s) {
    if constexpr (ZL) {
        if (a.W <= 96) return launch_bwd_tiled_ws<VU, CPLX, ZL, 96>(h, a, s);
    }
    return launch_bwd_tiled_ws<VU, CPLX, ZL, 128>(h, a, s);
}

}  // namespace

int launch_das_backward(const PlanHost& h, const DasArgs& a, int mode, cudaStream_t s) {
    const bool cplx = a.dtype == RCBF_CF32;
    if (mode == 0) {
        const long long n_vox = (long long)a.n_u * a.n_v * a.n_w;
        const unsigned grid = (unsigned)((n_vox + 127) / 128);
        if (cplx) das_bwd_plain_kernel<true><<<grid, 128, 0, s>>>(a);
        else das_bwd_plain_kernel<false><<<grid, 128, 0, s>>>(a);
        return check_launch("das_bwd_plain_kernel");
    }
    if (mode == 2) {
        if (a.bu != 32) return set_error(RCBF_EINVAL, "das_backward: the adjoint tile needs 32 voxels along u");
        return cplx ? launch_bwd_tiled<1, true, true>(h, a, s) : launch_bwd_tiled<1, false, true>(h, a, s);
    }
    switch (h.vu) {
        case 1: return cplx ? launch_bwd_tiled<1, true, false>(h, a, s) : launch_bwd_tiled<1, false, false>(h, a, s);
        case 2: return cplx ? launch_bwd_tiled<2, true, false>(h, a, s) : launch_bwd_tiled<2, false, false>(h, a, s);
        default: return cplx ? launch_bwd_tiled<4, true, false>(h, a, s) : launch_bwd_tiled<4, false, false>(h, a, s);
    }
}

}  // namespace rcbf

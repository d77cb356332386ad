// das_tile.cuh — one work unit (a voxel tile x a range of receive channels)
// of the delay-and-sum of Eq. (1) (§THEORY "Synthetic Aperture Imaging";
// §OPTIMIZATIONS "DAS").
//
// A CTA of 256 threads beamforms a tile of 1024 voxels, 4 per thread, and
// walks its part of the (transmit, channel) plane in stages of CI x CJ
// windows. A plan may split the channels of a tile over several units (to
// fill every SM); each unit then writes a partial image and a reduce kernel
// adds the partials in a fixed order, or (the batch form) adds its sums into
// the image itself once the previous split of its tile has (tile_flags).
//
// Delays. For the tile centre q_ref the FP64 reference distance of every
// element is split into an integer sample K and a fractional remainder; a
// voxel's delay to element e is then
//   K_e + rho_e + (d_e(v) - d_e(ref)) * fs / c,
//   d_e(v) - d_e(ref) = (dL (2L + dL) + dZ (2Z + dZ)) / (d_e(v) + d_e(ref))
// evaluated in FP32 (no cancellation: dL, dZ are the voxel's offsets from
// q_ref, L = lat(q_ref) - e, Z = z(q_ref)). The separable row-column delay
// s_ij = A_i + B_j (transmit line i, receive line j) needs one such term per
// (voxel, transmit) and per (voxel, channel), never per (voxel, i, j).
//
// Cubic Hermite (CUBIC): each window copy starts one sample earlier and the
// pieces hold the interval's cubic in its local fraction f,
//   r(f) = a0 + f (a1 + f (a2 + f a3)),  a0 = r[n], a1 = m_n,
//   a2 = 3 (r[n+1] - r[n]) - 2 m_n - m_{n+1},  a3 = 2 (r[n] - r[n+1]) + m_n + m_{n+1},
// with the central-difference slopes m_k = (r[k+1] - r[k-1]) / 2; the inner
// loop takes f from the same rounding of t (one 16-byte load, three FMAs).
//
// IQ beamforming (IQ, complex data demodulated at f_d): each interpolated
// baseband sample is multiplied by e^{j 2 pi r s}, r = f_d / f_s, s the
// absolute fractional sample. Per window the phase of its start, frac(r S0),
// is taken in FP64 when the window is rewritten; per term the phase is
// frac(that + r u) (u the window-relative position), and the rotation is one
// sincos and a complex product.
//
// 2D receive aperture (D2, HERCULES read as a 2D array): the receive path of
// row i and column j is d = sqrt(P_i + Q_j), P_i = (lat_tx - e_i)^2 + z^2 and
// Q_j = (lat_rx - e_j)^2, so the tables keep P per (tile row, transmit) and Q
// per (voxel, channel) where the separable form keeps alpha and beta, and a
// sum costs P + Q, one approximate square root and one FMA more.
// Each (i, j) window starts below the smallest delay that the tile's bounding
// box admits (the box minima of P and Q and of the transmit wave's path: a
// plane wave's path is linear, a diverging wave's convex, so both have exact
// box bounds); P, Q and the transmit path are clamped to their box bounds per
// voxel, so every index lands inside the window.
//
// Windows. Every (i, j) trace is read only inside the window
// [K_i + K_j + lo, K_i + K_j + lo + W] that the tile can reach (W from the
// tile radius, a 1-Lipschitz bound of the distances). The 1-D TMA bulk engine
// copies each window into shared memory, where it is rewritten as W line
// pieces (c_n, slope_n): r(x) = c_n + u * slope_n on sample interval n, u
// being the window-centred position. The inner loop per voxel and (i, j) is
// then: u = alpha_i + beta_j; t = u + 2^23 + H (the low bits of t are the
// interval n); one 8-byte shared load; one FMA for the interpolated sample;
// one add (or FMA with the apodization weight a_j(v) of Eq. (2)-(3)).
//
// Pipeline (no CTA-wide barrier per stage): two raw-window buffers and three
// line-piece buffers, each with a "full" and an "empty" mbarrier. In stage s a
// thread (i) if it issues copies, waits until the raw buffer of stage s is
// drained and refills it with stage s+2, (ii) rewrites its share of the raw
// windows of stage s+1 once they have landed and the line-piece buffer of
// stage s-2 is free, (iii) sums stage s once every share of it is written.
// Warps drift apart by up to a stage instead of meeting at a barrier.
#pragma once

#include <type_traits>

#include "internal.cuh"

namespace rcbf {

template <int I, int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

template <int VU, int WS, bool CPLX, bool CUBIC = false, bool D2 = false, bool APOD = false, bool IQ = false>
struct DasCfg {
    static constexpr int VR = 4 / VU;              // tile rows per thread
    static constexpr int ROWS = 8 * VR;            // tile rows (one warp covers VR rows)
    static constexpr int BU = 32 * VU;             // tile extent along u
    // transmits per stage, so that three line-piece buffers and two raw
    // buffers fit two CTAs per SM for every window class
    static constexpr int CI_BASE = (WS <= 48 ? 8 : WS <= 96 ? 4 : 2) / (CPLX ? 2 : 1) / (CUBIC ? 2 : 1);
    static constexpr int CI = CI_BASE > 0 ? CI_BASE : 1;
    static constexpr int CJ = 8;                   // channels per stage
    static constexpr int NWIN = CI * CJ;           // windows per stage
    static constexpr int COPIES = NWIN * (CPLX ? 2 : 1);   // bulk copies per stage (windows x planes)
    static constexpr int NB = 3;                   // line-piece buffers
    static constexpr int PAIR_BYTES = (CPLX ? 16 : 8) * (CUBIC ? 2 : 1);   // one piece (all planes)
    static constexpr int SHIFT = CPLX ? (CUBIC ? 5 : 4) : (CUBIC ? 4 : 3);  // log2(PAIR_BYTES)
    static constexpr int RAWS = WS + (CUBIC ? 16 : 8);   // raw samples per window plane (max)
    static constexpr int RAW_WIN_BYTES = RAWS * 4 * (CPLX ? 2 : 1);
    static constexpr int PAIR_BUF = NWIN * WS * PAIR_BYTES;
    static constexpr int ALPHA_N = CI * ROWS;      // transmit terms per stage
    // transmit terms ordered by warp (VR rows), then transmit, then row, so a
    // warp reads the CI x VR terms of its rows from consecutive words
    static __device__ __forceinline__ int alpha_index(int ii, int row) {
        return (row / VR) * (CI * VR) + ii * VR + row % VR;
    }
    static constexpr int OFF_PAIRS = 0;                                // NB line-piece buffers
    static constexpr int OFF_RAW = OFF_PAIRS + NB * PAIR_BUF;          // 2 raw window buffers
    static constexpr int OFF_TX = OFF_RAW + 2 * NWIN * RAW_WIN_BYTES;  // float4[kMaxOrder]
    static constexpr int OFF_RX = OFF_TX + kMaxOrder * 16;             // float4[kMaxChannels]
    static constexpr int OFF_ALPHA = OFF_RX + kMaxChannels * 16;       // float[NB][CI][ROWS]
    static constexpr int OFF_WOFF = OFF_ALPHA + NB * ALPHA_N * 4;      // int[2][NWIN]
    static constexpr int OFF_WPH = OFF_WOFF + 2 * NWIN * 4;            // float[NB][NWIN]: 2D IQ window phases
    static constexpr int OFF_WS0 = OFF_WPH + (IQ && D2 ? NB * NWIN * 4 : 0);   // float[NB][NWIN]: 2D window starts
    static constexpr int OFF_ACT = OFF_WS0 + (D2 ? NB * NWIN * 4 : 0); // int[chunks + 1]: active channel chunks, count (APOD)
    // IQ: carrier phases (cycles) of the transmit and receive parts of every
    // window start
    static constexpr int OFF_TXPH = ((OFF_ACT + (APOD ? (kMaxChannels / CJ + 1) * 4 : 0) + 7) / 8) * 8;  // float[kMaxOrder]
    static constexpr bool IQ_SEP = IQ && !D2;    // separable delays: the rotation factorises
    static constexpr int OFF_RXPH = OFF_TXPH + (IQ_SEP ? kMaxOrder * 4 : 0);                          // float[kMaxChannels]
    static constexpr int OFF_BAR = OFF_RXPH + (IQ_SEP ? kMaxChannels * 4 : 0);                        // uint64[10]
    static constexpr int OFF_ABORT = OFF_BAR + 80;                     // int: a bounded wait expired
    static constexpr int SMEM = OFF_ABORT + 16;
    static_assert(ALPHA_N <= kDasThreads, "one thread per transmit term");
    static_assert(COPIES <= kDasThreads, "one issuing thread per copy");
    static_assert(OFF_RAW % 128 == 0 && OFF_TX % 16 == 0 && OFF_BAR % 8 == 0, "alignment");
    static_assert(2 * SMEM + 2048 <= 232448, "two CTAs per SM");
};

template <int OFF>
__device__ __forceinline__ float2 lds_f2(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0,%1}, [%2+%3];" : "=f"(v.x), "=f"(v.y) : "r"(addr), "n"(OFF));
    return v;
}
template <int OFF>
__device__ __forceinline__ float4 lds_f4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4+%5];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr), "n"(OFF));
    return v;
}

// Packed FP32 pairs (sm_100+ f32x2 arithmetic): two voxels per instruction.
typedef unsigned long long f2x;
__device__ __forceinline__ f2x pk(float lo, float hi) {
    f2x r;
    asm("mov.b64 %0, {%1,%2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(f2x v, float& lo, float& hi) {
    asm("mov.b64 {%0,%1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2x add2(f2x a, f2x b) {
    f2x r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c) {
    f2x r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Eq. (3) window at u = F# |lat| / |z|, support test F# |lat| < 0.5 |z|.
__device__ __forceinline__ float hann_weight(float f_number, float lat, float z) {
    const float al = f_number * fabsf(lat), az = fabsf(z);
    if (!(al < 0.5f * az)) return 0.0f;
    const float cs = cospif(al / az);
    return cs * cs;
}

template <class T> __device__ __forceinline__ float to_f32(T v, float scale);
template <> __device__ __forceinline__ float to_f32<float>(float v, float) { return v; }
template <> __device__ __forceinline__ float to_f32<__half>(__half v, float) { return __half2float(v); }
template <> __device__ __forceinline__ float to_f32<int>(int v, float scale) { return (float)v * scale; }

// Raw windows of one stage -> line pieces, a half-warp per window (a warp
// covers two windows per pass), K = WS / 16 intervals per lane. In the
// 48-interval class, and for complex pieces in every class, lane l takes
// intervals l, l + 16, l + 32, ..: each load of the half-warp reads 16
// consecutive staged samples, so a warp's load touches 16-18 words (one
// shared wavefront; 4-frame B-scan batch +1.1 %), and a half-warp's 16-byte
// complex pieces go to 256 consecutive bytes (K consecutive pieces per lane
// put lanes 4 apart on the same banks: two-way conflicts). The longer real
// classes take K consecutive intervals K l .. K l + K - 1 per lane from K + 1
// staged samples (fewer loads and conversions; the strided form cost the
// 96-interval volume and the mixed stream 2-3 %). Intervals past the window's
// W are written too (from staged samples inside the buffer) and never read.
template <class T, bool CPLX, int WS, int NWIN, int RAWS, int RAW_WIN_BYTES>
__device__ __forceinline__ void rewrite_windows_hw(const unsigned char* rawb, const int* woff,
                                                   unsigned char* pairs, int W, float hp, float scale,
                                                   int warp, int lane) {
    constexpr int K = WS / 16;
    static_assert(K * 16 == WS && NWIN % 2 == 0, "a half-warp per window");
    const int half = lane >> 4, l = lane & 15;
    if constexpr (WS == 48 || CPLX) {
        for (int w2 = warp; w2 < NWIN / 2; w2 += kDasThreads / 32) {
            const int win = 2 * w2 + half;
            const T* r = reinterpret_cast<const T*>(rawb + win * RAW_WIN_BYTES) + woff[win] + l;
            [[maybe_unused]] const T* ri =
                reinterpret_cast<const T*>(rawb + win * RAW_WIN_BYTES + RAWS * 4) + woff[win] + l;
            // every load first (all inside the staged buffer), then the pieces
            T x0[K], x1[K];
            [[maybe_unused]] T y0[K], y1[K];
#pragma unroll
            for (int e = 0; e < K; ++e) {
                x0[e] = r[16 * e];
                x1[e] = r[16 * e + 1];
                if constexpr (CPLX) {
                    y0[e] = ri[16 * e];
                    y1[e] = ri[16 * e + 1];
                }
            }
#pragma unroll
            for (int e = 0; e < K; ++e) {
                if (16 * e >= W) break;                       // uniform: W is the stage's window length
                const int n = l + 16 * e;
                const float a0 = to_f32<T>(x0[e], scale), sl = to_f32<T>(x1[e], scale) - a0;
                const float h = hp - (float)n;
                if constexpr (CPLX) {
                    const float b0 = to_f32<T>(y0[e], scale), si = to_f32<T>(y1[e], scale) - b0;
                    reinterpret_cast<float4*>(pairs + (size_t)win * WS * 16)[n] =
                        make_float4(fmaf(h, sl, a0), sl, fmaf(h, si, b0), si);
                } else {
                    reinterpret_cast<float2*>(pairs + (size_t)win * WS * 8)[n] = make_float2(fmaf(h, sl, a0), sl);
                }
            }
        }
    } else {
        const int n0 = K * l;
        const float hn0 = hp - (float)n0;                   // hp - n of this lane's first interval
        for (int w2 = warp; w2 < NWIN / 2; w2 += kDasThreads / 32) {
            const int win = 2 * w2 + half;
            if (n0 >= W) continue;
            const int off = woff[win] + n0;
            const T* r = reinterpret_cast<const T*>(rawb + win * RAW_WIN_BYTES) + off;
            float rv[K + 1];
            if constexpr (std::is_same<T, __half>::value && !CPLX) {
                // FP16 samples by 32-bit loads: the K + 2 samples from the even
                // sample at or before the first, pairs realigned by a byte
                // permute when the first is odd (K even: K / 2 + 1 words)
                constexpr int NW = K / 2 + 1;
                const uint32_t* rw = reinterpret_cast<const uint32_t*>(rawb + win * RAW_WIN_BYTES) + (off >> 1);
                uint32_t wv[NW + 1];
#pragma unroll
                for (int q = 0; q < NW; ++q) wv[q] = rw[q];
                wv[NW] = 0u;
                const uint32_t sel = (off & 1) ? 0x5432u : 0x3210u;
#pragma unroll
                for (int q = 0; q < NW; ++q) {
                    const uint32_t pr = __byte_perm(wv[q], wv[q + 1], sel);
                    rv[2 * q] = __half2float(__ushort_as_half((unsigned short)(pr & 0xffffu)));
                    if (2 * q + 1 <= K) rv[2 * q + 1] = __half2float(__ushort_as_half((unsigned short)(pr >> 16)));
                }
            } else {
#pragma unroll
                for (int e = 0; e <= K; ++e) rv[e] = to_f32<T>(r[e], scale);
            }
            if constexpr (CPLX) {
                const T* ri = reinterpret_cast<const T*>(rawb + win * RAW_WIN_BYTES + RAWS * 4) + off;
                float iv[K + 1];
#pragma unroll
                for (int e = 0; e <= K; ++e) iv[e] = to_f32<T>(ri[e], scale);
                float4* p = reinterpret_cast<float4*>(pairs + (size_t)(win * WS + n0) * 16);
#pragma unroll
                for (int e = 0; e < K; ++e) {
                    const float sr = rv[e + 1] - rv[e], si = iv[e + 1] - iv[e];
                    const float h = hn0 - (float)e;
                    p[e] = make_float4(fmaf(h, sr, rv[e]), sr, fmaf(h, si, iv[e]), si);
                }
            } else {
                float2* p = reinterpret_cast<float2*>(pairs + (size_t)(win * WS + n0) * 8);
#pragma unroll
                for (int e = 0; e < K; ++e) {
                    const float sl = rv[e + 1] - rv[e];
                    p[e] = make_float2(fmaf(hn0 - (float)e, sl, rv[e]), sl);
                }
            }
        }
    }
}

// The same for cubic Hermite pieces: the copy starts one sample before the
// window, so interval n reads staged samples n .. n+3 (after the offset) and
// K intervals read K + 3 samples per plane. Complex 96-interval windows take
// a whole warp (K = 3), which keeps the staged samples of a lane in registers.
template <class T, bool CPLX, int WS, int NWIN, int RAWS, int RAW_WIN_BYTES>
__device__ __forceinline__ void rewrite_windows_cubic_hw(const unsigned char* rawb, const int* woff,
                                                         unsigned char* pairs, int W, float scale,
                                                         int warp, int lane) {
    constexpr int LPW = (CPLX && WS == 96) ? 32 : 16;    // lanes per window
    constexpr int K = WS / LPW;
    constexpr int WPP = 32 / LPW;                         // windows per warp pass
    static_assert(K * LPW == WS && NWIN % WPP == 0, "whole windows per warp pass");
    auto coeffs = [](float p0, float p1, float p2, float p3) {
        const float m1 = 0.5f * (p2 - p0), m2 = 0.5f * (p3 - p1);
        const float d = p2 - p1;
        return make_float4(p1, m1, fmaf(3.0f, d, -(2.0f * m1 + m2)), fmaf(-2.0f, d, m1 + m2));
    };
    const int half = lane / LPW, n0 = K * (lane % LPW);
    for (int w2 = warp; w2 < NWIN / WPP; w2 += kDasThreads / 32) {
        const int win = WPP * w2 + half;
        if (n0 >= W) continue;
        const int off = woff[win] + n0;
        const T* r = reinterpret_cast<const T*>(rawb + win * RAW_WIN_BYTES) + off;
        float q[K + 3];
#pragma unroll
        for (int e = 0; e < K + 3; ++e) q[e] = to_f32<T>(r[e], scale);
        float4* p = reinterpret_cast<float4*>(pairs + (size_t)(win * WS + n0) * (CPLX ? 32 : 16));
        if constexpr (CPLX) {
            const T* ri = reinterpret_cast<const T*>(rawb + win * RAW_WIN_BYTES + RAWS * 4) + off;
            float qi[K + 3];
#pragma unroll
            for (int e = 0; e < K + 3; ++e) qi[e] = to_f32<T>(ri[e], scale);
#pragma unroll
            for (int e = 0; e < K; ++e) {
                p[2 * e] = coeffs(q[e], q[e + 1], q[e + 2], q[e + 3]);
                p[2 * e + 1] = coeffs(qi[e], qi[e + 1], qi[e + 2], qi[e + 3]);
            }
        } else {
#pragma unroll
            for (int e = 0; e < K; ++e) p[e] = coeffs(q[e], q[e + 1], q[e + 2], q[e + 3]);
        }
    }
}

// mbarrier slots (8 bytes each) of a DAS CTA: raw-window buffers (2) and
// line-piece buffers (3), each with a "full" and an "empty" barrier.
enum : int { kRawFull = 0, kRawEmpty = 2, kPieceFull = 4, kPieceEmpty = 7, kNumBars = 10 };

// State of a CTA running DAS units: the number of stages it ran before the
// current unit. Every barrier phase follows from the CTA-wide stage index
// k = base + s: raw buffers (two) complete phase k/2 for stage k, line-piece
// buffers (three) phase k/3, and each "empty" barrier starts with one
// pre-completed phase. So any thread may wait on any phase without keeping
// its own phase bits.
struct DasPipe {
    uint32_t base;
};

// Division by a small runtime count (transmit groups per channel chunk, tile
// rows per depth row): floor(s / n) = umulhi(s, ceil(2^32 / n)), exact
// whenever s n < 2^32 (the indices stay below 2^16, n below 2^10).
struct StageDiv {
    int n;
    uint32_t mul;
    __device__ __forceinline__ explicit StageDiv(int n_)
        : n(n_), mul(n_ > 1 ? (uint32_t)((0x100000000ull + (unsigned)n_ - 1u) / (unsigned)n_) : 0u) {}
    __device__ __forceinline__ int div(int s) const { return n > 1 ? (int)__umulhi((uint32_t)s, mul) : s; }
    __device__ __forceinline__ int mod(int s) const { return s - div(s) * n; }
};

// Initialise the CTA's mbarriers (thread 0) and pre-complete the first phase
// of every "empty" barrier so that the first fill of each buffer needs no
// special case. Ends with a CTA barrier.
template <int COPIES>
__device__ __forceinline__ void das_pipe_init(unsigned char* bar_base, volatile int* abort) {
    const uint32_t bar0 = smem_u32(bar_base);
    if (threadIdx.x == 0) {
        mbar_init(bar0 + 8 * (kRawFull + 0), COPIES);
        mbar_init(bar0 + 8 * (kRawFull + 1), COPIES);
        for (int k = kRawEmpty; k < kNumBars; ++k) mbar_init(bar0 + 8 * k, kDasThreads);
        *abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    for (int k = 0; k < 2; ++k) mbar_arrive(bar0 + 8 * (kRawEmpty + k));
    for (int k = 0; k < 3; ++k) mbar_arrive(bar0 + 8 * (kPieceEmpty + k));
}

// One work unit: channel part unit / tiles of tile unit % tiles, the tile's
// channels split into n_split parts, written to partial image `slice` (-1:
// the image itself when n_split is 1, else partial image unit / tiles).
// Returns false when a bounded wait expired (the CTA must stop; the caller
// records the status).
template <int VU, int WS, bool CPLX, bool APOD, bool CUBIC = false, bool IQ = false, bool D2 = false>
__device__ __forceinline__ bool das_unit(const DasArgs& a, int unit, int n_split, unsigned char* smem,
                                         DasPipe& pipe, int slice = -1) {
    using C = DasCfg<VU, WS, CPLX, CUBIC, D2, APOD, IQ>;
    static_assert(!IQ || CPLX, "IQ beamforming reads two planes");
    float* s_ws0 = reinterpret_cast<float*>(smem + C::OFF_WS0);
    float* s_txph = reinterpret_cast<float*>(smem + C::OFF_TXPH);
    float* s_rxph = reinterpret_cast<float*>(smem + C::OFF_RXPH);
    float* s_wph = reinterpret_cast<float*>(smem + C::OFF_WPH);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float4* s_tx = reinterpret_cast<float4*>(smem + C::OFF_TX);
    float4* s_rx = reinterpret_cast<float4*>(smem + C::OFF_RX);
    float* s_alpha = reinterpret_cast<float*>(smem + C::OFF_ALPHA);
    int* s_woff = reinterpret_cast<int*>(smem + C::OFF_WOFF);
    const uint32_t bar0 = smem_u32(smem + C::OFF_BAR);
    const uint32_t pairs_u32 = smem_u32(smem + C::OFF_PAIRS);
    unsigned char* raw = smem + C::OFF_RAW;
    const int es = (a.dtype == RCBF_F16) ? 2 : 4;

    // ---- unit -> (tile, channel split)
    const int n_tiles = a.tiles_u * a.tiles_v * a.tiles_w;
    const int tile = unit % n_tiles;
    const int split = unit / n_tiles;
    const int n_ic = a.n_tx / C::CI;
    const StageDiv sdiv(n_ic);        // stage -> (transmit group, channel chunk) without a division
    const StageDiv bvdiv(a.bv);       // tile row -> (v, w) offsets
    const int js = (a.n_ch / C::CJ) / n_split;       // channel chunks of this unit
    const int jc0 = split * js;
    int* s_act = reinterpret_cast<int*>(smem + C::OFF_ACT);

    // ---- tile position and FP64 reference delays
    const int tu = tile % a.tiles_u;
    const int tv = (tile / a.tiles_u) % a.tiles_v;
    const int tw = tile / (a.tiles_u * a.tiles_v);
    const int u0 = tu * C::BU, v0 = tv * a.bv, w0 = tw * a.bw;
    const double cu = u0 + 0.5 * (C::BU - 1), cv = v0 + 0.5 * (a.bv - 1), cw = w0 + 0.5 * (a.bw - 1);
    const double qx = a.q0[0] + a.Gu[0] * cu + a.Gv[0] * cv + a.Gw[0] * cw;
    const double qy = a.q0[1] + a.Gu[1] * cu + a.Gv[1] * cv + a.Gw[1] * cw;
    const double zr = a.q0[2] + a.Gu[2] * cu + a.Gv[2] * cv + a.Gw[2] * cw;
    const double lat_tx_ref = a.tx_axis ? qy : qx, lat_rx_ref = a.rx_axis ? qy : qx;
    const int j_lo = jc0 * C::CJ, n_rx = js * C::CJ;
    // 2D: the transmit wave's reference path splits into Kt + Eref (integer
    // and fractional samples); windows are placed relative to Kt. [elo, ehi]:
    // the path's bounds over the tile's bounding box (samples, relative to Kt,
    // with a slack for the FP32 evaluation per voxel)
    auto half_ext = [&](int d) {
        return 0.5 * (fabs(a.Gu[d]) * (C::BU - 1) + fabs(a.Gv[d]) * (a.bv - 1) + fabs(a.Gw[d]) * (a.bw - 1));
    };
    int Kt = 0;
    float Eref = 0.f, elo = 0.f, ehi = 0.f;
    if constexpr (D2) {
        double dw, dlo, dhi;
        if (a.tx_wave == RCBF_TX_PLANE) {
            const float2 sc = a.tx_dir[0];
            dw = zr * (double)sc.y + lat_tx_ref * (double)sc.x;
            const double hw = fabs((double)sc.y) * half_ext(2) + fabs((double)sc.x) * half_ext(a.tx_axis);
            dlo = dw - hw;
            dhi = dw + hw;
        } else {
            // source at (0, 0, f): nearest point of the box and farthest corner
            const double zf = zr - a.tx_focus, hx = half_ext(0), hy = half_ext(1), hz = half_ext(2);
            const double nx = fmax(fabs(qx) - hx, 0.0), ny = fmax(fabs(qy) - hy, 0.0), nz = fmax(fabs(zf) - hz, 0.0);
            const double fx = fabs(qx) + hx, fy = fabs(qy) + hy, fz = fabs(zf) + hz;
            dw = sqrt(qx * qx + qy * qy + zf * zf) + a.tx_focus;
            dlo = sqrt(nx * nx + ny * ny + nz * nz) + a.tx_focus;
            dhi = sqrt(fx * fx + fy * fy + fz * fz) + a.tx_focus;
        }
        const double A = dw * a.fs_over_c - a.t0fs;
        const double K = floor(A);
        Kt = (int)K;
        Eref = (float)(A - K);
        elo = (float)(dlo * a.fs_over_c - a.t0fs - K) - a.reach_a;
        ehi = (float)(dhi * a.fs_over_c - a.t0fs - K) + a.reach_a;
    }
    __syncthreads();   // the previous unit of this CTA no longer reads the tables
    if constexpr (D2) {
        // squared-distance bounds over the tile's bounding box (half extents
        // along each array axis): transmit rows (L, P_min, P_max), receive
        // columns (L, Q_min, Q_max), L the reference lateral offset
        auto sq_lo = [](double x, double h) { const double m = fabs(x) - h; return m > 0.0 ? m * m : 0.0; };
        auto sq_hi = [](double x, double h) { const double m = fabs(x) + h; return m * m; };
        const double ht = half_ext(a.tx_axis), hr = half_ext(a.rx_axis), hz = half_ext(2);
        const double z2lo = sq_lo(zr, hz), z2hi = sq_hi(zr, hz);
        for (int e = tid; e < a.n_tx + n_rx; e += kDasThreads) {
            if (e < a.n_tx) {
                const double L = lat_tx_ref - (a.tx_e0 + e * a.tx_pitch);
                // the floor keeps every P + Q positive (a finite reciprocal root)
                s_tx[e] = make_float4((float)L, (float)fmax(sq_lo(L, ht) + z2lo, 1e-14), (float)(sq_hi(L, ht) + z2hi), 0.f);
            } else {
                const int j = j_lo + e - a.n_tx;
                const double L = lat_rx_ref - (a.rx_e0 + j * a.rx_pitch);
                s_rx[j] = make_float4((float)L, (float)sq_lo(L, hr), (float)sq_hi(L, hr), 0.f);
            }
        }
    } else
    for (int e = tid; e < a.n_tx + n_rx; e += kDasThreads) {
        if (e < a.n_tx) {
            float tx0, tx1;
            const double d = tx_ref_distance(a, e, lat_tx_ref, zr, &tx0, &tx1);
            const double A = d * a.fs_over_c - a.t0fs;
            const double K = floor(A);
            // remainder with the window offset, the half-sample shift of the
            // rounding trick and the window centring folded in
            const float rho = (float)(A - K - (double)a.lo - 0.5 - (double)a.H);
            s_tx[e] = make_float4(tx0, tx1, rho, __int_as_float((int)K));
            if (C::IQ_SEP) {
                // carrier phase of the transmit part of every window start of
                // this transmit: S0 = K_i + K_j + lo, at u = 0 the sample
                // S0 + 0.5 + H for linear pieces (cubic positions include it)
                const double x = a.iq_ratio * (K + (double)a.lo + (CUBIC ? 0.0 : 0.5 + (double)a.H));
                s_txph[e] = (float)(x - floor(x));
            }
        } else {
            const int j = j_lo + e - a.n_tx;
            const double L = lat_rx_ref - (a.rx_e0 + j * a.rx_pitch);
            const double d = sqrt(L * L + zr * zr);
            const double B = d * a.fs_over_c;
            const double K = floor(B);
            s_rx[j] = make_float4((float)L, (float)d, (float)(B - K), __int_as_float((int)K));
            if (C::IQ_SEP) {
                const double x = a.iq_ratio * K;
                s_rxph[j] = (float)(x - floor(x));
            }
        }
    }

    // ---- voxel offsets from the reference in FP32 (exact half-integer index
    // offsets times the FP32 voxel steps)
    const float Zf = (float)zr;
    const float Zfoc = (float)(zr - a.tx_focus);   // reference depth below the virtual line sources
    const float fsc = (float)a.fs_over_c;
    const float gur = (float)(a.rx_axis ? a.Gu[1] : a.Gu[0]);
    const float gvr = (float)(a.rx_axis ? a.Gv[1] : a.Gv[0]);
    const float gwr = (float)(a.rx_axis ? a.Gw[1] : a.Gw[0]);
    const float guz = (float)a.Gu[2], gvz = (float)a.Gv[2], gwz = (float)a.Gw[2];
    // transmit-lateral steps of the tile rows (converted once, not per stage)
    const float gvt_row = (float)(a.tx_axis ? a.Gv[1] : a.Gv[0]), gwt_row = (float)(a.tx_axis ? a.Gw[1] : a.Gw[0]);
    auto voxel_offsets = [&](int k, float& dlr, float& dz) {
        const int ku = k % VU, kr = k / VU;
        const int row = warp * C::VR + kr;
        const float du = (float)(lane + 32 * ku) - 0.5f * (C::BU - 1);
        const float dv = (float)bvdiv.mod(row) - 0.5f * (a.bv - 1);
        const float dw = (float)bvdiv.div(row) - 0.5f * (a.bw - 1);
        dlr = gur * du + gvr * dv + gwr * dw;
        dz = guz * du + gvz * dv + gwz * dw;
    };
    // 2D: first window sample of (i, j) relative to Kt, one below the
    // smallest delay of the box (FP32, the same in every thread)
    auto win_start = [&](int i, int j) -> int {
        const float lowd = sqrtf(s_tx[i].y + s_rx[j].y);
        return (int)floorf(fmaf(lowd, fsc, elo)) - 1;
    };
    // Channel chunks of this unit with a nonzero F# window somewhere in the
    // tile (Eq. (2)-(3) skip test, on the tile's bounding box: a chunk is
    // skipped only if F# |lat - e_j| >= |z| / 2 at every voxel for all its
    // channels, so skipping changes nothing); all chunks without a window
    if (APOD && a.f_number > 0.f) {
        const double hr = 0.5 * (fabs(a.rx_axis ? a.Gu[1] : a.Gu[0]) * (C::BU - 1) +
                                 fabs(a.rx_axis ? a.Gv[1] : a.Gv[0]) * (a.bv - 1) +
                                 fabs(a.rx_axis ? a.Gw[1] : a.Gw[0]) * (a.bw - 1));
        const double zmax = fabs(zr) + 0.5 * (fabs(a.Gu[2]) * (C::BU - 1) + fabs(a.Gv[2]) * (a.bv - 1) +
                                              fabs(a.Gw[2]) * (a.bw - 1));
        for (int c = tid; c < js; c += kDasThreads) {
            int act = 0;
            for (int jj = 0; jj < C::CJ; ++jj) {
                const double L = lat_rx_ref - (a.rx_e0 + ((jc0 + c) * C::CJ + jj) * a.rx_pitch);
                act |= (double)a.f_number * fmax(fabs(L) - hr, 0.0) < 0.5 * zmax + 1e-9;
            }
            s_act[c] = act;
        }
        __syncthreads();
        if (tid == 0) {
            int n = 0;
            for (int c = 0; c < js; ++c)
                if (s_act[c]) s_act[n++] = jc0 + c;
            s_act[kMaxChannels / C::CJ] = n;
        }
    } else if (APOD && tid == 0) {
        for (int c = 0; c < js; ++c) s_act[c] = jc0 + c;
        s_act[kMaxChannels / C::CJ] = js;
    }
    __syncthreads();   // reference tables and the chunk list ready
    // channel chunk of stage s (forms without weights never skip a chunk)
    auto chunk_of = [&](int s) -> int { return APOD ? s_act[sdiv.div(s)] : jc0 + sdiv.div(s); };
    const int NS = n_ic * (APOD ? s_act[kMaxChannels / C::CJ] : js);

    volatile int* abort = reinterpret_cast<volatile int*>(smem + C::OFF_ABORT);
    auto wait = [&](int slot, uint32_t phase) -> bool {
        return mbar_wait_or_abort(bar0 + 8 * slot, phase & 1u, abort, a.wait_ns);
    };
    auto raw_phase = [&](int s) -> uint32_t { return (pipe.base + (uint32_t)s) >> 1; };
    auto piece_phase = [&](int s) -> uint32_t { return (pipe.base + (uint32_t)s) / 3u; };
    auto raw_buf = [&](int s) -> int { return (int)((pipe.base + (uint32_t)s) & 1u); };
    auto piece_buf = [&](int s) -> int { return (int)((pipe.base + (uint32_t)s) % 3u); };

    // ---- producer: one thread per bulk copy (window, plane) of stage s into
    // the raw buffer of stage s, once every thread has rewritten that buffer's previous stage
    // the copy-issuing and transmit-term roles rotate over the warps from
    // stage to stage, so that no warp carries the extra work every stage
    auto issue = [&](int s) -> bool {
        const int copy = (tid + kDasThreads - (s * C::COPIES) % kDasThreads) % kDasThreads;
        if (copy >= C::COPIES) return true;
        // test hook (rcbf_plan_set_wait): the first copy of the unit is never
        // requested, so the unit's first wait on its windows runs out
        if (a.withhold && s == 0 && copy == 0) return true;
        const int b = raw_buf(s);
        if (!wait(kRawEmpty + b, raw_phase(s))) return false;
        const int win = CPLX ? (copy >> 1) : copy;
        const int plane = CPLX ? (copy & 1) : 0;
        const int ii = win / C::CJ, jj = win % C::CJ;
        const int i = sdiv.mod(s) * C::CI + ii, j = chunk_of(s) * C::CJ + jj;
        // first staged sample (cubic: one before the window, for the stencil)
        const int S0 = (D2 ? Kt + win_start(i, j) : __float_as_int(s_tx[i].w) + __float_as_int(s_rx[j].w) + a.lo) -
                       (CUBIC ? 1 : 0);
        const int A = S0 & ~7;
        if (plane == 0) s_woff[b * C::NWIN + win] = S0 - A;
        const int lo_s = max(A, 0);
        const int hi_s = min(A + a.raw_samples, a.n_s);
        unsigned char* dst = raw + (b * C::NWIN + win) * C::RAW_WIN_BYTES + plane * C::RAWS * 4;
        const int pre = (min(lo_s, A + a.raw_samples) - A) * es;       // bytes of zeros before
        const int body = hi_s > lo_s ? (hi_s - lo_s) * es : 0;
        const int total = a.raw_samples * es;
        for (int o = 0; o < pre; o += 16) *reinterpret_cast<uint4*>(dst + o) = make_uint4(0, 0, 0, 0);
        for (int o = pre + body; o < total; o += 16) *reinterpret_cast<uint4*>(dst + o) = make_uint4(0, 0, 0, 0);
        fence_proxy_async_smem();
        const uint32_t bar = bar0 + 8 * (kRawFull + b);
        mbar_arrive_expect_tx(bar, (uint32_t)body);
        if (body > 0) {
            const char* src = static_cast<const char*>(a.rf) +
                ((long long)plane * a.plane_stride + ((long long)i * a.n_ch + j) * a.n_s + lo_s) * es;
            bulk_g2s(smem_u32(dst + pre), src, (uint32_t)body, bar);
        }
        return true;
    };

    // ---- stage preparation: once its raw windows have landed and the
    // line-piece buffer is free, rewrite this thread's share of the windows
    // and of the transmit-term table, then release both buffers
    const float hp = 0.5f + (float)a.H;
    auto prepare = [&](int s) -> bool {
        const int b = raw_buf(s), pb = piece_buf(s);
        if (!wait(kRawFull + b, raw_phase(s))) return false;
        if (!wait(kPieceEmpty + pb, piece_phase(s))) return false;
        const unsigned char* rawb = raw + b * C::NWIN * C::RAW_WIN_BYTES;
        unsigned char* pairs = smem + C::OFF_PAIRS + pb * C::PAIR_BUF;
        const int* woff = s_woff + b * C::NWIN;
        if (CUBIC) {
            if (a.dtype == RCBF_F16)
                rewrite_windows_cubic_hw<__half, CPLX, WS, C::NWIN, C::RAWS, C::RAW_WIN_BYTES>(rawb, woff, pairs, a.W, a.scale, warp, lane);
            else if (a.dtype == RCBF_I32)
                rewrite_windows_cubic_hw<int, CPLX, WS, C::NWIN, C::RAWS, C::RAW_WIN_BYTES>(rawb, woff, pairs, a.W, a.scale, warp, lane);
            else
                rewrite_windows_cubic_hw<float, CPLX, WS, C::NWIN, C::RAWS, C::RAW_WIN_BYTES>(rawb, woff, pairs, a.W, a.scale, warp, lane);
        } else if (a.dtype == RCBF_F16)
            rewrite_windows_hw<__half, CPLX, WS, C::NWIN, C::RAWS, C::RAW_WIN_BYTES>(rawb, woff, pairs, a.W, hp, a.scale, warp, lane);
        else if (a.dtype == RCBF_I32)
            rewrite_windows_hw<int, CPLX, WS, C::NWIN, C::RAWS, C::RAW_WIN_BYTES>(rawb, woff, pairs, a.W, hp, a.scale, warp, lane);
        else
            rewrite_windows_hw<float, CPLX, WS, C::NWIN, C::RAWS, C::RAW_WIN_BYTES>(rawb, woff, pairs, a.W, hp, a.scale, warp, lane);
        if (D2 && tid < C::NWIN) {
            const int win = tid;
            const int i = sdiv.mod(s) * C::CI + win / C::CJ, j = chunk_of(s) * C::CJ + win % C::CJ;
            const int w0 = win_start(i, j);
            s_ws0[pb * C::NWIN + win] = -(float)w0;
            if (IQ) {
                // the delay is not separable here: the carrier phase (cycles) of
                // the window's reference position, rotated per term (the sample
                // at u = 0 is Kt + w0 + 0.5 + H for linear pieces; cubic
                // positions already include 0.5 + H)
                const double x = a.iq_ratio * ((double)(Kt + w0) + (CUBIC ? 0.0 : 0.5 + (double)a.H));
                s_wph[pb * C::NWIN + win] = (float)(x - floor(x));
            }
        }
        const int ae = (tid + kDasThreads - (s * C::ALPHA_N + kDasThreads / 2) % kDasThreads) % kDasThreads;
        if (ae < C::ALPHA_N) {
            // transmit terms of this stage for every tile row (alpha depends on the row only)
            const int ii = ae / C::ROWS, row = ae % C::ROWS;
            const float dv = (float)bvdiv.mod(row) - 0.5f * (a.bv - 1);
            const float dw = (float)bvdiv.div(row) - 0.5f * (a.bw - 1);
            const float dL = gvt_row * dv + gwt_row * dw;
            const float dz = gvz * dv + gwz * dw;
            const float4 tx = s_tx[sdiv.mod(s) * C::CI + ii];
            if constexpr (D2) {
                // P = (lat_tx - e_i)^2 + z^2 of the row, clamped to its box bounds
                const float Lt = tx.x + dL, Zv = Zf + dz;
                s_alpha[pb * C::ALPHA_N + C::alpha_index(ii, row)] = fminf(fmaxf(fmaf(Lt, Lt, Zv * Zv), tx.y), tx.z);
            } else {
                const float al = tx_offset(a.tx_wave, tx, dL, dz, Zf, Zfoc, fsc);
                s_alpha[pb * C::ALPHA_N + C::alpha_index(ii, row)] = fminf(fmaxf(al, tx.z - a.reach_a), tx.z + a.reach_a);
            }
        }
        mbar_arrive(bar0 + 8 * (kRawEmpty + b));
        mbar_arrive(bar0 + 8 * (kPieceFull + pb));
        return true;
    };

    // voxel pairs (k, k+1) are packed in f32x2 registers: receive terms,
    // weights and accumulators
    f2x acc2[2] = {0ull, 0ull};
    float acci[4] = {0.f, 0.f, 0.f, 0.f};
    f2x acci2[2] = {0ull, 0ull};      // complex: imaginary sums of the voxel pairs
    [[maybe_unused]] float iq_re[4] = {0.f, 0.f, 0.f, 0.f}, iq_im[4] = {0.f, 0.f, 0.f, 0.f};   // IQ sums
    f2x beta2[2][C::CJ];
    f2x apw2[2][C::CJ];
    const float magic = CUBIC ? 8388607.5f : 8388608.0f + (float)a.H;     // 2^23 + H (cubic: on u + 0.5 + H)
    const f2x magic2 = pk(magic, magic);
    constexpr int SHIFT = C::SHIFT;
    const float iqr = (float)a.iq_ratio;
    const f2x fsc2 = pk(fsc, fsc);
    // 2D: per voxel the transmit wave's path in samples relative to Kt
    // (cancellation-free offset from the reference, clamped to its reach),
    // with the linear pieces' centring folded in
    f2x E2[2] = {0ull, 0ull};
    if constexpr (D2) {
        const float gut = (float)(a.tx_axis ? a.Gu[1] : a.Gu[0]);
        const float gvt = (float)(a.tx_axis ? a.Gv[1] : a.Gv[0]);
        const float gwt = (float)(a.tx_axis ? a.Gw[1] : a.Gw[0]);
        const float shift = CUBIC ? 0.0f : hp;
        float ev[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float dlr, dz;
            voxel_offsets(k, dlr, dz);
            const int ku = k % VU, kr = k / VU;
            const int row = warp * C::VR + kr;
            const float du = (float)(lane + 32 * ku) - 0.5f * (C::BU - 1);
            const float dv = (float)bvdiv.mod(row) - 0.5f * (a.bv - 1);
            const float dw = (float)bvdiv.div(row) - 0.5f * (a.bw - 1);
            const float dlt = gut * du + gvt * dv + gwt * dw;
            float de;
            if (a.tx_wave == RCBF_TX_PLANE) {
                const float2 sc = a.tx_dir[0];
                de = fmaf(dz, sc.y, dlt * sc.x) * fsc;
            } else {
                // point source at (0, 0, f) of the array frame
                const float X = (float)lat_rx_ref, Y = (float)lat_tx_ref, Zq = (float)(zr - a.tx_focus);
                const float Xv = X + dlr, Yv = Y + dlt, Zv = Zq + dz;
                const float dv3 = sqrtf(Xv * Xv + Yv * Yv + Zv * Zv);
                const float dr3 = sqrtf(X * X + Y * Y + Zq * Zq);
                const float num = dlr * (2.0f * X + dlr) + dlt * (2.0f * Y + dlt) + dz * (2.0f * Zq + dz);
                de = __fdividef(num, dv3 + dr3) * fsc;
            }
            ev[k] = fminf(fmaxf(Eref + de, elo), ehi) - shift;
        }
        E2[0] = pk(ev[0], ev[1]);
        E2[1] = pk(ev[2], ev[3]);
    }

    // ---- prologue: stages 0 and 1 in flight, stage 0 rewritten
    bool ok = true;
    if (!APOD || NS > 0) {          // a weighted unit may have no active chunk
        ok = issue(0);
        if (ok && NS > 1) ok = issue(1);
        if (ok) ok = prepare(0);
    }
    int issued = NS > 1 ? 1 : 0;      // last stage this thread's copies were requested for
    int landed = 0;                   // last stage whose raw windows this thread waited for

    for (int s = 0; ok && s < NS; ++s) {
        const int ic = sdiv.mod(s), jc = chunk_of(s);
        const int pb = piece_buf(s);
        if (ic == 0) {
            // per-voxel receive terms (and apodization) for this channel chunk
#pragma unroll
            for (int kp = 0; kp < 2; ++kp) {
                float dlr[2], dz[2];
                voxel_offsets(2 * kp, dlr[0], dz[0]);
                voxel_offsets(2 * kp + 1, dlr[1], dz[1]);
#pragma unroll
                for (int jj = 0; jj < C::CJ; ++jj) {
                    const int j = jc * C::CJ + jj;
                    const float4 rx = s_rx[j];
                    const float wj = APOD && a.apod ? __ldg(a.apod + j) : 1.0f;
                    float bt[2], aw[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if constexpr (D2) {
                            // Q = (lat_rx - e_j)^2, clamped to its box bounds (no F# window)
                            const float Lv = rx.x + dlr[h];
                            bt[h] = fminf(fmaxf(Lv * Lv, rx.y), rx.z);
                            aw[h] = wj;
                            continue;
                        }
                        const float Lv = rx.x + dlr[h], Zv = Zf + dz[h];
                        const float d = sqrtf(Lv * Lv + Zv * Zv);
                        const float num = dlr[h] * (2.0f * rx.x + dlr[h]) + dz[h] * (2.0f * Zf + dz[h]);
                        const float b0 = rx.z + __fdividef(num, d + rx.y) * fsc;
                        // (cubic: + 0.5 + H, the position in interval units)
                        bt[h] = fminf(fmaxf(b0, rx.z - a.reach_b), rx.z + a.reach_b) + (CUBIC ? hp : 0.0f);
                        aw[h] = a.f_number > 0.f ? wj * hann_weight(a.f_number, Lv, Zv) : wj;
                    }
                    beta2[kp][jj] = pk(bt[0], bt[1]);
                    if (APOD) apw2[kp][jj] = pk(aw[0], aw[1]);
                }
            }
        }
        if (s + 2 < NS) { if (!(ok = issue(s + 2))) break; issued = s + 2; }
        if (s + 1 < NS) { if (!(ok = prepare(s + 1))) break; landed = s + 1; }
        if (!(ok = wait(kPieceFull + pb, piece_phase(s)))) break;

        // ---- the sum: 4 voxels x CI transmits x CJ channels from buffer pb
        const uint32_t pbase = pairs_u32 + pb * C::PAIR_BUF - (0x4B000000u << SHIFT);
        const float* alb = s_alpha + pb * C::ALPHA_N + warp * (C::CI * C::VR);   // this warp's rows, all transmits
        // real linear pieces: two transmits per iteration, four in the
        // 48-interval class (more independent loads in flight; measured on the
        // batched B-scan +2.7 % and +1.3 %; four cost the 96 class 4-7 %); the
        // wider forms stay at one (register budget)
        if constexpr (C::IQ_SEP) {
            // IQ beamforming: the carrier phase of a term splits into a
            // transmit part P_i(row) = txph_i + r alpha_i(row) and a receive
            // part Q_j(voxel) = rxph_j + r beta_j(voxel), so the rotation
            // e^{j 2 pi (P + Q)} is the product of a factor per (row,
            // transmit) and a factor per (voxel, channel), the latter computed
            // once per stage and used for G transmits: the terms of a transmit
            // are summed rotated by the receive factor, and the sum is rotated
            // by the transmit factor
            constexpr int G = C::CI < 2 ? C::CI : 2;
            const int j0 = chunk_of(s) * C::CJ, i0 = sdiv.mod(s) * C::CI;
#pragma unroll 1
            for (int ig = 0; ig < C::CI; ig += G) {
                f2x alg[G][2];
                float ec[G][C::VR], es[G][C::VR];          // transmit factors of this thread's rows
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    float al[C::VR];
                    const float txph = s_txph[i0 + ig + g];
#pragma unroll
                    for (int kr = 0; kr < C::VR; ++kr) {
                        al[kr] = alb[(ig + g) * C::VR + kr];
                        const float x = fmaf(iqr, al[kr], txph);
                        __sincosf(6.28318530717958648f * (x - rintf(x)), &es[g][kr], &ec[g][kr]);
                    }
                    alg[g][0] = pk(al[0 / VU], al[1 / VU]);
                    alg[g][1] = pk(al[2 / VU], al[3 / VU]);
                }
                float sr[G][4], si[G][4];
#pragma unroll
                for (int g = 0; g < G; ++g)
#pragma unroll
                    for (int k = 0; k < 4; ++k) sr[g][k] = si[g][k] = 0.f;
                static_for<0, C::CJ>([&](auto jjc) {
                    constexpr int jj = decltype(jjc)::value;
                    constexpr int OFF = jj * WS * C::PAIR_BYTES;
                    // receive factors e^{j 2 pi Q} of the four voxels (times the weights)
                    const float qj = s_rxph[j0 + jj];
                    float bt[4], fc[4], fs[4];
                    upk(beta2[0][jj], bt[0], bt[1]);
                    upk(beta2[1][jj], bt[2], bt[3]);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float x = fmaf(iqr, bt[k], qj);
                        __sincosf(6.28318530717958648f * (x - rintf(x)), &fs[k], &fc[k]);
                    }
                    if (APOD) {
                        float w[4];
                        upk(apw2[0][jj], w[0], w[1]);
                        upk(apw2[1][jj], w[2], w[3]);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            fc[k] *= w[k];
                            fs[k] *= w[k];
                        }
                    }
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        const uint32_t pb_g = pbase + (ig + g) * (C::CJ * WS * C::PAIR_BYTES);
#pragma unroll
                        for (int kp = 0; kp < 2; ++kp) {
                            const f2x u2 = add2(alg[g][kp], beta2[kp][jj]);
                            const f2x t2 = add2(u2, magic2);
                            float u[2], t[2], f[2];
                            upk(u2, u[0], u[1]);
                            upk(t2, t[0], t[1]);
                            if (CUBIC) upk(fma2(add2(t2, pk(-8388608.0f, -8388608.0f)), pk(-1.0f, -1.0f), u2), f[0], f[1]);
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int k = 2 * kp + h;
                                const uint32_t addr = (__float_as_uint(t[h]) << SHIFT) + pb_g;
                                float vr, vi;
                                if (CUBIC) {
                                    const float4 p = lds_f4<OFF>(addr);
                                    const float4 q = lds_f4<OFF + 16>(addr);
                                    vr = fmaf(fmaf(fmaf(p.w, f[h], p.z), f[h], p.y), f[h], p.x);
                                    vi = fmaf(fmaf(fmaf(q.w, f[h], q.z), f[h], q.y), f[h], q.x);
                                } else {
                                    const float4 p = lds_f4<OFF>(addr);
                                    vr = fmaf(u[h], p.y, p.x);
                                    vi = fmaf(u[h], p.w, p.z);
                                }
                                sr[g][k] = fmaf(vr, fc[k], fmaf(-vi, fs[k], sr[g][k]));
                                si[g][k] = fmaf(vr, fs[k], fmaf(vi, fc[k], si[g][k]));
                            }
                        }
                    }
                });
#pragma unroll
                for (int g = 0; g < G; ++g)
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float c = ec[g][k / VU], sn = es[g][k / VU];
                        iq_re[k] = fmaf(c, sr[g][k], fmaf(-sn, si[g][k], iq_re[k]));
                        iq_im[k] = fmaf(c, si[g][k], fmaf(sn, sr[g][k], iq_im[k]));
                    }
            }
        } else {
#pragma unroll(CPLX || CUBIC ? 1 : WS <= 48 ? 4 : 2)
        for (int ii = 0; ii < C::CI; ++ii) {
            float al[C::VR];
#pragma unroll
            for (int kr = 0; kr < C::VR; ++kr) al[kr] = alb[ii * C::VR + kr];
            const f2x al2[2] = {pk(al[0 / VU], al[1 / VU]), pk(al[2 / VU], al[3 / VU])};
            const uint32_t pb_ii = pbase + ii * (C::CJ * WS * C::PAIR_BYTES);
            static_for<0, C::CJ>([&](auto jjc) {
                constexpr int jj = decltype(jjc)::value;
                constexpr int OFF = jj * WS * C::PAIR_BYTES;
                [[maybe_unused]] const float ws0 = D2 ? s_ws0[pb * C::NWIN + ii * C::CJ + jj] : 0.0f;
                [[maybe_unused]] const float phw = (IQ && D2) ? s_wph[pb * C::NWIN + ii * C::CJ + jj] : 0.0f;
                // 2D IQ: e^{j 2 pi (phw + r u)} applied to (vr, vi)
                [[maybe_unused]] auto iq_rotate = [&](float uu, float& vr, float& vi) {
                    const float x = fmaf(iqr, uu, phw);
                    float sn, cs;
                    __sincosf(6.28318530717958648f * (x - rintf(x)), &sn, &cs);
                    const float r0 = vr * cs - vi * sn;
                    vi = fmaf(vr, sn, vi * cs);
                    vr = r0;
                };
#pragma unroll
                for (int kp = 0; kp < 2; ++kp) {
                    f2x u2;
                    if constexpr (D2) {
                        // window position: sqrt(P + Q) fs/c + E - S0 (the square root
                        // by the approximate PTX instruction: one special-function
                        // operation, no multiply; measured faster than x rsqrt(x))
                        const f2x x2 = add2(al2[kp], beta2[kp][jj]);
                        float xa, xb, sa, sb;
                        upk(x2, xa, xb);
                        asm("sqrt.approx.f32 %0, %1;" : "=f"(sa) : "f"(xa));
                        asm("sqrt.approx.f32 %0, %1;" : "=f"(sb) : "f"(xb));
                        u2 = fma2(pk(sa, sb), fsc2, add2(E2[kp], pk(ws0, ws0)));
                    } else {
                        u2 = add2(al2[kp], beta2[kp][jj]);
                    }
                    const f2x t2 = add2(u2, magic2);
                    float u[2], t[2];
                    upk(u2, u[0], u[1]);
                    upk(t2, t[0], t[1]);
                    if (CUBIC) {
                        // u here is u + 0.5 + H: fraction f = u - (t - 2^23)
                        const f2x f2 = fma2(add2(t2, pk(-8388608.0f, -8388608.0f)), pk(-1.0f, -1.0f), u2);
                        float f[2];
                        upk(f2, f[0], f[1]);
                        float vr[2], vi[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const uint32_t addr = (__float_as_uint(t[h]) << SHIFT) + pb_ii;
                            const float4 p = lds_f4<OFF>(addr);
                            vr[h] = fmaf(fmaf(fmaf(p.w, f[h], p.z), f[h], p.y), f[h], p.x);
                            if (CPLX) {
                                const float4 q = lds_f4<OFF + 16>(addr);
                                vi[h] = fmaf(fmaf(fmaf(q.w, f[h], q.z), f[h], q.y), f[h], q.x);
                            }
                        }
                        if constexpr (IQ && D2) {
#pragma unroll
                            for (int h = 0; h < 2; ++h) iq_rotate(u[h], vr[h], vi[h]);
                        }
                        if (CPLX) {
                            const f2x vr2 = pk(vr[0], vr[1]), vi2 = pk(vi[0], vi[1]);
                            acc2[kp] = APOD ? fma2(apw2[kp][jj], vr2, acc2[kp]) : add2(acc2[kp], vr2);
                            acci2[kp] = APOD ? fma2(apw2[kp][jj], vi2, acci2[kp]) : add2(acci2[kp], vi2);
                        } else {
                            const f2x v2 = pk(vr[0], vr[1]);
                            acc2[kp] = APOD ? fma2(apw2[kp][jj], v2, acc2[kp]) : add2(acc2[kp], v2);
                        }
                    } else if (CPLX) {
                        float vr[2], vi[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const uint32_t addr = (__float_as_uint(t[h]) << SHIFT) + pb_ii;
                            const float4 p = lds_f4<OFF>(addr);
                            vr[h] = fmaf(u[h], p.y, p.x);
                            vi[h] = fmaf(u[h], p.w, p.z);
                            if constexpr (IQ && D2) iq_rotate(u[h], vr[h], vi[h]);
                        }
                        const f2x vr2 = pk(vr[0], vr[1]), vi2 = pk(vi[0], vi[1]);
                        acc2[kp] = APOD ? fma2(apw2[kp][jj], vr2, acc2[kp]) : add2(acc2[kp], vr2);
                        acci2[kp] = APOD ? fma2(apw2[kp][jj], vi2, acci2[kp]) : add2(acci2[kp], vi2);
                    } else {
                        const uint32_t ad0 = (__float_as_uint(t[0]) << SHIFT) + pb_ii;
                        const uint32_t ad1 = (__float_as_uint(t[1]) << SHIFT) + pb_ii;
                        const float2 p0 = lds_f2<OFF>(ad0);
                        const float2 p1 = lds_f2<OFF>(ad1);
                        const f2x v2 = pk(fmaf(u[0], p0.y, p0.x), fmaf(u[1], p1.y, p1.x));
                        acc2[kp] = APOD ? fma2(apw2[kp][jj], v2, acc2[kp]) : add2(acc2[kp], v2);
                    }
                }
            });
        }
        }
        mbar_arrive(bar0 + 8 * (kPieceEmpty + pb));
    }
    if (!ok) {
        // a bounded wait expired somewhere in the CTA: give the copies this
        // thread still expects a bounded chance to land, then stop
        for (int k = landed + 1; k <= issued; ++k)
            mbar_wait_parity(bar0 + 8 * (kRawFull + raw_buf(k)), raw_phase(k) & 1u, a.wait_ns);
        return false;
    }
    pipe.base += (uint32_t)NS;

    if constexpr (CPLX && !C::IQ_SEP) {
        upk(acci2[0], acci[0], acci[1]);
        upk(acci2[1], acci[2], acci[3]);
    }
    if constexpr (C::IQ_SEP) {
        acc2[0] = pk(iq_re[0], iq_re[1]);
        acc2[1] = pk(iq_re[2], iq_re[3]);
#pragma unroll
        for (int k = 0; k < 4; ++k) acci[k] = iq_im[k];
    }
    float acc[4];
    upk(acc2[0], acc[0], acc[1]);
    upk(acc2[1], acc[2], acc[3]);
    if (a.tile_flags && n_split > 1) {
        // ---- ordered accumulation of the channel splits of this tile: split
        // s adds its sums to the image once splits 0 .. s-1 have (the wait is
        // on a unit with a smaller ticket, which is running or done)
        int* flag = a.tile_flags + tile;
        int ok = 1;
        if (split > 0 && tid == 0) {
            const unsigned long long t0 = globaltimer_ns();
            for (;;) {
                int v;
                asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
                if (v >= split) break;
                if (globaltimer_ns() - t0 > (unsigned long long)a.wait_ns) { ok = 0; break; }
                __nanosleep(100);
            }
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(a.status, kStatusWaitExpired);
            return false;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int ku = k % VU, kr = k / VU;
            const int row = warp * C::VR + kr;
            const int iu = u0 + lane + 32 * ku, iv = v0 + bvdiv.mod(row), iw = w0 + bvdiv.div(row);
            if (iu < a.n_u && iv < a.n_v && iw < a.n_w) {
                const long long o = (long long)iw * a.out_sw + (long long)iv * a.out_sv + (long long)iu * a.out_su;
                a.image[o] = split ? __ldcg(a.image + o) + acc[k] : acc[k];
                if (CPLX) a.image[a.image_plane + o] = split ? __ldcg(a.image + a.image_plane + o) + acci[k] : acci[k];
            }
        }
        __syncthreads();                       // every store of this split precedes the release
        if (tid == 0) {
            __threadfence();
            asm volatile("st.release.gpu.global.s32 [%0], %1;" :: "l"(flag), "r"(split + 1) : "memory");
        }
        return true;
    }

    // ---- store the tile (or this unit's partial of it)
    float* out = slice >= 0 ? a.partial + (long long)slice * a.partial_stride
               : n_split > 1 ? a.partial + (long long)split * a.partial_stride : a.image;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int ku = k % VU, kr = k / VU;
        const int row = warp * C::VR + kr;
        const int iu = u0 + lane + 32 * ku, iv = v0 + bvdiv.mod(row), iw = w0 + bvdiv.div(row);
        if (iu < a.n_u && iv < a.n_v && iw < a.n_w) {
            const long long o = (long long)iw * a.out_sw + (long long)iv * a.out_sv + (long long)iu * a.out_su;
            out[o] = acc[k];
            if (CPLX) out[a.image_plane + o] = acci[k];
        }
    }
    return true;
}

}  // namespace rcbf

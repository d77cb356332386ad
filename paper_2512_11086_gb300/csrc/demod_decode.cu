// demod_decode.cu — quadrature demodulation fused into the decode's load
// (§OPTIMIZATIONS "Filtering & Demodulation": filter and decimate first, the
// samples reused from shared memory; Eq. (demodulation)), followed in the same
// kernel by the exact Hadamard decode of both planes (§OPTIMIZATIONS
// "Decoding"). The demodulated int16 planes never leave the SM.
//
// Tile: one receive channel c and 64 consecutive demodulated samples m0 ..
// m0 + 63, all n acquisitions. With f_s = 4 f_d and D = 4 or 8, every
// output m sits at raw index m D = 0 (mod 4), so the mixer phase of the raw
// sample m D - k depends on the tap k only: folding the mixer (1, -j, -1, j)
// and the complex taps h = hr + j hi into two real tap sets gives
//   I[m] = sum_k a[k] x[m D - k],  Q[m] = sum_k b[k] x[m D - k],
//   k even: a = s_k hr, b = s_k hi;  k odd: a = -s_k hi, b = s_k hr,
//   s_k = +1 for k = 0, 1 (mod 4), -1 for k = 2, 3 (mod 4)
// (real taps: a is zero at odd k, b at even k). Exact in 32-bit integers
// (sum |hr| + sum |hi| <= 65535), then the rounding right shift (ties to
// even) and int16 saturation of rcbf_demodulate.
//
// Per tile: (1) all threads stage the raw window x[k][c][m0 D - HALO ..
// m0 D + 64 D) of every acquisition k in shared memory, polyphase and
// transposed ([phase][q][k], k fastest), zero outside the record; (2) thread
// (k, output group) computes its N / 8 outputs of row k by a register-blocked
// convolution: for each tap class r = k mod 4 the taps a[4v + r] run over a
// window of phase-(-r mod 4) samples held in registers, so one shared load
// feeds up to 8 taps x N / 8 outputs; (3) the I and Q int16 outputs form one
// 128-column staged tile (I in columns 0-63, Q in 64-127) that the exact
// split-byte FP16 tensor-core decode (as in decode_mma_f16_kernel) turns into
// D / n for both planes, written as the two FP32 planes of RCBF_CF32.
#include "decode_tile.cuh"

namespace rcbf {

namespace {

constexpr int kFdThreads = 512;
constexpr int kFdDecodeWarps = 8;     // warps of the decode step (the mma.sync layout of 8 warps)
constexpr int kFdOut = 64;            // demodulated samples per tile
constexpr int kFdTapBlock = 8;        // taps of one class per register window

__device__ __forceinline__ int16_t fd_round_shift_sat(int acc, int shift) {
    int q = acc;
    if (shift > 0) {
        q = acc >> shift;                                      // floor (arithmetic shift)
        const int rem = acc - (q << shift);                    // 0 <= rem < 2^shift
        const int half = 1 << (shift - 1);
        if (rem > half || (rem == half && (q & 1))) q += 1;
    }
    return (int16_t)max(-32768, min(32767, q));
}

struct FdLayout {
    int halo;        // raw samples kept before the tile's first output position (32 vb: >= the padded taps)
    int wl;          // raw window length: 64 D + halo (multiple of 8)
    int ql;          // samples per phase row: wl / 4
    int vb;          // tap blocks per class: ceil(ceil(T / 4) / 8)
    size_t raw_bytes, stage_bytes, taps_bytes, total;
};

__host__ __device__ inline FdLayout fd_layout(int n, int D, int n_taps) {
    FdLayout L;
    L.vb = ((n_taps + 3) / 4 + kFdTapBlock - 1) / kFdTapBlock;
    // the padded tap range reaches k = 32 vb - 1: a halo of 32 vb samples keeps
    // every window index of every tap block inside the staged window
    L.halo = 4 * kFdTapBlock * L.vb;
    L.wl = kFdOut * D + L.halo;
    L.ql = L.wl / 4;
    L.raw_bytes = (size_t)4 * L.ql * n * sizeof(int16_t);
    L.stage_bytes = (size_t)n * kRowPitch;
    L.taps_bytes = (size_t)2 * 4 * L.vb * kFdTapBlock * sizeof(int);
    L.total = L.raw_bytes + L.stage_bytes + L.taps_bytes;
    return L;
}

// taps a (I) and b (Q), folded with the mixer, by class r = k mod 4 and index v = k / 4:
// ta[r][v], tb[r][v] (zero past the last tap)
template <int N, int DQ, bool CPLX>
__global__ void __launch_bounds__(kFdThreads, 1)
demod_decode_kernel(const int16_t* __restrict__ rf, float* __restrict__ out, const int16_t* __restrict__ taps,
                    const int16_t* __restrict__ taps_im, const uint32_t* __restrict__ afrag16,
                    const int* __restrict__ hsum, int n_taps, int shift, int D, int n_ch, int n_s, float inv_n) {
    using DC = DecodeCfg<N>;
    constexpr int OPT = kFdOut * N / kFdThreads;               // outputs per thread and component
    constexpr int GROUPS = kFdThreads / N;                     // output groups of a row
    static_assert(OPT * GROUPS == kFdOut, "tile split");
    extern __shared__ __align__(128) unsigned char smem[];
    const FdLayout L = fd_layout(N, D, n_taps);
    int16_t* raw = reinterpret_cast<int16_t*>(smem);                                  // [4][ql][N]
    unsigned char* stage = smem + L.raw_bytes;                                         // [N][kRowPitch]
    int* ta = reinterpret_cast<int*>(smem + L.raw_bytes + L.stage_bytes);             // [4][vb * 8]
    int* tb = ta + 4 * L.vb * kFdTapBlock;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long n_in = (long long)n_s * D;
    const int n_blocks = (n_s + kFdOut - 1) / kFdOut;
    const long long n_tiles = (long long)n_ch * n_blocks;
    const int TV = L.vb * kFdTapBlock;

    for (int q = tid; q < 4 * TV; q += kFdThreads) {
        const int r = q / TV, v = q % TV, k = 4 * v + r;
        int a = 0, b = 0;
        if (k < n_taps) {
            const int hr = taps[k], hi = CPLX ? (int)taps_im[k] : 0;
            const int sg = (r < 2) ? 1 : -1;
            if ((k & 1) == 0) { a = sg * hr; b = sg * hi; }
            else { a = -sg * hi; b = sg * hr; }
        }
        ta[q] = a;
        tb[q] = b;
    }

    const int krow = tid % N, grp = tid / N;
    const int o0 = grp * OPT;
    const uint32_t sb = smem_u32(stage);

    // ---- (1) raw window of a tile, polyphase and transposed: raw[(p * ql + q) * N + k] =
    // x[w0 + 4q + p], by threads tix of nthr. Each thread first loads up to 8 of its 16-byte
    // chunks, then scatters them, so that its global loads are in flight together.
    auto stage_raw = [&](long long tl, int tix, int nthr) {
        const int c = (int)(tl / n_blocks);
        const long long w0 = (long long)((int)(tl % n_blocks) * kFdOut) * D - L.halo;   // multiple of 8
        const int chunks = L.wl / 8;                           // 16-byte chunks per row
        const int total = N * chunks;
        for (int t0 = 0; t0 < total; t0 += 8 * nthr) {
            uint32_t wv[8][4];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int t = t0 + tix + u * nthr;
                wv[u][0] = wv[u][1] = wv[u][2] = wv[u][3] = 0u;
                if (t < total) {
                    const int k = t % N, ch = t / N;
                    const long long i0 = w0 + 8LL * ch;
                    const int16_t* src = rf + ((long long)k * n_ch + c) * n_in;
                    if (i0 >= 0 && i0 + 8 <= n_in) {
                        const int4 v = __ldg(reinterpret_cast<const int4*>(src + i0));
                        wv[u][0] = (uint32_t)v.x; wv[u][1] = (uint32_t)v.y;
                        wv[u][2] = (uint32_t)v.z; wv[u][3] = (uint32_t)v.w;
                    } else {
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const uint32_t w = (i0 + e >= 0 && i0 + e < n_in) ? (uint32_t)(uint16_t)src[i0 + e] : 0u;
                            wv[u][e >> 1] |= w << (16 * (e & 1));
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int t = t0 + tix + u * nthr;
                if (t >= total) break;
                const int k = t % N, ch = t / N;
                // samples 8 ch + e -> phase e % 4, q = 2 ch + e / 4
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int16_t val = (int16_t)((wv[u][e >> 1] >> (16 * (e & 1))) & 0xFFFFu);
                    raw[((e & 3) * L.ql + 2 * ch + (e >> 2)) * N + k] = val;
                }
            }
        }
    };

    // The decode of a tile reads only the staged tile, so while warps 0-7 decode tile t the
    // other warps stage the raw window of the CTA's next tile.
    if (blockIdx.x < n_tiles) stage_raw(blockIdx.x, tid, kFdThreads);
    __syncthreads();
    for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int c = (int)(tile / n_blocks);
        const int m0 = (int)(tile % n_blocks) * kFdOut;
        // ---- (2) FIR of row krow, outputs o0 .. o0 + OPT - 1 (tile-local), both components
        {
            int accI[OPT], accQ[OPT];
#pragma unroll
            for (int j = 0; j < OPT; ++j) accI[j] = accQ[j] = 0;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                // output o, tap k = 4 v + r reads window sample o D + halo - k
                //   = 4 q + ph,  q = o DQ - v + base,  ph = (-r) mod 4,  base = (halo - r - ph) / 4
                // (D = 4 DQ and halo are multiples of 4)
                constexpr int PH_OF[4] = {0, 3, 2, 1};
                const int ph = PH_OF[r];
                const int base = (L.halo - r - ph) / 4;
                const int16_t* prow = raw + (size_t)ph * L.ql * N + krow;
                const int* tar = ta + r * TV;
                const int* tbr = tb + r * TV;
                // real taps: class r feeds only I (r even) or only Q (r odd)
                const bool useI = CPLX || (r & 1) == 0, useQ = CPLX || (r & 1) == 1;
#pragma unroll 1
                for (int vb = 0; vb < L.vb; ++vb) {
                    const int v0 = vb * kFdTapBlock;
                    // window: q = (o0 + j) DQ - v + base for j in [0, OPT), v in [v0, v0 + 8)
                    //   -> win[t] = q_lo + t, q_lo = o0 DQ - v0 - 7 + base (>= 0: halo = 32 vb)
                    constexpr int WN = (OPT - 1) * DQ + kFdTapBlock;
                    int win[WN];
                    const int qlo = o0 * DQ - v0 - (kFdTapBlock - 1) + base;
#pragma unroll
                    for (int t = 0; t < WN; ++t) win[t] = prow[(size_t)(qlo + t) * N];
#pragma unroll
                    for (int vv = 0; vv < kFdTapBlock; ++vv) {
                        const int a = useI ? tar[v0 + vv] : 0, b = useQ ? tbr[v0 + vv] : 0;
#pragma unroll
                        for (int j = 0; j < OPT; ++j) {
                            const int x = win[j * DQ - vv + kFdTapBlock - 1];
                            if (useI) accI[j] += a * x;
                            if (useQ) accQ[j] += b * x;
                        }
                    }
                }
            }
            // ---- (3) int16 I / Q into the staged tile: row krow, columns o (I) and 64 + o (Q)
            int16_t* srow = reinterpret_cast<int16_t*>(stage + (size_t)krow * kRowPitch);
#pragma unroll
            for (int j = 0; j < OPT; ++j) {
                const bool valid = m0 + o0 + j < n_s;
                srow[o0 + j] = valid ? fd_round_shift_sat(accI[j], shift) : (int16_t)0;
                srow[kFdOut + o0 + j] = valid ? fd_round_shift_sat(accQ[j], shift) : (int16_t)0;
            }
        }
        __syncthreads();                                       // raw window consumed, staged tile ready
        if (warp >= kFdDecodeWarps) {
            const long long next = tile + gridDim.x;
            if (next < n_tiles) stage_raw(next, tid - 32 * kFdDecodeWarps, kFdThreads - 32 * kFdDecodeWarps);
        } else {
        // ---- (4) exact decode of the staged tile (split-byte FP16 mma.sync), two FP32 planes
            const int mg = warp % DC::MG, ng = warp / DC::MG;
            const int g = lane >> 2, t4 = lane & 3;
            constexpr int KF = N / 16;
            const uint4* fr4 = reinterpret_cast<const uint4*>(afrag16);
            auto frag = [&](int m, int kc, uint32_t (&rr)[4]) {
                const uint4 v = __ldg(fr4 + ((mg * 2 + m) * KF + kc) * 32 + lane);
                rr[0] = v.x; rr[1] = v.y; rr[2] = v.z; rr[3] = v.w;
            };
            int corr[2][2];
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                corr[m][0] = hsum[(mg * 2 + m) * 16 + g] * 295936;
                corr[m][1] = hsum[(mg * 2 + m) * 16 + g + 8] * 295936;
            }
#pragma unroll 1
            for (int jn = 0; jn < DC::NT; ++jn) {
                const int nt = ng * DC::NT + jn;              // n8 tile of the 128 staged columns
                float hi[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
                float lo[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll 1
                for (int kc = 0; kc < N / 32; ++kc) {
                    const int kr = kc * 32 + (lane >> 3) * 8 + (lane & 7);
                    uint32_t x[4];
                    ldsm_x4_trans(sb + kr * kRowPitch + nt * 16, x[0], x[1], x[2], x[3]);
                    uint32_t bh[4], bl[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        bl[q] = prmt(x[q], 0x64646464u, 0x4240);
                        bh[q] = prmt(x[q] ^ 0x80008000u, 0x64646464u, 0x4341);
                    }
#pragma unroll
                    for (int m = 0; m < 2; ++m) {
                        uint32_t a0[4], a1[4];
                        frag(m, 2 * kc, a0);
                        frag(m, 2 * kc + 1, a1);
                        mma_f16(hi[m], a0, bh[0], bh[1]);
                        mma_f16(lo[m], a0, bl[0], bl[1]);
                        mma_f16(hi[m], a1, bh[2], bh[3]);
                        mma_f16(lo[m], a1, bl[2], bl[3]);
                    }
                }
                // staged column col -> plane col / 64, sample m0 + col % 64
                const int col = nt * 8 + 2 * t4;
                const int plane = col / kFdOut, mm = m0 + col % kFdOut;
#pragma unroll
                for (int m = 0; m < 2; ++m) {
#pragma unroll
                    for (int hlf = 0; hlf < 2; ++hlf) {
                        const int row = (mg * 2 + m) * 16 + g + 8 * hlf;
                        const int d0 = __float2int_rn(hi[m][2 * hlf]) * 256 + __float2int_rn(lo[m][2 * hlf]) -
                                       corr[m][hlf];
                        const int d1 = __float2int_rn(hi[m][2 * hlf + 1]) * 256 +
                                       __float2int_rn(lo[m][2 * hlf + 1]) - corr[m][hlf];
                        float* dst = out + (((long long)plane * N + row) * n_ch + c) * n_s + mm;
                        // n_s is a multiple of 8, so a column pair is inside or outside the record together
                        if (mm < n_s)
                            *reinterpret_cast<float2*>(dst) =
                                make_float2(__int2float_rn(d0) * inv_n, __int2float_rn(d1) * inv_n);
                    }
                }
            }
        }
        __syncthreads();                                       // staged tile decoded, next raw window staged
    }
}

template <int N, int DQ, bool CPLX>
int fd_launch(const PlanHost& h, const int16_t* rf, float* out, cudaStream_t s, bool configure) {
    const int D = (int)h.p.demod_decimation, n_taps = (int)h.p.demod_n_taps;
    const FdLayout L = fd_layout(N, D, n_taps);
    auto k = demod_decode_kernel<N, DQ, CPLX>;
    if (configure) {
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total) != cudaSuccess)
            return check_launch("demod_decode: set shared memory");
        return RCBF_OK;
    }
    const long long tiles = (long long)h.p.n_ch * ((h.p.n_samples + kFdOut - 1) / kFdOut);
    long long grid = h.n_sms > 0 ? h.n_sms : 1;
    if (grid > tiles) grid = tiles;
    k<<<(unsigned)grid, kFdThreads, L.total, s>>>(rf, out, h.d_taps, h.d_taps_im, h.d_afrag16, h.d_hsum, n_taps,
                                                  (int)h.p.demod_shift, D, (int)h.p.n_ch, (int)h.p.n_samples,
                                                  1.0f / (float)h.p.n_tx);
    return check_launch("demod_decode_kernel");
}

template <int DQ>
int fd_dispatch_dq(const PlanHost& h, const int16_t* rf, float* out, cudaStream_t s, bool configure) {
    const bool cplx = h.d_taps_im != nullptr;
    switch (h.p.n_tx) {
        case 32: return cplx ? fd_launch<32, DQ, true>(h, rf, out, s, configure) : fd_launch<32, DQ, false>(h, rf, out, s, configure);
        case 64: return cplx ? fd_launch<64, DQ, true>(h, rf, out, s, configure) : fd_launch<64, DQ, false>(h, rf, out, s, configure);
        case 128: return cplx ? fd_launch<128, DQ, true>(h, rf, out, s, configure) : fd_launch<128, DQ, false>(h, rf, out, s, configure);
        default: return set_error(RCBF_EUNSUPPORTED, "rcbf_demod_decode: n_tx must be 32, 64 or 128");
    }
}

int fd_dispatch(const PlanHost& h, const int16_t* rf, float* out, cudaStream_t s, bool configure) {
    switch (h.p.demod_decimation) {
        case 4: return fd_dispatch_dq<1>(h, rf, out, s, configure);
        case 8: return fd_dispatch_dq<2>(h, rf, out, s, configure);
        default: return set_error(RCBF_EUNSUPPORTED, "rcbf_demod_decode: the decimation must be 4 or 8");
    }
}

}  // namespace

// Whether the fused form takes the plan (host only); *why says why not.
bool demod_decode_supported(const PlanHost& h, std::string* why) {
    const rcbf_params& p = h.p;
    if (!p.demod_decimation || !p.hadamard_order || p.decoded_dtype != RCBF_CF32) {
        *why = "rcbf_demod_decode: the plan needs demodulation, a Hadamard order and RCBF_CF32 output";
        return false;
    }
    if (p.demod_decimation != 4 && p.demod_decimation != 8) {
        *why = "rcbf_demod_decode: the decimation must be 4 or 8 (a multiple of 4 puts every output at mixer "
               "phase 0; larger ones exceed the register window)";
        return false;
    }
    if (!(p.n_tx == 32 || p.n_tx == 64 || p.n_tx == 128) || !h.d_afrag16) {
        *why = "rcbf_demod_decode: n_tx must be 32, 64 or 128";
        return false;
    }
    const FdLayout L = fd_layout((int)p.n_tx, (int)p.demod_decimation, (int)p.demod_n_taps);
    if (L.total > 227 * 1024) {
        *why = "rcbf_demod_decode: the raw window of 64 outputs (64 D + taps samples per acquisition) exceeds "
               "shared memory; use rcbf_demodulate and rcbf_decode";
        return false;
    }
    return true;
}

int configure_demod_decode(const PlanHost& h) {
    std::string why;
    if (!demod_decode_supported(h, &why)) return RCBF_OK;    // the entry point reports why at call time
    return fd_dispatch(h, nullptr, nullptr, nullptr, true);
}

int launch_demod_decode(const PlanHost& h, const int16_t* rf, float* out, cudaStream_t s) {
    return fd_dispatch(h, rf, out, s, false);
}

}  // namespace rcbf

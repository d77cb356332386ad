// decode.cu — Hadamard aperture decode D = H^T S across the transmit axis
// (§THEORY "Synthetic Aperture Imaging"; §OPTIMIZATIONS "Decoding").
//
// The tensor-core form treats the decode as one GEMM with M = K = n (the
// order) and N = n_ch * n_samples columns, exact in integer arithmetic:
//   each int16 sample v is split into a signed high byte h = v >> 8 and an
//   unsigned low byte l = v & 0xff (v = 256 h + l), and
//   D = 256 * (H^T . S_hi) + (H^T . S_lo)
// with two int8 mma.sync products accumulated in int32 (|partial| <= 256*255).
// The int8 tensor op of the 5th-generation tcgen05 path is not available on
// sm_103a, so the warp-level mma.sync.m16n8k32 s8/u8 form is used.
//
// Layout: S is [n][n_cols] int16 (columns contiguous). A CTA streams tiles of
// n rows x 128 columns through a cp.async pipeline into padded shared memory;
// ldmatrix.trans delivers, per thread, pairs of consecutive acquisitions of
// one column, which two byte permutes turn into the hi / lo B fragments. The
// B fragment's k order is therefore a fixed permutation of the acquisitions;
// the A = H^T fragments are built on the host in the same permuted order.
#include "decode_tile.cuh"

namespace rcbf {

namespace {

template <int N, int DT>
__global__ void __launch_bounds__(kDecodeThreads, 1)
decode_mma_kernel(DecodeArgs a) {
    using C = DecodeCfg<N>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int mg = warp % C::MG, ng = warp / C::MG;
    const int g = lane >> 2, t = lane & 3;
    const long long n_cols = a.n_cols;
    const long long n_tiles = (n_cols + kDecodeCols - 1) / kDecodeCols;

    // A = H^T fragments of this warp's two m16 tiles, all k chunks, held in registers
    uint32_t afr[2][C::KC][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int kc = 0; kc < C::KC; ++kc) {
            const uint4 v = reinterpret_cast<const uint4*>(a.afrag)[((mg * 2 + m) * C::KC + kc) * 32 + lane];
            afr[m][kc][0] = v.x; afr[m][kc][1] = v.y; afr[m][kc][2] = v.z; afr[m][kc][3] = v.w;
        }

    const uint32_t sbase = smem_u32(smem);
    auto issue = [&](long long tile, int stage) {
        const long long col0 = tile * kDecodeCols;
        const uint32_t dst0 = sbase + stage * C::STAGE_BYTES;
#pragma unroll
        for (int q = 0; q < C::CHUNKS_PER_THREAD; ++q) {
            const int chunk = tid + q * kDecodeThreads;
            const int row = chunk / (kDecodeCols / 8);
            const int cc = chunk % (kDecodeCols / 8);
            const long long col = col0 + cc * 8;
            const bool valid = (tile < n_tiles) && (col < n_cols);
            const int16_t* src = a.rf + (valid ? (long long)row * n_cols + col : 0);
            cp_async16(dst0 + row * kRowPitch + cc * 16, src, valid);
        }
    };

    long long tile = blockIdx.x;
    const long long step = gridDim.x;
#pragma unroll
    for (int s = 0; s < C::STAGES - 1; ++s) {
        issue(tile + s * step, s);
        cp_async_commit();
    }
    for (int it = 0; tile < n_tiles; ++it, tile += step) {
        cp_async_wait<C::STAGES - 2>();
        __syncthreads();
        issue(tile + (C::STAGES - 1) * step, (it + C::STAGES - 1) % C::STAGES);
        cp_async_commit();

        const uint32_t sb = sbase + (it % C::STAGES) * C::STAGE_BYTES;
        const long long col0 = tile * kDecodeCols;
#pragma unroll 1
        for (int j = 0; j < C::NT; ++j) {
            const int nt = ng * C::NT + j;           // n8 tile within the CTA tile
            const long long colb = col0 + nt * 8;
            if (colb >= n_cols) break;
            int acc_hi[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
            int acc_lo[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
#pragma unroll
            for (int kc = 0; kc < C::KC; ++kc) {
                // matrix q = lane / 8 covers acquisitions kc*32 + 8q .. +7; lane % 8 picks the row
                const int krow = kc * 32 + (lane >> 3) * 8 + (lane & 7);
                uint32_t x0, x1, x2, x3;
                ldsm_x4_trans(sb + krow * kRowPitch + nt * 16, x0, x1, x2, x3);
                const uint32_t bh0 = prmt(x0, x1, 0x7531), bl0 = prmt(x0, x1, 0x6420);
                const uint32_t bh1 = prmt(x2, x3, 0x7531), bl1 = prmt(x2, x3, 0x6420);
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    mma_s8s8(acc_hi[m], afr[m][kc], bh0, bh1);
                    mma_s8u8(acc_lo[m], afr[m][kc], bl0, bl1);
                }
            }
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int row = (mg * 2 + m) * 16 + g;
                const long long col = colb + 2 * t;
                const int d0 = acc_hi[m][0] * 256 + acc_lo[m][0];
                const int d1 = acc_hi[m][1] * 256 + acc_lo[m][1];
                const int d2 = acc_hi[m][2] * 256 + acc_lo[m][2];
                const int d3 = acc_hi[m][3] * 256 + acc_lo[m][3];
                store_pair<DT>(a.out, (long long)row * n_cols + col, d0, d1, a.inv_n);
                store_pair<DT>(a.out, (long long)(row + 8) * n_cols + col, d2, d3, a.inv_n);
            }
        }
    }
    cp_async_wait<0>();
}

// Byte-split FP16 form. The sample is offset to unsigned, u = v + 32768 =
// 256 U + l (U, l in [0, 255]); each byte b is placed in an FP16 as 1024 + b
// (exponent 10, exact), so with h_i = sum_k H[k][i]
//   D_i = 256 * sum_k H (1024 + U) + sum_k H (1024 + l) - (256*1024 + 1024 + 32768) h_i,
// both sums exact in the FP32 accumulators (|sum| <= 256 * 1279 < 2^24).
// ldmatrix.trans yields the k16 B fragments in natural order, so the A = H^T
// fragments need no permutation here.
template <int N, int DT>
__global__ void __launch_bounds__(kDecodeThreads, 1)
decode_mma_f16_kernel(DecodeArgs a) {
    using C = DecodeCfg<N>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int mg = warp % C::MG, ng = warp / C::MG;
    const int g = lane >> 2, t = lane & 3;
    const long long n_cols = a.n_cols;
    const long long n_tiles = (n_cols + kDecodeCols - 1) / kDecodeCols;
    constexpr int K16 = N / 16;

    uint32_t afr[2][K16][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int kc = 0; kc < K16; ++kc) {
            const uint4 v = reinterpret_cast<const uint4*>(a.afrag16)[((mg * 2 + m) * K16 + kc) * 32 + lane];
            afr[m][kc][0] = v.x; afr[m][kc][1] = v.y; afr[m][kc][2] = v.z; afr[m][kc][3] = v.w;
        }
    int corr[2][2];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        corr[m][0] = a.hsum[(mg * 2 + m) * 16 + g] * 295936;
        corr[m][1] = a.hsum[(mg * 2 + m) * 16 + g + 8] * 295936;
    }

    const uint32_t sbase = smem_u32(smem);
    auto issue = [&](long long tile, int stage) {
        const long long col0 = tile * kDecodeCols;
        const uint32_t dst0 = sbase + stage * C::STAGE_BYTES;
#pragma unroll
        for (int q = 0; q < C::CHUNKS_PER_THREAD; ++q) {
            const int chunk = tid + q * kDecodeThreads;
            const int row = chunk / (kDecodeCols / 8);
            const int cc = chunk % (kDecodeCols / 8);
            const long long col = col0 + cc * 8;
            const bool valid = (tile < n_tiles) && (col < n_cols);
            const int16_t* src = a.rf + (valid ? (long long)row * n_cols + col : 0);
            cp_async16(dst0 + row * kRowPitch + cc * 16, src, valid);
        }
    };

    long long tile = blockIdx.x;
    const long long step = gridDim.x;
#pragma unroll
    for (int s = 0; s < C::STAGES - 1; ++s) {
        issue(tile + s * step, s);
        cp_async_commit();
    }
    for (int it = 0; tile < n_tiles; ++it, tile += step) {
        cp_async_wait<C::STAGES - 2>();
        __syncthreads();
        issue(tile + (C::STAGES - 1) * step, (it + C::STAGES - 1) % C::STAGES);
        cp_async_commit();

        const uint32_t sb = sbase + (it % C::STAGES) * C::STAGE_BYTES;
        const long long col0 = tile * kDecodeCols;
#pragma unroll 1
        for (int j = 0; j < C::NT; ++j) {
            const int nt = ng * C::NT + j;
            const long long colb = col0 + nt * 8;
            if (colb >= n_cols) break;
            float acc_hi[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
            float acc_lo[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
            for (int kc = 0; kc < N / 32; ++kc) {
                const int krow = kc * 32 + (lane >> 3) * 8 + (lane & 7);
                uint32_t x[4];
                ldsm_x4_trans(sb + krow * kRowPitch + nt * 16, x[0], x[1], x[2], x[3]);
                uint32_t bh[4], bl[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    bl[q] = prmt(x[q], 0x64646464u, 0x4240);                 // 1024 + low byte
                    bh[q] = prmt(x[q] ^ 0x80008000u, 0x64646464u, 0x4341);   // 1024 + high byte of v + 32768
                }
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    mma_f16(acc_hi[m], afr[m][2 * kc], bh[0], bh[1]);
                    mma_f16(acc_lo[m], afr[m][2 * kc], bl[0], bl[1]);
                    mma_f16(acc_hi[m], afr[m][2 * kc + 1], bh[2], bh[3]);
                    mma_f16(acc_lo[m], afr[m][2 * kc + 1], bl[2], bl[3]);
                }
            }
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int row = (mg * 2 + m) * 16 + g;
                const long long col = colb + 2 * t;
                int d[4];
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    d[r] = __float2int_rn(acc_hi[m][r]) * 256 + __float2int_rn(acc_lo[m][r]) - corr[m][r >> 1];
                store_pair<DT>(a.out, (long long)row * n_cols + col, d[0], d[1], a.inv_n);
                store_pair<DT>(a.out, (long long)(row + 8) * n_cols + col, d[2], d[3], a.inv_n);
            }
        }
    }
    cp_async_wait<0>();
}

// Plain CUDA-core form: one thread per (column, block of 16 decoded rows),
// int32 sums over all acquisitions, H read through the read-only cache.
template <int DT>
__global__ void __launch_bounds__(256)
decode_plain_kernel(DecodeArgs a) {
    const int n = a.n;
    const long long col = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int i0 = blockIdx.y * 16;
    if (col >= a.n_cols) return;
    int acc[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) acc[r] = 0;
    for (int k = 0; k < n; ++k) {
        const int v = a.rf[(long long)k * a.n_cols + col];
#pragma unroll
        for (int r = 0; r < 16; ++r) acc[r] += (int)__ldg(a.hmat + k * n + i0 + r) * v;
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const long long idx = (long long)(i0 + r) * a.n_cols + col;
        if (DT == RCBF_I32) static_cast<int*>(a.out)[idx] = acc[r];
        else if (DT == RCBF_F32) static_cast<float*>(a.out)[idx] = __int2float_rn(acc[r]) * a.inv_n;
        else static_cast<__half*>(a.out)[idx] = __float2half_rn(__int2float_rn(acc[r]) * a.inv_n);
    }
}

template <int N, int DT, bool F16>
int configure_mma(int* grid_per_sm) {
    using C = DecodeCfg<N>;
    auto k = F16 ? decode_mma_f16_kernel<N, DT> : decode_mma_kernel<N, DT>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) != cudaSuccess)
        return check_launch("decode: set shared memory");
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kDecodeThreads, C::SMEM) != cudaSuccess)
        return check_launch("decode: occupancy");
    *grid_per_sm = per_sm < 1 ? 1 : per_sm;
    return RCBF_OK;
}

template <int N, int DT, bool F16>
int launch_mma(const PlanHost& h, const DecodeArgs& a, cudaStream_t s) {
    using C = DecodeCfg<N>;
    const long long tiles = (a.n_cols + kDecodeCols - 1) / kDecodeCols;
    long long grid = (long long)h.n_sms * h.decode_blocks_per_sm;
    if (grid > tiles) grid = tiles;
    if (grid < 1) grid = 1;
    if (F16) decode_mma_f16_kernel<N, DT><<<(unsigned)grid, kDecodeThreads, C::SMEM, s>>>(a);
    else decode_mma_kernel<N, DT><<<(unsigned)grid, kDecodeThreads, C::SMEM, s>>>(a);
    return check_launch("decode_mma_kernel");
}

template <int DT, bool F16>
int launch_mma_dt(const PlanHost& h, const DecodeArgs& a, cudaStream_t s) {
    switch (a.n) {
        case 32: return launch_mma<32, DT, F16>(h, a, s);
        case 64: return launch_mma<64, DT, F16>(h, a, s);
        case 128: return launch_mma<128, DT, F16>(h, a, s);
        case 256: return launch_mma<256, DT, F16>(h, a, s);
        default: return set_error(RCBF_EUNSUPPORTED, "decode: tensor-core form needs n_tx in {32, 64, 128, 256}");
    }
}

template <int DT, bool F16>
int configure_dt(int n, int* per_sm) {
    switch (n) {
        case 32: return configure_mma<32, DT, F16>(per_sm);
        case 64: return configure_mma<64, DT, F16>(per_sm);
        case 128: return configure_mma<128, DT, F16>(per_sm);
        case 256: return configure_mma<256, DT, F16>(per_sm);
        default: return set_error(RCBF_EUNSUPPORTED, "decode: tensor-core form needs n_tx in {32, 64, 128, 256}");
    }
}

template <int DT>
int launch_plain(const DecodeArgs& a, cudaStream_t s) {
    dim3 grid((unsigned)((a.n_cols + 255) / 256), (unsigned)(a.n / 16));
    decode_plain_kernel<DT><<<grid, 256, 0, s>>>(a);
    return check_launch("decode_plain_kernel");
}

}  // namespace

int launch_decode(const PlanHost& h, const int16_t* rf, void* out, cudaStream_t s) {
    if (h.p.decoded_dtype == RCBF_CF32) {
        // demodulated data: each int16 plane decodes to its FP32 plane (D / N)
        PlanHost hp = h;
        hp.p.decoded_dtype = RCBF_F32;
        const long long plane = (long long)h.p.n_tx * h.p.n_ch * h.p.n_samples;
        for (int p = 0; p < 2; ++p) {
            const int rc = launch_decode(hp, rf + p * plane, static_cast<float*>(out) + p * plane, s);
            if (rc != RCBF_OK) return rc;
        }
        return RCBF_OK;
    }
    DecodeArgs a;
    a.rf = rf;
    a.out = out;
    a.afrag = h.d_afrag;
    a.hmat = h.d_hmat;
    a.n = (int)h.p.n_tx;
    a.n_cols = (long long)h.p.n_ch * h.p.n_samples;
    a.dtype = (int)h.p.decoded_dtype;
    a.inv_n = 1.0f / (float)h.p.n_tx;
    a.afrag16 = h.d_afrag16;
    a.hsum = h.d_hsum;
    const int v = (int)h.p.decode_variant;
    if (v == RCBF_DECODE_TC) return launch_decode_tc(h, a.dtype, rf, out, s);
    switch (a.dtype) {
        case RCBF_I32: return v == RCBF_DECODE_PLAIN ? launch_plain<RCBF_I32>(a, s)
                            : v == RCBF_DECODE_MMA_F16 ? launch_mma_dt<RCBF_I32, true>(h, a, s)
                            : launch_mma_dt<RCBF_I32, false>(h, a, s);
        case RCBF_F32: return v == RCBF_DECODE_PLAIN ? launch_plain<RCBF_F32>(a, s)
                            : v == RCBF_DECODE_MMA_F16 ? launch_mma_dt<RCBF_F32, true>(h, a, s)
                            : launch_mma_dt<RCBF_F32, false>(h, a, s);
        case RCBF_F16: return v == RCBF_DECODE_PLAIN ? launch_plain<RCBF_F16>(a, s)
                            : v == RCBF_DECODE_MMA_F16 ? launch_mma_dt<RCBF_F16, true>(h, a, s)
                            : launch_mma_dt<RCBF_F16, false>(h, a, s);
        default: return set_error(RCBF_EUNSUPPORTED, "decode: output dtype must be RCBF_I32, RCBF_F32 or RCBF_F16");
    }
}

// Plan-time set-up of the tensor-core decode: shared-memory opt-in and the
// persistent grid (CTAs per SM) for the plan's order and output type.
int configure_decode(PlanHost& h) {
    if (h.p.hadamard_order == 0 || h.p.decode_variant == RCBF_DECODE_PLAIN) return RCBF_OK;
    if (h.p.decode_variant == RCBF_DECODE_TC)
        return configure_decode_tc(h, h.p.decoded_dtype == RCBF_CF32 ? (int)RCBF_F32 : (int)h.p.decoded_dtype);
    const int n = (int)h.p.n_tx;
    const bool f16 = h.p.decode_variant == RCBF_DECODE_MMA_F16;
    switch (h.p.decoded_dtype == RCBF_CF32 ? (uint32_t)RCBF_F32 : h.p.decoded_dtype) {
        case RCBF_I32: return f16 ? configure_dt<RCBF_I32, true>(n, &h.decode_blocks_per_sm)
                                  : configure_dt<RCBF_I32, false>(n, &h.decode_blocks_per_sm);
        case RCBF_F32: return f16 ? configure_dt<RCBF_F32, true>(n, &h.decode_blocks_per_sm)
                                  : configure_dt<RCBF_F32, false>(n, &h.decode_blocks_per_sm);
        case RCBF_F16: return f16 ? configure_dt<RCBF_F16, true>(n, &h.decode_blocks_per_sm)
                                  : configure_dt<RCBF_F16, false>(n, &h.decode_blocks_per_sm);
        default: return RCBF_OK;
    }
}

}  // namespace rcbf

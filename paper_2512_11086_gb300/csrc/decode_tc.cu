// decode_tc.cu — the exact Hadamard decode D = H^T S (§THEORY "Synthetic
// Aperture Imaging"; §OPTIMIZATIONS "Decoding") on the 5th-generation tensor
// cores: tcgen05.mma with the accumulators in tensor memory, the int16 tiles
// brought in by TMA tensor loads and the decoded tiles written by TMA stores.
//
// Arithmetic (the split-byte FP16 reading of the exact decode): the sample v
// is offset to unsigned, u = v + 32768 = 256 U + l with bytes U, l in
// [0, 255], and each byte b is held as the FP16 1024 + b (exponent 10, the
// byte in the mantissa: exact, one byte permute per two samples). With the
// Hadamard entries +-1 exact in FP16 and h_i = sum_k H[k][i],
//   D_i = 256 sum_k H[k][i] (1024 + U_k) + sum_k H[k][i] (1024 + l_k) - 295936 h_i.
// The two sums accumulate in separate FP32 accumulators in tensor memory;
// each partial sum is an integer of magnitude at most n * 1279 < 2^24, so
// every addition is exact and D is exact for every int16 input.
//
// One CTA per SM, persistent over tiles of 64 columns (one 128-byte row of
// int16 per acquisition). Warp roles:
//   warp 0     TMA producer: S tiles (n rows x 64 columns, 128-byte swizzle)
//              into a ring of raw tiles (as many as shared memory holds, 2-8)
//              that runs ahead of the converters;
//   warp 1     owns the tensor memory (256 columns: two accumulator sets of
//              lo 64 + hi 64 columns) and issues the MMAs: M = 128 (rows i;
//              rows >= n of A are zero), N = 128 (the lo and the hi operand
//              tile of the same 64 columns side by side, so that one
//              instruction, one read of A, serves both byte planes), K = 16 per
//              instruction, A = H^T K-major, B MN-major (samples contiguous,
//              as they arrive), both 128-byte swizzled;
//   warps 2-5  convert a landed tile: each 16-byte chunk of int16 becomes
//              the FP16 lo bytes and the FP16 hi bytes at the same offset of a
//              (lo, hi) operand pair of a 2-deep ring (int16 and FP16 are both
//              2 bytes, so the swizzled layout carries over);
//   warps 6-13 epilogue: tcgen05.ld of 32 accumulator lanes (rows) by 32
//              columns each, D = 256 hi + lo - correction, the output
//              conversion, a 128-byte-swizzled staging tile (double-buffered)
//              and one TMA store per tile.
// Every mbarrier wait is bounded (global timer); an expired wait records
// kStatusWaitExpired in the plan's status word, stops the CTA's loop, drains
// what it issued (bounded) and frees the tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "internal.cuh"

namespace rcbf {

namespace {

constexpr int kTcThreads = 448;
constexpr int kTcCols = 64;          // columns per tile
constexpr int kTcTmemCols = 256;     // two accumulator sets of (lo 64 + hi 64) FP32 columns
constexpr int kTcConvThreads = 128;  // warps 2-5
constexpr int kTcEpiThreads = 256;   // warps 6-13
constexpr int kTcSmemMax = 232448;   // opt-in shared memory per CTA

template <int N, int ES>
struct TcCfg {
    static constexpr int KATOMS = N > 64 ? N / 64 : 1;      // 64-wide K atoms of A (K-major, swizzled)
    static constexpr int A_BYTES = KATOMS * 128 * 128;      // 128 rows x 128 bytes per atom
    static constexpr int TILE_BYTES = N * 128;              // n rows x 64 int16 / FP16
    static constexpr int ROWS = N < 128 ? N : 128;          // output rows of a tile
    static constexpr int BOXES = kTcCols * ES / 128;        // 128-byte store boxes per tile
    static constexpr int STAGING = BOXES * ROWS * 128;      // one output tile (two of them, double-buffered)
    // raw int16 tiles in flight: as many as the remaining shared memory holds (2..8)
    static constexpr int FIXED = A_BYTES + 2 * 2 * TILE_BYTES + 2 * STAGING + 2048 + 1024;
    static constexpr int RS_FIT = (kTcSmemMax - FIXED) / TILE_BYTES;
    static constexpr int RS = RS_FIT > 8 ? 8 : RS_FIT;
    static_assert(RS >= 2, "shared memory holds at least two raw tiles");
    static constexpr int OFF_A = 0;
    static constexpr int OFF_RAW = OFF_A + A_BYTES;                // RS raw tiles (TMA destination)
    static constexpr int OFF_B = OFF_RAW + RS * TILE_BYTES;        // 2 x (lo, hi) FP16 operand tiles
    static constexpr int OFF_STAGING = OFF_B + 2 * 2 * TILE_BYTES; // 2 output staging tiles
    static constexpr int OFF_BAR = OFF_STAGING + 2 * STAGING;
    // raw_full[RS], raw_empty[RS], b_full[2], b_empty[2], accf[2], acce[2], a_full
    static constexpr int NBAR = 2 * RS + 9;
    static constexpr int OFF_MISC = OFF_BAR + 8 * NBAR;     // tmem address, abort flag
    // + alignment slack of the dynamic base; at least 120 KB so that one CTA
    // holds an SM (two would not fit) and the tensor-memory allocation of a
    // CTA never waits for another CTA of the kernel
    static constexpr int SMEM_USED = OFF_MISC + 16 + 1024;
    static constexpr int SMEM = SMEM_USED > 120 * 1024 ? SMEM_USED : 120 * 1024;
    static_assert(SMEM <= kTcSmemMax, "shared memory budget");
    static_assert(TILE_BYTES % 1024 == 0 && A_BYTES % 1024 == 0 && STAGING % 1024 == 0, "1024-byte atoms");
};

// ---- PTX wrappers (tcgen05, TMA tensor copies)

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;                       // descriptor version of sm_100 and later
    d |= (uint64_t)2 << 61;                       // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar) : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, uint32_t src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
                 :: "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(src) : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(bar) : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 lanes (one row per thread)
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void named_sync(int id, int n) {
    asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(n) : "memory");
}

// Named barrier over n threads that also ANDs a predicate across them.
__device__ __forceinline__ bool named_sync_and(int id, int n, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r) : "r"((uint32_t)v), "r"(id), "r"(n) : "memory");
    return r != 0;
}

__device__ __forceinline__ uint32_t prmt32(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// The decoded value from the two accumulators, exactly, in FP32: with
// 295936 = 256 * 1156, D = 256 (hi - 1156 h_i) + lo, where hi - 1156 h_i =
// sum_k H[k][i] (U_k - 132) is an integer below 2^15 in magnitude and
// |D| < 2^23, so the subtraction and the fused multiply-add are exact.
__device__ __forceinline__ float decoded_value(float hi, float lo, float c1) {
    return fmaf(256.0f, hi - c1, lo);
}

template <int N, int DT>
__global__ void __launch_bounds__(kTcThreads, 1)
decode_tc_kernel(const __grid_constant__ CUtensorMap map_in, const __grid_constant__ CUtensorMap map_out,
                 const uint16_t* __restrict__ atc, const int* __restrict__ hsum, long long n_cols, float inv_n,
                 int* status, long long wait_ns) {
    constexpr int ES = DT == RCBF_F16 ? 2 : 4;
    using C = TcCfg<N, ES>;
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte alignment of every swizzled buffer
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const uint32_t sbase = smem_u32(smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar0 = sbase + C::OFF_BAR;
    constexpr int RS = C::RS;
    auto raw_full = [&](int s) { return bar0 + 8u * s; };
    auto raw_empty = [&](int s) { return bar0 + 8u * (RS + s); };
    auto b_full = [&](int b) { return bar0 + 8u * (2 * RS + b); };
    auto b_empty = [&](int b) { return bar0 + 8u * (2 * RS + 2 + b); };
    auto accf_bar = [&](int a) { return bar0 + 8u * (2 * RS + 4 + a); };
    auto acce_bar = [&](int a) { return bar0 + 8u * (2 * RS + 6 + a); };
    const uint32_t a_full = bar0 + 8u * (2 * RS + 8);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + C::OFF_MISC);
    volatile int* abort = reinterpret_cast<volatile int*>(smem + C::OFF_MISC + 4);
    auto raw_buf = [&](int s) { return sbase + C::OFF_RAW + (uint32_t)(s * C::TILE_BYTES); };
    auto lo_buf = [&](int b) { return sbase + C::OFF_B + (uint32_t)(b * 2 * C::TILE_BYTES); };
    auto hi_buf = [&](int b) { return lo_buf(b) + (uint32_t)C::TILE_BYTES; };
    const long long n_tiles = (n_cols + kTcCols - 1) / kTcCols;
    const int my_tiles = blockIdx.x < n_tiles ? (int)((n_tiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;

    // ---- set-up: barriers; A = H^T (FP16 +-1, K-major, 128-byte swizzle, rows >= n
    // zero), prepared with the plan, arrives by one bulk copy while the
    // tensor memory is allocated; tensor memory
    if (tid == 0) {
        for (int s = 0; s < RS; ++s) {
            mbar_init(raw_full(s), 1);
            mbar_init(raw_empty(s), kTcConvThreads);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(b_full(b), kTcConvThreads);
            mbar_init(b_empty(b), 1);
            mbar_init(accf_bar(b), 1);
            mbar_init(acce_bar(b), kTcEpiThreads);
        }
        mbar_init(a_full, 1);
        *abort = 0;
        fence_mbar_init();
        asm volatile("prefetch.tensormap [%0];" :: "l"(reinterpret_cast<uint64_t>(&map_in)) : "memory");
        asm volatile("prefetch.tensormap [%0];" :: "l"(reinterpret_cast<uint64_t>(&map_out)) : "memory");
        mbar_arrive_expect_tx(a_full, (uint32_t)C::A_BYTES);
        bulk_g2s(sbase + C::OFF_A, atc, (uint32_t)C::A_BYTES, a_full);
        // the first raw tiles are requested before the tensor memory is
        // allocated: their latency overlaps the rest of the set-up
        for (int j = 0; j < RS && j < my_tiles; ++j) {
            const long long tile = blockIdx.x + (long long)j * gridDim.x;
            mbar_arrive_expect_tx(raw_full(j), (uint32_t)C::TILE_BYTES);
            tma_load_2d(raw_buf(j), &map_in, (int)(tile * kTcCols), 0, raw_full(j));
        }
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(s_tmem)), "r"(kTcTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    auto wait = [&](uint32_t bar, int use) -> bool {
        return mbar_wait_or_abort(bar, (uint32_t)use & 1u, abort, wait_ns);
    };
    bool ok = true;

    if (warp == 0) {
        // ---- TMA producer: raw tiles run up to RS ahead of the converters
        if (lane == 0) {
            int issued = my_tiles < RS ? my_tiles : RS;     // requested during the set-up
            for (int j = issued; j < my_tiles && ok; ++j) {
                const int s = j % RS;
                if (!(ok = wait(raw_empty(s), j / RS - 1))) break;
                const long long tile = blockIdx.x + (long long)j * gridDim.x;
                mbar_arrive_expect_tx(raw_full(s), (uint32_t)C::TILE_BYTES);
                tma_load_2d(raw_buf(s), &map_in, (int)(tile * kTcCols), 0, raw_full(s));
                issued = j + 1;
            }
            // drain: every issued load lands before the CTA may exit
            for (int j = (issued > RS ? issued - RS : 0); j < issued; ++j)
                mbar_wait_parity(raw_full(j % RS), (uint32_t)(j / RS) & 1u, wait_ns);
        }
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            // kind::f16: F32 accumulator, F16 A and B, A K-major, B MN-major, N = 128 (the lo and the
            // hi operand tile side by side: two 64-column swizzle atoms LBO apart), M = 128
            const uint32_t idesc = (1u << 4) | (1u << 16) | ((uint32_t)(2 * kTcCols >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
            const uint32_t a_base = sbase + C::OFF_A;
            int committed = 0;
            ok = wait(a_full, 0);
            for (int j = 0; j < my_tiles && ok; ++j) {
                const int b = j & 1;
                if (!(ok = wait(b_full(b), j / 2))) break;
                if (j >= 2 && !(ok = wait(acce_bar(b), j / 2 - 1))) break;
                tc_fence_after();
                // accumulator columns b * 128 + [0, 64): lo sums, + [64, 128): hi sums
                const uint32_t d = tmem + (uint32_t)(b * 128);
#pragma unroll
                for (int kk = 0; kk < N / 16; ++kk) {
                    // A: K atom kk / 4, 32 bytes per k16 step inside the swizzled row (SBO: 8-row groups)
                    const uint64_t ad = smem_desc(a_base + (uint32_t)((kk >> 2) * 16384 + (kk & 3) * 32), 16, 1024);
                    // B: 16 rows (two 8-row groups, SBO 1024) per k16 step; the lo atom, then the hi
                    // atom LBO = one tile further
                    const uint64_t bd = smem_desc(lo_buf(b) + (uint32_t)(kk * 2048), (uint32_t)C::TILE_BYTES, 1024);
                    tc_mma(d, ad, bd, idesc, kk > 0 ? 1u : 0u);
                }
                tc_commit(b_empty(b));
                tc_commit(accf_bar(b));
                committed = j + 1;
            }
            // the tensor memory is freed below only after the last MMAs completed
            if (committed > 0)
                mbar_wait_parity(accf_bar((committed - 1) & 1), (uint32_t)((committed - 1) / 2) & 1u, wait_ns);
        }
    } else if (warp < 6) {
        // ---- converters: int16 -> FP16 (1024 + byte): lo and hi operand tiles in the raw tile's
        // swizzled layout (int16 and FP16 are both 2 bytes). Eight chunks are loaded before any
        // is converted and stored, so that the loads overlap.
        const int t = tid - 64;
        constexpr int CPT = N * 8 / kTcConvThreads;          // 16-byte chunks per thread and tile
        constexpr int BATCH = CPT < 8 ? CPT : 8;
        for (int j = 0; j < my_tiles && ok; ++j) {
            const int s = j % RS, b = j & 1;
            if (!(ok = wait(raw_full(s), j / RS))) break;
            if (j >= 2 && !(ok = wait(b_empty(b), j / 2 - 1))) break;
            const uint4* raw = reinterpret_cast<const uint4*>(smem + (raw_buf(s) - sbase));
            uint4* lo = reinterpret_cast<uint4*>(smem + (lo_buf(b) - sbase));
            uint4* hi = reinterpret_cast<uint4*>(smem + (hi_buf(b) - sbase));
#pragma unroll
            for (int c0 = 0; c0 < CPT; c0 += BATCH) {
                uint4 v[BATCH];
#pragma unroll
                for (int u = 0; u < BATCH; ++u) v[u] = raw[t + kTcConvThreads * (c0 + u)];
#pragma unroll
                for (int u = 0; u < BATCH; ++u) {
                    const uint32_t in[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
                    uint32_t l[4], h[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        l[e] = prmt32(in[e], 0x64646464u, 0x4240);                 // 1024 + low byte
                        h[e] = prmt32(in[e] ^ 0x80008000u, 0x64646464u, 0x4341);   // 1024 + high byte of v + 32768
                    }
                    lo[t + kTcConvThreads * (c0 + u)] = make_uint4(l[0], l[1], l[2], l[3]);
                    hi[t + kTcConvThreads * (c0 + u)] = make_uint4(h[0], h[1], h[2], h[3]);
                }
            }
            mbar_arrive(raw_empty(s));
            fence_proxy_async_smem();
            mbar_arrive(b_full(b));
        }
    } else {
        // ---- epilogue: warp 6 + 4 hc + j' (q = warp % 4) reads accumulator lanes (rows) 32q .. 32q + 31,
        // columns 32 hc .. 32 hc + 31 of the tile
        const int e = tid - 192, q = warp & 3, hc = (warp - 6) >> 2, row = 32 * q + lane;
        const bool active = 32 * q < N;                       // warp-uniform
        const float c1 = (active && row < N) ? 1156.0f * (float)hsum[row] : 0.0f;
        for (int j = 0; j < my_tiles && ok; ++j) {
            const int a = j & 1;
            const long long tile = blockIdx.x + (long long)j * gridDim.x;
            unsigned char* stg = smem + C::OFF_STAGING + a * C::STAGING;
            bool got = wait(accf_bar(a), j / 2);
            if (e == 0) bulk_wait_read1();                    // the store of tile j - 2 has read this staging tile
            // one decision for the whole group, so that every epilogue thread
            // reaches the same named barriers
            if (!(ok = named_sync_and(1, kTcEpiThreads, got))) break;
            tc_fence_after();
            if (active) {
                float vh[32], vl[32];
                const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(a * 128 + 32 * hc);
                tc_ld32(taddr, vl);
                tc_ld32(taddr + 64, vh);
                tc_wait_ld();
                if (row < N) {
#pragma unroll
                    for (int g = 0; g < 32 * ES / 16; ++g) {
                        // 16-byte chunk g of this thread's 32 columns
                        constexpr int PER = 16 / ES;
                        uint32_t w[4];
#pragma unroll
                        for (int k = 0; k < PER; k += (ES == 2 ? 2 : 1)) {
                            const int col = g * PER + k;
                            const float d0 = decoded_value(vh[col], vl[col], c1);
                            if (DT == RCBF_F16) {
                                const float d1 = decoded_value(vh[col + 1], vl[col + 1], c1);
                                const __half2 h2 = __floats2half2_rn(d0 * inv_n, d1 * inv_n);
                                w[k >> 1] = *reinterpret_cast<const uint32_t*>(&h2);
                            } else if (DT == RCBF_F32) {
                                w[k] = __float_as_uint(d0 * inv_n);      // exact: power-of-two scale
                            } else {
                                w[k] = (uint32_t)__float2int_rn(d0);
                            }
                        }
                        const int colg = 32 * hc + g * PER;                // first column of the chunk
                        const int box = colg * ES / 128, cb = (colg * ES % 128) / 16;
                        const uint32_t off = box * (C::ROWS * 128) + row * 128 + ((cb ^ (row & 7)) << 4);
                        *reinterpret_cast<uint4*>(stg + off) = make_uint4(w[0], w[1], w[2], w[3]);
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(acce_bar(a));
            fence_proxy_async_smem();
            named_sync(1, kTcEpiThreads);
            if (e == 0) {
#pragma unroll
                for (int b = 0; b < C::BOXES; ++b)
                    tma_store_2d(&map_out, (int)(tile * kTcCols) + b * (128 / ES), 0,
                                 sbase + C::OFF_STAGING + (uint32_t)(a * C::STAGING + b * C::ROWS * 128));
                bulk_commit();
            }
        }
        if (e == 0) bulk_wait0();
    }
    if (!ok) {
        *abort = 1;
        if (lane == 0) atomicOr(status, kStatusWaitExpired);
    }
    // the copy of A lands before the CTA may exit (it normally did long ago)
    if (tid == 0) mbar_wait_parity(a_full, 0, wait_ns);
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcTmemCols) : "memory");
    }
}

// ---- host: tensor maps through the driver entry point (no link to libcuda)

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 2-D map of a row-major [rows][n_cols] matrix, box = box_cols x box_rows, 128-byte swizzle
int make_map(CUtensorMap* map, CUtensorMapDataType dt, int es, const void* base, long long n_cols, int rows,
             int box_cols, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return set_error(RCBF_ECUDA, "decode (tcgen05): cuTensorMapEncodeTiled is not available");
    const cuuint64_t dims[2] = {(cuuint64_t)n_cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(n_cols * es)};
    const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(RCBF_ECUDA, "decode (tcgen05): cuTensorMapEncodeTiled failed");
    return RCBF_OK;
}

template <int N, int DT>
int tc_launch_job(const TcJob& job, int* status, long long wait_ns, cudaStream_t s) {
    constexpr int ES = DT == RCBF_F16 ? 2 : 4;
    decode_tc_kernel<N, DT><<<job.grid, kTcThreads, TcCfg<N, ES>::SMEM, s>>>(
        job.in_map, job.out_map, job.atc, job.hsum, job.n_cols, job.inv_n, status, wait_ns);
    return check_launch("decode_tc_kernel");
}

template <int N, int DT>
int tc_prepare(const PlanHost& h, const int16_t* rf, void* out, TcJob* job) {
    constexpr int ES = DT == RCBF_F16 ? 2 : 4;
    using C = TcCfg<N, ES>;
    const long long n_cols = (long long)h.p.n_ch * h.p.n_samples;
    if (n_cols > 2147483647LL - kTcCols)
        return set_error(RCBF_EUNSUPPORTED, "decode (tcgen05): n_ch * n_samples must stay below 2^31 (TMA coordinates)");
    // int16 samples moved as 16-bit words (TMA has no signed 16-bit type; only the bits matter)
    int rc = make_map(&job->in_map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, rf, n_cols, N, kTcCols, N);
    if (rc != RCBF_OK) return rc;
    const CUtensorMapDataType odt = DT == RCBF_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                  : DT == RCBF_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_INT32;
    if ((rc = make_map(&job->out_map, odt, ES, out, n_cols, N, 128 / ES, C::ROWS)) != RCBF_OK) return rc;
    const long long tiles = (n_cols + kTcCols - 1) / kTcCols;
    long long grid = h.n_sms > 0 ? h.n_sms : 1;
    if (grid > tiles) grid = tiles;
    if (!h.d_atc) return set_error(RCBF_EUNSUPPORTED, "decode (tcgen05): the plan holds no A operand image (order above 128)");
    job->atc = h.d_atc;
    job->hsum = h.d_hsum;
    job->n_cols = n_cols;
    job->inv_n = 1.0f / (float)h.p.n_tx;
    job->n = N;
    job->dtype = DT;
    job->grid = (unsigned)grid;
    return RCBF_OK;
}

template <int N, int DT>
int tc_launch(const PlanHost& h, const int16_t* rf, void* out, cudaStream_t s) {
    TcJob job;
    const int rc = tc_prepare<N, DT>(h, rf, out, &job);
    return rc != RCBF_OK ? rc : tc_launch_job<N, DT>(job, h.d_status, h.das.wait_ns, s);
}

template <int N, int DT>
int tc_configure() {
    constexpr int ES = DT == RCBF_F16 ? 2 : 4;
    if (cudaFuncSetAttribute(decode_tc_kernel<N, DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TcCfg<N, ES>::SMEM) != cudaSuccess)
        return check_launch("decode (tcgen05): set shared memory");
    return RCBF_OK;
}

// op: 0 configure, 1 launch, 2 prepare a job, 3 run a job
template <int DT>
int tc_dispatch(int n, int op, const PlanHost* h, const int16_t* rf, void* out, cudaStream_t s, TcJob* job,
                int* status, long long wait_ns) {
#define RCBF_TC_OPS(NN)                                                                              \
    switch (op) {                                                                                    \
        case 0: return tc_configure<NN, DT>();                                                       \
        case 1: return tc_launch<NN, DT>(*h, rf, out, s);                                            \
        case 2: return tc_prepare<NN, DT>(*h, rf, out, job);                                         \
        default: return tc_launch_job<NN, DT>(*job, status, wait_ns, s);                             \
    }
    switch (n) {
        case 32: RCBF_TC_OPS(32)
        case 64: RCBF_TC_OPS(64)
        case 128: RCBF_TC_OPS(128)
        default: return set_error(RCBF_EUNSUPPORTED, "decode (tcgen05): n_tx must be 32, 64 or 128");
    }
#undef RCBF_TC_OPS
}

int tc_by_dtype(int dtype, int n, int op, const PlanHost* h, const int16_t* rf, void* out, cudaStream_t s,
                TcJob* job, int* status, long long wait_ns) {
    switch (dtype) {
        case RCBF_I32: return tc_dispatch<RCBF_I32>(n, op, h, rf, out, s, job, status, wait_ns);
        case RCBF_F32: return tc_dispatch<RCBF_F32>(n, op, h, rf, out, s, job, status, wait_ns);
        case RCBF_F16: return tc_dispatch<RCBF_F16>(n, op, h, rf, out, s, job, status, wait_ns);
        default: return set_error(RCBF_EUNSUPPORTED, "decode (tcgen05): output dtype must be RCBF_I32, RCBF_F32 or RCBF_F16");
    }
}

}  // namespace

int launch_decode_tc(const PlanHost& h, int dtype, const int16_t* rf, void* out, cudaStream_t s) {
    return tc_by_dtype(dtype, (int)h.p.n_tx, 1, &h, rf, out, s, nullptr, nullptr, 0);
}

int configure_decode_tc(const PlanHost& h, int dtype) {
    if (!encode_fn()) return set_error(RCBF_EUNSUPPORTED, "decode (tcgen05): no tensor-map encoder in the driver");
    return tc_by_dtype(dtype, (int)h.p.n_tx, 0, &h, nullptr, nullptr, nullptr, nullptr, nullptr, 0);
}

int decode_tc_prepare(const PlanHost& h, int dtype, const int16_t* rf, void* out, TcJob* job) {
    return tc_by_dtype(dtype, (int)h.p.n_tx, 2, &h, rf, out, nullptr, job, nullptr, 0);
}

int decode_tc_run(const TcJob& job, int* status, long long wait_ns, cudaStream_t s) {
    return tc_by_dtype(job.dtype, job.n, 3, nullptr, nullptr, nullptr, s, const_cast<TcJob*>(&job), status, wait_ns);
}

}  // namespace rcbf

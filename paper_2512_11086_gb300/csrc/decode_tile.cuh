// decode_tile.cuh — shared pieces of the Hadamard decode (§THEORY
// "Synthetic Aperture Imaging"; §OPTIMIZATIONS "Decoding"): staging layout,
// PTX wrappers (cp.async, ldmatrix, prmt, int8 / FP16 mma.sync), the
// exact output conversion, and a single-tile decode used by the persistent
// batch kernel. The pipelined whole-frame kernels live in decode.cu.
#pragma once

#include "internal.cuh"

namespace rcbf {

constexpr int kRowPitch = kDecodeCols * 2 + 16;   // bytes per staged row (padding kills ldmatrix conflicts)

template <int N> struct DecodeCfg {
    static constexpr int MG = N / 32;              // warp groups along M (2 m16 tiles each)
    static constexpr int NG = 8 / MG;              // warp groups along N
    static constexpr int NT = (kDecodeCols / 8) / NG;   // n8 tiles per warp
    static constexpr int KC = N / 32;              // k32 chunks
    static constexpr int STAGES = (N >= 256) ? 2 : 3;
    static constexpr int STAGE_BYTES = N * kRowPitch;
    static constexpr int SMEM = STAGES * STAGE_BYTES;
    static constexpr int CHUNKS = N * (kDecodeCols / 8);          // 16-byte chunks per stage
    static constexpr int CHUNKS_PER_THREAD = CHUNKS / kDecodeThreads;
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(dst), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" :: "n"(K) : "memory");
}

__device__ __forceinline__ void ldsm_x4_trans(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

__device__ __forceinline__ void mma_s8s8(int (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma_s8u8(int (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int DT>
__device__ __forceinline__ void store_pair(void* out, long long idx, int d0, int d1, float inv_n) {
    if (DT == RCBF_I32) {
        *reinterpret_cast<int2*>(static_cast<int*>(out) + idx) = make_int2(d0, d1);
    } else if (DT == RCBF_F32) {
        // |d| < 2^24, so the conversion is exact and the power-of-two scale too
        *reinterpret_cast<float2*>(static_cast<float*>(out) + idx) =
            make_float2(__int2float_rn(d0) * inv_n, __int2float_rn(d1) * inv_n);
    } else {
        // one rounding of the exact value d / n
        *reinterpret_cast<__half2*>(static_cast<__half*>(out) + idx) =
            __floats2half2_rn(__int2float_rn(d0) * inv_n, __int2float_rn(d1) * inv_n);
    }
}

__device__ __forceinline__ void mma_f16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One 128-column tile of D = H^T S, staged once (no pipeline), for the
// persistent batch kernel. F16 selects the split-byte FP16 form, else the
// split-byte int8 form; both are exact. Leaves the staging buffer free.
template <int N, int DT, bool F16>
__device__ __forceinline__ void decode_one_tile(const DecodeArgs& a, long long tile, unsigned char* smem) {
    using C = DecodeCfg<N>;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int mg = warp % C::MG, ng = warp / C::MG;
    const int g = lane >> 2, t = lane & 3;
    const long long n_cols = a.n_cols;
    const uint32_t sb = smem_u32(smem);
    const long long col0 = tile * kDecodeCols;
#pragma unroll
    for (int q = 0; q < C::CHUNKS_PER_THREAD; ++q) {
        const int chunk = tid + q * kDecodeThreads;
        const int row = chunk / (kDecodeCols / 8);
        const int cc = chunk % (kDecodeCols / 8);
        const long long col = col0 + cc * 8;
        const bool valid = col < n_cols;
        const int16_t* src = a.rf + (valid ? (long long)row * n_cols + col : 0);
        cp_async16(sb + row * kRowPitch + cc * 16, src, valid);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    // A fragments are read per k chunk (L1-resident) rather than held for the
    // whole tile, so that the batch kernel keeps its registers for the DAS
    constexpr int KF = F16 ? N / 16 : N / 32;
    const uint4* fr4 = reinterpret_cast<const uint4*>(F16 ? a.afrag16 : a.afrag);
    auto frag = [&](int m, int kc, uint32_t (&r)[4]) {
        const uint4 v = __ldg(fr4 + ((mg * 2 + m) * KF + kc) * 32 + lane);
        r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
    };
    int corr[2][2] = {{0, 0}, {0, 0}};
    if (F16) {
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            corr[m][0] = a.hsum[(mg * 2 + m) * 16 + g] * 295936;
            corr[m][1] = a.hsum[(mg * 2 + m) * 16 + g + 8] * 295936;
        }
    }
#pragma unroll 1
    for (int j = 0; j < C::NT; ++j) {
        const int nt = ng * C::NT + j;
        const long long colb = col0 + nt * 8;
        if (colb >= n_cols) break;
        int d[2][4];
        if (F16) {
            float hi[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
            float lo[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll 1
            for (int kc = 0; kc < N / 32; ++kc) {
                const int krow = kc * 32 + (lane >> 3) * 8 + (lane & 7);
                uint32_t x[4];
                ldsm_x4_trans(sb + krow * kRowPitch + nt * 16, x[0], x[1], x[2], x[3]);
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
#pragma unroll
            for (int m = 0; m < 2; ++m)
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    d[m][r] = __float2int_rn(hi[m][r]) * 256 + __float2int_rn(lo[m][r]) - corr[m][r >> 1];
        } else {
            int hi[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
            int lo[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
#pragma unroll 1
            for (int kc = 0; kc < N / 32; ++kc) {
                const int krow = kc * 32 + (lane >> 3) * 8 + (lane & 7);
                uint32_t x0, x1, x2, x3;
                ldsm_x4_trans(sb + krow * kRowPitch + nt * 16, x0, x1, x2, x3);
                const uint32_t bh0 = prmt(x0, x1, 0x7531), bl0 = prmt(x0, x1, 0x6420);
                const uint32_t bh1 = prmt(x2, x3, 0x7531), bl1 = prmt(x2, x3, 0x6420);
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    uint32_t a0[4];
                    frag(m, kc, a0);
                    mma_s8s8(hi[m], a0, bh0, bh1);
                    mma_s8u8(lo[m], a0, bl0, bl1);
                }
            }
#pragma unroll
            for (int m = 0; m < 2; ++m)
#pragma unroll
                for (int r = 0; r < 4; ++r) d[m][r] = hi[m][r] * 256 + lo[m][r];
        }
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int row = (mg * 2 + m) * 16 + g;
            const long long col = colb + 2 * t;
            store_pair<DT>(a.out, (long long)row * n_cols + col, d[m][0], d[m][1], a.inv_n);
            store_pair<DT>(a.out, (long long)(row + 8) * n_cols + col, d[m][2], d[m][3], a.inv_n);
        }
    }
    __syncthreads();   // the staging buffer may be reused
}

}  // namespace rcbf

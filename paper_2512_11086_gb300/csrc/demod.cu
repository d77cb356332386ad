// demod.cu — quadrature demodulation with an integer FIR and decimation,
// Eq. (demodulation) of §OPTIMIZATIONS "Filtering & Demodulation":
//   IQ[m] = sum_k h[k] x[mD - k],  x[n] = s[n] e^{-j pi n / 2}   (f_s = 4 f_d)
// then a right shift with rounding (ties to even) and saturation to int16.
//
// The mixer is 1, -j, -1, j for n mod 4 = 0..3, so a mixed sample is real
// for even n and imaginary for odd n: with e[n] = s[n] * (+1, -1, -1, +1)[n mod 4]
// the I output sums the taps k with n - k even and the Q output the others.
// A CTA stages the sign-mixed samples of one trace segment in shared memory
// (kDemodOut outputs need kDemodOut * D + N_f samples, loaded and converted
// once, zero outside the record: the paper's LDS reuse) and every thread
// computes four outputs, sharing each tap load between them. Accumulation is
// exact in 32 bits (sum |h| <= 65535 is checked at plan time).
#include "internal.cuh"

namespace rcbf {

namespace {

constexpr int kDemodThreads = 256;
constexpr int kDemodPer = 4;                                  // outputs per thread
constexpr int kDemodOut = kDemodThreads * kDemodPer;          // outputs per CTA

__device__ __forceinline__ int16_t round_shift_sat(int acc, int shift) {
    int q = acc;
    if (shift > 0) {
        q = acc >> shift;                                      // floor (arithmetic shift)
        const int rem = acc - (q << shift);                    // 0 <= rem < 2^shift
        const int half = 1 << (shift - 1);
        if (rem > half || (rem == half && (q & 1))) q += 1;
    }
    return (int16_t)max(-32768, min(32767, q));
}

// grid: (traces, segments of kDemodOut outputs)
__global__ void __launch_bounds__(kDemodThreads)
demod_kernel(const int16_t* __restrict__ rf, int16_t* __restrict__ iq, const int16_t* __restrict__ taps,
             int n_taps, int shift, int D, long long n_in, long long n_out, long long n_traces) {
    extern __shared__ int sm[];
    const int n_taps2 = (n_taps + 1) & ~1;                     // even, zero-padded
    int* h = sm;                                               // [n_taps2]
    int* e = sm + n_taps2;                                     // sign-mixed samples
    const long long tr = blockIdx.x;
    const long long m0 = (long long)blockIdx.y * kDemodOut;
    const long long base = m0 * D - (n_taps2 - 1);             // input index of e[0]
    const int L = (kDemodOut - 1) * D + n_taps2;
    const int16_t* x = rf + tr * n_in;
    for (int k = threadIdx.x; k < n_taps2; k += kDemodThreads) h[k] = k < n_taps ? (int)taps[k] : 0;
    for (int p = threadIdx.x; p < L; p += kDemodThreads) {
        const long long n = base + p;
        int v = 0;
        if (n >= 0 && n < n_in) {
            v = (int)x[n];
            const int r = (int)(n & 3);
            if (r == 1 || r == 2) v = -v;
        }
        e[p] = v;
    }
    __syncthreads();
    // output m = m0 + t + 256 r reads e at (m - m0) D + (n_taps2 - 1) - k
    int acc_even[kDemodPer], acc_odd[kDemodPer];
    int pos[kDemodPer];
#pragma unroll
    for (int r = 0; r < kDemodPer; ++r) {
        acc_even[r] = 0;
        acc_odd[r] = 0;
        pos[r] = (threadIdx.x + kDemodThreads * r) * D + (n_taps2 - 1);
    }
    for (int k = 0; k < n_taps2; k += 2) {
        const int h0 = h[k], h1 = h[k + 1];
#pragma unroll
        for (int r = 0; r < kDemodPer; ++r) {
            acc_even[r] += h0 * e[pos[r] - k];          // n - k with k even
            acc_odd[r] += h1 * e[pos[r] - k - 1];       // k odd
        }
    }
#pragma unroll
    for (int r = 0; r < kDemodPer; ++r) {
        const long long m = m0 + threadIdx.x + kDemodThreads * r;
        if (m >= n_out) continue;
        // n = m D: even n takes I from the even taps, odd n from the odd ones
        const bool even = ((m * D) & 1) == 0;
        const int ai = even ? acc_even[r] : acc_odd[r];
        const int aq = even ? acc_odd[r] : acc_even[r];
        iq[tr * n_out + m] = round_shift_sat(ai, shift);
        iq[(n_traces + tr) * n_out + m] = round_shift_sat(aq, shift);
    }
}

}  // namespace

int launch_demodulate(const PlanHost& h, const int16_t* rf, int16_t* iq, cudaStream_t s) {
    const int D = (int)h.p.demod_decimation, n_taps = (int)h.p.demod_n_taps;
    const long long n_out = h.p.n_samples, n_in = n_out * D;
    const long long n_traces = (long long)h.p.n_tx * h.p.n_ch;
    const int n_taps2 = (n_taps + 1) & ~1;
    const size_t smem = (size_t)(n_taps2 + (kDemodOut - 1) * D + n_taps2) * sizeof(int);
    if (cudaFuncSetAttribute(demod_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return check_launch("demodulate: set shared memory");
    dim3 grid((unsigned)n_traces, (unsigned)((n_out + kDemodOut - 1) / kDemodOut));
    demod_kernel<<<grid, kDemodThreads, smem, s>>>(rf, iq, h.d_taps, n_taps, (int)h.p.demod_shift, D, n_in,
                                                    n_out, n_traces);
    return check_launch("demod_kernel");
}

}  // namespace rcbf

// demod.cu — quadrature demodulation with an integer FIR and decimation,
// Eq. (demodulation) of §OPTIMIZATIONS "Filtering & Demodulation":
//   IQ[m] = sum_k h[k] x[mD - k],  x[n] = s[n] e^{-j pi n / 2}   (f_s = 4 f_d)
// then a right shift with rounding (ties to even) and saturation to int16.
//
// The mixer is 1, -j, -1, j for n mod 4 = 0..3, so a mixed sample is real
// for even n and imaginary for odd n: with e[n] = s[n] * (+1, -1, -1, +1)[n mod 4]
// the I output sums the taps k with n - k even and the Q output the others.
// A CTA stages the sign-mixed samples of one trace segment in shared memory
// (kDemodOut outputs need about kDemodOut * D + N_f samples, loaded and
// converted once, zero outside the record: the paper's LDS reuse) and every
// thread computes four outputs, sharing each tap load between them.
// Complex taps h + j hq (a matched filter with a phase correction) add the
// sums of hq. Accumulation is exact in 32 bits (sum |h| + sum |hq| <= 65535 is
// checked at plan time).
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

// Shared layout (polyphase): the staged samples e[p] (p from the segment's
// first needed input) are stored as D rows, e_ph[p mod D][p / D], so that for
// a tap k = a D + b the 32 threads of a warp (consecutive outputs, inputs D
// apart) read consecutive words of one row: no bank conflicts.
// grid: (traces, segments of kDemodOut outputs)
template <bool CPLX>
__global__ void __launch_bounds__(kDemodThreads)
demod_kernel(const int16_t* __restrict__ rf, int16_t* __restrict__ iq, const int16_t* __restrict__ taps,
             const int16_t* __restrict__ taps_im, int n_taps, int shift, int D, int Q, long long n_in,
             long long n_out, long long n_traces) {
    extern __shared__ int sm[];
    const int n_taps2 = (n_taps + 1) & ~1;                     // even, zero-padded
    const int PD = (n_taps2 - 1 + D - 1) / D;                  // rows of history before the first output
    int* h = sm;                                               // [n_taps2] real parts
    int* hq = sm + n_taps2;                                    // [n_taps2] imaginary parts (complex taps)
    int* e_ph = sm + (CPLX ? 2 : 1) * n_taps2;                 // [D][Q]
    const long long tr = blockIdx.x;
    const long long m0 = (long long)blockIdx.y * kDemodOut;
    const long long base = (m0 - PD) * D;                      // input index of e[0]
    const int L = (kDemodOut + PD) * D;                        // staged samples, D * (rows used)
    const int16_t* x = rf + tr * n_in;
    for (int k = threadIdx.x; k < n_taps2; k += kDemodThreads) {
        h[k] = k < n_taps ? (int)taps[k] : 0;
        if (CPLX) hq[k] = k < n_taps ? (int)taps_im[k] : 0;
    }
    for (int p = threadIdx.x; p < L; p += kDemodThreads) {
        const long long n = base + p;
        int v = 0;
        if (n >= 0 && n < n_in) {
            v = (int)x[n];
            const int r = (int)(n & 3);
            if (r == 1 || r == 2) v = -v;                      // mixer 1, -j, -1, j: real / imaginary sign
        }
        e_ph[(p % D) * Q + p / D] = v;
    }
    __syncthreads();
    // output m (local index mi = m - m0) and tap k = a D + b read
    // e[(mi + PD) D - k] = e_ph[b ? D - b : 0][mi + PD - a - (b ? 1 : 0)]
    // sums over the even and the odd taps k, of the real parts h and (complex
    // taps) of the imaginary parts hq
    int acc_even[kDemodPer], acc_odd[kDemodPer], accq_even[kDemodPer], accq_odd[kDemodPer];
#pragma unroll
    for (int r = 0; r < kDemodPer; ++r) acc_even[r] = acc_odd[r] = accq_even[r] = accq_odd[r] = 0;
    const int astep = (D & 1) ? 2 : 1;                         // odd D: the parity of k alternates with a
    for (int b = 0; b < D; ++b) {
        const int* row = e_ph + (b ? D - b : 0) * Q + PD - (b ? 1 : 0) + threadIdx.x;
        for (int a0 = 0; a0 < astep; ++a0) {
            int acc[kDemodPer], accq[kDemodPer];
#pragma unroll
            for (int r = 0; r < kDemodPer; ++r) acc[r] = accq[r] = 0;
            for (int a = a0; a * D + b < n_taps2; a += astep) {
                const int hk = h[a * D + b];
                const int hqk = CPLX ? hq[a * D + b] : 0;
#pragma unroll
                for (int r = 0; r < kDemodPer; ++r) {
                    const int e = row[kDemodThreads * r - a];
                    acc[r] += hk * e;
                    if (CPLX) accq[r] += hqk * e;
                }
            }
            const bool odd = ((a0 * D + b) & 1) != 0;         // parity of every k of this loop
#pragma unroll
            for (int r = 0; r < kDemodPer; ++r) {
                acc_even[r] += odd ? 0 : acc[r];
                acc_odd[r] += odd ? acc[r] : 0;
                if (CPLX) {
                    accq_even[r] += odd ? 0 : accq[r];
                    accq_odd[r] += odd ? accq[r] : 0;
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < kDemodPer; ++r) {
        const long long m = m0 + threadIdx.x + kDemodThreads * r;
        if (m >= n_out) continue;
        // n = m D: a mixed sample n - k is real (re) for n - k even, imaginary
        // (im) for odd; (h + j hq)(re + j im): I = sum h re - sum hq im,
        // Q = sum h im + sum hq re
        const bool even = ((m * D) & 1) == 0;
        const int re_h = even ? acc_even[r] : acc_odd[r], im_h = even ? acc_odd[r] : acc_even[r];
        const int re_q = even ? accq_even[r] : accq_odd[r], im_q = even ? accq_odd[r] : accq_even[r];
        const int ai = CPLX ? re_h - im_q : re_h;
        const int aq = CPLX ? im_h + re_q : im_h;
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
    const int PD = (n_taps2 - 1 + D - 1) / D;
    const int Q = (kDemodOut + PD) | 1;          // row length (odd: rows start in different banks)
    const bool cplx = h.d_taps_im != nullptr;
    const size_t smem = (size_t)((cplx ? 2 : 1) * n_taps2 + D * Q) * sizeof(int);
    auto k = cplx ? demod_kernel<true> : demod_kernel<false>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return check_launch("demodulate: set shared memory");
    dim3 grid((unsigned)n_traces, (unsigned)((n_out + kDemodOut - 1) / kDemodOut));
    k<<<grid, kDemodThreads, smem, s>>>(rf, iq, h.d_taps, h.d_taps_im, n_taps, (int)h.p.demod_shift, D, Q, n_in,
                                        n_out, n_traces);
    return check_launch("demod_kernel");
}

}  // namespace rcbf

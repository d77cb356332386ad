/*
 * rcbf.h — C ABI of the GB300 row-column / TOBE beamformer hot path.
 *
 * The library implements the data-parallel core of the realtime beamformer of
 * Palamar et al., "An Open Source Realtime GPU Beamformer for Row-Column and
 * TOBE Arrays" (arXiv 2512.11086):
 *
 *   decode   Hadamard aperture decode of FORCES / HERCULES acquisitions
 *            (§THEORY "Synthetic Aperture Imaging"; §OPTIMIZATIONS "Decoding"):
 *            a matrix product across the transmit axis.
 *   das      synthetic-aperture delay-and-sum, Eq. (1), with the constant-F#
 *            receive apodization of Eq. (2) and the Hanning window of Eq. (3)
 *            (§OPTIMIZATIONS "DAS").
 *   backward the adjoint of das with respect to the RF samples, the speed of
 *            sound and the per-channel apodization weights (Eq. (1)
 *            differentiated; the paper has no adjoint, it serves
 *            speed-of-sound autofocus).
 *   batch    many frames of uneven size in one persistent launch
 *            (§METHODS "Data Processing": several pre-uploaded parameter sets).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * Layouts. Encoded RF is int16 [n_tx][n_ch][n_samples], samples fastest
 *    (n_tx = acquisitions = Hadamard order). Decoded RF has the same shape;
 *    row i is the decoded transmit element i. A complex decoded RF (RCBF_CF32)
 *    is two planes [2][n_tx][n_ch][n_samples] (real, then imaginary).
 *    Images are float32 [nz][ny][nx], x fastest; a complex image is two such
 *    planes (real, then imaginary).
 *  * Memory. Every data pointer passed to decode / das / backward / batch is
 *    a DEVICE pointer owned by the caller; the library never frees it. It must
 *    be 16-byte aligned. A plan owns the device tables it creates in
 *    rcbf_plan (decode matrix fragments) and frees them in rcbf_destroy.
 *  * Streams. `stream` is a cudaStream_t passed as void* (NULL = legacy
 *    default stream). Work is enqueued asynchronously; no entry point except
 *    rcbf_plan, rcbf_batch_create and rcbf_batch_status synchronises the host.
 *  * Errors. Every int-returning entry point returns 0 on success or a
 *    negative RCBF_E* code. Arguments are validated on the host before any
 *    launch; on error nothing is enqueued. rcbf_last_error() returns a
 *    thread-local, human-readable message for the last failure on the calling
 *    thread.
 *  * Geometry. All lengths in metres, times in seconds, rates in Hz. The array
 *    frame has z along the array normal and its origin at the centre of the
 *    array: transmit element i (a line element) sits at lateral coordinate
 *    (i - (n_tx-1)/2) * tx_pitch, receive element j at
 *    (j - (n_ch-1)/2) * rx_pitch, both at z = 0. A row element spans x, so
 *    its lateral coordinate is y; a column element spans y, so its lateral
 *    coordinate is x. The paper's corner-element origin is one translation
 *    away, expressible through xdc_transform.
 *  * Delays. For a voxel at array-frame position q and line elements with
 *    lateral coordinates e_i (transmit) and e_j (receive):
 *        d_tx = sqrt((lat_tx(q) - e_i)^2 + q_z^2)
 *        d_rx = sqrt((lat_rx(q) - e_j)^2 + q_z^2)
 *        s_ij = ((d_tx + d_rx) / c - t0) * fs          (fractional sample)
 *    and DAS reads the decoded trace r_ij at s_ij by linear interpolation or
 *    by the 4-point cubic Hermite spline (§THEORY "Interpolation &
 *    Sampling"), with r_ij[n] = 0 for n outside [0, n_samples-1].
 *  * Cubic Hermite reading. On [n, n+1] (n = floor(s), f = s - n) the cubic
 *    with values r[n], r[n+1] and slopes m_k = (r[k+1] - r[k-1]) / 2 at both
 *    ends: the paper names the Hermite basis and 4 points but not the
 *    tangents; central differences are the 4-point choice.
 */
#ifndef RCBF_H
#define RCBF_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define RCBF_OK             0
#define RCBF_EINVAL        -1  /* bad argument: NULL, zero size, misaligned, inconsistent */
#define RCBF_EUNSUPPORTED  -2  /* dtype / mode / size combination not built */
#define RCBF_ECUDA         -3  /* CUDA runtime or launch error (message in rcbf_last_error) */
#define RCBF_ENOMEM        -4  /* device allocation failed */
#define RCBF_ETIMEOUT      -5  /* a bounded device-side wait expired (rcbf_plan_status, rcbf_batch_status,
                                  rcbf_pipeline_wait, rcbf_das_noalloc_status) */

/* ---- enumerations -------------------------------------------------------- */
enum rcbf_dtype {
    RCBF_I16  = 0,   /* int16 (encoded RF only) */
    RCBF_I32  = 1,   /* int32: exact decode sum H^T S, unscaled */
    RCBF_F32  = 2,   /* float32: (H^T S) / N, exact for N a power of two */
    RCBF_F16  = 3,   /* float16: (H^T S) / N rounded once to nearest-even */
    RCBF_CF32 = 4    /* complex float32 as two planes (DAS input only) */
};

enum rcbf_acq_kind {
    RCBF_FORCES      = 0,  /* Hadamard-encoded transmit aperture */
    RCBF_HERCULES    = 1,  /* Hadamard-encoded receive rows; same separable delays */
    RCBF_HERCULES_2D = 2   /* decoded rows x columns as a 2D receive aperture for one transmit wave
                              (tx_wave RCBF_TX_PLANE with tx_angles[0], or RCBF_TX_POINT): index i is
                              the receive row at lateral e_i (tx_orientation's axis), j the column;
                              d_rx = sqrt((lat_rx - e_j)^2 + (lat_tx - e_i)^2 + z^2), not separable;
                              the F# window uses the radial lateral distance. Tiled DAS form with
                              windows from the tile's bounding box (one voxel per thread along u,
                              tile 32 x bv x bw) when f_number == 0, the tile reaches at most 128
                              samples and rows and columns lie along different axes; otherwise
                              the plain form. */
};

enum rcbf_orientation {
    RCBF_ROWS    = 0,   /* line elements span x: lateral coordinate is y */
    RCBF_COLUMNS = 1    /* line elements span y: lateral coordinate is x */
};

enum rcbf_tx_wave {
    RCBF_TX_LINE  = 0,  /* line element i: d_tx = sqrt((lat_tx - e_i)^2 + z^2) */
    RCBF_TX_PLANE = 1,  /* plane wave i: d_tx = z cos(a_i) + lat_tx sin(a_i) (crosses the array at t = 0) */
    RCBF_TX_VLS   = 2,  /* virtual line source above line i at depth f:
                           d_tx = f + sgn(z - f) sqrt((lat_tx - e_i)^2 + (z - f)^2), sgn(0) = +1.
                           Off axis the delay jumps at z = f: the voxel tiles whose depth
                           range reaches f run the plain DAS form, all others the tiled one
                           (rcbf_das_backward runs the plain form for such an image). */
    RCBF_TX_POINT = 3   /* RCBF_HERCULES_2D only: diverging wave from a virtual point at depth f < 0 on the
                           array axis: d_tx = sqrt(x^2 + y^2 + (z - f)^2) + f */
};

enum rcbf_interp {
    RCBF_LINEAR = 0,    /* (1 - f) r[n] + f r[n+1] */
    RCBF_CUBIC  = 1     /* 4-point cubic Hermite spline, central-difference slopes (rcbf_das only) */
};

enum rcbf_decode_variant {
    RCBF_DECODE_MMA_I8  = 0,  /* split-byte int8 tensor-core GEMM (mma.sync s8/u8), exact */
    RCBF_DECODE_PLAIN   = 1,  /* plain CUDA-core form: one thread per output, int32 sums */
    RCBF_DECODE_MMA_F16 = 2,  /* split-byte FP16 tensor-core GEMM (bytes and +-1 exact in
                                 FP16, FP32 accumulation exact below 2^24), exact */
    RCBF_DECODE_TC      = 3   /* the split-byte FP16 GEMM on the 5th-generation tensor cores:
                                 tcgen05.mma with accumulators in tensor memory, TMA tensor
                                 loads of the int16 tiles and TMA stores of the output; exact;
                                 n_tx in {32, 64, 128}. In a batch such a frame is decoded by its
                                 own tcgen05 launch ahead of the persistent launch. */
};

enum rcbf_das_variant {
    RCBF_DAS_TILED = 0,  /* voxel tiles, per-tile FP64 reference delays, shared-memory windows */
    RCBF_DAS_PLAIN = 1   /* plain FP32 form: one thread per voxel, FP32 delays, global loads */
};

/* ---- parameter block ------------------------------------------------------
 * Caller-owned; rcbf_plan copies it. Zero-initialise and fill what you use:
 * an all-zero xdc_transform / voxel_transform means "not given". */
typedef struct rcbf_params {
    uint32_t n_tx;            /* decoded transmits (rows of RF) */
    uint32_t n_ch;            /* receive channels */
    uint32_t n_samples;       /* samples per (transmit, channel) trace */
    uint32_t hadamard_order;  /* 0: RF is not encoded (decode unavailable); else == n_tx */
    uint32_t acq_kind;        /* enum rcbf_acq_kind (FORCES and HERCULES share separable delays) */
    uint32_t tx_orientation;  /* enum rcbf_orientation of the transmit line elements */
    uint32_t rx_orientation;  /* enum rcbf_orientation of the receive line elements */
    uint32_t decoded_dtype;   /* enum rcbf_dtype: decode output and DAS input
                                 (RCBF_I32, RCBF_F32, RCBF_F16, RCBF_CF32) */
    uint32_t interp;          /* enum rcbf_interp */
    uint32_t decode_variant;  /* enum rcbf_decode_variant */
    uint32_t das_variant;     /* enum rcbf_das_variant */
    uint32_t out_dims[3];     /* nx, ny, nz (>= 1 each) */
    uint32_t tile[3];         /* DAS voxel tile (bu, bv, bw); all 0 = choose automatically.
                                 bu (32, 64 or 128) runs along the image axis parallel to the
                                 transmit line elements (x for rows, y for columns), bv along
                                 the other lateral image axis, bw along z; bu*bv*bw = 1024. */
    uint32_t reserved;
    double   fs;              /* sampling rate [Hz] */
    double   c;               /* speed of sound [m/s] (DAS may override per call) */
    double   t0;              /* time of sample 0 relative to emission [s] */
    double   fc;              /* centre frequency [Hz] (informational) */
    double   tx_pitch;        /* transmit element pitch [m] */
    double   rx_pitch;        /* receive element pitch [m] */
    double   xdc_transform[16]; /* row-major 4x4 affine, world -> array frame; zeros = identity */
    double   out_min[3];      /* world position of voxel (0,0,0) [m] */
    double   out_max[3];      /* world position of voxel (nx-1,ny-1,nz-1) [m] (inclusive linspace) */
    double   voxel_transform[16]; /* row-major 4x4 affine, voxel index -> world; zeros = use out_min/out_max */
    double   f_number;        /* F# of Eq. (2); 0 disables the window (all weights 1) */
    const int8_t* decode_matrix; /* optional HOST pointer to an n_tx x n_tx +-1 matrix H,
                                    row-major H[k][i] (k = acquisition, i = decoded element),
                                    copied by rcbf_plan; NULL = Sylvester H[k][i] = (-1)^popcount(k&i) */
    /* Quadrature demodulation ahead of the decode (rcbf_demodulate, §OPTIMIZATIONS
     * "Filtering & Demodulation"). 0 = none. With D = demod_decimation >= 1 the raw RF
     * has n_samples * D samples per trace, sampled at 4 f_d; n_samples, fs and t0
     * describe the demodulated data (fs = raw rate / D). A Hadamard-encoded plan with
     * demodulation decodes the two int16 planes into RCBF_CF32. */
    uint32_t demod_decimation;  /* D in [1, 16], or 0 */
    uint32_t demod_n_taps;      /* FIR length, 1..1024 */
    int32_t  demod_shift;       /* right shift (rounding ties to even) back to int16, 0..30 */
    uint32_t reserved2;
    const int16_t* demod_taps;  /* HOST pointer to the int16 taps h[0..n_taps-1], copied by rcbf_plan;
                                   sum |h| <= 65535 (exact 32-bit accumulation) */
    double   iq_freq;           /* > 0: the decoded data is baseband IQ demodulated at this frequency
                                   (RCBF_CF32 only): rcbf_das multiplies each interpolated sample by
                                   e^{j 2 pi (iq_freq / fs) s} (IQ beamforming). 0 = RF data. */
    /* Transmit wave of each transmit index (§CAPABILITIES: FORCES / TPW / VLS row-column
     * methods); every one keeps the delay separable (it depends on lat_tx and z only). */
    uint32_t tx_wave;           /* enum rcbf_tx_wave */
    uint32_t reserved3;
    double   tx_focus;          /* RCBF_TX_VLS: depth f of the virtual line sources [m] */
    const double* tx_angles;    /* RCBF_TX_PLANE: HOST pointer to n_tx steering angles [rad], |angle| < pi/2,
                                   copied by rcbf_plan */
    /* Receive channels as a slice of a larger array (a channel-sharded frame: Eq. (1) is a
     * sum over channels, so each GPU beamforms its slice and one reduce-sum adds the
     * partial images):
     * channel j of this plan is element rx_channel_offset + j of rx_channels_total.
     * 0 / 0 = the plan's channels are the whole array. */
    uint32_t rx_channel_offset;
    uint32_t rx_channels_total;
    /* Imaginary parts of complex demodulation taps h = demod_taps + j demod_taps_imag (a
     * baseband matched filter that also applies a phase correction, §OPTIMIZATIONS
     * "Filtering & Demodulation"): HOST pointer to demod_n_taps int16 values, copied by
     * rcbf_plan; NULL = real taps. With complex taps sum |h_re| + sum |h_im| <= 65535. */
    const int16_t* demod_taps_imag;
} rcbf_params;

typedef struct rcbf_plan_s*  rcbf_plan_t;
typedef struct rcbf_batch_s* rcbf_batch_t;
typedef struct rcbf_pipeline_s* rcbf_pipeline_t;

/* rcbf_plan — validate `params`, copy it, build the device decode tables and
 * pick the DAS tile. Allocates a few KB of device memory on the current
 * device; synchronises once. Decode requires hadamard_order == n_tx with
 * n_tx a multiple of 32 in [32, 256] (any +-1 matrix if decode_matrix is
 * given, else n_tx a power of two). Errors: RCBF_EINVAL (NULL, zero sizes,
 * non-power-of-two order without a matrix, entries not +-1, tile product),
 * RCBF_EUNSUPPORTED (dtype / variant), RCBF_ENOMEM, RCBF_ECUDA.
 * Passage: §METHODS "Data Processing" (data description, array geometry,
 * image region and resolution) and Fig. "das_dispatch" (voxel-index affine). */
int rcbf_plan(const rcbf_params* params, rcbf_plan_t* out_plan);

/* What a plan chose, for callers that size, schedule or count work. */
typedef struct rcbf_plan_info {
    uint32_t tile[3];          /* DAS voxel tile (bu, bv, bw) */
    uint32_t tiled;            /* 1 if rcbf_das runs the tiled form at params.c, 0 if the plain form */
    uint32_t window;           /* samples per (transmit, channel) window of a tile at params.c */
    uint32_t n_split;          /* channels of a tile split over this many work units (1 = none); the
                                  units of the grid's last 3/4 wave run in up to four channel parts */
    uint32_t das_launches;     /* kernels one rcbf_das call enqueues at params.c */
    uint32_t decode_launches;  /* kernels one rcbf_decode call enqueues (0 without Hadamard order) */
    uint64_t workspace_bytes;  /* device memory the plan owns */
    uint32_t bwd_tile[3];      /* voxel tile rcbf_das_backward uses at params.c */
    uint32_t bwd_mode;         /* rcbf_das_backward at params.c: 0 plain form, 1 tiled with lanes along the
                                  tile's u axis, 2 tiled with lanes over z (tile 32 x bv x bw, bv * bw = 32) */
} rcbf_plan_info;

/* rcbf_plan_query — describe a plan (host only, no CUDA call).
 * Errors: RCBF_EINVAL (NULL plan or info). */
int rcbf_plan_query(rcbf_plan_t plan, rcbf_plan_info* info);

/* rcbf_destroy — free the plan's device tables. NULL is accepted. Must not be
 * called while work using the plan is still pending on a stream. */
void rcbf_destroy(rcbf_plan_t plan);

/* rcbf_demodulate — Eq. (demodulation), IQ[n] = LPF{s[n] e^{-j 2 pi f_d n / f_s}}
 * (§OPTIMIZATIONS "Filtering & Demodulation"), at quadrature sampling f_s = 4 f_d,
 * where the mixer e^{-j pi n / 2} is 1, -j, -1, j for n mod 4 = 0..3. The LPF is
 * the causal FIR y[n] = sum_k h[k] x[n - k] with the plan's int16 taps (x = 0
 * outside the record), evaluated at n = m D (decimation); each component is
 * shifted right by demod_shift with rounding ties to even and saturated to
 * int16. Exact integer arithmetic, so the result is reproducible bit for bit.
 *   rf  device int16 [n_tx][n_ch][n_samples * D] (raw traces, any encoding)
 *   iq  device int16 [2][n_tx][n_ch][n_samples]: I plane, then Q plane
 * Errors: RCBF_EINVAL (NULL, misaligned, plan without demodulation), RCBF_ECUDA. */
int rcbf_demodulate(rcbf_plan_t plan, const int16_t* rf, int16_t* iq, void* stream);

/* rcbf_demod_decode — rcbf_demodulate followed by rcbf_decode in one kernel,
 * the demodulation fused into the decode's load (§OPTIMIZATIONS "Filtering &
 * Demodulation": the raw samples are filtered and decimated from shared
 * memory before anything else; Eq. (demodulation); §OPTIMIZATIONS
 * "Decoding"). Per channel and block of 64 demodulated samples, the raw
 * window of every acquisition is staged once in shared memory, the FIR with
 * the quadrature mixer (real or complex taps) gives the int16 I and Q samples
 * with the same rounding and saturation as rcbf_demodulate, and the exact
 * split-byte tensor-core decode turns them into both decoded planes; the
 * demodulated planes never reach device memory. The result equals
 * rcbf_demodulate then rcbf_decode bit for bit.
 *   rf       device int16 [n_tx][n_ch][n_samples * D] (raw, Hadamard-encoded)
 *   decoded  device float32 [2][n_tx][n_ch][n_samples]: D / N of the I plane,
 *            then of the Q plane (RCBF_CF32)
 * Needs a plan with demodulation, a Hadamard order, decoded_dtype RCBF_CF32,
 * D = demod_decimation 4 or 8, n_tx in {32, 64, 128} and a raw window
 * (64 D + 32 ceil(ceil(n_taps / 4) / 8) samples per acquisition) that fits
 * shared memory. Errors: RCBF_EINVAL (NULL, misaligned), RCBF_EUNSUPPORTED
 * (plan or sizes outside that set), RCBF_ECUDA. */
int rcbf_demod_decode(rcbf_plan_t plan, const int16_t* rf, float* decoded, void* stream);

/* rcbf_decode — D = H^T S over the transmit axis (§THEORY "Synthetic Aperture
 * Imaging": decoded data behaves as one transmit per element; §OPTIMIZATIONS
 * "Decoding": a matrix product across transmits).
 *   rf       device int16 [n_tx][n_ch][n_samples] (encoded acquisitions k), or
 *            with demodulation the two int16 planes [2][n_tx][n_ch][n_samples]
 *            that rcbf_demodulate writes (decoded as RCBF_CF32: each plane D / N)
 *   decoded  device [n_tx][n_ch][n_samples] of params.decoded_dtype:
 *            RCBF_I32 = D exactly; RCBF_F32 = D / N exactly (|D| < 2^24 always
 *            holds for int16 input and N <= 256); RCBF_F16 = D / N rounded once.
 * Exact for every int16 input (integer arithmetic throughout).
 * n_samples must be a multiple of 8. The RCBF_DECODE_TC form's waits are
 * bounded like the tiled DAS's (rcbf_plan_set_wait) and an expiry is reported
 * by rcbf_plan_status. Errors: RCBF_EINVAL (NULL, misaligned, plan without
 * Hadamard order), RCBF_EUNSUPPORTED (CF32 output), RCBF_ECUDA. */
int rcbf_decode(rcbf_plan_t plan, const int16_t* rf, void* decoded, void* stream);

/* rcbf_das — delay-and-sum of Eq. (1) with a_tx = 1 and receive apodization
 *   a_j(v) = w_j * W(F# * |lat_rx(v) - e_j| / |z(v)|)   (Eq. (2), Eq. (3), W(u)=cos^2(pi u) for |u|<0.5)
 * (a_j = w_j when f_number == 0):
 *   image(v) = sum_i sum_j a_j(v) * lerp(r_ij, s_ij(v)).
 *   decoded  device decoded RF of params.decoded_dtype (RCBF_I32 data is
 *            scaled by 1/n_tx; RCBF_CF32 gives a complex image)
 *   apod     device float32 [n_ch] per-channel weights w_j, or NULL (all 1)
 *   c        speed of sound for this call; <= 0 uses params.c
 *   image    device float32 [nz][ny][nx] (x2 planes for RCBF_CF32), overwritten
 * IQ beamforming (params.iq_freq > 0, RCBF_CF32): the interpolated baseband
 * sample is multiplied by e^{j 2 pi (iq_freq / fs) s} before the sum, which
 * restores the carrier that the index-based demodulation mixer removed.
 * Accumulation is FP32. The tiled form (params.das_variant = RCBF_DAS_TILED)
 * needs n_tx % 8 == 0 (4 for complex), n_ch % 8 == 0, an image axis parallel
 * to the transmit line elements, and voxel tiles that reach at most 128
 * samples of a trace (any grid finer than about a quarter of the pulse
 * length); a grid too coarse for that runs the plain form instead. With
 * f_number > 0 the tiled form skips, per voxel tile, every chunk of 8
 * channels whose window W is zero at all of the tile's voxels (the test of
 * Eq. (2)-(3) on the tile's bounding box; the result is unchanged).
 * Status: the tiled form's waits on its staged windows are bounded (one second
 * by default, see rcbf_plan_set_wait); a wait that expires stops its voxel
 * tile, leaving that part of the image unwritten, and records the expiry in
 * the plan's status word, which rcbf_plan_status reads and clears.
 * Errors: RCBF_EINVAL, RCBF_EUNSUPPORTED, RCBF_ECUDA. */
int rcbf_das(rcbf_plan_t plan, const void* decoded, const float* apod, float c,
             float* image, void* stream);

/* rcbf_das_backward — adjoint of rcbf_das (Eq. (1) differentiated) for an
 * upstream gradient G = dL/dimage:
 *   grad_rf[i][j][n]  = sum_v a_j(v) G(v) * lerp-weight of sample n at s_ij(v)
 *   grad_c            = sum_v sum_ij a_j(v) G(v) * (r_ij[n+1]-r_ij[n]) * ds_ij/dc,
 *                       ds_ij/dc = -(d_tx + d_rx) * fs / c^2
 *   grad_apod[j]      = sum_v sum_i (a_j(v)/w_j) G(v) * lerp(r_ij, s_ij(v))
 * (complex data: the real and imaginary planes contribute independently).
 *   decoded    device RF as for rcbf_das (RCBF_F32 or RCBF_CF32 only)
 *   grad_image device float32 image-shaped (x2 planes for complex)
 *   grad_rf    device float32 RF-shaped, overwritten; NULL = not computed
 *   grad_c     device float32 scalar, overwritten; NULL = not computed
 *   grad_apod  device float32 [n_ch], overwritten; NULL = not computed
 * Delays are recomputed per voxel tile, never stored. The tiled form sums a
 * tile's terms per (transmit, channel) window in 32-bit fixed point (scale
 * 2^e chosen so a window cannot overflow; a term is rounded to about 2e-6 of
 * max|w| max|G|) and adds windows into grad_rf, grad_c and grad_apod with
 * float atomics, so the order of those sums (and their last bits) varies
 * between runs. A 16-byte aligned grad_rf takes four-float reductions; any
 * 4-byte aligned one is accepted. rcbf_plan_query reports the tile used.
 * Built for RF data with linear interpolation: IQ or cubic plans return
 * RCBF_EUNSUPPORTED. Bounded waits and the status word as for rcbf_das: an
 * expired wait leaves the gradients incomplete and the next rcbf_plan_status
 * returns RCBF_ETIMEOUT.
 * Errors: RCBF_EINVAL, RCBF_EUNSUPPORTED (dtype), RCBF_ECUDA. */
int rcbf_das_backward(rcbf_plan_t plan, const void* decoded, const float* apod, float c,
                      const float* grad_image, float* grad_rf, float* grad_c,
                      float* grad_apod, void* stream);

/* rcbf_plan_status — synchronise `stream` and return the plan's status word:
 * RCBF_OK, or RCBF_ETIMEOUT when a bounded device-side wait of one of the
 * plan's kernels (tiled rcbf_das, rcbf_das_backward, the RCBF_DECODE_TC
 * decode) expired since the previous rcbf_plan_status call; the output of that
 * call is then incomplete. Reading clears the word (a synchronous 4-byte
 * memset when it was set), so each expiry is reported once. The word is
 * shared by all calls on the plan, whichever stream they use.
 * Errors: RCBF_EINVAL (NULL plan), RCBF_ECUDA. */
int rcbf_plan_status(rcbf_plan_t plan, void* stream);

/* rcbf_plan_set_wait — bound of every device-side wait of the plan's tiled
 * DAS, adjoint and RCBF_DECODE_TC kernels (default one second; at most ten),
 * and a test hook
 * for failure detection: withhold = 1 makes every voxel tile of the tiled
 * rcbf_das omit the request of its first window copy, so that the tile's
 * first wait runs out, the kernel stops that tile and returns, and
 * rcbf_plan_status reports RCBF_ETIMEOUT while the context stays usable;
 * withhold = 0 restores normal operation. Batches created from the plan are
 * not affected. Host only.
 * Errors: RCBF_EINVAL (NULL plan, wait_ns == 0, withhold not 0 or 1). */
int rcbf_plan_set_wait(rcbf_plan_t plan, uint64_t wait_ns, int32_t withhold);

/* rcbf_batch_create — bind n_frames (plan, buffers) triples into one batch
 * that persistent kernels process: for every frame with a
 * Hadamard order, decode rf[f] into decoded[f] (with the plan's tensor-core
 * decode form; an RCBF_DECODE_TC frame by its own tcgen05 launch, enqueued by
 * rcbf_batch_run ahead of the persistent launches, the other forms as work
 * items of the persistent kernel), then DAS decoded[f] into images[f] (frames with
 * hadamard_order == 0 skip the decode and read decoded[f] directly). Plans
 * may differ in transmit count, samples, grid, orientation and tile; all
 * must use decoded_dtype RCBF_F32 or RCBF_F16 and the tiled DAS with no F#
 * window. Frames are grouped into phases by DAS window class (48, 64, 96 or
 * 128 samples) and tile extent along u (tile[0]); each phase is one
 * persistent launch, the later ones launched as programmatic dependents so
 * that a phase's CTAs start on the SMs the previous phase frees at its tail
 * (all frames of one class and tile extent: one launch). Each frame is beamformed at its
 * plan's speed of sound, without channel weights. The plans must outlive the
 * batch. Pointer arrays are HOST arrays of DEVICE pointers, copied; rf may be
 * NULL when no frame is encoded.
 * Passage: §METHODS "Data Processing" (pre-uploaded parameter sets) and
 * §OPTIMIZATIONS "Data Transfer" (frames kept in flight).
 * Allocates the device work list; synchronises once. Errors: RCBF_EINVAL,
 * RCBF_EUNSUPPORTED (dtype, variant, F#, window longer than 128 samples),
 * RCBF_ENOMEM, RCBF_ECUDA. */
int rcbf_batch_create(const rcbf_plan_t* plans, uint32_t n_frames,
                      const int16_t* const* rf, void* const* decoded,
                      float* const* images, rcbf_batch_t* out_batch);

/* rcbf_batch_run — enqueue the whole batch on `stream`: a counter reset, one
 * tcgen05 decode launch per RCBF_DECODE_TC frame, then one persistent launch
 * per phase. Contains no host synchronisation and no allocation, so it can
 * be captured in a CUDA graph. The persistent kernels' waits on per-frame
 * decode completion are bounded; on expiry they record RCBF_ETIMEOUT in the
 * batch's device status word (see rcbf_batch_status). */
int rcbf_batch_run(rcbf_batch_t batch, void* stream);

/* rcbf_batch_status — synchronise `stream` and return the device status word
 * of the last run: RCBF_OK or RCBF_ETIMEOUT. */
int rcbf_batch_status(rcbf_batch_t batch, void* stream);

/* rcbf_batch_set_wait — bound of a DAS item's wait for its frame's decode
 * (default one second; at most ten), and a test hook: withhold_frame >= 0
 * makes that frame's decode completion count unreachable, so that its DAS
 * items wait out the bound and the run reports RCBF_ETIMEOUT through
 * rcbf_batch_status while the context stays usable; -1 disables the hook.
 * Host only. Errors: RCBF_EINVAL (NULL batch, wait_ns == 0, frame out of range). */
int rcbf_batch_set_wait(rcbf_batch_t batch, uint64_t wait_ns, int32_t withhold_frame);

/* rcbf_batch_destroy — free the batch's device work list. NULL is accepted. */
void rcbf_batch_destroy(rcbf_batch_t batch);

/* rcbf_pipeline_create — the upload ring of §OPTIMIZATIONS "Data Transfer"
 * (several frames in flight so that uploads never stall the GPU):
 * n_slots (2..8; the paper keeps 3) sets of device buffers for a batch of
 * n_frames frames, each set bound to its own rcbf_batch (plans validated as
 * for rcbf_batch_create) and captured once as a CUDA graph, plus three streams
 * (host->device copies, compute, device->host copies). Allocates the buffers
 * and synchronises once. The plans must outlive the pipeline.
 * Errors: RCBF_EINVAL, RCBF_EUNSUPPORTED (as rcbf_batch_create), RCBF_ENOMEM, RCBF_ECUDA. */
int rcbf_pipeline_create(const rcbf_plan_t* plans, uint32_t n_frames, uint32_t n_slots,
                         rcbf_pipeline_t* out_pipeline);

/* rcbf_pipeline_submit — one step through the next slot: copy each frame's
 * input from host memory (encoded int16 RF [n_tx][n_ch][n_samples] for a plan
 * with a Hadamard order, else the decoded data of the plan's dtype), run the
 * batch, and copy each image [nz][ny][nx] back to host_images[f]. Returns
 * once the work is enqueued; the copies of one step overlap the compute of
 * the step before. Before reusing a slot the call waits on the host until
 * that slot's previous step has finished (so at most n_slots steps are in
 * flight) and folds its batch status into the pipeline's status. Host
 * buffers (arrays of HOST pointers, one per frame) must stay valid and
 * unchanged until the step completes; page-locked memory makes the copies
 * asynchronous (pageable memory works but serialises them).
 * Errors: RCBF_EINVAL, RCBF_ECUDA. */
int rcbf_pipeline_submit(rcbf_pipeline_t pipeline, const void* const* host_inputs, float* const* host_images);

/* rcbf_pipeline_wait — wait for every submitted step; RCBF_ETIMEOUT if the
 * bounded per-frame wait of any step's batch expired since the last call
 * (the status is then cleared). Errors: RCBF_EINVAL, RCBF_ECUDA, RCBF_ETIMEOUT. */
int rcbf_pipeline_wait(rcbf_pipeline_t pipeline);

/* rcbf_pipeline_destroy — wait for the pipeline, then free its buffers,
 * batches, graphs, events and streams. NULL is accepted. */
void rcbf_pipeline_destroy(rcbf_pipeline_t pipeline);

/* rcbf_das_noalloc — rcbf_das without a plan, for callers that must not
 * allocate device memory: code that owns every device allocation through its
 * own pool, or real-time loops that forbid allocation after start-up.
 * rcbf_plan allocates (decode tables,
 * a status word, the channel-split partial images), so those callers cannot
 * make a plan. This entry point takes the parameter block itself, validates
 * and sets up the geometry on the host, and calls no cudaMalloc, cudaFree or
 * other allocating routine. The scratch the DAS kernels need (the partial
 * images of a channel-split tile pass and the status word) is a fixed,
 * file-scope device array of 16 MiB, which every GPU that loads the library
 * holds until the process exits. There is no counterpart in the paper.
 *   params, decoded, apod, c, image, stream: as for rcbf_plan + rcbf_das.
 * The first call on a device looks up that device's address of the array
 * (once per device, on the host). All calls share the one array: calls
 * whose work overlaps on the GPU (other streams, other host threads) race on
 * it, so serialise them. A bounded wait of the tiled kernel that expires is
 * reported by rcbf_das_noalloc_status. Errors: as rcbf_plan and rcbf_das
 * (RCBF_EUNSUPPORTED for a tiled form the geometry does not admit, and for
 * plane waves, whose direction table needs a plan), and RCBF_EINVAL when the
 * partial images would exceed the 16 MiB array. */
int rcbf_das_noalloc(const rcbf_params* params, const void* decoded, const float* apod, float c,
                     float* image, void* stream);

/* rcbf_das_noalloc_status — synchronise `stream` and return the status of the
 * last rcbf_das_noalloc call on the current device: RCBF_OK, or RCBF_ETIMEOUT
 * when a bounded wait of its tiled DAS expired (the image is then
 * incomplete). The status word lives in the same static array as the scratch,
 * so it is cleared by the next rcbf_das_noalloc call on the device and shared
 * by every caller on it. Allocates nothing.
 * Errors: RCBF_ECUDA. */
int rcbf_das_noalloc_status(void* stream);

/* rcbf_measure_ceilings — on-chip ceilings of the current device, measured
 * by microbenchmark kernels run at the tiled DAS kernel's occupancy (two CTAs
 * of 256 threads per SM, one per resident slot): the denominators of the DAS
 * roofline, which is bound on chip, not by HBM (the paper's own optimisation
 * section discusses the DAS as the stage with the most operations, without a
 * roofline). Fields:
 *   lds64_bytes_per_s    conflict-free 8-byte shared-memory loads (one line
 *                        piece (c_n, slope_n) per DAS sum);
 *   ffma_lane_ops_per_s  scalar FP32 FMAs, lanes x instructions per second;
 *   ffma2_lane_ops_per_s packed f32x2 FMAs, two lane operations each;
 *   red_shared_per_s     warp-wide shared integer reductions (red.shared.add.s32)
 *                        to 32 distinct addresses, warp instructions per second;
 *   sm_clock_hz          SM clock during the loads: clock64 cycles over
 *                        global-timer time in one thread (0 if the timer
 *                        did not advance).
 * Runs four short kernels (a few ms each, bounded loops, no waits) on `stream`
 * and synchronises it. Errors: RCBF_EINVAL (NULL out), RCBF_ECUDA. */
typedef struct rcbf_ceilings {
    double lds64_bytes_per_s;
    double ffma_lane_ops_per_s;
    double ffma2_lane_ops_per_s;
    double red_shared_per_s;
    double sm_clock_hz;
} rcbf_ceilings;

int rcbf_measure_ceilings(rcbf_ceilings* out, void* stream);

/* rcbf_last_error — message for the last failure on this thread ("" if none). */
const char* rcbf_last_error(void);

/* rcbf_version — library version string. */
const char* rcbf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RCBF_H */

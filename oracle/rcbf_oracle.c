/*
 * rcbf_oracle.c — plain, slow FP64 CPU oracle of the beamformer hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library, its kernels or its Python
 * binding may include, link or call this file; only the tests, the smoke
 * check and the benchmark's CPU-baseline leg use it. It shares no header,
 * table or helper with the CUDA path.
 *
 * Every function writes out the paper's definition directly, loop by loop,
 * in double precision (int64 for the decode), with no blocking, fusion or
 * reordering beyond the definition:
 *
 *   oracle_hadamard  Sylvester Hadamard matrix H[k][i] = (-1)^popcount(k & i).
 *   oracle_decode    D[i][c] = sum_k H[k][i] * S[k][c]          (§THEORY
 *                    "Synthetic Aperture Imaging": decoding is a matrix
 *                    product across transmits; after decoding, row i behaves
 *                    as a transmit on element i).
 *   oracle_das       HR(v) = sum_i a_tx sum_j a_j(v) r_ij(ToF_ij(v))  Eq. (1),
 *                    a_tx = 1, a_j(v) = w_j W(F# |lat_rx(v) - e_j| / |z(v)|)
 *                    Eq. (2), W(u) = cos^2(pi u) for |u| < 0.5, else 0  Eq. (3);
 *                    r_ij read at fractional sample s = (ToF - t0) fs by linear
 *                    or 4-point cubic Hermite interpolation (§THEORY
 *                    "Interpolation & Sampling"), zero outside the record.
 *   oracle_das_grad  the derivatives of oracle_das with respect to the RF
 *                    samples, the speed of sound c and the weights w_j.
 *   oracle_demodulate  IQ[n] = LPF{s[n] e^{-j 2 pi f_d n / f_s}} (§OPTIMIZATIONS
 *                    "Filtering & Demodulation", Eq. (demodulation)) at
 *                    quadrature sampling f_s = 4 f_d, with an integer FIR
 *                    (int16 taps, real or complex, a rounding right shift back
 *                    to int16) and decimation, in exact integer arithmetic.
 *   IQ beamforming   oracle_das with iq_freq = f_d > 0 reads the two planes as
 *                    the baseband signal and multiplies each interpolated
 *                    sample by e^{j 2 pi (f_d / f_s) s}, which restores the
 *                    carrier that the index-based mixer removed.
 *
 * Geometry (the readings used by the whole project): line elements centred
 * on the origin, e_i = (i - (n-1)/2) pitch at z = 0; a row element's lateral
 * coordinate is y, a column element's is x; the distance from a point q to a
 * line element is sqrt((lat(q) - e)^2 + q_z^2). Voxel positions come from an
 * inclusive linspace (or a 4x4 voxel-index affine), then a 4x4 world-to-array
 * affine.
 *
 * Transmit waves (the row-column methods of §CAPABILITIES: FORCES, TPW,
 * VLS): the transmit path of line (or wave) i to a point q is
 *   line element     d_tx = sqrt((lat_tx(q) - e_i)^2 + q_z^2)
 *   plane wave       d_tx = q_z cos(theta_i) + lat_tx(q) sin(theta_i)
 *   virtual line     d_tx = f + sgn(q_z - f) sqrt((lat_tx(q) - e_i)^2 + (q_z - f)^2)
 *                    (a line focus at depth f above line element i; sgn(0) = +1)
 * and every one of them depends on (lat_tx, z) only, so s_ij = A_i + B_j
 * stays separable.
 *
 * HERCULES with its 2D receive aperture (acq_kind 2; §THEORY: after decoding
 * the data is that of a 2D matrix array receiving one plane or diverging
 * wave): index i is the receive row at lateral e_i (rows' lateral axis),
 * index j the column at e_j (columns' axis); for each (i, j) the receive path
 * is the point distance sqrt((lat_rx - e_j)^2 + (lat_tx - e_i)^2 + z^2), and
 * one transmit wave reaches the point after
 *   plane wave       d_tx = z cos(a) + lat_tx sin(a)      (a = tx_angles[0])
 *   diverging wave   d_tx = sqrt(x^2 + y^2 + (z - f)^2) + f   (virtual point at depth f < 0)
 * so the delay is not a sum of a row term and a column term. The F# window of
 * Eq. (2) is applied to the radial lateral distance to element (i, j).
 *
 * Window reading: the window is non-zero exactly when F# |lat - e_j| < 0.5 |z|
 * (|u| < 0.5 written without a division), so a voxel at z = 0 gets weight 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct oracle_geom {
    int64_t n_tx, n_ch, n_samples;
    int64_t tx_orientation, rx_orientation;  /* 0 rows (lateral y), 1 columns (lateral x) */
    int64_t dims[3];                          /* nx, ny, nz */
    int64_t has_voxel_transform, has_xdc_transform;
    double fs, c, t0;
    double tx_pitch, rx_pitch;
    double f_number;
    double out_min[3], out_max[3];
    double voxel_transform[16];               /* row-major, index -> world */
    double xdc_transform[16];                 /* row-major, world -> array */
    int64_t interp;                           /* 0 linear, 1 cubic Hermite */
    double iq_freq;                           /* 0: RF planes; > 0: baseband IQ demodulated at this frequency */
    int64_t tx_wave;                          /* 0 line elements, 1 plane waves, 2 virtual line sources */
    double tx_focus;                          /* virtual line source depth f [m] */
    const double* tx_angles;                  /* plane-wave angles theta_i [rad], n_tx of them */
    int64_t acq_kind;                         /* 2: HERCULES with a 2D receive aperture */
} oracle_geom;

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- decode */

void oracle_hadamard(int64_t n, int8_t* H) {
    for (int64_t k = 0; k < n; ++k)
        for (int64_t i = 0; i < n; ++i)
            H[k * n + i] = (__builtin_popcountll((unsigned long long)(k & i)) & 1) ? -1 : 1;
}

/* D[i][c] = sum_k H[k][i] S[k][c]; S is [n][n_cols] int16, D is [n][n_cols] int64. */
void oracle_decode(int64_t n, int64_t n_cols, const int16_t* S, const int8_t* H, int64_t* D) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t* out = D + i * n_cols;
        for (int64_t c = 0; c < n_cols; ++c) out[c] = 0;
        for (int64_t k = 0; k < n; ++k) {
            const int64_t h = (int64_t)H[k * n + i];
            const int16_t* row = S + k * n_cols;
            for (int64_t c = 0; c < n_cols; ++c) out[c] += h * (int64_t)row[c];
        }
    }
}

/* ------------------------------------------------------------- geometry */

static void voxel_position(const oracle_geom* g, int64_t v, double q[3]) {
    const int64_t nx = g->dims[0], ny = g->dims[1];
    const int64_t ix = v % nx, iy = (v / nx) % ny, iz = v / (nx * ny);
    const double idx[3] = {(double)ix, (double)iy, (double)iz};
    double p[3];
    if (g->has_voxel_transform) {
        for (int r = 0; r < 3; ++r) {
            const double* m = g->voxel_transform + 4 * r;
            p[r] = m[0] * idx[0] + m[1] * idx[1] + m[2] * idx[2] + m[3];
        }
    } else {
        for (int d = 0; d < 3; ++d) {
            if (g->dims[d] > 1)
                p[d] = g->out_min[d] + idx[d] * (g->out_max[d] - g->out_min[d]) / (double)(g->dims[d] - 1);
            else
                p[d] = g->out_min[d];
        }
    }
    if (g->has_xdc_transform) {
        for (int r = 0; r < 3; ++r) {
            const double* m = g->xdc_transform + 4 * r;
            q[r] = m[0] * p[0] + m[1] * p[1] + m[2] * p[2] + m[3];
        }
    } else {
        q[0] = p[0]; q[1] = p[1]; q[2] = p[2];
    }
}

static double lateral(const double q[3], int64_t orientation) {
    return orientation == 0 ? q[1] : q[0];
}

static double element_position(int64_t index, int64_t count, double pitch) {
    return ((double)index - (double)(count - 1) / 2.0) * pitch;
}

/* Transmit path of wave i to the point (lat_tx, z). */
static double transmit_distance(const oracle_geom* g, int64_t i, double lat_tx, double z) {
    if (g->tx_wave == 1) {
        const double th = g->tx_angles[i];
        return z * cos(th) + lat_tx * sin(th);
    }
    const double dx = lat_tx - element_position(i, g->n_tx, g->tx_pitch);
    if (g->tx_wave == 2) {
        const double dz = z - g->tx_focus;
        return g->tx_focus + (dz >= 0.0 ? 1.0 : -1.0) * sqrt(dx * dx + dz * dz);
    }
    return sqrt(dx * dx + z * z);
}

/* Eq. (3) evaluated at u = F# |delta| / |z|, with the support test written
 * as F# |delta| < 0.5 |z|. */
static double window_weight(double f_number, double delta, double z) {
    if (f_number <= 0.0) return 1.0;
    const double a = f_number * fabs(delta);
    if (!(a < 0.5 * fabs(z))) return 0.0;
    const double cs = cos(M_PI * a / fabs(z));
    return cs * cs;
}

/* r at fractional sample s: (1-f) r[n] + f r[n+1], n = floor(s), zero outside. */
static double sample_linear(const double* trace, int64_t n_s, double s) {
    const double fl = floor(s);
    const double f = s - fl;
    const int64_t n = (int64_t)fl;
    const double a = (n >= 0 && n < n_s) ? trace[n] : 0.0;
    const double b = (n + 1 >= 0 && n + 1 < n_s) ? trace[n + 1] : 0.0;
    return (1.0 - f) * a + f * b;
}

static double sample_at(const double* trace, int64_t n_s, int64_t k) {
    return (k >= 0 && k < n_s) ? trace[k] : 0.0;
}

/* 4-point cubic Hermite spline at fractional sample s (§THEORY
 * "Interpolation & Sampling"): on [n, n+1], n = floor(s), f = s - n, the
 * cubic with values r[n], r[n+1] and slopes m_k = (r[k+1] - r[k-1]) / 2 at
 * both ends (central differences; the paper names the Hermite basis but not
 * its tangents), in the Hermite basis h00 = 2f^3 - 3f^2 + 1,
 * h10 = f^3 - 2f^2 + f, h01 = -2f^3 + 3f^2, h11 = f^3 - f^2; zero outside. */
static double sample_cubic(const double* trace, int64_t n_s, double s) {
    const double fl = floor(s);
    const double f = s - fl;
    const int64_t n = (int64_t)fl;
    const double p0 = sample_at(trace, n_s, n - 1), p1 = sample_at(trace, n_s, n);
    const double p2 = sample_at(trace, n_s, n + 1), p3 = sample_at(trace, n_s, n + 2);
    const double m1 = 0.5 * (p2 - p0), m2 = 0.5 * (p3 - p1);
    const double f2 = f * f, f3 = f2 * f;
    const double h00 = 2.0 * f3 - 3.0 * f2 + 1.0, h10 = f3 - 2.0 * f2 + f;
    const double h01 = -2.0 * f3 + 3.0 * f2, h11 = f3 - f2;
    return h00 * p1 + h10 * m1 + h01 * p2 + h11 * m2;
}

/* HERCULES 2D: transmit path of the frame's one wave (tx_wave 1 plane,
 * 3 diverging) to q, and the receive path to element (row i, column j). */
static double hercules_transmit(const oracle_geom* g, const double q[3]) {
    if (g->tx_wave == 1) {
        const double a = g->tx_angles[0];
        return q[2] * cos(a) + lateral(q, g->tx_orientation) * sin(a);
    }
    const double dz = q[2] - g->tx_focus;
    return sqrt(q[0] * q[0] + q[1] * q[1] + dz * dz) + g->tx_focus;
}

static double hercules_receive(const oracle_geom* g, int64_t i, int64_t j, const double q[3], double* radial) {
    const double dr = lateral(q, g->rx_orientation) - element_position(j, g->n_ch, g->rx_pitch);
    const double dt = lateral(q, g->tx_orientation) - element_position(i, g->n_tx, g->tx_pitch);
    *radial = sqrt(dr * dr + dt * dt);
    return sqrt(dr * dr + dt * dt + q[2] * q[2]);
}

/* ------------------------------------------------------------------ DAS */

/* rf: [n_planes][n_tx][n_ch][n_s] doubles; w: [n_ch] or NULL; c > 0.
 * vox: n_vox voxel linear indices (z-major, x fastest) or NULL for all voxels
 * (then n_vox must equal nx*ny*nz). out: [n_planes][n_vox]. */
void oracle_das(const oracle_geom* g, const double* rf, int64_t n_planes, const double* w,
                double c, int64_t n_vox, const int64_t* vox, double* out) {
    const int64_t n_tx = g->n_tx, n_ch = g->n_ch, n_s = g->n_samples;
    const int iq = g->iq_freq > 0.0 && n_planes == 2;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < n_vox; ++t) {
        const int64_t v = vox ? vox[t] : t;
        double q[3];
        voxel_position(g, v, q);
        const double lat_tx = lateral(q, g->tx_orientation);
        const double lat_rx = lateral(q, g->rx_orientation);
        double acc[2] = {0.0, 0.0};
        const int h2d = g->acq_kind == 2;
        const double d_wave = h2d ? hercules_transmit(g, q) : 0.0;
        for (int64_t i = 0; i < n_tx; ++i) {
            const double d_tx = h2d ? d_wave : transmit_distance(g, i, lat_tx, q[2]);
            for (int64_t j = 0; j < n_ch; ++j) {
                double d_rx, lat_off;
                if (h2d) {
                    d_rx = hercules_receive(g, i, j, q, &lat_off);
                } else {
                    lat_off = lat_rx - element_position(j, n_ch, g->rx_pitch);
                    d_rx = sqrt(lat_off * lat_off + q[2] * q[2]);
                }
                const double a = (w ? w[j] : 1.0) * window_weight(g->f_number, lat_off, q[2]);
                if (a == 0.0) continue;
                const double tof = (d_tx + d_rx) / c;
                const double s = (tof - g->t0) * g->fs;
                double val[2] = {0.0, 0.0};
                for (int64_t p = 0; p < n_planes; ++p) {
                    const double* trace = rf + ((p * n_tx + i) * n_ch + j) * n_s;
                    val[p] = g->interp == 1 ? sample_cubic(trace, n_s, s) : sample_linear(trace, n_s, s);
                }
                if (iq) {
                    /* (I + jQ) e^{j 2 pi (f_d / f_s) s} */
                    const double ph = 2.0 * M_PI * (g->iq_freq / g->fs) * s;
                    const double cr = cos(ph), sr = sin(ph);
                    acc[0] += a * (val[0] * cr - val[1] * sr);
                    acc[1] += a * (val[0] * sr + val[1] * cr);
                } else {
                    for (int64_t p = 0; p < n_planes; ++p) acc[p] += a * val[p];
                }
            }
        }
        for (int64_t p = 0; p < n_planes; ++p) out[p * n_vox + t] = acc[p];
    }
}

/* Gradients of L with dL/dHR = G (G: [n_planes][nx*ny*nz], all voxels):
 *   grad_rf[p][i][j][n] = sum_v a_j(v) G_p(v) dlerp/dr[n]
 *   grad_c              = sum_p sum_v sum_ij a_j(v) G_p(v) (r[n+1] - r[n]) ds/dc,
 *                         ds/dc = -(d_tx + d_rx) fs / c^2
 *   grad_w[j]           = sum_p sum_v sum_i W_j(v) G_p(v) lerp(r_ij, s)
 * with n = floor(s) (the right derivative at integer s). Any output may be NULL.
 * Parallel over transmits: each thread owns grad_rf rows of its transmits. */
void oracle_das_grad(const oracle_geom* g, const double* rf, int64_t n_planes, const double* w,
                     double c, const double* G, double* grad_rf, double* grad_c, double* grad_w) {
    const int64_t n_tx = g->n_tx, n_ch = g->n_ch, n_s = g->n_samples;
    const int64_t n_vox = g->dims[0] * g->dims[1] * g->dims[2];
    if (grad_rf) memset(grad_rf, 0, sizeof(double) * (size_t)(n_planes * n_tx * n_ch * n_s));
    double gc_total = 0.0;
    double* gw_total = (double*)calloc((size_t)n_ch, sizeof(double));
#pragma omp parallel
    {
        double gc = 0.0;
        double* gw = (double*)calloc((size_t)n_ch, sizeof(double));
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < n_tx; ++i) {
            for (int64_t v = 0; v < n_vox; ++v) {
                double q[3];
                voxel_position(g, v, q);
                const double lat_tx = lateral(q, g->tx_orientation);
                const double lat_rx = lateral(q, g->rx_orientation);
                const double d_tx = transmit_distance(g, i, lat_tx, q[2]);
                for (int64_t j = 0; j < n_ch; ++j) {
                    const double dx_r = lat_rx - element_position(j, n_ch, g->rx_pitch);
                    const double d_rx = sqrt(dx_r * dx_r + q[2] * q[2]);
                    const double W = window_weight(g->f_number, dx_r, q[2]);
                    if (W == 0.0) continue;
                    const double a = (w ? w[j] : 1.0) * W;
                    const double s = ((d_tx + d_rx) / c - g->t0) * g->fs;
                    const double dsdc = -(d_tx + d_rx) * g->fs / (c * c);
                    const double fl = floor(s);
                    const double f = s - fl;
                    const int64_t n = (int64_t)fl;
                    for (int64_t p = 0; p < n_planes; ++p) {
                        const double Gv = G[p * n_vox + v];
                        if (Gv == 0.0) continue;
                        const int64_t base = ((p * n_tx + i) * n_ch + j) * n_s;
                        const double* trace = rf + base;
                        const double r0 = (n >= 0 && n < n_s) ? trace[n] : 0.0;
                        const double r1 = (n + 1 >= 0 && n + 1 < n_s) ? trace[n + 1] : 0.0;
                        if (grad_rf) {
                            if (n >= 0 && n < n_s) grad_rf[base + n] += a * Gv * (1.0 - f);
                            if (n + 1 >= 0 && n + 1 < n_s) grad_rf[base + n + 1] += a * Gv * f;
                        }
                        gc += a * Gv * (r1 - r0) * dsdc;
                        gw[j] += W * Gv * ((1.0 - f) * r0 + f * r1);
                    }
                }
            }
        }
#pragma omp critical
        {
            gc_total += gc;
            for (int64_t j = 0; j < n_ch; ++j) gw_total[j] += gw[j];
        }
        free(gw);
    }
    if (grad_c) *grad_c = gc_total;
    if (grad_w) for (int64_t j = 0; j < n_ch; ++j) grad_w[j] = gw_total[j];
    free(gw_total);
}

/* ------------------------------------------------------------ demodulation */

/* Round x / 2^shift to the nearest integer, ties to even. */
static int64_t round_shift_even(int64_t x, int64_t shift) {
    if (shift <= 0) return x;
    const int64_t d = (int64_t)1 << shift;
    int64_t q = x >= 0 ? x / d : -((-x + d - 1) / d);     /* floor(x / d) */
    const int64_t rem = x - q * d;                          /* 0 <= rem < d */
    if (2 * rem > d || (2 * rem == d && (q & 1))) q += 1;
    return q;
}

/* Eq. (demodulation) at f_d = f_s / 4: e^{-j 2 pi n / 4} = cos(pi n / 2) - j sin(pi n / 2)
 * is 1, -j, -1, j for n mod 4 = 0, 1, 2, 3. The LPF is the causal FIR
 * y[n] = sum_k h[k] x[n - k] (x = 0 outside the record); decimation keeps
 * n = m D. The taps may be complex, h[k] = h_re[k] + j h_im[k] (a baseband
 * matched filter that also applies a phase correction); the product
 * h[k] x[n - k] is the complex product. Each output component is rounded
 * (ties to even) after a right shift and saturated to int16.
 * s: [n_traces][n_in] int16; h_re, h_im: [n_taps] int16 (h_im NULL = real
 * taps); out: [2][n_traces][n_out] (I plane, then Q plane), n_out * D <= n_in. */
void oracle_demodulate_complex(int64_t n_traces, int64_t n_in, const int16_t* s, const int16_t* h_re,
                               const int16_t* h_im, int64_t n_taps, int64_t shift, int64_t decimation,
                               int64_t n_out, int16_t* out) {
#pragma omp parallel for schedule(static)
    for (int64_t tr = 0; tr < n_traces; ++tr) {
        const int16_t* x = s + tr * n_in;
        for (int64_t m = 0; m < n_out; ++m) {
            const int64_t n = m * decimation;
            int64_t acc_i = 0, acc_q = 0;
            for (int64_t k = 0; k < n_taps; ++k) {
                const int64_t idx = n - k;
                if (idx < 0 || idx >= n_in) continue;
                const int64_t v = x[idx];
                /* x[idx] e^{-j pi idx / 2} */
                int64_t re = 0, im = 0;
                switch (idx & 3) {
                    case 0: re = v; break;
                    case 1: im = -v; break;
                    case 2: re = -v; break;
                    default: im = v; break;
                }
                const int64_t hr = h_re[k], hi = h_im ? h_im[k] : 0;
                /* (hr + j hi)(re + j im) */
                acc_i += hr * re - hi * im;
                acc_q += hr * im + hi * re;
            }
            int64_t oi = round_shift_even(acc_i, shift), oq = round_shift_even(acc_q, shift);
            oi = oi > 32767 ? 32767 : oi < -32768 ? -32768 : oi;
            oq = oq > 32767 ? 32767 : oq < -32768 ? -32768 : oq;
            out[tr * n_out + m] = (int16_t)oi;
            out[(n_traces + tr) * n_out + m] = (int16_t)oq;
        }
    }
}

/* The same with real taps. */
void oracle_demodulate(int64_t n_traces, int64_t n_in, const int16_t* s, const int16_t* h, int64_t n_taps,
                       int64_t shift, int64_t decimation, int64_t n_out, int16_t* out) {
    oracle_demodulate_complex(n_traces, n_in, s, h, NULL, n_taps, shift, decimation, n_out, out);
}

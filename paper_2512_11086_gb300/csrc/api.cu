// api.cu — the C ABI of include/rcbf.h: argument validation, plan
// construction (geometry affine, decode fragments, DAS tile choice), error
// reporting and dispatch to the kernels. Every check happens on the host
// before a launch; on error nothing is enqueued.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

namespace rcbf {

namespace {
thread_local std::string g_last_error;

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
bool aligned4(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }
bool is_pow2(uint32_t n) { return n && !(n & (n - 1)); }
bool all_zero(const double* m, int n) {
    for (int k = 0; k < n; ++k) if (m[k] != 0.0) return false;
    return true;
}
}  // namespace

int set_error(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int check_launch(const char* what) {
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return RCBF_OK;
    return set_error(e == cudaErrorMemoryAllocation ? RCBF_ENOMEM : RCBF_ECUDA,
                     std::string(what) + ": " + cudaGetErrorString(e));
}

namespace {

// A = H^T fragments of mma.m16n8k32 (row-major A, int8) in the k order that
// ldmatrix.trans + byte permutes give the B fragments: fragment position p of
// a k32 chunk holds acquisition 16*(p>>4) + 8*((p&3)>>1) + 2*((p>>2)&3) + (p&1).
std::vector<uint32_t> build_afrag(const std::vector<int8_t>& H, int n) {
    const int MT = n / 16, KC = n / 32;
    std::vector<uint32_t> out((size_t)MT * KC * 32 * 4);
    for (int mt = 0; mt < MT; ++mt)
        for (int kc = 0; kc < KC; ++kc)
            for (int lane = 0; lane < 32; ++lane) {
                const int g = lane >> 2, t = lane & 3;
                for (int r = 0; r < 4; ++r) {
                    uint32_t word = 0;
                    for (int m = 0; m < 4; ++m) {
                        const int row = mt * 16 + g + ((r & 1) ? 8 : 0);
                        const int pos = ((r >= 2) ? 16 : 0) + 4 * t + m;
                        const int kk = 16 * (pos >> 4) + 8 * ((pos & 3) >> 1) + 2 * ((pos >> 2) & 3) + (pos & 1);
                        const int k = kc * 32 + kk;
                        const int8_t v = H[(size_t)k * n + row];    // A[row][k] = H[k][row]
                        word |= (uint32_t)(uint8_t)v << (8 * m);
                    }
                    out[(((size_t)mt * KC + kc) * 32 + lane) * 4 + r] = word;
                }
            }
    return out;
}

// A = H^T fragments of mma.m16n8k16 (row-major A, FP16 +-1): register r of
// lane (g, t) holds rows g (+8 for r odd) and k pair 2t, 2t+1 (+8 for r >= 2).
// A = H^T as the tcgen05 decode's shared-memory operand: FP16 +-1, K-major,
// 128-byte swizzled. Per K atom of 64 acquisitions (atoms = max(1, n / 64)),
// row i of 128 (rows >= n zero) holds eight 16-byte chunks c of the
// acquisitions k = 64 atom + 8 c + 0..7; chunk c of row i sits at
// 1024 (i / 8) + 128 (i % 8) + 16 (c xor (i % 8)) within the 16 KB atom.
std::vector<uint16_t> build_a_tc(const std::vector<int8_t>& H, int n) {
    const int atoms = n > 64 ? n / 64 : 1;
    std::vector<uint16_t> a((size_t)atoms * 128 * 64, 0);
    for (int atom = 0; atom < atoms; ++atom)
        for (int i = 0; i < 128; ++i)
            for (int c = 0; c < 8; ++c)
                for (int e = 0; e < 8; ++e) {
                    const int k = atom * 64 + c * 8 + e;
                    if (i >= n || k >= n) continue;
                    const size_t off = (size_t)atom * 16384 + (size_t)(i >> 3) * 1024 + (size_t)(i & 7) * 128 +
                                       (size_t)((c ^ (i & 7)) << 4);
                    a[off / 2 + e] = H[(size_t)k * n + i] > 0 ? 0x3C00u : 0xBC00u;
                }
    return a;
}

std::vector<uint32_t> build_afrag16(const std::vector<int8_t>& H, int n) {
    const int MT = n / 16, KC = n / 16;
    std::vector<uint32_t> out((size_t)MT * KC * 32 * 4);
    for (int mt = 0; mt < MT; ++mt)
        for (int kc = 0; kc < KC; ++kc)
            for (int lane = 0; lane < 32; ++lane) {
                const int g = lane >> 2, t = lane & 3;
                for (int r = 0; r < 4; ++r) {
                    const int row = mt * 16 + g + ((r & 1) ? 8 : 0);
                    const int k0 = kc * 16 + 2 * t + ((r >= 2) ? 8 : 0);
                    uint32_t word = 0;
                    for (int e = 0; e < 2; ++e) {
                        const int8_t v = H[(size_t)(k0 + e) * n + row];
                        const uint32_t bits = v > 0 ? 0x3C00u : 0xBC00u;   // FP16 +1 / -1
                        word |= bits << (16 * e);
                    }
                    out[(((size_t)mt * KC + kc) * 32 + lane) * 4 + r] = word;
                }
            }
    return out;
}

void mat_mul_3x4(const double* X /*4x4*/, const double* M /*4x4*/, double* G /*3x4*/) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 4; ++c) {
            double s = 0;
            for (int k = 0; k < 4; ++k) s += X[r * 4 + k] * M[k * 4 + c];
            G[r * 4 + c] = s;
        }
}

// Tile radius in the (lateral, z) plane of an element family: the largest
// distance from the tile centre to a tile corner (distances to a line element
// are 1-Lipschitz in that plane, so this bounds every delay offset).
double tile_radius(const double* G, int lat_axis, int ua, int va, int bu, int bv, int bw) {
    double best = 0;
    for (int sx = -1; sx <= 1; sx += 2)
        for (int sy = -1; sy <= 1; sy += 2)
            for (int sz = -1; sz <= 1; sz += 2) {
                const double du = sx * 0.5 * (bu - 1), dv = sy * 0.5 * (bv - 1), dw = sz * 0.5 * (bw - 1);
                const double dl = G[lat_axis * 4 + ua] * du + G[lat_axis * 4 + va] * dv + G[lat_axis * 4 + 2] * dw;
                const double dz = G[2 * 4 + ua] * du + G[2 * 4 + va] * dv + G[2 * 4 + 2] * dw;
                best = std::fmax(best, std::sqrt(dl * dl + dz * dz));
            }
    return best;
}

int validate(const rcbf_params* p) {
    if (!p) return set_error(RCBF_EINVAL, "rcbf_plan: params is NULL");
    if (p->n_tx < 1 || p->n_tx > (uint32_t)kMaxOrder)
        return set_error(RCBF_EINVAL, "rcbf_plan: n_tx must be in [1, 256]");
    if (p->n_ch < 1 || p->n_ch > (uint32_t)kMaxChannels)
        return set_error(RCBF_EINVAL, "rcbf_plan: n_ch must be in [1, 256]");
    if (p->n_samples < 8 || p->n_samples % 8)
        return set_error(RCBF_EINVAL, "rcbf_plan: n_samples must be a positive multiple of 8");
    if (p->n_samples > (1u << 24))
        return set_error(RCBF_EINVAL, "rcbf_plan: n_samples too large");
    for (int d = 0; d < 3; ++d)
        if (p->out_dims[d] < 1) return set_error(RCBF_EINVAL, "rcbf_plan: out_dims must be >= 1");
    if ((double)p->out_dims[0] * p->out_dims[1] * p->out_dims[2] > 2147483647.0)
        return set_error(RCBF_EINVAL, "rcbf_plan: too many voxels");
    if (!(p->fs > 0) || !(p->c > 0)) return set_error(RCBF_EINVAL, "rcbf_plan: fs and c must be > 0");
    if (!(p->f_number >= 0)) return set_error(RCBF_EINVAL, "rcbf_plan: f_number must be >= 0");
    if (p->tx_orientation > 1 || p->rx_orientation > 1)
        return set_error(RCBF_EINVAL, "rcbf_plan: orientation must be RCBF_ROWS or RCBF_COLUMNS");
    if (p->acq_kind > RCBF_HERCULES_2D) return set_error(RCBF_EINVAL, "rcbf_plan: unknown acq_kind");
    if (p->interp != RCBF_LINEAR && p->interp != RCBF_CUBIC)
        return set_error(RCBF_EUNSUPPORTED, "rcbf_plan: interp must be RCBF_LINEAR or RCBF_CUBIC");
    if (p->decoded_dtype != RCBF_I32 && p->decoded_dtype != RCBF_F32 && p->decoded_dtype != RCBF_F16 &&
        p->decoded_dtype != RCBF_CF32)
        return set_error(RCBF_EUNSUPPORTED, "rcbf_plan: decoded_dtype must be RCBF_I32, RCBF_F32, RCBF_F16 or RCBF_CF32");
    if (p->decode_variant > RCBF_DECODE_TC || p->das_variant > RCBF_DAS_PLAIN)
        return set_error(RCBF_EUNSUPPORTED, "rcbf_plan: unknown variant");
    if (p->hadamard_order) {
        if (p->hadamard_order != p->n_tx)
            return set_error(RCBF_EINVAL, "rcbf_plan: hadamard_order must equal n_tx");
        if (p->decoded_dtype == RCBF_CF32 && p->demod_decimation == 0)
            return set_error(RCBF_EUNSUPPORTED, "rcbf_plan: complex data is Hadamard-decoded only after rcbf_demodulate "
                                                "(demod_decimation > 0)");
        if (p->demod_decimation && p->decoded_dtype != RCBF_CF32)
            return set_error(RCBF_EUNSUPPORTED, "rcbf_plan: demodulated data decodes to RCBF_CF32");
        if (!p->decode_matrix && !is_pow2(p->n_tx))
            return set_error(RCBF_EINVAL, "rcbf_plan: a Sylvester order must be a power of two");
        if (p->decode_variant != RCBF_DECODE_PLAIN && !(p->n_tx == 32 || p->n_tx == 64 || p->n_tx == 128 || p->n_tx == 256))
            return set_error(RCBF_EUNSUPPORTED, "rcbf_plan: the tensor-core decode needs n_tx in {32, 64, 128, 256}");
        if (p->decode_variant == RCBF_DECODE_TC && !(p->n_tx == 32 || p->n_tx == 64 || p->n_tx == 128))
            return set_error(RCBF_EUNSUPPORTED, "rcbf_plan: the tcgen05 decode needs n_tx in {32, 64, 128}");
        if (p->decode_variant == RCBF_DECODE_PLAIN && p->n_tx % 16)
            return set_error(RCBF_EUNSUPPORTED, "rcbf_plan: the plain decode needs n_tx a multiple of 16");
        if (p->decode_matrix)
            for (uint32_t q = 0; q < p->n_tx * p->n_tx; ++q)
                if (p->decode_matrix[q] != 1 && p->decode_matrix[q] != -1)
                    return set_error(RCBF_EINVAL, "rcbf_plan: decode_matrix entries must be +1 or -1");
    }
    if (p->demod_decimation) {
        if (p->demod_decimation > 16) return set_error(RCBF_EINVAL, "rcbf_plan: demod_decimation must be in [1, 16]");
        if (!p->demod_taps || p->demod_n_taps < 1 || p->demod_n_taps > 1024)
            return set_error(RCBF_EINVAL, "rcbf_plan: demodulation needs 1..1024 taps (demod_taps, demod_n_taps)");
        if (p->demod_shift < 0 || p->demod_shift > 30)
            return set_error(RCBF_EINVAL, "rcbf_plan: demod_shift must be in [0, 30]");
        long long l1 = 0;
        for (uint32_t k = 0; k < p->demod_n_taps; ++k) {
            l1 += std::llabs((long long)p->demod_taps[k]);
            if (p->demod_taps_imag) l1 += std::llabs((long long)p->demod_taps_imag[k]);
        }
        if (l1 > 65535) return set_error(RCBF_EINVAL, "rcbf_plan: sum |taps| (real and imaginary parts) must be <= 65535");
        if ((double)p->n_samples * p->demod_decimation > (double)(1u << 24))
            return set_error(RCBF_EINVAL, "rcbf_plan: raw trace too long");
    }
    if (!(p->iq_freq >= 0.0)) return set_error(RCBF_EINVAL, "rcbf_plan: iq_freq must be >= 0");
    if (p->rx_channels_total ? (uint64_t)p->rx_channel_offset + p->n_ch > p->rx_channels_total
                             : p->rx_channel_offset != 0)
        return set_error(RCBF_EINVAL, "rcbf_plan: the channel slice must lie inside rx_channels_total");
    if (p->rx_channels_total && p->acq_kind == RCBF_HERCULES_2D)
        return set_error(RCBF_EUNSUPPORTED, "rcbf_plan: a 2D receive aperture is not sliced by channel");
    if (p->tx_wave > RCBF_TX_POINT) return set_error(RCBF_EINVAL, "rcbf_plan: unknown tx_wave");
    const bool h2d = p->acq_kind == RCBF_HERCULES_2D;
    if (h2d && p->tx_wave != RCBF_TX_PLANE && p->tx_wave != RCBF_TX_POINT)
        return set_error(RCBF_EINVAL, "rcbf_plan: a 2D receive aperture takes one plane or diverging wave");
    if (p->tx_wave == RCBF_TX_POINT && (!h2d || !(p->tx_focus < 0.0)))
        return set_error(RCBF_EINVAL, "rcbf_plan: RCBF_TX_POINT is a virtual point behind a 2D aperture (tx_focus < 0)");
    if (p->tx_wave == RCBF_TX_PLANE) {
        if (!p->tx_angles) return set_error(RCBF_EINVAL, "rcbf_plan: plane waves need tx_angles");
        for (uint32_t i = 0; i < (h2d ? 1u : p->n_tx); ++i)
            if (!(std::fabs(p->tx_angles[i]) < 1.5707963267948966))
                return set_error(RCBF_EINVAL, "rcbf_plan: plane-wave angles must satisfy |angle| < pi/2");
    }
    if (p->tx_wave == RCBF_TX_VLS && !std::isfinite(p->tx_focus))
        return set_error(RCBF_EINVAL, "rcbf_plan: tx_focus must be finite");
    if (p->iq_freq > 0.0 && p->decoded_dtype != RCBF_CF32)
        return set_error(RCBF_EINVAL, "rcbf_plan: IQ beamforming (iq_freq > 0) needs RCBF_CF32 data");
    const bool tile_given = p->tile[0] || p->tile[1] || p->tile[2];
    if (tile_given) {
        if (!(p->tile[0] == 32 || p->tile[0] == 64 || p->tile[0] == 128) ||
            p->tile[1] < 1 || p->tile[2] < 1 || p->tile[0] * p->tile[1] * p->tile[2] != (uint32_t)kTileVoxels)
            return set_error(RCBF_EINVAL, "rcbf_plan: tile must be (32|64|128, a, b) with product 1024");
    }
    return RCBF_OK;
}

// Geometry of a plan (host only, no CUDA call, no allocation): the voxel-index
// to array-frame affine, the lane axis, the DAS argument block and the tile.
void setup_geometry(PlanHost& h) {
    const rcbf_params& p = h.p;
    // ---- geometry: voxel index -> world (M), world -> array (X), G = X M
    double M[16] = {0}, X[16] = {0}, G[12];
    if (!all_zero(p.voxel_transform, 16)) {
        std::memcpy(M, p.voxel_transform, sizeof(M));
    } else {
        for (int d = 0; d < 3; ++d) {
            const double step = p.out_dims[d] > 1 ? (p.out_max[d] - p.out_min[d]) / (double)(p.out_dims[d] - 1) : 0.0;
            M[d * 4 + d] = step;
            M[d * 4 + 3] = p.out_min[d];
        }
        M[15] = 1.0;
    }
    if (!all_zero(p.xdc_transform, 16)) std::memcpy(X, p.xdc_transform, sizeof(X));
    else { X[0] = X[5] = X[10] = X[15] = 1.0; }
    mat_mul_3x4(X, M, G);

    const int tx_axis = p.tx_orientation == RCBF_ROWS ? 1 : 0;
    const int rx_axis = p.rx_orientation == RCBF_ROWS ? 1 : 0;
    // lane axis u: an index axis along which neither the transmit lateral
    // coordinate nor z changes (then the transmit delay depends on tile rows only)
    auto tx_invariant = [&](int ax) {
        const double scale = std::fabs(G[ax]) + std::fabs(G[4 + ax]) + std::fabs(G[8 + ax]);
        return std::fabs(G[tx_axis * 4 + ax]) <= 1e-12 * scale && std::fabs(G[8 + ax]) <= 1e-12 * scale;
    };
    int ua = -1;
    for (int ax = 0; ax < 2 && ua < 0; ++ax) if (tx_invariant(ax) && p.out_dims[ax] > 1) ua = ax;
    for (int ax = 0; ax < 2 && ua < 0; ++ax) if (tx_invariant(ax)) ua = ax;
    h.tiled_ok = ua >= 0 && p.n_ch % kCJ == 0 && p.n_tx % (p.decoded_dtype == RCBF_CF32 ? 4 : kCI) == 0;
    const bool h2d = p.acq_kind == RCBF_HERCULES_2D;
    if (h2d) {
        // the tiled 2D form takes no F# window (its weight is radial, per
        // (i, j)), needs the rows and columns along different axes, and
        // holds one voxel per thread along u
        h.force_plain = p.f_number > 0.0 || tx_axis == rx_axis || (p.tile[0] && p.tile[0] != 32);
    }
    if (ua < 0) ua = 0;
    const int va = 1 - ua;
    h.swap_uv = ua == 1;

    DasArgs& a = h.das;
    std::memset(&a, 0, sizeof(a));
    for (int d = 0; d < 3; ++d) {
        a.q0[d] = G[d * 4 + 3];
        a.Gu[d] = G[d * 4 + ua];
        a.Gv[d] = G[d * 4 + va];
        a.Gw[d] = G[d * 4 + 2];
    }
    const long long strides[3] = {1, (long long)p.out_dims[0], (long long)p.out_dims[0] * p.out_dims[1]};
    a.n_u = (int)p.out_dims[ua];
    a.n_v = (int)p.out_dims[va];
    a.n_w = (int)p.out_dims[2];
    a.out_su = strides[ua];
    a.out_sv = strides[va];
    a.out_sw = strides[2];
    a.n_tx = (int)p.n_tx;
    a.n_ch = (int)p.n_ch;
    a.n_s = (int)p.n_samples;
    a.tx_axis = tx_axis;
    a.rx_axis = rx_axis;
    a.tx_pitch = p.tx_pitch;
    a.rx_pitch = p.rx_pitch;
    a.tx_e0 = -0.5 * (double)(p.n_tx - 1) * p.tx_pitch;
    const uint32_t rx_total = p.rx_channels_total ? p.rx_channels_total : p.n_ch;
    a.rx_e0 = (-0.5 * (double)(rx_total - 1) + (double)p.rx_channel_offset) * p.rx_pitch;
    a.fs = p.fs;
    a.f_number = (float)p.f_number;
    a.iq_ratio = p.iq_freq / p.fs;
    a.tx_wave = (int)p.tx_wave;
    a.acq_kind = (int)p.acq_kind;
    a.tx_focus = p.tx_focus;
    a.tx_dir = nullptr;        // device directions, set by rcbf_plan
    a.interp = (int)p.interp;
    a.dtype = (int)p.decoded_dtype;
    a.scale = p.decoded_dtype == RCBF_I32 ? 1.0f / (float)p.n_tx : 1.0f;
    a.plane_stride = (long long)p.n_tx * p.n_ch * p.n_samples;
    a.image_plane = (long long)p.out_dims[0] * p.out_dims[1] * p.out_dims[2];
    a.wait_ns = kWaitNs;
    a.withhold = 0;

    // ---- DAS tile: given, or the shape with the smallest window at the plan's c
    auto radius_sum = [&](int bu, int bv, int bw) {
        return tile_radius(G, tx_axis, ua, va, bu, bv, bw) + tile_radius(G, rx_axis, ua, va, bu, bv, bw);
    };
    // 2D receive aperture: the receive path spans at most the tile's
    // bounding-box diagonal; the transmit wave's path spans, over a tile's
    // box, |cos a| 2 h_z + |sin a| 2 h_lat (plane) or the largest difference
    // between the farthest corner and the nearest point from the virtual
    // source (diverging wave, over every tile of the image)
    auto half_ext = [&](int d, int bu, int bv, int bw) {
        return 0.5 * (std::fabs(G[d * 4 + ua]) * (bu - 1) + std::fabs(G[d * 4 + va]) * (bv - 1) +
                      std::fabs(G[d * 4 + 2]) * (bw - 1));
    };
    auto box_diag = [&](int bu, int bv, int bw) {
        double e2 = 0.0;
        for (int d = 0; d < 3; ++d) e2 += 4.0 * half_ext(d, bu, bv, bw) * half_ext(d, bu, bv, bw);
        return std::sqrt(e2);
    };
    auto wave_spread = [&](int bu, int bv, int bw) {
        const double hx = half_ext(0, bu, bv, bw), hy = half_ext(1, bu, bv, bw), hz = half_ext(2, bu, bv, bw);
        if (p.tx_wave == RCBF_TX_PLANE) {
            const double ang = h.tx_angle0;
            const double cs = h.has_tx_angle0 ? std::fabs(std::cos(ang)) : 1.0;
            const double sn = h.has_tx_angle0 ? std::fabs(std::sin(ang)) : 1.0;
            return 2.0 * (cs * hz + sn * (tx_axis ? hy : hx));
        }
        const long long tu = ((long long)p.out_dims[ua] + bu - 1) / bu, tv = ((long long)p.out_dims[va] + bv - 1) / bv;
        const long long tw = ((long long)p.out_dims[2] + bw - 1) / bw;
        double spread = 0.0;
        for (long long w = 0; w < tw; ++w)
            for (long long v = 0; v < tv; ++v)
                for (long long u = 0; u < tu; ++u) {
                    const double cu = u * bu + 0.5 * (bu - 1), cv = v * bv + 0.5 * (bv - 1), cw = w * bw + 0.5 * (bw - 1);
                    double q[3];
                    for (int d = 0; d < 3; ++d) q[d] = G[d * 4 + 3] + G[d * 4 + ua] * cu + G[d * 4 + va] * cv + G[d * 4 + 2] * cw;
                    const double zf = std::fabs(q[2] - p.tx_focus);
                    const double nx = std::fmax(std::fabs(q[0]) - hx, 0.0), ny = std::fmax(std::fabs(q[1]) - hy, 0.0);
                    const double nz = std::fmax(zf - hz, 0.0);
                    const double fx = std::fabs(q[0]) + hx, fy = std::fabs(q[1]) + hy, fz = zf + hz;
                    spread = std::fmax(spread, std::sqrt(fx * fx + fy * fy + fz * fz) - std::sqrt(nx * nx + ny * ny + nz * nz));
                }
        return spread;
    };
    int best_bu = 64, best_bv = 1, best_bw = 16;
    if (h2d && !p.tile[0]) {
        const double spm = p.fs / p.c;
        double best_key = 1e300;
        best_bu = 32;
        for (int bv = 1; bv <= 32; bv *= 2) {
            const int bw = 32 / bv;
            if (bv > 1 && a.n_v == 1) continue;
            const double W = std::floor(4.0 + (box_diag(32, bv, bw) + wave_spread(32, bv, bw)) * spm + 0.02) + 1.0;
            const double cls = W <= 64 ? 0.0 : W <= 96 ? 1.0 : W <= 128 ? 2.0 : 3.0;
            const double key = cls * 1e6 + W;
            if (key < best_key) { best_key = key; best_bv = bv; best_bw = bw; }
        }
    } else if (p.tile[0]) {
        best_bu = (int)p.tile[0];
        best_bv = (int)p.tile[1];
        best_bw = (int)p.tile[2];
    } else {
        // window length (in samples) of a shape at the plan's speed of sound;
        // prefer the smallest window class (48, 64, 128 intervals: larger
        // stages), then more voxels per thread along u (fewer transmit-term
        // loads per sum), then the shorter window
        const double spm = p.fs / p.c;
        double best_key = 1e300;
        const int bus[3] = {128, 64, 32};
        for (int bi = 0; bi < 3; ++bi) {
            const int bu = bus[bi];
            const int rows = kTileVoxels / bu;
            for (int bv = 1; bv <= rows; bv *= 2) {
                const int bw = rows / bv;
                if (bv > 1 && a.n_v == 1) continue;
                const double W = std::floor(4.0 + 2.0 * radius_sum(bu, bv, bw) * spm + 0.01) + 1.0;
                const double cls = W <= 48 ? 0.0 : W <= 64 ? 1.0 : W <= 128 ? 2.0 : 3.0;
                const double key = cls * 1e6 + (cls < 2 ? (128 - bu) * 100.0 : 0.0) + W;
                if (key < best_key) { best_key = key; best_bu = bu; best_bv = bv; best_bw = bw; }
            }
        }
    }
    h.vu = best_bu / 32;
    a.bu = best_bu;
    a.bv = best_bv;
    a.bw = best_bw;
    a.tiles_u = (a.n_u + a.bu - 1) / a.bu;
    a.tiles_v = (a.n_v + a.bv - 1) / a.bv;
    a.tiles_w = (a.n_w + a.bw - 1) / a.bw;
    h.r_alpha_m = tile_radius(G, tx_axis, ua, va, a.bu, a.bv, a.bw);
    h.r_beta_m = tile_radius(G, rx_axis, ua, va, a.bu, a.bv, a.bw);
    if (h2d) {
        h.r_alpha_m = wave_spread(a.bu, a.bv, a.bw);    // the 2D form's transmit spread [m]
        h.r_beta_m = 0.0;
    }

    // adjoint tile: 32 voxels along u by 32 rows, lanes over the rows with z
    // fastest; the most z-rows whose window stays within 128 samples
    h.bwd_bv = h.bwd_bw = 0;
    h.bwd_r_alpha_m = h.bwd_r_beta_m = 0.0;
    for (int bv = 1; bv <= 4; bv *= 2) {
        const int bw = 32 / bv;
        if (bv > 1 && a.n_v == 1) break;
        const double ra = tile_radius(G, tx_axis, ua, va, 32, bv, bw);
        const double rb = tile_radius(G, rx_axis, ua, va, 32, bv, bw);
        if (std::floor(4.0 + 2.0 * (ra + rb) * p.fs / p.c + 0.01) + 1.0 <= 128.0) {
            h.bwd_bv = bv;
            h.bwd_bw = bw;
            h.bwd_r_alpha_m = ra;
            h.bwd_r_beta_m = rb;
            break;
        }
    }

    if (p.tx_wave == RCBF_TX_VLS) {
        // off the line's axis the virtual-line-source delay jumps by 2 |lat - e|
        // at the focal depth (converging above, diverging below), so tile
        // windows from the 1-Lipschitz radius bound hold only for tiles whose
        // whole box (ragged tiles included: the reference sits at the centre
        // of the full tile) lies on one side of it. The test is the kernels'
        // own (tile_across_focus), over every tile of the forward and of the
        // adjoint tiling.
        auto any_across = [&](int bu, int bv, int bw) {
            if (bv <= 0) return false;
            const long long tu_n = (a.n_u + bu - 1) / bu, tv_n = (a.n_v + bv - 1) / bv, tw_n = (a.n_w + bw - 1) / bw;
            const double hz = 0.5 * (std::fabs(a.Gu[2]) * (bu - 1) + std::fabs(a.Gv[2]) * (bv - 1) +
                                     std::fabs(a.Gw[2]) * (bw - 1));
            for (long long tw = 0; tw < tw_n; ++tw)
                for (long long tv = 0; tv < tv_n; ++tv)
                    for (long long tu = 0; tu < tu_n; ++tu) {
                        const double cu = tu * bu + 0.5 * (bu - 1), cv = tv * bv + 0.5 * (bv - 1),
                                     cw = tw * bw + 0.5 * (bw - 1);
                        const double zc = a.q0[2] + a.Gu[2] * cu + a.Gv[2] * cv + a.Gw[2] * cw;
                        if (std::fabs(p.tx_focus - zc) <= hz + 1e-9) return true;
                    }
            return false;
        };
        h.vls_split = any_across(a.bu, a.bv, a.bw);
        h.vls_split_bwd = any_across(32, h.bwd_bv, h.bwd_bw);
    }
}

}  // namespace

int plan_validate(const rcbf_params* p) { return validate(p); }
void plan_geometry(PlanHost& h) { setup_geometry(h); }

}  // namespace rcbf

using namespace rcbf;

extern "C" {

const char* rcbf_last_error(void) { return g_last_error.c_str(); }

const char* rcbf_version(void) { return "rcbf 0.1 (sm_103a)"; }

int rcbf_plan(const rcbf_params* params, rcbf_plan_t* out_plan) {
    g_last_error.clear();
    if (!out_plan) return set_error(RCBF_EINVAL, "rcbf_plan: out_plan is NULL");
    *out_plan = nullptr;
    int rc = validate(params);
    if (rc != RCBF_OK) return rc;

    rcbf_plan_s* plan = new rcbf_plan_s();
    PlanHost& h = plan->h;
    h.p = *params;
    h.p.decode_matrix = nullptr;   // the matrix is copied, never referenced later
    h.p.demod_taps = nullptr;      // so are the taps
    h.p.demod_taps_imag = nullptr;
    h.p.tx_angles = nullptr;       // and the plane-wave angles
    h.has_tx_angle0 = params->tx_angles != nullptr;
    h.tx_angle0 = params->tx_angles ? params->tx_angles[0] : 0.0;
    const rcbf_params& p = h.p;

    setup_geometry(h);
    DasArgs& a = h.das;

    // ---- device tables
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&h.n_sms, cudaDevAttrMultiProcessorCount, dev);
    auto fail = [&](int code, const std::string& msg) {
        rcbf_destroy(plan);
        return set_error(code, msg);
    };
    if (cudaMalloc(&h.d_status, sizeof(int)) != cudaSuccess) return fail(RCBF_ENOMEM, "rcbf_plan: cudaMalloc status");
    if (cudaMemset(h.d_status, 0, sizeof(int)) != cudaSuccess) return fail(RCBF_ECUDA, "rcbf_plan: cudaMemset");
    a.status = h.d_status;
    if (p.tx_wave == RCBF_TX_PLANE) {
        std::vector<float2> dir(p.n_tx);
        for (uint32_t i = 0; i < p.n_tx; ++i) {
            const double ang = params->tx_angles[p.acq_kind == RCBF_HERCULES_2D ? 0 : i];   // 2D: one wave
            dir[i] = make_float2((float)std::sin(ang), (float)std::cos(ang));
        }
        if (cudaMalloc(&h.d_tx_dir, dir.size() * sizeof(float2)) != cudaSuccess)
            return fail(RCBF_ENOMEM, "rcbf_plan: cudaMalloc directions");
        if (cudaMemcpy(h.d_tx_dir, dir.data(), dir.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(RCBF_ECUDA, "rcbf_plan: copy directions");
        a.tx_dir = h.d_tx_dir;
    }
    if (p.demod_decimation) {
        const size_t bytes = (size_t)p.demod_n_taps * sizeof(int16_t);
        if (cudaMalloc(&h.d_taps, bytes) != cudaSuccess) return fail(RCBF_ENOMEM, "rcbf_plan: cudaMalloc taps");
        if (cudaMemcpy(h.d_taps, params->demod_taps, bytes, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(RCBF_ECUDA, "rcbf_plan: copy taps");
        if (params->demod_taps_imag) {
            if (cudaMalloc(&h.d_taps_im, bytes) != cudaSuccess) return fail(RCBF_ENOMEM, "rcbf_plan: cudaMalloc taps");
            if (cudaMemcpy(h.d_taps_im, params->demod_taps_imag, bytes, cudaMemcpyHostToDevice) != cudaSuccess)
                return fail(RCBF_ECUDA, "rcbf_plan: copy taps");
        }
    }
    if (p.hadamard_order) {
        const int n = (int)p.n_tx;
        std::vector<int8_t> H((size_t)n * n);
        if (params->decode_matrix) std::memcpy(H.data(), params->decode_matrix, H.size());
        else
            for (int k = 0; k < n; ++k)
                for (int i = 0; i < n; ++i) H[(size_t)k * n + i] = (__builtin_popcount((unsigned)(k & i)) & 1) ? -1 : 1;
        if (cudaMalloc(&h.d_hmat, H.size()) != cudaSuccess) return fail(RCBF_ENOMEM, "rcbf_plan: cudaMalloc H");
        if (cudaMemcpy(h.d_hmat, H.data(), H.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(RCBF_ECUDA, "rcbf_plan: copy H");
        if (n % 32 == 0) {
            const std::vector<uint32_t> fr = build_afrag(H, n);
            if (cudaMalloc(&h.d_afrag, fr.size() * 4) != cudaSuccess) return fail(RCBF_ENOMEM, "rcbf_plan: cudaMalloc fragments");
            if (cudaMemcpy(h.d_afrag, fr.data(), fr.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
                return fail(RCBF_ECUDA, "rcbf_plan: copy fragments");
            const std::vector<uint32_t> f16 = build_afrag16(H, n);
            if (cudaMalloc(&h.d_afrag16, f16.size() * 4) != cudaSuccess) return fail(RCBF_ENOMEM, "rcbf_plan: cudaMalloc fragments");
            if (cudaMemcpy(h.d_afrag16, f16.data(), f16.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
                return fail(RCBF_ECUDA, "rcbf_plan: copy fragments");
            std::vector<int> hs(n, 0);
            for (int k = 0; k < n; ++k)
                for (int i = 0; i < n; ++i) hs[i] += H[(size_t)k * n + i];
            if (cudaMalloc(&h.d_hsum, hs.size() * 4) != cudaSuccess) return fail(RCBF_ENOMEM, "rcbf_plan: cudaMalloc sums");
            if (cudaMemcpy(h.d_hsum, hs.data(), hs.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
                return fail(RCBF_ECUDA, "rcbf_plan: copy sums");
            if (n <= 128) {
                const std::vector<uint16_t> at = build_a_tc(H, n);
                if (cudaMalloc(&h.d_atc, at.size() * 2) != cudaSuccess) return fail(RCBF_ENOMEM, "rcbf_plan: cudaMalloc A");
                if (cudaMemcpy(h.d_atc, at.data(), at.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess)
                    return fail(RCBF_ECUDA, "rcbf_plan: copy A");
            }
        }
        if ((rc = configure_decode(h)) != RCBF_OK) { std::string m = g_last_error; rcbf_destroy(plan); return set_error(rc, m); }
        if (p.demod_decimation && (rc = configure_demod_decode(h)) != RCBF_OK) {
            std::string m = g_last_error;
            rcbf_destroy(plan);
            return set_error(rc, m);
        }
    }
    if ((rc = configure_das(h)) != RCBF_OK) { std::string m = g_last_error; rcbf_destroy(plan); return set_error(rc, m); }
    {
        const int sp = std::max(std::max(das_slices(h, 0), das_slices(h, 1)), std::max(das_slices(h, 2), das_slices(h, 3)));
        if (sp > 1) {
            h.partial_floats = (size_t)sp * a.image_plane * (p.decoded_dtype == RCBF_CF32 ? 2 : 1);
            if (cudaMalloc(&h.d_partial, h.partial_floats * sizeof(float)) != cudaSuccess)
                return fail(RCBF_ENOMEM, "rcbf_plan: cudaMalloc partial images");
        }
    }
    *out_plan = plan;
    return RCBF_OK;
}

int rcbf_plan_query(rcbf_plan_t plan, rcbf_plan_info* info) {
    if (!plan || !info) return set_error(RCBF_EINVAL, "rcbf_plan_query: NULL argument");
    const PlanHost& h = plan->h;
    std::memset(info, 0, sizeof(*info));
    info->tile[0] = (uint32_t)h.das.bu;
    info->tile[1] = (uint32_t)h.das.bv;
    info->tile[2] = (uint32_t)h.das.bw;
    DasArgs a;
    std::string why;
    const bool fits = das_prepare(h, h.p.c, &a, &why) == RCBF_OK;
    const bool tiled = h.p.das_variant == RCBF_DAS_TILED && h.tiled_ok && fits;
    info->tiled = tiled ? 1u : 0u;
    info->window = (uint32_t)a.W;
    const int cls = das_class_index(a.W, h.p.acq_kind == RCBF_HERCULES_2D);
    const int sp = tiled ? std::max(1, h.n_split[cls]) : 1;
    info->n_split = (uint32_t)sp;
    info->das_launches = tiled && das_slices(h, cls) > 1 ? 2u : 1u;
    info->decode_launches = h.p.hadamard_order ? (h.p.decoded_dtype == RCBF_CF32 ? 2u : 1u) : 0u;
    uint64_t bytes = sizeof(int) + h.partial_floats * sizeof(float);
    if (h.p.hadamard_order) {
        const uint64_t n = h.p.n_tx;
        bytes += n * n + n * sizeof(int);
        if (n % 32 == 0) bytes += 2 * (n / 16) * (n / 32) * 32 * 16 + (n / 16) * (n / 16) * 32 * 16 / 2;
    }
    if (h.p.demod_decimation) bytes += (uint64_t)h.p.demod_n_taps * sizeof(int16_t) * (h.d_taps_im ? 2 : 1);
    info->workspace_bytes = bytes;
    int mode = 0;
    DasArgs b = a;
    if (h.p.das_variant == RCBF_DAS_TILED && h.tiled_ok) {
        if (!h.vls_split_bwd && h.bwd_bv > 0 &&
            das_prepare_tile(h, h.p.c, 32, h.bwd_bv, h.bwd_bw, h.bwd_r_alpha_m, h.bwd_r_beta_m, &b, &why) == RCBF_OK)
            mode = 2;
        else if (!h.vls_split && fits)
            mode = 1;
    }
    info->bwd_mode = (uint32_t)mode;
    info->bwd_tile[0] = mode == 2 ? 32u : (uint32_t)h.das.bu;
    info->bwd_tile[1] = mode == 2 ? (uint32_t)h.bwd_bv : (uint32_t)h.das.bv;
    info->bwd_tile[2] = mode == 2 ? (uint32_t)h.bwd_bw : (uint32_t)h.das.bw;
    return RCBF_OK;
}

void rcbf_destroy(rcbf_plan_t plan) {
    if (!plan) return;
    PlanHost& h = plan->h;
    if (h.d_afrag) cudaFree(h.d_afrag);
    if (h.d_hmat) cudaFree(h.d_hmat);
    if (h.d_afrag16) cudaFree(h.d_afrag16);
    if (h.d_hsum) cudaFree(h.d_hsum);
    if (h.d_atc) cudaFree(h.d_atc);
    if (h.d_status) cudaFree(h.d_status);
    if (h.d_partial) cudaFree(h.d_partial);
    if (h.d_taps) cudaFree(h.d_taps);
    if (h.d_taps_im) cudaFree(h.d_taps_im);
    if (h.d_tx_dir) cudaFree(h.d_tx_dir);
    delete plan;
}

int rcbf_demodulate(rcbf_plan_t plan, const int16_t* rf, int16_t* iq, void* stream) {
    if (!plan) return set_error(RCBF_EINVAL, "rcbf_demodulate: plan is NULL");
    const PlanHost& h = plan->h;
    if (!h.p.demod_decimation) return set_error(RCBF_EINVAL, "rcbf_demodulate: the plan has no demodulation");
    if (!rf || !iq) return set_error(RCBF_EINVAL, "rcbf_demodulate: NULL buffer");
    if (!aligned16(rf) || !aligned16(iq)) return set_error(RCBF_EINVAL, "rcbf_demodulate: buffers must be 16-byte aligned");
    return launch_demodulate(h, rf, iq, static_cast<cudaStream_t>(stream));
}

int rcbf_decode(rcbf_plan_t plan, const int16_t* rf, void* decoded, void* stream) {
    if (!plan) return set_error(RCBF_EINVAL, "rcbf_decode: plan is NULL");
    const PlanHost& h = plan->h;
    if (!h.p.hadamard_order) return set_error(RCBF_EINVAL, "rcbf_decode: the plan has no Hadamard order");
    if (!rf || !decoded) return set_error(RCBF_EINVAL, "rcbf_decode: NULL buffer");
    if (!aligned16(rf) || !aligned16(decoded)) return set_error(RCBF_EINVAL, "rcbf_decode: buffers must be 16-byte aligned");
    return launch_decode(h, rf, decoded, static_cast<cudaStream_t>(stream));
}

int rcbf_demod_decode(rcbf_plan_t plan, const int16_t* rf, float* decoded, void* stream) {
    if (!plan) return set_error(RCBF_EINVAL, "rcbf_demod_decode: plan is NULL");
    const PlanHost& h = plan->h;
    if (!rf || !decoded) return set_error(RCBF_EINVAL, "rcbf_demod_decode: NULL buffer");
    if (!aligned16(rf) || !aligned16(decoded))
        return set_error(RCBF_EINVAL, "rcbf_demod_decode: buffers must be 16-byte aligned");
    std::string why;
    if (!demod_decode_supported(h, &why)) return set_error(RCBF_EUNSUPPORTED, why);
    return launch_demod_decode(h, rf, decoded, static_cast<cudaStream_t>(stream));
}

int rcbf_das(rcbf_plan_t plan, const void* decoded, const float* apod, float c, float* image, void* stream) {
    if (!plan) return set_error(RCBF_EINVAL, "rcbf_das: plan is NULL");
    const PlanHost& h = plan->h;
    if (!decoded || !image) return set_error(RCBF_EINVAL, "rcbf_das: NULL buffer");
    if (!aligned16(decoded) || !aligned4(image) || (apod && !aligned4(apod)))
        return set_error(RCBF_EINVAL, "rcbf_das: decoded must be 16-byte aligned, image and apod 4-byte aligned");
    const double cc = c > 0.f ? (double)c : h.p.c;
    DasArgs a;
    std::string why;
    const bool tiled = h.p.das_variant == RCBF_DAS_TILED;
    if (tiled && !h.tiled_ok)
        return set_error(RCBF_EUNSUPPORTED, "rcbf_das: the tiled form needs n_ch % 8 == 0, n_tx % 8 == 0 "
                                            "(4 for complex) and an image axis parallel to the transmit elements");
    // a grid so coarse that a 1024-voxel tile reaches more than 128 samples
    // of a trace runs the plain GPU form (same result within the bound)
    const bool fits = das_prepare(h, cc, &a, &why) == RCBF_OK;
    a.rf = decoded;
    a.apod = apod;
    a.image = image;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!(tiled && fits)) return launch_das_plain(h, a, s);
    if (!h.vls_split) return launch_das(h, a, s);
    // VLS focal plane inside the image: the tiled form for every tile but
    // those across the focal depth, then the plain form for exactly those
    a.vls_split = 1;
    const int rc = launch_das(h, a, s);
    return rc != RCBF_OK ? rc : launch_das_plain(h, a, s);
}

int rcbf_das_backward(rcbf_plan_t plan, const void* decoded, const float* apod, float c,
                      const float* grad_image, float* grad_rf, float* grad_c, float* grad_apod, void* stream) {
    if (!plan) return set_error(RCBF_EINVAL, "rcbf_das_backward: plan is NULL");
    const PlanHost& h = plan->h;
    if (!decoded || !grad_image) return set_error(RCBF_EINVAL, "rcbf_das_backward: NULL buffer");
    if (!aligned16(decoded) || !aligned4(grad_image) || (grad_rf && !aligned4(grad_rf)) ||
        (grad_c && !aligned4(grad_c)) || (grad_apod && !aligned4(grad_apod)) || (apod && !aligned4(apod)))
        return set_error(RCBF_EINVAL, "rcbf_das_backward: decoded must be 16-byte aligned, float buffers 4-byte aligned");
    if (h.p.decoded_dtype != RCBF_F32 && h.p.decoded_dtype != RCBF_CF32)
        return set_error(RCBF_EUNSUPPORTED, "rcbf_das_backward: decoded_dtype must be RCBF_F32 or RCBF_CF32");
    if (h.p.interp != RCBF_LINEAR || h.p.iq_freq > 0.0 || h.p.acq_kind == RCBF_HERCULES_2D)
        return set_error(RCBF_EUNSUPPORTED, "rcbf_das_backward: the adjoint is built for separable RF data with "
                                            "linear interpolation");
    const double cc = c > 0.f ? (double)c : h.p.c;
    DasArgs a;
    std::string why;
    // the adjoint's own tile (lanes over z) where its window fits at this
    // speed of sound, else the plan's tile, else the plain form
    // (a VLS focal plane inside the image: the plain form throughout)
    int mode = 0;
    if (h.p.das_variant == RCBF_DAS_TILED && h.tiled_ok) {
        if (!h.vls_split_bwd && h.bwd_bv > 0 &&
            das_prepare_tile(h, cc, 32, h.bwd_bv, h.bwd_bw, h.bwd_r_alpha_m, h.bwd_r_beta_m, &a, &why) == RCBF_OK)
            mode = 2;
        else if (!h.vls_split && das_prepare(h, cc, &a, &why) == RCBF_OK)
            mode = 1;
    }
    if (mode == 0) das_prepare(h, cc, &a, &why);
    a.rf = decoded;
    a.apod = apod;
    a.grad_image = grad_image;
    a.grad_rf = grad_rf;
    a.grad_c = grad_c;
    a.grad_apod = grad_apod;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int planes = h.p.decoded_dtype == RCBF_CF32 ? 2 : 1;
    if (grad_rf && cudaMemsetAsync(grad_rf, 0, (size_t)a.plane_stride * planes * sizeof(float), s) != cudaSuccess)
        return check_launch("rcbf_das_backward: clear grad_rf");
    if (grad_c && cudaMemsetAsync(grad_c, 0, sizeof(float), s) != cudaSuccess)
        return check_launch("rcbf_das_backward: clear grad_c");
    if (grad_apod && cudaMemsetAsync(grad_apod, 0, (size_t)h.p.n_ch * sizeof(float), s) != cudaSuccess)
        return check_launch("rcbf_das_backward: clear grad_apod");
    return launch_das_backward(h, a, mode, s);
}

int rcbf_plan_status(rcbf_plan_t plan, void* stream) {
    if (!plan) return set_error(RCBF_EINVAL, "rcbf_plan_status: plan is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return check_launch("rcbf_plan_status: synchronize");
    int st = 0;
    if (cudaMemcpy(&st, plan->h.d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return check_launch("rcbf_plan_status: read status");
    if (!st) return RCBF_OK;
    if (cudaMemset(plan->h.d_status, 0, sizeof(int)) != cudaSuccess) return check_launch("rcbf_plan_status: clear status");
    return set_error(RCBF_ETIMEOUT, "rcbf_plan_status: a bounded device wait of the plan's kernels expired since the "
                                    "last status read; that call's output is incomplete");
}

int rcbf_plan_set_wait(rcbf_plan_t plan, uint64_t wait_ns, int32_t withhold) {
    if (!plan) return set_error(RCBF_EINVAL, "rcbf_plan_set_wait: plan is NULL");
    if (wait_ns == 0 || (withhold != 0 && withhold != 1))
        return set_error(RCBF_EINVAL, "rcbf_plan_set_wait: wait_ns must be > 0 and withhold 0 or 1");
    plan->h.das.wait_ns = (long long)std::min<uint64_t>(wait_ns, (uint64_t)10000000000ULL);
    plan->h.das.withhold = withhold;
    return RCBF_OK;
}

}  // extern "C"

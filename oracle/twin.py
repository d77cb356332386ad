"""Pure-Python brute-force twin of the C oracle, for tiny inputs only.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``). It restates
the same definitions with Python scalars and explicit loops so that the C
oracle can be checked against an independent transcription:

* decode: D[i][c] = sum_k H[k][i] S[k][c] with H[k][i] = (-1)^popcount(k & i)
  (§THEORY "Synthetic Aperture Imaging").
* DAS: Eq. (1) with a_tx = 1, receive apodization Eq. (2) and the Hanning
  window Eq. (3); linear interpolation at s = (ToF - t0) fs, zero outside.
"""
from __future__ import annotations

import math


def hadamard(n):
    return [[-1 if bin(k & i).count("1") % 2 else 1 for i in range(n)] for k in range(n)]


def decode(S, H=None):
    """S: nested lists [n][cols] of ints -> D [n][cols] ints."""
    n = len(S)
    H = hadamard(n) if H is None else H
    cols = len(S[0])
    return [[sum(H[k][i] * S[k][c] for k in range(n)) for c in range(cols)] for i in range(n)]


def _positions(g, ix, iy, iz):
    idx = (ix, iy, iz)
    p = []
    for d in range(3):
        if g.out_dims[d] > 1:
            p.append(g.out_min[d] + idx[d] * (g.out_max[d] - g.out_min[d]) / (g.out_dims[d] - 1))
        else:
            p.append(g.out_min[d])
    return p


def _lat(p, orientation):
    return p[1] if orientation == 0 else p[0]


def _window(fnum, delta, z):
    if fnum <= 0:
        return 1.0
    a = fnum * abs(delta)
    if not (a < 0.5 * abs(z)):
        return 0.0
    return math.cos(math.pi * a / abs(z)) ** 2


def _lerp(trace, s):
    n = math.floor(s)
    f = s - n
    ns = len(trace)
    a = trace[n] if 0 <= n < ns else 0.0
    b = trace[n + 1] if 0 <= n + 1 < ns else 0.0
    return (1 - f) * a + f * b


def das(g, rf, w=None, c=None):
    """rf: nested lists / array [n_tx][n_ch][n_s] of floats. Returns a flat
    list over voxels (x fastest, then y, then z)."""
    c = g.c if c is None else c
    out = []
    for iz in range(g.out_dims[2]):
        for iy in range(g.out_dims[1]):
            for ix in range(g.out_dims[0]):
                p = _positions(g, ix, iy, iz)
                acc = 0.0
                for i in range(g.n_tx):
                    ei = (i - (g.n_tx - 1) / 2) * g.tx_pitch
                    dt = math.sqrt((_lat(p, g.tx_orientation) - ei) ** 2 + p[2] ** 2)
                    for j in range(g.n_ch):
                        ej = (j - (g.n_ch - 1) / 2) * g.rx_pitch
                        delta = _lat(p, g.rx_orientation) - ej
                        dr = math.sqrt(delta ** 2 + p[2] ** 2)
                        a = (1.0 if w is None else float(w[j])) * _window(g.f_number, delta, p[2])
                        s = ((dt + dr) / c - g.t0) * g.fs
                        acc += a * _lerp(rf[i][j], s)
                out.append(acc)
    return out

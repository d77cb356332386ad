"""Cached synthetic frames and small helpers shared by the GPU tests."""
import functools

import numpy as np

import synth


@functools.lru_cache(maxsize=None)
def frame(name: str):
    return {
        "tiny": lambda: synth.tiny_bscan(1),
        "bscan": lambda: synth.full_bscan(2),
        "volume": lambda: synth.hercules_volume(3),
        "autofocus": lambda: synth.autofocus(5),
    }[name]()


def rel_l2(got, want) -> float:
    got = np.asarray(got, dtype=np.complex128 if np.iscomplexobj(want) else np.float64)
    want = np.asarray(want)
    return float(np.linalg.norm((got - want).ravel()) / np.linalg.norm(np.asarray(want).ravel()))


def sample_voxels(dims, count: int, seed: int) -> np.ndarray:
    """Random voxel indices plus the eight corners of the grid."""
    nx, ny, nz = dims
    n = nx * ny * nz
    rng = np.random.default_rng(seed)
    corners = [((z * ny) + y) * nx + x for z in (0, nz - 1) for y in (0, ny - 1) for x in (0, nx - 1)]
    vox = np.unique(np.concatenate([rng.choice(n, size=min(count, n), replace=False), corners]))
    return vox.astype(np.int64)

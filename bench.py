"""Benchmark of the row-column / TOBE beamformer hot path on GB300.

Workload: the FORCES full-aperture B-scan (128 Hadamard-encoded transmits x
128 channels x 4096 int16 samples, 512 x 1024 image, 8.59e9 voxel-channel-
transmit sums per frame), synthetic point-scatterer data. One step = one
batch of B frames (default 4) through the whole path, replayed from one CUDA
graph: the exact Hadamard decode of each frame on the tcgen05 tensor cores
(FP16-stored output), then the tiled DAS (FP32 accumulation) of all frames in
one persistent launch, voxel tile from the autotuner.

Reported: value = whole-job DAS sums/s over the full step (decode included),
frames/s, the same step with the split-byte int8 mma.sync decode inside the
persistent kernel, the forms unbatched (per-kernel CUDA-event times), the
plain FP32 form on the same GPU, the roofline of the dominant kernel and of
the decode, an end-to-end figure through the C ABI with host buffers, clocks
during the timed region, the volume / stream / autofocus configurations, and
the CPU leg (N = 1, rank 0): the FP64 oracle timed on a bounded sample and the
parity stamps of the timed outputs.

--impl reference times the FP64 CPU oracle itself (the reference arm) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "DAS G voxel·chan·tx sums/s & frames/s vs plain FP32 at <=1e-4 rel-L2"
UNIT = "Gsums/s"
WORKLOAD = "FORCES 2D full aperture: 128 tx (H128) x 128 ch x 4096 int16 samples -> 512x1024 FP32 image"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)),
                "src": "of measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "src": "of fallback"}


def recorded_traffic(kernel: str, frames_per_launch: int):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, only
    while the kernel's sources still hash to the value recorded with it."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.md")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    for line in lines:
        if not line.startswith("TRAFFIC %s " % kernel):
            continue
        fields = dict(f.split("=", 1) for f in line.split()[2:])
        if int(fields.get("frames_per_launch", -1)) != frames_per_launch:
            return None
        h = hashlib.sha1()
        for f in fields["files"].split(","):
            with open(os.path.join(ROOT, "paper_2512_11086_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
        return int(fields["bytes_per_launch"]) if h.hexdigest()[:16] == fields["sources"] else None
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(float(r[2]) for r in rows),
                "reasons": reasons, "samples": len(rows)}


def aggregate(local_ms: float, local_units: float, device=None):
    """Whole-job figures of a weak-scaling run: the slowest rank's time and
    the units all ranks processed (each rank beamforms its own frames; the
    only collective is this bookkeeping, never the data path)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return local_ms, local_units
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    u = torch.tensor([local_units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    dist.init_process_group("nccl")
    return rank, ws, local


def cpu_baseline(frame, target_s: float = 15.0, gpu_image=None, gpu_decoded=None):
    """The CPU leg: the FP64 oracle as it stands, timed on a bounded sample of
    the frame (the decode of a slice of columns and the DAS of a random voxel
    subset, both the same fraction phi of the frame, sized to about target_s
    seconds), and, outside its timing, the parity stamp of the GPU's output:
    the decoded frame compared bit for bit with the oracle's decode, and the
    image at the sampled voxels against the oracle's DAS of the same
    FP16-rounded decoded data (the DAS input of the tuned form), plus the
    FP16 storage error against the exact decode on up to 2048 voxels.
    Returns (Gsums/s, details)."""
    import oracle
    g = frame.geometry
    cores = oracle.threads()
    D = _exact_int(frame)                  # inputs of the DAS sample (not timed)
    data16 = oracle.decoded_as(D, g.n_tx, "f16")
    r16 = data16.astype(np.float64)
    rng = np.random.default_rng(0)
    flat = frame.rf.reshape(g.n_tx, -1)
    nv = 256
    while True:
        vox = np.sort(rng.choice(g.n_vox, size=nv, replace=False)).astype(np.int64)
        ncol = max(8, int(round(nv / g.n_vox * flat.shape[1])))
        t0 = time.perf_counter()
        oracle.decode(flat[:, :ncol])
        want = oracle.das(g, r16, voxels=vox)
        t = time.perf_counter() - t0
        if t >= 0.5 * target_s or nv >= g.n_vox:
            break
        nv = min(g.n_vox, int(nv * max(2.0, target_s / max(t, 1e-3))))
    value = nv * g.n_tx * g.n_ch / t / 1e9
    det = {"cores": cores, "seconds": t,
           "sample": "%d of %d voxels (%.4f of the frame) plus the same fraction of the decode "
                     "columns: %.1f s of oracle time" % (nv, g.n_vox, nv / g.n_vox, t)}
    if gpu_image is not None:
        got = np.asarray(gpu_image, dtype=np.float64).ravel()[vox]
        sub = vox[:: max(1, vox.size // 2048)]
        exact = oracle.das(g, D.astype(np.float64) / g.n_tx, voxels=sub)
        det["parity"] = {
            "das_rel_l2": rel_l2(got, want), "das_max_abs": float(np.max(np.abs(got - want))),
            "peak": float(np.max(np.abs(want))), "voxels": int(vox.size), "tol": 1e-4,
            "reference": "FP64 oracle DAS of the FP16-rounded exact decode (the DAS input of the timed form)",
            "fp16_storage_rel_l2": rel_l2(np.asarray(gpu_image, dtype=np.float64).ravel()[sub], exact),
            "decode_bit_exact": None if gpu_decoded is None else
            bool(np.array_equal(np.asarray(gpu_decoded).view(np.uint16), data16.view(np.uint16))),
        }
    return value, det


def rel_l2(got, want) -> float:
    got = np.asarray(got)
    want = np.asarray(want)
    return float(np.linalg.norm((got - want).ravel()) / max(np.linalg.norm(want.ravel()), 1e-300))


_EXACT = {}


def _exact_int(frame):
    """The oracle's exact integer decode of the frame (cached)."""
    key = id(frame)
    if key not in _EXACT:
        import oracle
        _EXACT[key] = oracle.decode(frame.rf)
    return _EXACT[key]


def _exact_decoded(frame):
    return _exact_int(frame).astype(np.float64) / frame.geometry.n_tx


def headline_config(B: int, ws: int) -> dict:
    """The `config` of the headline line, shared by both arms."""
    return {"workload": WORKLOAD, "frames_per_step": B, "global_batch": B * ws,
            "l2": "inputs larger than L2: %d frames of 128 MB int16 RF + 128 MB FP16 decoded per step "
                  "(129 MB L2)" % B,
            "parallelism": "independent frames per GPU" if ws > 1 else "1 GPU"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle timed on the host cores."""
    rank, ws, _ = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), 0
    if rank != 0:
        return
    import oracle
    import synth
    # the default B-scan, or (for the oracle's own timing on the other
    # configurations) the tiny B-scan, the HERCULES volume or the complex
    # autofocus frame; each step times a bounded random voxel sample
    workload = args.workload if args.workload in ("tiny", "volume", "autofocus") else "bscan"
    frame = {"bscan": lambda: synth.full_bscan(seed=2), "tiny": lambda: synth.tiny_bscan(1),
             "volume": lambda: synth.hercules_volume(3), "autofocus": lambda: synth.autofocus(5)}[workload]()
    g = frame.geometry
    oracle.build()
    cores = oracle.threads()
    if frame.rf is not None:
        exact = _exact_decoded(frame)
    else:
        exact = frame.decoded.astype(np.complex128 if np.iscomplexobj(frame.decoded) else np.float64)
    rng = np.random.default_rng(1)
    nv = min(32768, g.n_vox)                   # voxels per step (a bounded sample, ~0.3 s of oracle time)
    phi = nv / g.n_vox
    ncol = int(round(phi * g.n_ch * g.n_samples))
    times = []
    for step in range(args.warmup + args.steps):
        vox = np.sort(rng.choice(g.n_vox, size=nv, replace=False)).astype(np.int64)
        t0 = time.perf_counter()
        if frame.rf is not None:
            oracle.decode(frame.rf.reshape(g.n_tx, -1)[:, :ncol])
        oracle.das(g, exact, voxels=vox)
        t1 = time.perf_counter()
        if step >= args.warmup:
            times.append(t1 - t0)
    per = float(np.mean(times))
    value = nv * g.n_tx * g.n_ch / per / 1e9
    sample = "%d random voxels (%.5f of the frame)%s per step" % (
        nv, phi, " and the same fraction of decode columns" if frame.rf is not None else " (complex, two planes)")
    if workload == "bscan":
        config = headline_config(max(1, args.batch), ws)
    else:
        config = {"workload": "FORCES tiny B-scan: 32 tx (H32) x 32 ch x 1024 int16 samples -> 128x128 FP32 image"
                  if workload == "tiny" else OTHER_WORKLOADS[workload]}
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config,
        "frames_per_s": value * 1e9 / g.sums,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


OTHER_WORKLOADS = {
    "volume": "HERCULES volume: 128 tx x 128 ch x 2048 int16 samples -> 128x128x256 FP32 voxels",
    "stream": "realtime stream: 64 frames of uneven size (32/64/128 tx, 2048-4096 samples, 256x512 to "
              "512x1024 grids, 16 cross-plane pairs) in one persistent launch",
    "autofocus": "differentiable DAS: complex 128 tx x 128 ch x 2048 decoded RF -> 256x512 image, "
                 "forward + adjoint (dRF, dc, dw) per step",
    "hercules2d": "HERCULES 2D receive aperture (non-separable delays, tiled form): decoded FP16 128 rows x 128 "
                  "columns x 2048 samples, one plane wave -> 128x128x256 FP32 voxels",
    "iq": "IQ pipeline: FORCES 128 tx x 128 ch x 4096 int16 at 4 f_d -> quadrature demodulation (166-tap "
          "integer FIR, decimation 4) fused with the exact decode of both planes -> cubic IQ DAS to 512x1024 "
          "(complex)",
}


def _alu_peak_tops(sms: int) -> float:
    """FP32 lane-operations per second of the whole GPU at the maximum SM clock (T)."""
    return sms * 128 * _peaks()["sm_max_mhz"] * 1e6 / 1e12


def _time_steps(step, steps: int, warmup: int, stream):
    """Warm-up, then CUDA-event time of `steps` calls of step() on `stream`,
    with the clocks sampled during the timed region. Returns (ms/step, clocks)."""
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = _events(2)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, clocks.stop()


def _graph_of(batch):
    """A CUDA graph of one batch run (warm-up launch outside the capture)."""
    import torch
    stream = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        batch.run(stream=side)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.run()
    return graph


def measure_batched(name: str, args, parity: bool = True) -> dict:
    """The HERCULES volume (4 volumes per step) or the 64-frame stream, per
    step one CUDA graph: the exact tcgen05 decode of each frame to FP16, then
    the tiled DAS of all frames in one persistent launch, tiles from the
    autotuner. The roofline fraction is that of the whole step. Parity stamp
    (outside the timed region): decode bit-exact and sampled voxels against
    the FP64 oracle of the same FP16 decoded data, for the first frame of
    every frame class."""
    import torch
    import paper_2512_11086_gb300 as rc
    from paper_2512_11086_gb300 import tune
    import synth
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    out = {}
    if name == "volume":
        fr = synth.hercules_volume(3)
        frames = [fr] * max(1, args.batch)
        tiles = [tune.tune_tile(fr.geometry, "f16")] * len(frames)
    else:
        cache = {}
        frames = []
        for g, seed, box in synth.stream_geometries():
            key = (g.n_tx, g.n_samples, g.out_dims, g.tx_orientation)
            if key not in cache:                      # one synthetic content per frame class
                cache[key] = synth.make_frame(g, seed, 16, **box)
            frames.append(cache[key])
        tiles = tune.tune_stream([f.geometry for f in frames], "f16")
        out["content"] = "frames of one class share synthetic content (distinct buffers)"
    plans, rf, dec, img = [], [], [], []
    for fr, t in zip(frames, tiles):
        g = fr.geometry
        plans.append(rc.Plan(rc.make_params(g, decoded_dtype="f16", decode_variant=rc.DECODE_TC, tile=t)))
        rf.append(torch.from_numpy(fr.rf).to(dev))
        dec.append(torch.empty(g.n_tx, g.n_ch, g.n_samples, dtype=torch.float16, device=dev))
        img.append(torch.empty(g.out_dims[2], g.out_dims[1], g.out_dims[0], device=dev))
    batch = rc.Batch(plans, rf, dec, img)
    graph = _graph_of(batch)
    ms, clk = _time_steps(graph.replay, args.steps, args.warmup, stream)
    if batch.status() != rc.OK:
        raise RuntimeError("%s: batch status %d" % (name, batch.status()))
    sums = sum(f.geometry.sums for f in frames)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    achieved = 5 * sums / (ms * 1e-3) / 1e12
    out.update({"workload": OTHER_WORKLOADS[name], "value": sums / (ms * 1e-3) / 1e9, "unit": UNIT,
                "ms_per_step": ms, "frames_per_step": len(frames),
                ("volumes_per_s" if name == "volume" else "frames_per_s"): len(frames) * 1e3 / ms,
                "tiles": sorted({tuple(t) for t in tiles}),
                "roofline": {"bound": "alu", "achieved": achieved, "peak": _alu_peak_tops(sms), "unit": "TOP/s",
                             "frac": achieved / _alu_peak_tops(sms), "kernel": "batch_kernel",
                             "ops_per_sum": 5, "traffic": None},
                "clocks": clk})
    if parity:
        import oracle
        checked, worst, exact_all = 0, 0.0, True
        seen = set()
        for k, fr in enumerate(frames):
            if id(fr) in seen:
                continue
            seen.add(id(fr))
            g = fr.geometry
            want16 = oracle.decoded_as(oracle.decode(fr.rf), g.n_tx, "f16")
            exact_all &= bool(np.array_equal(dec[k].cpu().numpy().view(np.uint16), want16.view(np.uint16)))
            vox = np.sort(np.random.default_rng(k).choice(g.n_vox, size=min(512, g.n_vox), replace=False))
            got = img[k].cpu().numpy().astype(np.float64).ravel()[vox]
            worst = max(worst, rel_l2(got, oracle.das(g, want16.astype(np.float64), voxels=vox)))
            checked += 1
        out["parity"] = {"decode_bit_exact": exact_all, "das_rel_l2_max": worst, "tol": 1e-4,
                         "frames_checked": checked, "voxels_per_frame": 512,
                         "reference": "FP64 oracle: decode, then DAS of the FP16-rounded decode"}
    return out


def measure_autofocus(args, parity: bool = True) -> dict:
    """Speed-of-sound autofocus step: complex forward DAS and its adjoint
    (dRF, dc, dw) for L = -sum |I|^2. Parity stamp: the forward at sampled
    voxels and dL/dc, dL/dw against the FP64 oracle (whose own image gives its
    upstream gradient)."""
    import torch
    import paper_2512_11086_gb300 as rc
    from paper_2512_11086_gb300 import tune
    import synth
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    fr = synth.autofocus(5)
    g = fr.geometry
    tile = tune.tune_tile(g, "cf32")
    plan = rc.Plan(rc.make_params(g, decoded_dtype="cf32", tile=tile))
    d = torch.from_numpy(np.stack([fr.decoded.real, fr.decoded.imag]).astype(np.float32)).to(dev)
    w = torch.ones(g.n_ch, device=dev)
    out = torch.empty((2,) + plan.image_shape, device=dev)
    grad_rf = torch.empty_like(d)
    res = {}

    def forward():
        plan.das(d, apod=w, c=1540.0, out=out)

    # the adjoint is linear in its upstream gradient: the step passes G = I
    # (no elementwise kernel between the two calls), and the gradients of
    # L = -sum |I|^2 (G = -2 I) are -2 times its outputs
    def step():
        plan.das(d, apod=w, c=1540.0, out=out)
        res["g"] = plan.das_backward(d, out, apod=w, c=1540.0, out_rf=grad_rf)

    ms, clk = _time_steps(step, args.steps, args.warmup, stream)
    fwd_ms, _ = _time_steps(forward, args.steps, 2, stream)
    if plan.status() != rc.OK:
        raise RuntimeError("autofocus: plan status %d" % plan.status())
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    achieved = 7 * g.sums / (fwd_ms * 1e-3) / 1e12
    line = {"workload": OTHER_WORKLOADS["autofocus"], "value": g.sums / (ms * 1e-3) / 1e9, "unit": UNIT,
            "ms_per_step": ms, "forward_ms": fwd_ms, "adjoint_ms": ms - fwd_ms,
            "sums": "complex voxel x channel x transmit sums (two real planes each)",
            "tile": list(tile), "adjoint_tile": list(plan.info()["bwd_tile"]),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": _alu_peak_tops(sms), "unit": "TOP/s",
                         "frac": achieved / _alu_peak_tops(sms), "kernel": "das_tiled_kernel (forward, complex)",
                         "ops_per_sum": 7, "traffic": None},
            "clocks": clk}
    if parity:
        import oracle
        step()
        torch.cuda.synchronize()
        im = out.cpu().numpy().astype(np.float64)
        im = im[0] + 1j * im[1]
        _, gc, gw = res["g"]
        gc, gw = -2.0 * gc.item(), -2.0 * gw.cpu().numpy().astype(np.float64)
        ref = fr.decoded.astype(np.complex128)
        want_im = oracle.das(g, ref, c=1540.0)
        _, want_c, want_w = oracle.das_grad(g, ref, -2.0 * want_im, c=1540.0, want_rf=False)
        line["parity"] = {"das_rel_l2": rel_l2(im, want_im), "grad_c_rel": abs(gc - want_c) / abs(want_c),
                          "grad_apod_rel_l2": rel_l2(gw, want_w), "tol": {"das": 1e-4, "grad": 1e-3},
                          "reference": "FP64 oracle forward and gradients (L = -sum |I|^2) on the same complex RF"}
    return line


def measure_iq(args, parity: bool = True) -> dict:
    """The IQ pipeline on the B-scan acquisition (128 x 128 x 4096 int16 at
    4 f_d): quadrature demodulation (166-tap FIR, D = 4) fused into the exact
    decode of both planes (one launch), then the cubic IQ DAS. The stages are
    also timed apart, beside the unfused demodulate + decode. Parity stamp: the
    fused decoded planes bit for bit against oracle.demodulate then
    oracle.decode, and the image at sampled voxels against the oracle's IQ DAS
    of those planes."""
    import torch
    import paper_2512_11086_gb300 as rc
    import synth
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    fr = synth.full_bscan(2)
    g_raw = fr.geometry
    D, taps, shift = 4, synth.lowpass_taps(166, 0.12, shift=14), 14
    gd = (taps.size - 1) / 2
    g = dataclasses.replace(g_raw, n_samples=g_raw.n_samples // D, fs=g_raw.fs / D,
                            t0=g_raw.t0 - gd / g_raw.fs, iq_freq=g_raw.fs / 4, interp="cubic")
    plan = rc.Plan(rc.make_params(g, decoded_dtype="cf32", demod=(D, taps, shift)))
    rf = torch.from_numpy(fr.rf).to(dev)
    iq = torch.empty((2,) + plan.rf_shape, dtype=torch.int16, device=dev)
    dec = torch.empty((2,) + plan.rf_shape, dtype=torch.float32, device=dev)
    out = torch.empty((2,) + plan.image_shape, device=dev)

    def step():
        plan.demod_decode(rf, out=dec)
        plan.das(dec, out=out)

    ms, clk = _time_steps(step, args.steps, args.warmup, stream)
    stages = {"demod_decode_fused": lambda: plan.demod_decode(rf, out=dec),
              "demodulate": lambda: plan.demodulate(rf, out=iq),
              "decode_two_planes": lambda: plan.decode(iq, out=dec),
              "iq_das_cubic": lambda: plan.das(dec, out=out)}
    stage_ms = {k: _time_steps(f, max(3, min(args.steps, 10)), 2, stream)[0] for k, f in stages.items()}
    rec = {"workload": OTHER_WORKLOADS["iq"], "value": g.sums / (ms * 1e-3) / 1e9, "unit": UNIT,
           "ms_per_step": ms, "stage_ms": stage_ms,
           "unfused_demod_plus_decode_ms": stage_ms["demodulate"] + stage_ms["decode_two_planes"],
           "sums": "complex voxel x channel x transmit sums of the IQ DAS",
           "form": "rcbf_demod_decode (demodulation fused into the decode's load) + cubic IQ DAS",
           "plan": plan.info(), "clocks": clk}
    if parity:
        import oracle
        plan.demod_decode(rf, out=dec)
        torch.cuda.synchronize()
        got = dec.cpu().numpy()
        iq_o = oracle.demodulate(fr.rf, taps, shift, D)
        want = np.stack([oracle.decoded_as(oracle.decode(iq_o[p]), g.n_tx, "f32") for p in range(2)])
        plan.das(dec, out=out)
        torch.cuda.synchronize()
        img = out.cpu().numpy().astype(np.float64)
        img = (img[0] + 1j * img[1]).ravel()
        vox = np.sort(np.random.default_rng(3).choice(g.n_vox, size=512, replace=False))
        ref = oracle.das(g, want[0].astype(np.float64) + 1j * want[1].astype(np.float64), voxels=vox)
        rec["parity"] = {"demod_decode_bit_exact": bool(np.array_equal(got, want)),
                         "iq_das_rel_l2": rel_l2(img[vox], ref), "tol": 1e-4, "voxels": int(vox.size),
                         "reference": "oracle.demodulate then oracle.decode (bit for bit); FP64 IQ DAS"}
    return rec


def run_other_workload(args):
    """Another configuration on its own line, timed like the headline (CUDA
    events, warm-up, clocks)."""
    import torch
    import paper_2512_11086_gb300 as rc
    from paper_2512_11086_gb300 import build as rbuild
    import synth
    rbuild.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    if args.workload in ("volume", "stream", "autofocus", "iq"):
        rec = (measure_autofocus(args) if args.workload == "autofocus" else
               measure_iq(args) if args.workload == "iq" else measure_batched(args.workload, args))
        value, ms, clk = rec.pop("value"), rec.pop("ms_per_step"), rec.pop("clocks")
        rec.pop("unit")
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": rec.pop("workload")}, "clocks": clk}
        line.update(rec)
        print(json.dumps(line))
        return
    extra = {}
    if args.workload == "hercules2d":
        g = dataclasses.replace(synth.hercules_volume_geometry(), acq_kind=synth.HERCULES_2D, hadamard_order=0,
                                tx_wave="plane", tx_angles=(0.0,))
        plan = rc.Plan(rc.make_params(g, decoded_dtype="f16"))
        rng = np.random.default_rng(7)
        dec = torch.from_numpy(rng.normal(size=(g.n_tx, g.n_ch, g.n_samples)).astype(np.float16)).to(dev)
        out = torch.empty(plan.image_shape, device=dev)

        def step():
            plan.das(dec, out=out)
        sums = g.sums
        extra["plan"] = plan.info()
        extra["data"] = "seeded Gaussian decoded samples (timing only)"
    ms, clk = _time_steps(step, args.steps, args.warmup, stream)
    line = {"metric": METRIC, "value": sums / (ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict({"workload": OTHER_WORKLOADS[args.workload]}, **extra), "clocks": clk}
    print(json.dumps(line))


def run_channel_shard(args):
    """One B-scan per step split over the ranks by receive channel (Eq. (1) is
    a sum over channels): rank r decodes and beamforms its contiguous slice
    of channels with a plan over that slice of the array, and one NCCL
    all-reduce sums the partial images (2 MB), the only exchange of the path.
    Total work is fixed as N grows ("strong" scaling). At N = 1 it is the
    unbatched decode + DAS of one frame."""
    import torch
    rank, ws, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2512_11086_gb300 import build as rbuild
    if rank == 0:
        rbuild.build()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    import paper_2512_11086_gb300 as rc
    from paper_2512_11086_gb300 import shard, tune
    import synth
    frame = synth.full_bscan(seed=2)
    g = frame.geometry
    tile = tune.tune_tile(g, "f16")
    off, cnt = shard.channel_slices(g.n_ch, ws)[rank]
    plan = rc.Plan(shard.shard_params(g, rank, ws, decoded_dtype="f16", decode_variant=rc.DECODE_TC,
                                      das_variant=rc.DAS_TILED, tile=tile))
    host = torch.from_numpy(np.ascontiguousarray(frame.rf[:, off:off + cnt, :])).pin_memory()
    rf = host.to(dev)
    dec = torch.empty(g.n_tx, cnt, g.n_samples, dtype=torch.float16, device=dev)
    img = torch.empty(plan.image_shape, dtype=torch.float32, device=dev)
    img_host = torch.empty(plan.image_shape, dtype=torch.float32).pin_memory()
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def step():
        plan.decode(rf, out=dec)
        plan.das(dec, out=img)
        shard.reduce_image(img)

    def e2e_step():
        rf.copy_(host, non_blocking=True)
        step()
        if rank == 0:
            img_host.copy_(img, non_blocking=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = _events(2)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    total_ms, _ = aggregate(e0.elapsed_time(e1), 0.0, device=dev)
    ms = total_ms / args.steps
    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    q0, q1 = _events(2)
    q0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    q1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms, _ = aggregate(q0.elapsed_time(q1), 0.0, device=dev)
    e2e_ms /= args.steps
    if plan.status() != rc.OK:
        raise RuntimeError("rank %d: plan status %d" % (rank, plan.status()))
    line = {"metric": METRIC, "value": g.sums / (ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "frames_per_step": 1, "global_batch": 1,
                       "parallelism": "receive channels split over %d GPU(s), partial images summed by one "
                                      "all-reduce" % ws,
                       "l2": "one 128 MB int16 frame per step (129 MB L2; decoded FP16 written and re-read)"},
            "form": "per rank: tcgen05 decode of its channel slice to FP16, tiled DAS of the slice, "
                    "NCCL all-reduce of the partial image",
            "tile": list(tile), "frames_per_s": 1e3 / ms,
            "e2e": {"value": g.sums / (e2e_ms * 1e-3) / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": int(frame.rf.nbytes), "d2h_bytes_per_step": int(img_host.numel() * 4),
                    "ms_per_step": e2e_ms,
                    "form": "each rank uploads its RF slice from pinned memory, rank 0 reads the image back"},
            "gpu_launches": args.steps * (1 + plan.info()["das_launches"]),
            "plan": plan.info(), "clocks": clk}
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _graph_ms(batch, steps: int, warmup: int, stream) -> float:
    """CUDA-event time of one replay of a graph of batch.run() (after warm-up)."""
    import torch
    graph = _graph_of(batch)
    for _ in range(warmup):
        graph.replay()
    torch.cuda.synchronize()
    e0, e1 = _events(2)
    e0.record(stream)
    for _ in range(steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _events(n):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--batch", type=int, default=4, help="frames per step (one persistent launch)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the CPU leg (the oracle's timing and the parity stamps)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the volume, stream and autofocus records of the default line")
    ap.add_argument("--shard", default="frames", choices=["frames", "channels"],
                    help="frames: each GPU beamforms its own frames (no collective); channels: one B-scan "
                         "split over the GPUs by receive channel, partial images summed by one all-reduce")
    ap.add_argument("--workload", default="bscan", choices=["bscan", "tiny"] + sorted(OTHER_WORKLOADS),
                    help="bscan (the headline) or another configuration on its own line "
                         "(tiny: the 32-transmit B-scan, reference arm only)")
    args = ap.parse_args()
    if args.workload == "tiny" and args.impl != "reference":
        ap.error("--workload tiny times the oracle only (--impl reference)")
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload != "bscan":
        run_other_workload(args)
        return
    if args.shard == "channels":
        run_channel_shard(args)
        return

    import torch
    rank, ws, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2512_11086_gb300 import build as rbuild
    if rank == 0:
        rbuild.build()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    import paper_2512_11086_gb300 as rc
    from paper_2512_11086_gb300 import tune
    import synth

    B = max(1, args.batch)
    frame = synth.full_bscan(seed=2)
    g = frame.geometry
    sums = g.sums
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if ws == 1:
            return x
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    # ---- the batched, precision-tuned form: B frames per step, the exact
    # decode on the tcgen05 tensor cores to FP16 (one launch per frame), then
    # the tiled FP32 DAS of all frames in one persistent launch, the whole step
    # replayed from a CUDA graph; the voxel tile comes from the autotuner
    tile = tune.tune_tile(g, "f16")
    tuned = rc.Plan(rc.make_params(g, decoded_dtype="f16", decode_variant=rc.DECODE_TC,
                                   das_variant=rc.DAS_TILED, tile=tile))
    rf_host = torch.from_numpy(frame.rf)
    rf = [rf_host.to(dev) for _ in range(B)]
    dec16 = [torch.empty(g.n_tx, g.n_ch, g.n_samples, dtype=torch.float16, device=dev) for _ in range(B)]
    imgs = [torch.empty(tuned.image_shape, dtype=torch.float32, device=dev) for _ in range(B)]
    batch = rc.Batch([tuned] * B, rf, dec16, imgs)
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        batch.run(stream=side)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.run()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    if batch.status() != rc.OK:
        raise RuntimeError("batch status %d after warm-up" % batch.status())
    ev = _events(args.steps + 1)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    ev[0].record(stream)
    for s in range(args.steps):
        graph.replay()
        ev[s + 1].record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    total_ms, job_sums = aggregate(ev[0].elapsed_time(ev[-1]), float(B * sums * args.steps), device=dev)
    ms_step = total_ms / args.steps
    t_batch = float(np.mean([ev[s].elapsed_time(ev[s + 1]) for s in range(args.steps)]))
    value = job_sums / (total_ms * 1e-3) / 1e9
    if batch.status() != rc.OK:
        raise RuntimeError("batch status %d after the timed steps" % batch.status())
    # the last timed step's output, for the parity stamp of the CPU leg
    last_image = imgs[B - 1].cpu().numpy()
    last_decoded = dec16[B - 1].cpu().numpy()

    # ---- the persistent DAS kernel alone (the dominant kernel): the same batch
    # over the decoded frames, without their decode
    g_dec = dataclasses.replace(g, hadamard_order=0)
    das_only = rc.Batch([rc.Plan(rc.make_params(g_dec, decoded_dtype="f16", das_variant=rc.DAS_TILED,
                                                tile=tile))] * B, None, dec16, imgs)
    t_batch_kernel = _graph_ms(das_only, args.steps, args.warmup, stream)

    # ---- the same batch with the split-byte int8 mma.sync decode as work items
    # of the persistent kernel (the int8 tensor-core form of the decode)
    i8 = rc.Plan(rc.make_params(g, decoded_dtype="f16", decode_variant=rc.DECODE_MMA_I8,
                                das_variant=rc.DAS_TILED, tile=tile))
    batch_i8 = rc.Batch([i8] * B, rf, dec16, imgs)
    t_batch_i8 = _graph_ms(batch_i8, args.steps, args.warmup, stream)
    if batch_i8.status() != rc.OK or das_only.status() != rc.OK:
        raise RuntimeError("batch status after the variant timings")

    # ---- the same form unbatched: decode and DAS launched per frame
    ub_steps = max(3, min(args.steps, 10))
    for s in range(3):
        tuned.das(tuned.decode(rf[s % B], out=dec16[s % B]), out=imgs[0])
    torch.cuda.synchronize()
    ue = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(ub_steps)]
    for s in range(ub_steps):
        ue[s][0].record(stream)
        tuned.decode(rf[s % B], out=dec16[s % B])
        ue[s][1].record(stream)
        tuned.das(dec16[s % B], out=imgs[0])
        ue[s][2].record(stream)
    torch.cuda.synchronize()
    t_dec = float(np.mean([e[0].elapsed_time(e[1]) for e in ue]))
    t_das = float(np.mean([e[1].elapsed_time(e[2]) for e in ue]))

    # ---- the other exact decode forms, same output: split-byte int8 and FP16 mma.sync
    def decode_ms(plan):
        for s in range(3):
            plan.decode(rf[s % B], out=dec16[s % B])
        q0, q1 = _events(2)
        torch.cuda.synchronize()
        q0.record(stream)
        for s in range(ub_steps):
            plan.decode(rf[s % B], out=dec16[s % B])
        q1.record(stream)
        torch.cuda.synchronize()
        return q0.elapsed_time(q1) / ub_steps
    t_dec_tc = decode_ms(tuned)          # back-to-back launches over the rotating frames: the kernel's rate
    t_dec_i8 = decode_ms(i8)
    t_dec_f16 = decode_ms(rc.Plan(rc.make_params(g, decoded_dtype="f16", decode_variant=rc.DECODE_MMA_F16,
                                                 das_variant=rc.DAS_TILED, tile=tile)))

    # ---- cubic Hermite interpolation (the paper's measured setting): the DAS
    # alone on the same FP16 decoded frame, its own tuned tile
    gcub = dataclasses.replace(g, interp="cubic")
    ctile = tune.tune_tile(gcub, "f16")
    cub = rc.Plan(rc.make_params(gcub, decoded_dtype="f16", das_variant=rc.DAS_TILED, tile=ctile))
    for s in range(3):
        cub.das(dec16[s % B], out=imgs[0])
    c0, c1 = _events(2)
    torch.cuda.synchronize()
    c0.record(stream)
    for s in range(ub_steps):
        cub.das(dec16[s % B], out=imgs[0])
    c1.record(stream)
    torch.cuda.synchronize()
    t_cubic = c0.elapsed_time(c1) / ub_steps

    # ---- F# = 1 (the receive window of Eq. (2)-(3) active): sums/s counts
    # every term of the sum ("effective" throughput) although channel chunks
    # outside a tile's aperture are skipped
    fn1 = rc.Plan(rc.make_params(g, decoded_dtype="f16", das_variant=rc.DAS_TILED, tile=tile, f_number=1.0))
    for s in range(3):
        fn1.das(dec16[s % B], out=imgs[0])
    f0, f1 = _events(2)
    torch.cuda.synchronize()
    f0.record(stream)
    for s in range(ub_steps):
        fn1.das(dec16[s % B], out=imgs[0])
    f1.record(stream)
    torch.cuda.synchronize()
    t_fn1 = f0.elapsed_time(f1) / ub_steps

    # ---- plain FP32 form on the same GPU (same frames, same timing)
    plain = rc.Plan(rc.make_params(g, decoded_dtype="f32", decode_variant=rc.DECODE_PLAIN,
                                   das_variant=rc.DAS_PLAIN))
    dec32 = torch.empty(g.n_tx, g.n_ch, g.n_samples, dtype=torch.float32, device=dev)
    plain_steps = max(3, min(args.steps, 6))
    for s in range(2):
        plain.das(plain.decode(rf[s % B], out=dec32), out=imgs[0])
    p0, p1 = _events(2)
    torch.cuda.synchronize()
    p0.record(stream)
    for s in range(plain_steps):
        plain.das(plain.decode(rf[s % B], out=dec32), out=imgs[0])
    p1.record(stream)
    torch.cuda.synchronize()
    plain_ms = max_over_ranks(p0.elapsed_time(p1)) / plain_steps
    plain_value = sums / (plain_ms * 1e-3) / 1e9

    # ---- end to end through the C ABI with host buffers: every step copies
    # the B encoded frames from pinned host memory, runs the batch and reads
    # the B images back. Through the upload ring (rcbf_pipeline, 3 slots) the
    # copies of one step overlap the compute of the previous one; the serial
    # form (one stream: copy, replay, copy) is reported beside it.
    pinned = [rf_host.pin_memory() for _ in range(B)]
    img_host = [[torch.empty(tuned.image_shape, dtype=torch.float32).pin_memory() for _ in range(B)]
                for _ in range(3)]

    def e2e_serial_step():
        for b in range(B):
            rf[b].copy_(pinned[b], non_blocking=True)
        graph.replay()
        for b in range(B):
            img_host[0][b].copy_(imgs[b], non_blocking=True)

    for _ in range(2):
        e2e_serial_step()
    torch.cuda.synchronize()
    e0, e1 = _events(2)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        e2e_serial_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_serial_ms = max_over_ranks(e0.elapsed_time(e1)) / args.steps

    pipe = rc.Pipeline([tuned] * B, n_slots=3)
    for s in range(3):
        pipe.submit(pinned, img_host[s % 3])
    pipe.wait()
    barrier()
    torch.cuda.synchronize()
    t_start = time.perf_counter()
    for s in range(args.steps):
        pipe.submit(pinned, img_host[s % 3])
    pipe.wait()
    e2e_ms = max_over_ranks((time.perf_counter() - t_start) * 1e3) / args.steps
    pipe.close()
    e2e_value = B * sums * ws / (e2e_ms * 1e-3) / 1e9

    # ---- roofline: the dominant kernel (the persistent batch kernel) against
    # the FP32 ALU peak; the decode against HBM
    peaks = _peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    ops_per_sum = 5   # add (A_i + B_j), floor, fraction, interpolation FMA, accumulate
    alu_peak = sms * 128 * peaks["sm_max_mhz"] * 1e6 / 1e12   # FP32 lane-ops/s in T
    achieved = ops_per_sum * B * sums / (t_batch_kernel * 1e-3) / 1e12
    dec_bytes = g.n_tx * g.n_ch * g.n_samples * (2 + 2)       # int16 in + FP16 out
    info = tuned.info()
    # the same launch against HBM: compulsory bytes per frame if nothing stayed
    # on chip (RF read, FP16 decoded written and read back once, image written),
    # and the window bytes the DAS copies from L2 per frame (every tile stages
    # raw_samples FP16 samples of every (transmit, channel) trace)
    n_tiles = -(-g.out_dims[0] // tile[0]) * -(-g.out_dims[1] // tile[1]) * -(-g.out_dims[2] // tile[2])
    raw_samples = ((info["window"] + 8 + 7) // 8) * 8
    frame_bytes = g.n_tx * g.n_ch * g.n_samples * (2 + 2 + 2) + g.n_vox * 4
    window_bytes = n_tiles * g.n_tx * g.n_ch * raw_samples * 2
    traffic = recorded_traffic("batch_kernel", B)
    traffic_dec = recorded_traffic("decode_tc_kernel", 1)
    # on-chip ceilings measured on this GPU (microbenchmarks at the DAS
    # kernel's occupancy): one 8-byte line piece per sum from shared memory
    ceil = rc.measure_ceilings()
    das_alone = sums / (t_das * 1e-3)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": headline_config(B, ws),
        "form": "per step (one CUDA graph): exact split-byte decode to FP16 on the tcgen05 tensor cores "
                "(TMEM accumulators, TMA tiles), one launch per frame, then the tiled TMA-window FP32 DAS of "
                "all frames in one persistent launch",
        "tile": list(tile),
        "frames_per_s": B * ws * 1e3 / ms_step,
        "kernel_ms": {"step": t_batch, "batch_kernel_das_only": t_batch_kernel,
                      "unbatched_decode_tc": t_dec, "unbatched_das": t_das, "decode_tc": t_dec_tc,
                      "decode_i8_mma": t_dec_i8, "decode_f16_mma": t_dec_f16},
        "batched_i8_decode": {"value": B * sums / (t_batch_i8 * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": t_batch_i8,
                              "form": "the same step with the split-byte int8 mma.sync decode as work items of "
                                      "the persistent kernel (one launch per step)"},
        "unbatched": {"value": sums / ((t_dec + t_das) * 1e-3) / 1e9, "unit": UNIT,
                      "das_only": sums / (t_das * 1e-3) / 1e9},
        "f_number_1": {"value": sums / (t_fn1 * 1e-3) / 1e9, "unit": UNIT, "ms_per_frame": t_fn1,
                       "form": "tiled DAS alone with F# = 1 (effective: every term counted; channel chunks "
                               "outside a tile's aperture skipped)"},
        "cubic": {"value": sums / (t_cubic * 1e-3) / 1e9, "unit": UNIT, "ms_per_frame": t_cubic,
                  "tile": list(ctile), "window": cub.info()["window"],
                  "form": "tiled DAS alone, 4-point cubic Hermite, FP16 decoded frame"},
        "plain_fp32": {"value": plain_value, "unit": UNIT, "ms_per_frame": plain_ms,
                       "speedup_of_tuned": value / ws / plain_value},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TOP/s",
                     "frac": achieved / alu_peak, "traffic": traffic,
                     "kernel": "batch_kernel (the persistent DAS launch of the step, timed alone)",
                     "peak_src": "%d SMs x 128 FP32 lanes x %.0f MHz" % (sms, peaks["sm_max_mhz"]),
                     "ops_per_sum": ops_per_sum,
                     "binding": "shared-memory data path: one 8-byte line piece per sum (16 sums per clock per "
                                "SM); the fraction of that measured ceiling is ceilings.frac_lds_batched"},
        "roofline_memory": {"bound": "hbm", "achieved": B * frame_bytes / (t_batch_kernel * 1e-3) / 1e9,
                            "peak": peaks["hbm_gbs"], "unit": "GB/s",
                            "frac": B * frame_bytes / (t_batch_kernel * 1e-3) / 1e9 / peaks["hbm_gbs"],
                            "traffic": traffic,
                            "traffic_GBps": None if traffic is None else traffic / (t_batch_kernel * 1e-3) / 1e9,
                            "l2_window_GBps": B * window_bytes / (t_batch_kernel * 1e-3) / 1e9,
                            "kernel": "batch_kernel", "peak_src": peaks["src"],
                            "bytes_per_frame": frame_bytes},
        "ceilings": {"lds64_TBps": ceil["lds64_bytes_per_s"] / 1e12,
                     "ffma_TOPs": ceil["ffma_lane_ops_per_s"] / 1e12,
                     "ffma2_TOPs": ceil["ffma2_lane_ops_per_s"] / 1e12,
                     "red_shared_G_per_s": ceil["red_shared_per_s"] / 1e9,
                     "sm_mhz": ceil["sm_clock_hz"] / 1e6,
                     "lds_sums_per_s_ceiling": ceil["lds64_bytes_per_s"] / 8.0,
                     "frac_lds_batched": B * sums / (t_batch_kernel * 1e-3) * 8.0 / ceil["lds64_bytes_per_s"],
                     "frac_lds_das_alone": das_alone * 8.0 / ceil["lds64_bytes_per_s"],
                     "frac_ffma_batched": achieved * 1e12 / ceil["ffma_lane_ops_per_s"],
                     "source": "rcbf_measure_ceilings (this GPU, 2 CTAs x 256 threads per SM)"},
        "roofline_decode": {"bound": "hbm", "achieved": dec_bytes / (t_dec_tc * 1e-3) / 1e9,
                            "peak": peaks["hbm_gbs"], "unit": "GB/s",
                            "frac": dec_bytes / (t_dec_tc * 1e-3) / 1e9 / peaks["hbm_gbs"], "traffic": traffic_dec,
                            "kernel": "decode_tc_kernel (tcgen05, back-to-back launches over four frames)", "peak_src": peaks["src"],
                            "bytes_per_launch": dec_bytes},
        "roofline_decode_i8": {"bound": "tensor (int8 mma.sync rate)", "achieved_GBps": dec_bytes / (t_dec_i8 * 1e-3) / 1e9,
                               "peak": peaks["hbm_gbs"], "unit": "GB/s",
                               "frac": dec_bytes / (t_dec_i8 * 1e-3) / 1e9 / peaks["hbm_gbs"],
                               "kernel": "decode_mma_kernel (split-byte int8 mma.sync, unbatched)"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(B * rf_host.numel() * 2),
                "d2h_bytes_per_step": int(B * img_host[0][0].numel() * 4), "ms_per_step": e2e_ms,
                "form": "rcbf_pipeline upload ring, 3 slots (host wall clock between full waits)",
                "serial_ms_per_step": e2e_serial_ms},
        "gpu_launches": args.steps * (1 + B),
        "plan": info,
        "clocks": clk,
    }
    if rank == 0 and ws == 1 and not args.no_configs:
        # the other configurations, each timed like the headline and stamped
        # with its own parity check (outside its timed region)
        line["configs"] = {
            "volume": measure_batched("volume", args, parity=not args.no_cpu_baseline),
            "stream": measure_batched("stream", args, parity=not args.no_cpu_baseline),
            "autofocus": measure_autofocus(args, parity=not args.no_cpu_baseline),
            "iq": measure_iq(args, parity=not args.no_cpu_baseline),
        }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, det = cpu_baseline(frame, gpu_image=last_image, gpu_decoded=last_decoded)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": det["cores"], "kind": "oracle",
                                "sample": det["sample"]}
        line["parity"] = det["parity"]
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Frames/s of the dense-field phase-to-space (DF-P2S) simulator on one GB300.

Default workload: a 512 x 512 x 3 frame (seeded rectangles and edges), J = 36
Zernike fields on a 1024 x 1024 FFT grid, D/r0 cycling over {1, 2, 4}, K = 100
basis PSFs of 33 x 33, learned P2S (network weights in the P2S handle).  A step
is one frame: fields (noise -> FFT -> spectral multiply -> inverse FFT -> mix)
-> tilt warp -> P2S weights -> basis blur, with the input image resident in HBM.
The e2e figure runs the public simulate_frame call with the image copied in
from pinned host memory and the frame copied back every step, the copies of
neighbouring frames overlapping the computation (two buffers, copy streams).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload 512|4k|256|64]
                  [--mode learned|exact] [--impl ours|reference]

Under torchrun every rank simulates its own frames (weak scaling, no
collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (H, W, C, image kind, K, D/r0 list, description)
    "512": (512, 512, 3, "shapes", 100, [1.0, 2.0, 4.0], "512x512x3 shapes, J=36, N=1024, K=100, D/r0 in {1,2,4}"),
    "4k": (2160, 3840, 3, "texture", 100, [4.0], "3840x2160x3 1/f^2 texture, J=36, N=4096, K=100, D/r0=4"),
    "256": (256, 256, 3, "blobs", 100, [3.0], "256x256x3 blobs, J=36, N=512, K=100, D/r0=3"),
    "64": (64, 64, 1, "smooth_noise", 16, [2.0], "64x64x1 smoothed noise, J=36, N=128, K=16, D/r0=2"),
}
J = 36
PIX_PER_D = 8.0
L2_BYTES = 129 * 1024 * 1024


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            # nvidia-smi's start-up briefly stalls the device: wait for its first sample
            t0 = time.time()
            while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.05)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, val in zip(names, r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "window": "0.4 s of the same frames untimed, then the timed frames"}


def setup_ours(workload: str, mode: str, device, train_steps: int = 60000):
    """Untimed setup: spectral factor, SVD basis of 2000 exact PSFs and (learned mode) the trained surrogate,
    all built on the device."""
    import torch
    import paper_2210_06713_gb300 as d
    from inputs import synthetic

    H, W, C, kind, K, dlist, _ = WORKLOADS[workload]
    N = d.grid_size(H, W, PIX_PER_D)
    img = torch.as_tensor(synthetic.image_for(kind, H, W, C, seed=0), device=device).contiguous()
    t0 = time.perf_counter()
    factor = d.SpectralFactor(J, N, PIX_PER_D)
    t_factor = time.perf_counter() - t0
    t0 = time.perf_counter()
    basis, sig, sweeps = d.build_basis(factor, K, 2000, tuple(dlist), seed=0)
    t_basis = time.perf_counter() - t0
    P = d.P2S(J, basis)
    info = {"factor_s": t_factor, "basis_s": t_basis, "basis_sweeps": sweeps}
    if mode == "learned":
        t0 = time.perf_counter()
        rep = d.mlp_train(P, factor, n_pairs=1 << 20, D_over_r0=tuple(dlist), seed=1, batch=2048,
                          steps=train_steps, lr=2e-3)
        info.update({"train_s": time.perf_counter() - t0, "train_steps": rep["steps"],
                     "val_weight_rel_l2": rep["val_weight_rel_l2"]})
    sim = d.Simulator(factor, P, C, H, W)
    return d, dict(H=H, W=W, C=C, K=K, N=N, dlist=dlist, img=img, factor=factor, P=P, P_basis=basis, sim=sim,
                   info=info)


def accuracy_vs_exact(d, S, seed):
    """rel-L2 of the learned frame against the exact-P2S FP32 frame, one frame per D/r0."""
    out = {}
    for dr in S["dlist"]:
        ex = S["sim"].simulate_frame(S["img"], dr, seed, 0, d.P2S_EXACT).double()
        le = S["sim"].simulate_frame(S["img"], dr, seed, 0, d.P2S_LEARNED).double()
        out[str(dr)] = float((le - ex).norm() / ex.norm())
    S["P"].check()
    return out


# ---- the multi-rank host logic: frames are independent, each rank draws its own Philox streams (a seed base of
# its own), times its frames, and rank 0 reports the whole job from the slowest rank's time (no data collective)
def rank_seed_base(rank: int) -> int:
    return 1000 * rank


def max_over_ranks(value: float, world: int, device) -> float:
    if world == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_frames_per_s(world: int, steps: int, max_total_ms: float) -> float:
    return world * steps / (max_total_ms * 1e-3)


def stage_roofline(name, ms, args, peaks, peak_kind, H, W, C, K):
    """Roofline of one single-launch stage of the frame (its CUDA events bracket one kernel launch)."""
    npix = H * W
    learned = args.mode == "learned"
    if name == "blur" and learned:
        # Eq. (varying blur) as a dense contraction on the tensor cores: 2 x 33^2 x K MACs per pixel and
        # channel; the events bracket the one k_blur_tc launch of the frame (C <= 3)
        flops = 2.0 * 1089 * K * C * npix
        # DRAM traffic is not measured in this process (ncu captures only, reported beside the bench)
        roof = {"kernel": "k_blur_tc", "bound": "tensor", "achieved": flops / (ms * 1e-3) / 1e12,
                "peak": peaks["bf16_tflops"], "unit": "TFLOP/s", "traffic": None,
                "peak_source": peak_kind + " (burst bf16 GEMM)"}
    elif name == "blur":
        flops = 2.0 * 1089 * (K + C) * npix  # per-pixel PSF form on FP32 CUDA cores
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        roof = {"kernel": "k_blur_psf", "bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12,
                "peak": peak, "unit": "TFLOP/s", "traffic": None,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"}
    elif name.startswith("p2s") and learned:
        # the surrogate MLP on the tensor cores: 2 (256 J + 256^2 + 256 K) FLOP per pixel, one k_mlp_tc launch
        flops = npix * 2.0 * (J * 256 + 256 * 256 + 256 * K)
        roof = {"kernel": "k_mlp_tc", "bound": "tensor", "achieved": flops / (ms * 1e-3) / 1e12,
                "peak": peaks["bf16_tflops"], "unit": "TFLOP/s", "traffic": None,
                "peak_source": peak_kind + " (burst bf16 GEMM)"}
    elif name.startswith("p2s"):
        flops = npix * (2.0 * 1089 * (J - 2) + 2 * 8.0 * 33 ** 3 + 2.0 * 1089 * K)
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        roof = {"kernel": "k_p2s_exact", "bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12,
                "peak": peak, "unit": "TFLOP/s", "traffic": None,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"}
    elif learned:
        wq = (W + 127) // 128 * 128 + 64
        byt = 4.0 * npix * (2 + C) + 16.0 * C * (H + 32) * wq  # tilts and image in, eight BF16 planes out
        roof = {"kernel": "k_warp_pad_shifted", "bound": "hbm", "achieved": byt / (ms * 1e-3) / 1e9,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "traffic": None, "peak_source": peak_kind}
    else:
        byt = 4.0 * npix * (2 + 2 * C)  # tilt fields a2, a3 and the image in, the warped image out
        roof = {"kernel": "k_tilt_warp", "bound": "hbm", "achieved": byt / (ms * 1e-3) / 1e9,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "traffic": None, "peak_source": peak_kind}

    roof["frac"] = roof["achieved"] / roof["peak"]
    return roof


def large_frame(d, S, device, stream, flush):
    """The other half of the metric: a 3840 x 2160 x 3 frame (1/f^2 texture, J = 36, N = 4096, K = 100,
    D/r0 = 4) with this run's basis and trained network, learned and exact P2S on the same GPU, frames/s of
    each (CUDA events on this stream, L2 flushed between frames) and the learned frame's rel-L2 against the
    exact frame."""
    import torch
    from inputs import synthetic
    H, W, C, kind, K, dlist, desc = WORKLOADS["4k"]
    N = d.grid_size(H, W, PIX_PER_D)
    img = torch.as_tensor(synthetic.image_for(kind, H, W, C, seed=0), device=device).contiguous()
    factor = d.SpectralFactor(J, N, PIX_PER_D)
    sim = d.Simulator(factor, S["P"], C, H, W)
    out = torch.empty(C, H, W, device=device)
    dr = dlist[0]
    res = {"workload": desc}
    for name, mode, nw, nt in (("learned", d.P2S_LEARNED, 3, 10), ("exact", d.P2S_EXACT, 1, 3)):
        for i in range(nw):
            sim.simulate_frame(img, dr, 500, i, mode, out=out, stream=stream)
        torch.cuda.synchronize()
        sim.stage_timing(nt)
        for i in range(nt):
            flush.zero_()
            sim.simulate_frame(img, dr, 500, nw + i, mode, out=out, stream=stream)
        st = sim.stage_times(nt).astype(np.float64)
        sim.stage_timing(0)
        ms = float(st.sum(axis=1).mean())
        res[name] = {"frames_per_s": 1e3 / ms, "ms_per_frame": ms, "frames": nt,
                     "stage_ms": dict(zip(["fields", "warp", "p2s", "blur"], st.mean(axis=0).tolist()))}
    ex = sim.simulate_frame(img, dr, 77, 0, d.P2S_EXACT).double()
    le = sim.simulate_frame(img, dr, 77, 0, d.P2S_LEARNED).double()
    S["P"].check()
    res["rel_l2_learned_vs_exact"] = float((le - ex).norm() / ex.norm())
    res["learned_over_exact"] = res["learned"]["frames_per_s"] / res["exact"]["frames_per_s"]
    del sim, factor, ex, le
    torch.cuda.empty_cache()
    return res


def full_sampler_frames(d, S, device, stream, flush):
    """512 x 512 x 3 learned frames whose fields come from the full cross-spectral density (no approximation):
    frames/s with the stage events (L2 flushed between frames) and rel-L2 against the exact frame at D/r0 = 4."""
    import torch
    H, W, C = S["H"], S["W"], S["C"]
    sim = d.Simulator(d.SpectralFactor(J, S["N"], PIX_PER_D, kind=d.FACTOR_FULL), S["P"], C, H, W)
    sim.set_field_sampler(d.FIELDS_FULL)
    out = torch.empty(C, H, W, device=device)
    for i in range(3):
        sim.simulate_frame(S["img"], 2.0, 600, i, d.P2S_LEARNED, out=out, stream=stream)
    torch.cuda.synchronize()
    nt = 10
    sim.stage_timing(nt)
    for i in range(nt):
        flush.zero_()
        sim.simulate_frame(S["img"], S["dlist"][i % len(S["dlist"])], 600, 3 + i, d.P2S_LEARNED, out=out,
                           stream=stream)
    st = sim.stage_times(nt).astype(np.float64)
    sim.stage_timing(0)
    ms = float(st.sum(axis=1).mean())
    ex = sim.simulate_frame(S["img"], 4.0, 77, 0, d.P2S_EXACT).double()
    le = sim.simulate_frame(S["img"], 4.0, 77, 0, d.P2S_LEARNED).double()
    S["P"].check()
    res = {"workload": "512x512x3, J=36, N=1024, K=100, fields of the full cross-spectral density",
           "frames_per_s": 1e3 / ms, "ms_per_frame": ms,
           "stage_ms": dict(zip(["fields", "warp", "p2s", "blur"], st.mean(axis=0).tolist())),
           "rel_l2_learned_vs_exact_dr4": float((le - ex).norm() / ex.norm())}
    del sim
    torch.cuda.empty_cache()
    return res


def full_sampler_timing(d, device, stream, flush, peak_gbs):
    """The exact sampler of the full cross-spectral density (no approximation) against the factored sampler with
    its mixing pass, J = 36, at the 512 x 512 frame's grid (N = 1024) and at 3840 x 2160 (N = 4096): ms per
    call (CUDA events on this stream, L2 flushed before each call) and the full sampler's HBM roofline over its
    algorithmic bytes (order fields written and read once, column spectra written and read, fields written,
    Cholesky table read once)."""
    import torch
    out = {}
    for name, H, W in (("512x512", 512, 512), ("3840x2160", 2160, 3840)):
        N = d.grid_size(H, W, PIX_PER_D)
        t0 = time.perf_counter()
        f = d.SpectralFactor(J, N, PIX_PER_D, kind=d.FACTOR_FULL)
        setup_s = time.perf_counter() - t0
        fields = torch.empty(J, H, W, device=device)
        res = {"N": N, "setup_s": setup_s}
        for label, fn in (("full", d.sample_zernike_fields_full), ("factored", d.sample_zernike_fields)):
            for i in range(3):
                fn(f, 2.0, 9, i, H, W, out=fields, stream=stream)
            e = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
            for i, (a, b) in enumerate(e):
                flush.zero_()
                a.record(stream)
                fn(f, 2.0, 9, 10 + i, H, W, out=fields, stream=stream)
                b.record(stream)
            torch.cuda.synchronize()
            res[label + "_ms"] = float(np.median([a.elapsed_time(b) for a, b in e]))
        R = 8
        half = N // 2 + 1
        noct = half * (half + 1) // 2
        alg = (2 * R * half * N * 8 + 2 * J * half * H * 8 + J * H * W * 4 + noct * (R * (R + 1) // 2) * 4)
        res["full_roofline"] = {"bound": "hbm", "bytes": alg, "achieved": alg / (res["full_ms"] * 1e-3) / 1e9,
                                "peak": peak_gbs, "unit": "GB/s",
                                "frac": alg / (res["full_ms"] * 1e-3) / 1e9 / peak_gbs}
        out[name] = res
        del f, fields
        torch.cuda.empty_cache()
    # the subharmonic levels of the factored sampler (nine, the tilt's low-frequency compensation) at 512 x 512
    f0 = d.SpectralFactor(J, 1024, PIX_PER_D)
    f9 = d.SpectralFactor(J, 1024, PIX_PER_D, subharmonics=9)
    fields = torch.empty(J, 512, 512, device=device)
    res = {}
    for label, f in (("levels_0", f0), ("levels_9", f9)):
        for i in range(3):
            d.sample_zernike_fields(f, 2.0, 9, i, 512, 512, out=fields, stream=stream)
        e = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
        for i, (a, b) in enumerate(e):
            flush.zero_()
            a.record(stream)
            d.sample_zernike_fields(f, 2.0, 9, 10 + i, 512, 512, out=fields, stream=stream)
            b.record(stream)
        torch.cuda.synchronize()
        res[label + "_ms"] = float(np.median([a.elapsed_time(b) for a, b in e]))
    out["subharmonics_512x512"] = res
    # the dense per-frequency root (FP64 Jacobi at setup, the J x J product per frame) at 512 x 512
    t0 = time.perf_counter()
    fd = d.SpectralFactor(J, 1024, PIX_PER_D, kind=d.FACTOR_DENSE)
    torch.cuda.synchronize()
    dres = {"setup_s": time.perf_counter() - t0}
    for i in range(3):
        d.sample_zernike_fields_dense(fd, 2.0, 9, i, 512, 512, out=fields, stream=stream)
    e = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
    for i, (a, b) in enumerate(e):
        flush.zero_()
        a.record(stream)
        d.sample_zernike_fields_dense(fd, 2.0, 9, 10 + i, 512, 512, out=fields, stream=stream)
        b.record(stream)
    torch.cuda.synchronize()
    dres["ms"] = float(np.median([a.elapsed_time(b) for a, b in e]))
    half = 513 * 1024
    dbytes = J * J * half * 4 + 2 * J * half * 8 + 2 * J * half * 512 * 8 // 1024 + J * 512 * 512 * 4
    dres["roofline"] = {"bound": "hbm", "bytes": dbytes, "achieved": dbytes / (dres["ms"] * 1e-3) / 1e9,
                        "peak": peak_gbs, "unit": "GB/s", "frac": dbytes / (dres["ms"] * 1e-3) / 1e9 / peak_gbs}
    out["dense_root_512x512"] = dres
    del f0, f9, fd, fields
    torch.cuda.empty_cache()
    return out


def batched_uneven(d, S, device, stream, seed_base=0, train_steps=20000):
    """The batched workload: 64 requests, image sides uniform in {256, 512, 768, 1024} (x 3 channels), D/r0 uniform
    in [1, 5], J in {15, 36}, 8 frames each with independent seeds, learned P2S, through one engine call
    (per-shape-class frame graphs, autotuned field column pass). The J = 36 handle is this run's; a J = 15 basis
    and network are built on the device the same way (train_steps, 20 000 by default). Returns frames/s of whole
    runs."""
    import torch
    from inputs import synthetic
    rng = np.random.default_rng(4)
    sides = [256, 512, 768, 1024]
    reqs_spec = [(int(rng.choice(sides)), float(rng.uniform(1.0, 5.0)), int(rng.choice([15, 36]))) for _ in range(64)]
    f15 = d.SpectralFactor(15, 1024, PIX_PER_D)
    b15, _, _ = d.build_basis(f15, 100, 2000, (1.0, 2.0, 3.0, 4.0, 5.0), seed=0)
    P15 = d.P2S(15, b15)
    d.mlp_train(P15, f15, n_pairs=1 << 20, D_over_r0=(1.0, 2.0, 3.0, 4.0, 5.0), seed=1, batch=2048,
                steps=train_steps, lr=2e-3)
    imgs = {sd: torch.as_tensor(synthetic.shapes(sd, sd, 3, seed=sd), device=device) for sd in sides}
    reqs = [{"img": imgs[sd], "J": J, "D_over_r0": dr, "seed": seed_base + 500 + r, "n_frames": 8,
             "mode": d.P2S_LEARNED, "out": torch.empty(8, 3, sd, sd, device=device)}
            for r, (sd, dr, J) in enumerate(reqs_spec)]
    nframes = 64 * 8
    pix = sum(8 * sd * sd for sd, _, _ in reqs_spec)
    res = {"workload": "64 requests, sides {256,512,768,1024}x3, D/r0 U[1,5], J {15,36}, 8 frames each, learned P2S",
           "frames": nframes, "megapixels": pix / 1e6, "l2": "not flushed (512 frames per run)"}
    for name, graphs in (("graphs", True), ("no_graphs", False)):
        eng = d.Engine([P15, S["P"]], PIX_PER_D, graphs=graphs, autotune=True)
        eng.run(reqs, stream=stream)  # builds the classes, tunes them, instantiates the graphs
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ts = []
        for _ in range(3):
            e0.record(stream)
            eng.run(reqs, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = float(np.median(ts))
        info = eng.info()
        res[name] = {"ms_per_run": ms, "frames_per_s": nframes / (ms * 1e-3), "megapixels_per_s": pix / 1e6 / (ms * 1e-3),
                     "graph_launches": info["graph_launches"], "graph_updates": info["graph_updates"]}
        if graphs:
            res["classes"] = [{k: c[k] for k in ("J", "H", "N", "column_pass", "tuned_ms")} for c in info["classes"]]
        eng.close()
    S["P"].check()
    P15.check()
    del reqs
    torch.cuda.empty_cache()
    return res


def run_ours(args, rank, world, device):
    import torch
    d, S = setup_ours(args.workload, args.mode, device, args.train_steps)
    H, W, C, K = S["H"], S["W"], S["C"], S["K"]
    mode = d.P2S_LEARNED if args.mode == "learned" else d.P2S_EXACT
    wdt = d.W_F32
    stream = torch.cuda.current_stream()
    out = torch.empty(C, H, W, device=device)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=device)
    seed_base = rank_seed_base(rank)

    def step(i):
        # one frame through the library's frame call (the C ABI's dfp2s_simulate_frame); with stage timing on,
        # it records CUDA events between the field, warp, P2S and blur stages on this stream
        dr = S["dlist"][i % len(S["dlist"])]
        S["sim"].simulate_frame(S["img"], dr, seed_base, i, mode, out=out, stream=stream)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    S["sim"].stage_timing(args.steps)
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
        # the timed region lasts milliseconds: the same frames run untimed for about 0.4 s first, so that the
        # clock record (100 ms samples) covers the device under this load up to the timed frames
        t_load = time.perf_counter()
        i = 0
        while time.perf_counter() - t_load < 0.4:
            step(args.warmup + args.steps + i)
            i += 1
            if i % 50 == 0:
                torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()  # evict L2 between timed frames (outside the events)
        step(args.warmup + i)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop() if clocks else None
    stage_ms = S["sim"].stage_times(args.steps).astype(np.float64)
    S["sim"].stage_timing(0)
    frame_ms = stage_ms.sum(axis=1)
    total_ms = max_over_ranks(float(frame_ms.sum()), world, device)

    # end to end through simulate_frame with host buffers: every frame copies its image in from pinned host memory
    # and its result out to pinned host memory; frames are pipelined the way a streaming caller runs them (copy-in
    # of frame i+1 and copy-out of frame i-1 on their own streams while frame i computes, two buffers each, events
    # guarding their reuse)
    img_h = S["img"].cpu().pin_memory()
    out_h = [torch.empty(C, H, W, pin_memory=True) for _ in range(2)]
    img_d = [torch.empty_like(S["img"]) for _ in range(2)]
    out_d = [torch.empty_like(S["img"]) for _ in range(2)]
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    for k in range(2):  # all buffers free at the start
        ev_done[k].record(stream)
        ev_out[k].record(stream)

    def e2e_frame(i):
        b = i % 2
        s_in.wait_event(ev_done[b])  # frame i-2 has finished reading img_d[b]
        with torch.cuda.stream(s_in):
            img_d[b].copy_(img_h, non_blocking=True)
        ev_in[b].record(s_in)
        stream.wait_event(ev_in[b])
        stream.wait_event(ev_out[b])  # out_d[b] of frame i-2 has reached the host
        S["sim"].simulate_frame(img_d[b], S["dlist"][i % len(S["dlist"])], seed_base + 1, i, mode, out=out_d[b],
                                stream=stream)
        ev_done[b].record(stream)
        s_out.wait_event(ev_done[b])
        with torch.cuda.stream(s_out):
            out_h[b].copy_(out_d[b], non_blocking=True)
        ev_out[b].record(s_out)

    e2e_steps = max(3, min(args.steps, 20))
    for i in range(2):
        e2e_frame(i)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    for i in range(e2e_steps):
        e2e_frame(2 + i)
    e1.record(s_out)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / e2e_steps, world, device)  # per frame, the slowest rank

    # the other P2S form on the same GPU (the metric compares them): whole frames through simulate_frame
    other = d.P2S_EXACT if mode == d.P2S_LEARNED else (d.P2S_LEARNED if S["P"].has_mlp else None)
    other_line = None
    if other is not None:
        n_other = 3 if other == d.P2S_EXACT else 10
        S["sim"].simulate_frame(S["img"], S["dlist"][0], seed_base + 2, 0, other, out=out)
        torch.cuda.synchronize()
        o0, o1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        o0.record(stream)
        for i in range(n_other):
            S["sim"].simulate_frame(S["img"], S["dlist"][i % len(S["dlist"])], seed_base + 2, i, other, out=out)
        o1.record(stream)
        torch.cuda.synchronize()
        oms = o0.elapsed_time(o1) / n_other
        other_line = {"p2s": "exact" if other == d.P2S_EXACT else "learned", "frames_per_s": 1e3 / oms,
                      "ms_per_frame": oms, "frames": n_other}
    # field statistics (Sec. III-D): lagged covariances of one frame's fields at four lags, FP32 FMA-bound
    stat = None
    try:
        fl = d.sample_zernike_fields(S["factor"], S["dlist"][0], seed_base + 3, 0, H, W)
        lags = [(0, 0), (0, 1), (1, 0), (4, -4)]
        d.field_covariance(fl, lags)
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(5):
            d.field_covariance(fl, lags)
        s1.record(stream)
        torch.cuda.synchronize()
        sms = s0.elapsed_time(s1) / 5
        fmas = float(J * J) * sum((H - abs(a)) * (W - abs(b)) for a, b in lags)
        mhz = _peaks()[0].get("sm_max_mhz", 2070.0)
        alu = 152 * 128 * 2 * mhz * 1e6 / 1e12
        stat = {"what": "dfp2s_field_covariance, J x J at 4 lags of one frame's fields", "ms": sms,
                "achieved_tflops": 2 * fmas / (sms * 1e-3) / 1e12, "alu_peak_tflops": alu,
                "frac": 2 * fmas / (sms * 1e-3) / 1e12 / alu}
        # Sec. IV-B validation: structure function + LE/SE OTFs of every fourth pixel's vector (two 64 x 64 FFTs
        # each), and the tilt correlation / DTV at lags 0..64 along both axes
        for name, fn in (("aperture_statistics", lambda: d.aperture_statistics(fl, 4)),
                         ("tilt_statistics", lambda: d.tilt_statistics(fl, 64))):
            fn()
            torch.cuda.synchronize()
            s0.record(stream)
            for _ in range(3):
                fn()
            s1.record(stream)
            torch.cuda.synchronize()
            stat[name + "_ms"] = s0.elapsed_time(s1) / 3
        nreal = ((H + 3) // 4) * ((W + 3) // 4)
        stat["aperture_statistics_realisations_per_s"] = nreal / (stat["aperture_statistics_ms"] * 1e-3)
        del fl
    except RuntimeError as exc:
        stat = {"unavailable": str(exc).splitlines()[0][:120]}
    # cuFFT (through torch.fft) on the field sampler's transforms, as a comparison: J real N x N noise planes ->
    # R2C 2-D FFT -> spectral multiply -> C2R 2-D inverse FFT, cropped to H x W (no noise, no mixing)
    cufft = None
    try:
        N = S["N"]
        noise_t = torch.randn(J, N, N, device=device)
        mult_t = torch.rand(J, N, N // 2 + 1, device=device)
        for _ in range(2):
            torch.fft.irfft2(torch.fft.rfft2(noise_t) * mult_t, s=(N, N))[:, :H, :W].contiguous()
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(5):
            torch.fft.irfft2(torch.fft.rfft2(noise_t) * mult_t, s=(N, N))[:, :H, :W].contiguous()
        c1.record(stream)
        torch.cuda.synchronize()
        cufft = {"what": "torch.fft rfft2 -> multiply -> irfft2 -> crop, J x N x N FP32", "ms": c0.elapsed_time(c1) / 5}
        del noise_t, mult_t
    except RuntimeError as exc:  # out of memory at the largest grids
        cufft = {"unavailable": str(exc).splitlines()[0][:120]}

    names = ["fields", "warp_and_blur_operand" if args.mode == "learned" else "warp", "p2s_" + args.mode, "blur"]
    acc = None
    if args.mode == "learned" and not args.no_accuracy:
        acc = accuracy_vs_exact(d, S, seed_base + 77)
    mean_stage = stage_ms.mean(axis=0)
    peaks, peak_kind = _peaks()
    # dominant kernel roofline: among the stages that are one kernel launch each (warp, P2S weights, blur
    # contraction); the field stage is two or three launches, each shorter than the blur contraction (ncu list)
    single = [1, 2, 3]
    dom = single[int(np.argmax(mean_stage[single]))]
    npix = H * W
    roofs = {i: stage_roofline(names[i], mean_stage[i], args, peaks, peak_kind, H, W, C, K) for i in single}
    roof = roofs[dom]
    # the field sampler as one HBM-bound stage: multiplier read (4 J N (N/2+1)), cropped columns written and read
    # (16 J H (N/2+1)), unit fields written (4 J H W) and, in exact frames, read and written by the mixing
    # pass (8 J H W; learned frames fold the mixing into the warp and the network); the noise is made in registers
    N = S["N"]
    half = N // 2 + 1
    learned = args.mode == "learned"
    fbytes = 4.0 * J * N * half + 16.0 * J * H * half + (4.0 if learned else 12.0) * J * npix
    fields_roof = {"kernels": "k_colgen + k_rowifft" + ("" if learned else " + k_mix"), "bound": "hbm",
                   "achieved": fbytes / (mean_stage[0] * 1e-3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s"}
    fields_roof["frac"] = fields_roof["achieved"] / fields_roof["peak"]
    value = whole_job_frames_per_s(world, args.steps, total_ms)
    line = {
        "metric": "dense-field frames/s at 512^2 and 4K: learned vs exact P2S, same GB300, at tol",
        "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16" if args.mode == "learned" else "f32", "data": "synthetic",
        "config": config_for(args.workload, args.mode, world),
        "stage_ms": {n: float(v) for n, v in zip(names, mean_stage)},
        "rel_l2_learned_vs_exact": acc,
        "roofline": roof,
        "fields_roofline": fields_roof,
        "stage_rooflines": {roofs[i]["kernel"]: {k: roofs[i][k] for k in ("bound", "achieved", "peak", "unit", "frac")}
                            for i in single},
        "e2e": {"value": world * 1e3 / e2e_ms, "unit": "frames/s", "h2d_bytes_per_step": int(4 * C * H * W),
                "d2h_bytes_per_step": int(4 * C * H * W)},
        # field launches (noise + column IFFT, row IFFT, and the mixing in exact frames), warp, P2S, blur
        "gpu_launches": args.steps * (5 if args.mode == "learned" else 6),
        "other_p2s": other_line,
        "cufft_fields_comparison": cufft,
        "field_statistics": stat,
        "setup": S["info"],
        "clocks": clk,
        "wall_s": wall,
    }
    if args.workload == "512" and args.mode == "learned" and not args.no_4k:
        try:
            line["workloads"] = {"3840x2160x3": large_frame(d, S, device, stream, flush)}
        except RuntimeError as exc:
            line["workloads"] = {"3840x2160x3": {"unavailable": str(exc).splitlines()[0][:160]}}
    if args.workload == "512" and args.mode == "learned" and not args.no_full_sampler:
        line.setdefault("workloads", {})
        try:
            line["workloads"]["full_cross_spectrum_fields"] = full_sampler_timing(d, device, stream, flush,
                                                                                  peaks["hbm_gbs"])
        except RuntimeError as exc:
            line["workloads"]["full_cross_spectrum_fields"] = {"unavailable": str(exc).splitlines()[0][:160]}
    if args.workload == "512" and args.mode == "learned" and not args.no_full_sampler:
        try:
            line["workloads"]["full_cross_spectrum_frames"] = full_sampler_frames(d, S, device, stream, flush)
        except RuntimeError as exc:
            line["workloads"]["full_cross_spectrum_frames"] = {"unavailable": str(exc).splitlines()[0][:160]}
    if args.workload == "512" and args.mode == "learned" and not args.no_batched:
        line.setdefault("workloads", {})
        try:
            line["workloads"]["batched_uneven"] = batched_uneven(d, S, device, stream, seed_base,
                                                                      min(20000, args.train_steps))
        except RuntimeError as exc:
            line["workloads"]["batched_uneven"] = {"unavailable": str(exc).splitlines()[0][:160]}
    return line, S


# ---- the FP64 oracle on the host cores: whole frames (oracle.frame.simulate_frame as it stands: fields,
# warp, network with the unit-flux projection, blur), independent frames on separate processes (spawn, one per
# core, as the GPU runs independent replicas), timed from the first submitted frame to the last finished one
_ORACLE = {}


def _oracle_worker_init(img, basis, net, J_, N, ppd):
    from oracle import spectrum
    _ORACLE.update(img=img, basis=basis, net=net, J=J_, N=N, ppd=ppd)
    spectrum.lambdas(J_, N, ppd)  # the radial spectrum table (cached per process): setup, not frame work


def _oracle_frame(dr, seed, frame):
    from oracle import frame as oframe
    o = _ORACLE
    t0 = time.perf_counter()
    out = oframe.simulate_frame(o["img"], dr, seed, frame, o["J"], o["basis"], o["ppd"], o["N"], net=o["net"])
    return time.perf_counter() - t0, float(np.abs(out["out"]).sum())


def _oracle_ping(sec):
    time.sleep(sec)
    return os.getpid()


def oracle_frames(img, basis, net, dlist, N, n_timed, n_warm, workers):
    """Whole oracle frames on `workers` host processes; returns (wall seconds of the n_timed frames, mean
    seconds of one frame on one core)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"  # one core per worker process (inherited at spawn)
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=ctx, initializer=_oracle_worker_init,
                                initargs=(img, basis, net, J, N, PIX_PER_D)) as ex:
        # start and initialise every worker before anything is timed
        list(ex.map(_oracle_ping, [1.0] * workers))
        list(ex.map(_oracle_frame, [dlist[i % len(dlist)] for i in range(n_warm)], [7] * n_warm, range(n_warm)))
        t0 = time.perf_counter()
        res = list(ex.map(_oracle_frame, [dlist[i % len(dlist)] for i in range(n_timed)], [7] * n_timed,
                          range(n_warm, n_warm + n_timed)))
        wall = time.perf_counter() - t0
    return wall, float(np.mean([r[0] for r in res]))


def oracle_inputs(workload, basis=None, net=None):
    """Image, basis and network for the oracle frames.  Without a device basis / trained network (the reference
    arm runs on the host alone) the oracle's own SVD basis of the same 2000 PSFs and a network of the trained
    shape with seeded weights (the frame's cost does not depend on their values)."""
    from oracle import p2s as op2s, sampler as osampler
    from inputs import synthetic
    H, W, C, kind, K, dlist, _ = WORKLOADS[workload]
    N = osampler.grid_size(H, W, PIX_PER_D)
    img = synthetic.image_for(kind, H, W, C, seed=0)
    if basis is None:
        basis = op2s.build_basis(0, J, K, 2000, dlist)
    if net is None:
        rng = np.random.default_rng(0)
        params = {"W1": rng.standard_normal((256, J)) / 6, "b1": np.zeros(256),
                  "W2": rng.standard_normal((256, 256)) / 16, "b2": np.zeros(256),
                  "W3": rng.standard_normal((K, 256)) / 16, "b3": np.zeros(K)}
        in_scale = np.ones(J)
        in_scale[:2] = 0
        net = {"params": params, "in_scale": in_scale, "out_scale": np.full(K, 0.01),
               "out_shift": op2s.weights(np.zeros(J), J, basis)}
    return img, basis, net, dlist, N


def read_network_file(path, J_, K):
    """The network file of dfp2s_mlp_save (magic, version, J, K, then float32 arrays) as oracle parameters."""
    raw = open(path, "rb").read()
    if raw[:8] != b"DFP2SMLP" or tuple(np.frombuffer(raw[8:20], dtype="<i4")) != (1, J_, K):
        raise ValueError(f"{path} is not a J = {J_}, K = {K} network file")
    v = np.frombuffer(raw[20:], dtype="<f4").astype(np.float64)
    out, o = {}, 0
    for name, shp in (("W1", (256, J_)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)), ("W3", (K, 256)),
                      ("b3", (K,)), ("in_scale", (J_,)), ("out_scale", (K,)), ("out_shift", (K,))):
        n = int(np.prod(shp))
        out[name] = v[o:o + n].reshape(shp)
        o += n
    return {"params": {k: out[k] for k in ("W1", "b1", "W2", "b2", "W3", "b3")}, "in_scale": out["in_scale"],
            "out_scale": out["out_scale"], "out_shift": out["out_shift"]}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def config_for(workload, mode, world, extra=None):
    """The workload description both arms print."""
    H, W, C, kind, K, dlist, desc = WORKLOADS[workload]
    from oracle import sampler as osampler  # grid-size rule only
    cfg = {"workload": desc, "p2s": mode, "H": H, "W": W, "C": C, "J": J, "K": K,
           "N": osampler.grid_size(H, W, PIX_PER_D), "D_over_r0": dlist,
           "l2": "flushed between timed frames (256 MB write)", "parallelism": f"replicas{world}"}
    if extra:
        cfg.update(extra)
    return cfg


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="512", choices=sorted(WORKLOADS))
    ap.add_argument("--mode", default="learned", choices=["learned", "exact"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--train-steps", type=int, default=60000)
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-4k", action="store_true", help="skip the 3840x2160x3 half of the metric")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched uneven-request workload")
    ap.add_argument("--no-full-sampler", action="store_true", help="skip the full cross-spectrum sampler timing")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        # the FP64 oracle on the host cores: every step one whole frame of the workload; the frames run
        # concurrently, one per core, so the K timed frames take about K / cores frame times
        img, basis, net, dlist, N = oracle_inputs(args.workload)
        if args.mode == "exact":
            net = None
        cores = min(host_cores(), max(1, args.steps))
        wall, per = oracle_frames(img, basis, net, dlist, N, args.steps, args.warmup, cores)
        v = args.steps / wall
        sample = (f"whole {args.workload} frames (oracle.frame.simulate_frame: fields on the {N}x{N} grid, warp, "
                  f"{args.mode} P2S with the oracle's SVD basis of 2000 PSFs{' and a seeded network of the trained shape' if net else ''}, blur), "
                  f"{args.steps} timed frames on {cores} processes, {per:.2f} s per frame on one core")
        line = {"impl": "reference", "metric": "dense-field frames/s at 512^2 and 4K: learned vs exact P2S, same "
                "GB300, at tol", "value": v, "unit": "frames/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config_for(args.workload, args.mode, args.gpus),
                "cpu_baseline": {"value": v, "unit": "frames/s", "cores": cores, "kind": "oracle", "sample": sample},
                "e2e": {"value": v, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    line, S = run_ours(args, rank, world, device)
    if rank == 0:
        if not args.no_cpu_baseline:
            # the oracle on this host's cores, on the same workload with this run's device basis and trained
            # network (read back through the network file): one round of whole frames, one per core
            import tempfile
            basis = S["P_basis"].cpu().numpy().astype(np.float64)
            net = None
            if args.mode == "learned":
                fd, path = tempfile.mkstemp(suffix=".bin")
                os.close(fd)
                S["P"].save_mlp(path)
                net = read_network_file(path, J, S["K"])
                os.unlink(path)
            img, _, _, dlist, N = oracle_inputs(args.workload, basis=basis, net=net or {})
            cores = host_cores()
            nfr = cores if args.mode == "learned" else max(1, cores // 4)
            wall, per = oracle_frames(img, basis, net, dlist, N, nfr, 0, cores)
            line["cpu_baseline"] = {
                "value": nfr / wall, "unit": "frames/s", "cores": cores, "kind": "oracle",
                "sample": f"{nfr} whole {args.workload} frames ({args.mode} P2S with this run's SVD basis"
                          f"{' and trained network' if net else ''}) on {cores} processes in {wall:.1f} s, "
                          f"{per:.2f} s per frame on one core"}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()

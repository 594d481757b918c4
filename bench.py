#!/usr/bin/env python
"""Throughput of the Magnetic Gaussian slice renderer on one B300.

One step = one training iteration of the FeTA-shaped plain fit (256^3
phantom at 0.5 mm; 3 orthogonal stacks of 64 slices of 256 x 256 at 0.5 mm,
2 mm slice profile; 200k Gaussians): record pass + tile binning + forward
render, the FP64 L1+L2 slice loss with its gradient, and the adjoint (moments
+ chain to the Gaussian parameters). All of it runs in this repository's
CUDA kernels through the C ABI.

metric: fwd+bwd Gaussian-voxel pairs/s = P / step time, P = (Gaussian record,
slice voxel) pairs inside the K = 3 ellipsoid of the profile-convolved
covariance, counted on the device by mg_render_pair_count for the step's
input. The evaluated (tile-level) pair count is reported beside it.

The line's "fitted" sub-record times the same step on the Gaussians after a
2000-iteration L1+L2 fit (the state a reconstruction spends its iterations in).
The "sampler" records (top level on the initial Gaussians, in "fitted" on the
fitted ones) time the inference sampling onto the workload's isotropic target
grid.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mgauss|reference]
Under torchrun each rank renders its own independent replica (seed = rank):
weak scaling, no collective on the data path (the step does not shard).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "fwd+bwd Gaussian-voxel pairs/s"
UNIT = "pairs/s"
# kernels per library stage (the scans are two kernels each)
KERNELS_PER_STAGE = {"slices": 1, "k1_count": 1, "scan_records": 2, "k1_emit": 1, "chunks": 1, "bin_hist": 2,
                     "bin_colscan": 1, "scan_tiles": 2, "bin_scatter": 2, "render_fwd": 1, "zero_moments": 1,
                     "render_bwd": 1, "chain": 1, "loss": 1, "pair_count": 1, "nrf_fwd": 1, "nrf_bwd": 1, "rec_geom": 1, "rec_fill": 1}
# Algorithmic per-pair work of the evaluation kernels (SIMT FP32 pipe ops,
# MUFU ex2 ops): forward q (2 FMA) + accumulate (1 FMA) + 1 ex2; backward q
# (2 FMA) + the running column sums a += g 2^q (1 FMA), z += a, zz += z (2
# adds) + 1 ex2 (batches of more than 16 records; smaller batches split rows
# over lanes and take one more FP32 op per pair).
PAIR_OPS = {"render_fwd": (3, 1), "render_bwd": (5, 1)}
# DRAM bytes (read + write) per launch of the evaluation kernels on the
# FeTA-shaped workload, from ncu captures of the kernels as built
# (dram__bytes_read.sum + dram__bytes_write.sum of the backward on the initial
# Gaussians, profiles/k_render_fwd_bwd_feta256_full.md); None where a kernel
# has changed since its last capture (the forward, and both kernels on the
# Gaussians of the 2000-iteration fit, whose last captures predate the
# dependent-launch wait at their entry).
PROFILED_TRAFFIC = {"initial": {"render_fwd": None, "render_bwd": (238.94 + 58.37) * 1e6},
                    "fitted": {"render_fwd": None, "render_bwd": None}}
# B300 unit counts per SM and clock: 148 SMs, 128 FP32 lanes per SM per
# clock, 2032 MHz maximum SM clock; ex2.approx issues at 32 per SM per clock
# (measured on this part: 9.5e12 ex2/s at 2032 MHz over 148 SMs).
N_SM, FP32_LANES, MUFU_LANES, SM_MHZ = 148, 128, 32, 2032.0


def alu_peak_pairs(kernel: str) -> float:
    fp32, mufu = PAIR_OPS[kernel]
    per_clk = min(FP32_LANES / fp32, MUFU_LANES / mufu)
    return N_SM * per_clk * SM_MHZ * 1e6


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.idx)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) >= 9:
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# whole-job throughput over ranks (independent replicas, no data-path collective)
# ---------------------------------------------------------------------------
def job_throughput(units_local: float, ms_local: float, steps: int, dist=None, device="cpu"):
    """(units/s of the whole job, ms per step of the slowest rank, units per
    step of the whole job): every rank ran ``steps`` steps of its own replica
    in ``ms_local`` ms, processing ``units_local`` units per step; the job's
    time is the slowest rank's and its units are the sum over ranks."""
    import torch

    ms, units = float(ms_local), float(units_local)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        u = torch.tensor([units], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        ms, units = float(t.item()), float(u.item())
    ms_step = ms / steps
    return units / (ms_step / 1e3), ms_step, units


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def build_workload(name: str, seed: int, device, keep_volume: bool = False):
    import torch

    import mg_synth as ms

    maker = {"feta": ms.feta_workload, "tiny": ms.tiny_workload, "motion": ms.motion_workload,
             "stress": ms.stress_workload}[name]
    wl = maker(seed)
    vol = wl.phantom.volume_torch(device=str(device))
    vs = wl.phantom.spacing
    data = [ms.simulate_stack(vol, vs, s, seed=seed * 100 + i, noise_sigma=wl.noise_sigma, device=str(device))
            for i, s in enumerate(wl.stacks)]
    target = torch.cat([d.reshape(-1) for d in data]).contiguous()
    if not keep_volume:
        del vol
        vol = None
    if name == "tiny":
        G = ms.devoxelised_gaussians(wl.stacks, [d.cpu().numpy() for d in data], wl.n_gaussians, seed=seed)
    else:
        G = ms.phantom_init_gaussians(wl, seed=seed)
    if keep_volume:
        return wl, G, target, vol
    return wl, G, target


def fitted_gaussians(wl, G, target, dev, iterations: int = 2000):
    """The workload's Gaussians after an L1+L2 fit of ``iterations`` Adam steps
    (the state a reconstruction step runs on: a few Gaussians grow over many
    slices and tiles)."""
    import mg_synth as ms
    import torch

    from paper_2603_00145_b300 import recon

    cfg = recon.FitConfig(iterations=iterations, log_every=0)
    model, _, _ = recon.fit(wl.stacks, target, G, (0.0, 0.0, 0.0), wl.phantom.fov_mm / 2, cfg, device=dev)
    with torch.no_grad():
        mean, q, s, a = (x.detach().float().contiguous().cpu().numpy() for x in model.gaussians())
    return ms.Gaussians(mean, q, s, a)


# ---------------------------------------------------------------------------
# the mgauss arm
# ---------------------------------------------------------------------------
def device_step_timing(G, wl, target, dev, args, dist=None, state="initial"):
    """The device-resident step on Gaussians G: record pass + binning + forward
    with the fused L1 + L2 loss + adjoint, captured once as a CUDA graph and
    replayed ``args.steps`` times (L2 flushed between steps, CUDA events on
    the launching stream), then the same steps launched one by one for the
    evaluation kernels' live times and the per-stage breakdown. Returns a dict
    with the renderer, buffers and all figures."""
    import torch

    from paper_2603_00145_b300 import SliceRenderer
    from paper_2603_00145_b300.ops import mg_profile_enable, mg_profile_read, mg_profile_stages

    m, q, s, a = (torch.from_numpy(x).to(dev) for x in (G.mean, G.quat, G.scale, G.alpha))
    R = SliceRenderer(wl.stacks, device=dev, check=True)
    out = R.forward(m, q, s, a)  # sizes the workspace (grows on overflow)
    st = R.stats()
    R.set_capacity(int(st["records"] * 1.1) + 64, int(st["entries"] * 1.1) + 256, G.n)
    R.forward(m, q, s, a, out=out)
    pairs_inside, pairs_eval = R.pair_count(m, q, s, a)
    R.check = False
    nv = target.numel()
    grad = torch.empty(nv, dtype=torch.float32, device=dev)
    loss = torch.empty(2, dtype=torch.float64, device=dev)

    def step(mm, qq, ss, aa):
        # forward with the L1 + L2 loss and its gradient fused, then the adjoint
        R.forward_l1l2(mm, qq, ss, aa, target, out, grad, loss)
        return R.backward(mm, qq, ss, aa, grad)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 126 MB L2
    for _ in range(args.warmup):
        step(m, q, s, a)
    torch.cuda.synchronize()
    # the step's launches captured once as a CUDA graph (the library's stage
    # events off) and replayed in the timed region
    mg_profile_enable(False)
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        step(m, q, s, a)
    torch.cuda.current_stream(dev).wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step(m, q, s, a)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record()
        graph.replay()
        ev[k][1].record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    # the roofline's live kernel times: the same steps launched one by one with
    # events around the two evaluation kernels only; the per-stage breakdown
    # from a third set with events around every stage (they cost about 5 % of
    # the step)
    mg_profile_read(reset=True)
    mg_profile_stages(["render_fwd", "render_bwd"])
    for k in range(args.steps):
        flush.fill_(float(k))
        step(m, q, s, a)
    torch.cuda.synchronize()
    mg_profile_enable(False)
    prof_eval = mg_profile_read(reset=True)
    mg_profile_enable(True)
    for k in range(args.steps):
        flush.fill_(float(k))
        step(m, q, s, a)
    torch.cuda.synchronize()
    mg_profile_enable(False)
    prof = mg_profile_read(reset=True)
    prof.update({k: v for k, v in prof_eval.items() if v[1] > 0})  # the evaluation kernels as timed
    ms_total = sum(e0.elapsed_time(e1) for e0, e1 in ev)
    value, ms_step, pairs_job = job_throughput(pairs_inside, ms_total, args.steps, dist, dev)
    st = R.stats()
    assert st["status"] == 0, f"device status {st['status']} during the timed steps"
    stages = {k: v for k, v in prof.items() if v[1] > 0}
    roof = roofline(stages, pairs_eval, traffic=PROFILED_TRAFFIC.get(state) if args.workload == "feta" else None)
    del flush, graph
    return {"R": R, "out": out, "grad": grad, "loss": loss, "dev_in": (m, q, s, a), "value": value,
            "ms_step": ms_step, "pairs_inside": pairs_inside, "pairs_eval": pairs_eval, "stats": st, "stages": stages,
            "roofline": roof, "clocks": clk}


def roofline(stages, pairs_eval, traffic=None):
    """Roofline of the dominant evaluation kernel from its live CUDA-event time."""
    dom = max(("render_fwd", "render_bwd"), key=lambda k: stages.get(k, (0, 0))[0])
    dom_ms = stages[dom][0] / stages[dom][1]
    achieved = pairs_eval / (dom_ms / 1e3)
    peak = alu_peak_pairs(dom)
    roof = {"bound": "alu", "kernel": dom, "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gpair/s",
            "frac": achieved / peak, "traffic": (traffic or {}).get(dom),
            "traffic_unit": "bytes per launch (ncu capture)",
            "peak_basis": (f"{N_SM} SMs x min({FP32_LANES}/{PAIR_OPS[dom][0]} FP32, {MUFU_LANES}/{PAIR_OPS[dom][1]} "
                           f"MUFU) pairs/clk x {SM_MHZ:.0f} MHz (nominal unit counts)"),
            "units_per_launch": pairs_eval, "ms_per_launch": dom_ms}
    other = {}
    for k in ("render_fwd", "render_bwd"):
        if k in stages and k != dom:
            t_ = stages[k][0] / stages[k][1]
            other[k] = {"ms": t_, "Gpair_s": pairs_eval / (t_ / 1e3) / 1e9,
                        "frac": pairs_eval / (t_ / 1e3) / alu_peak_pairs(k), "traffic": (traffic or {}).get(k)}
    roof["other"] = other
    return roof


# Tensor-core work of the hash-grid NRF per point (BF16 mma, FP32 accumulate):
# layers 32->64, 64->64, 64->1 = 6208 MAC forward; the training backward
# recomputes the forward, forms dW (6208 MAC) and the deltas of the hidden
# layers and the features (4096 + 2048 MAC).
NRF_FLOPS_FWD = 2 * (32 * 64 + 64 * 64 + 64)
NRF_FLOPS_BWD = NRF_FLOPS_FWD + 2 * (32 * 64 + 64 * 64 + 64) + 2 * (64 * 64 + 64 * 32)
# L2 requests per 2^20 points from one ncu capture of the BF16 grid kernels
# (profiles/nrf_grid_bf16.md): table gathers (forward) and table-gradient
# atomics (backward); None once a kernel changes.
NRF_PROFILED = {"fwd_gather_requests": 83408692, "bwd_red_requests": 101138216, "bwd_gather_requests": 3131437}


def sampler_timing(G, wl, dev, steps: int, warmup: int):
    """Inference sampling (mg_sample_volume: records, binning and the forward
    over the planes of the isotropic target grid) of Gaussians G onto the
    workload's target grid; CUDA events around each call, L2 flushed between
    calls. Evaluated pairs = (record, 8x8 tile) entries x 64 (the grid's edge is
    a multiple of 8)."""
    import torch

    from paper_2603_00145_b300.ops import VolumeSampler, _opts, mg_sample_volume

    m, q, s_, a = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (G.mean, G.quat, G.scale, G.alpha)]
    S = VolumeSampler(wl.target_G, wl.target_spacing, device=dev)
    out = torch.empty(wl.target_G ** 3, dtype=torch.float32, device=dev)
    S(m, q, s_, a, out=out)  # sizes the workspace
    o = _opts(S.K, S.f64, *S.caps)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    t = 0.0
    for k in range(warmup + steps):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mg_sample_volume(m, q, s_, a, S.centre, S.h, S.G, o, out, S.ws, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= warmup:
            t += e0.elapsed_time(e1)
    ms_ = t / steps
    st = S.last_stats
    pairs = int(st["entries"]) * 64
    return {"grid": f"{wl.target_G}^3 at {wl.target_spacing} mm", "gaussians": G.n, "ms": ms_,
            "voxels_per_s": wl.target_G ** 3 / (ms_ * 1e-3), "records": int(st["records"]),
            "entries": int(st["entries"]), "evaluated_pairs": pairs, "evaluated_pairs_per_s": pairs / (ms_ * 1e-3)}


def nrf_pair_timing(wl, dev, steps: int, warmup: int, n: int = 1 << 20):
    """The neural residual field's training pair as the reconstruction runs it
    once the field is on: mg_nrf_fwd_at (BF16 hash grid, adds r at 2^20 random
    slice voxels, storing the points' encoding) then mg_nrf_bwd_at (gradients
    of the parameters and the table, reading the encoding back), on the
    workload's voxel coordinates; CUDA events around each call."""
    import torch

    import mg_synth as ms
    from paper_2603_00145_b300 import recon
    from paper_2603_00145_b300.ops import NRF, mg_nrf_bwd_at, mg_nrf_fwd_at

    coords = recon.voxel_coords(wl.stacks, (0.0, 0.0, 0.0), wl.phantom.fov_mm / 2, device=dev)
    rows = coords.numel() // 3
    W, b, t = ms.nrf_init("grid", 0, bf16=True, last_gain=0.1)
    net = NRF("grid", "bf16", W, b, t, device=dev)
    acc = torch.zeros(rows, device=dev)
    ga = torch.randn(rows, device=dev)
    gp, gt = torch.empty_like(net.params), torch.empty_like(net.table)
    enc = net.enc_cache(n)
    tf = tb = 0.0
    for k in range(warmup + steps):
        idx = torch.randint(0, rows, (n,), device=dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        mg_nrf_fwd_at(net, coords, idx, n, acc, enc=enc)
        ev[1].record()
        mg_nrf_bwd_at(net, coords, idx, n, ga, gp, gt, enc=enc)
        ev[2].record()
        torch.cuda.synchronize()
        if k >= warmup:
            tf += ev[0].elapsed_time(ev[1])
            tb += ev[1].elapsed_time(ev[2])
    fwd_ms, bwd_ms = tf / steps, tb / steps
    peaks = measured_peaks()
    peak = float(peaks.get("bf16_tflops", 1800.0))
    ach_f = NRF_FLOPS_FWD * n / (fwd_ms * 1e-3) / 1e12
    ach_b = NRF_FLOPS_BWD * n / (bwd_ms * 1e-3) / 1e12
    dom = "nrf_bwd" if bwd_ms >= fwd_ms else "nrf_fwd"
    ach = ach_b if dom == "nrf_bwd" else ach_f
    return {"points": n, "encoding": "hash grid 16 x 2, 2 x 64 ReLU, BF16 mma.sync, FP32 accumulation",
            "fwd_at_ms": fwd_ms, "bwd_at_ms": bwd_ms, "pair_ms": fwd_ms + bwd_ms,
            "roofline": {"bound": "tensor", "kernel": dom, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach / peak, "peak_basis": "bf16_tflops of MEASURED_PEAKS.json (measured, burst)"
                         if "bf16_tflops" in peaks else "fallback 1.8 PFLOP/s",
                         "traffic": None,
                         "note": "the MLP is 64 wide; the kernels are bound by L2 requests (hash-table "
                                 "gathers forward, table-gradient atomics backward), not by the tensor pipe"},
            "l2_requests_profiled": NRF_PROFILED}


def run_mgauss(args, rank, world, local_rank):
    import torch

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    wl, G, target = build_workload(args.workload, args.seed + rank, dev)
    if args.only == "nrf":
        if rank == 0:
            print(json.dumps({"metric": "NRF training pair ms per 2^20 points", "workload": wl.name,
                              "nrf": nrf_pair_timing(wl, dev, args.steps, args.warmup)}), flush=True)
        return
    if args.gaussians:
        import mg_synth as ms

        z = np.load(args.gaussians)
        G = ms.Gaussians(z["mean"], z["quat"], z["scale"], z["alpha"])
    elif args.fitted:
        G = fitted_gaussians(wl, G, target, dev)
    if args.save_gaussians and rank == 0:
        np.savez(args.save_gaussians, mean=G.mean, quat=G.quat, scale=G.scale, alpha=G.alpha)
    T = device_step_timing(G, wl, target, dev, args, dist, state="fitted" if args.fitted else
                           "loaded" if args.gaussians else "initial")
    R, out, grad, loss = T["R"], T["out"], T["grad"], T["loss"]
    value, ms_step, pairs_inside, pairs_eval = T["value"], T["ms_step"], T["pairs_inside"], T["pairs_eval"]
    stages, roof, clk, st = T["stages"], T["roofline"], T["clocks"], T["stats"]
    nv = target.numel()
    from paper_2603_00145_b300.ops import mg_profile_enable

    # end to end through the C ABI with host buffers: every step copies its
    # inputs (Gaussian parameters and target slices) from pinned memory, runs,
    # and reads the loss and the gradients back, and the host waits for them.
    # Each step is one CUDA graph holding its copies and its compute: on a
    # copy stream forked from the graph's stream, the step's Gaussians (a fit
    # would update them on the host in between), then the NEXT step's target
    # slices into the other of two device buffers (they do not depend on this
    # step, so that 50 MB copy overlaps this step's compute); on the graph's
    # stream the compute, then the gradients and the loss copied back. The
    # Gaussians go ahead of the target on the copy stream (behind it they
    # would hold the step). The timed window holds exactly K steps: the first
    # step's own target is copied before its graph, the last step's graph
    # copies no target for a step after it.
    loss_ref = loss.cpu()  # the device-resident step's loss (a fixed-order reduction)
    host_in = [torch.from_numpy(x).pin_memory() for x in (G.mean, G.quat, G.scale, G.alpha)]
    host_tgt = target.cpu().pin_memory()
    dev_in = [torch.empty_like(x, device=dev) for x in host_in]
    for d_, h_ in zip(dev_in, host_in):
        d_.copy_(h_)
    host_out = [torch.empty((G.n, w), dtype=torch.float32).pin_memory() for w in (3, 4, 3)] + \
        [torch.empty(G.n, dtype=torch.float32).pin_memory()]
    dev_gout = [torch.empty(h_.shape, dtype=torch.float32, device=dev) for h_ in host_out]
    host_loss = torch.empty(2, dtype=torch.float64).pin_memory()
    h2d = sum(x.numel() * x.element_size() for x in host_in) + host_tgt.numel() * 4
    d2h = sum(x.numel() * x.element_size() for x in host_out) + 16
    tgt_buf = [target, torch.empty_like(target)]
    main = torch.cuda.current_stream(dev)
    side = torch.cuda.Stream(dev)
    mg_profile_enable(False)

    def capture_step(b, copy_next):
        gr_ = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr_):
            cap = torch.cuda.current_stream(dev)
            side.wait_stream(cap)
            with torch.cuda.stream(side):
                for d_, h_ in zip(dev_in, host_in):
                    d_.copy_(h_, non_blocking=True)
            cap.wait_stream(side)  # the compute waits for the Gaussians only
            if copy_next:
                with torch.cuda.stream(side):
                    tgt_buf[1 - b].copy_(host_tgt, non_blocking=True)
            R.forward_l1l2(*dev_in, tgt_buf[b], out, grad, loss)
            R.backward(*dev_in, grad, out=dev_gout)
            for h_, g_ in zip(host_out, dev_gout):
                h_.copy_(g_, non_blocking=True)
            host_loss.copy_(loss, non_blocking=True)
            cap.wait_stream(side)  # the next target's copy joins the graph's end
        return gr_

    # [parity][copies the next target]
    e2e_graphs = [[capture_step(b, c) for c in (False, True)] for b in range(2)]
    torch.cuda.synchronize()

    def run_e2e(n_steps):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(main)
        tgt_buf[0].copy_(host_tgt, non_blocking=True)
        for k in range(n_steps):
            e2e_graphs[k % 2][k + 1 < n_steps].replay()
            main.synchronize()  # the host reads this step's loss and gradients
        t1.record(main)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1)

    run_e2e(args.warmup)
    e2e_ms = run_e2e(args.steps)
    e2e_value, e2e_ms_step, _ = job_throughput(pairs_inside, e2e_ms, args.steps, dist, dev)
    e2e_ms = e2e_ms_step * args.steps

    launches = sum(KERNELS_PER_STAGE.get(k, 1) * v[1] for k, v in stages.items())

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded ellipsoid phantom, simulated stacks)",
            "config": {"workload": wl.name + ("-fitted" if args.fitted else "") +
                       ("-" + os.path.basename(args.gaussians) if args.gaussians else ""), "gaussians": G.n,
                       "stacks": len(wl.stacks),
                       "slices": sum(s_.n_slices for s_ in wl.stacks), "voxels": nv, "cutoff_k": 3.0,
                       "records": st["records"], "entries": st["entries"],
                       "pairs_inside_per_step": pairs_inside, "pairs_evaluated_per_step": pairs_eval,
                       "binning_efficiency": pairs_inside / max(pairs_eval, 1),
                       "l2": "flushed between timed steps (256 MiB write)", "launch": "CUDA graph of the step, replayed",
                       "parallelism": f"replicas x{world}"},
            "roofline": roof,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_ms / args.steps,
                    "loss_equals_device_step": bool(torch.equal(host_loss, loss_ref)),
                    "overlap": "each step one CUDA graph: its Gaussians, then step k+1's target slices, copied "
                               "on a forked copy stream (the target copy overlaps the compute), the compute, the "
                               "gradients and loss copied back; host sync every step"},
            "gpu_launches": launches,
            "stages_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()},
            "stages_note": "the timed steps replay a CUDA graph of the step; render_fwd and render_bwd timed "
                           "with events in the same steps launched one by one (events around those two kernels "
                           "only), the other stages in a third set with events around every stage",
            "clocks": clk}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(G, wl, args.cpu_seconds)
    del T, R, out, grad, e2e_graphs, dev_gout
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.fitted and args.fit_iters > 0:
        # the same step on the Gaussians after an L1 + L2 fit: the state a
        # reconstruction spends its iterations in (a few Gaussians grown over
        # whole slices, many tiles with few records)
        t0 = time.perf_counter()
        Gf = fitted_gaussians(wl, G, target, dev, iterations=args.fit_iters)
        fit_s = time.perf_counter() - t0
        F = device_step_timing(Gf, wl, target, dev, args, None, state="fitted")
        line["fitted"] = {"state": f"after {args.fit_iters} L1+L2 Adam iterations ({fit_s:.1f} s incl. set-up)",
                          "value": F["value"], "unit": UNIT, "ms_per_step": F["ms_step"],
                          "records": F["stats"]["records"], "entries": F["stats"]["entries"],
                          "pairs_inside_per_step": F["pairs_inside"], "pairs_evaluated_per_step": F["pairs_eval"],
                          "roofline": F["roofline"],
                          "stages_ms_per_step": {k: v[0] / args.steps for k, v in F["stages"].items()},
                          "clocks": F["clocks"]}
        del F
        torch.cuda.empty_cache()
        if args.sampler:
            line["fitted"]["sampler"] = sampler_timing(Gf, wl, dev, args.steps, args.warmup)
            torch.cuda.empty_cache()
    if rank == 0 and world == 1 and args.nrf:
        line["nrf"] = nrf_pair_timing(wl, dev, args.steps, args.warmup)
        torch.cuda.empty_cache()
    if rank == 0 and world == 1 and args.sampler:
        line["sampler"] = sampler_timing(G, wl, dev, args.steps, args.warmup)
        torch.cuda.empty_cache()
    if rank == 0 and world == 1 and args.recon_iters > 0:
        line["recon"] = run_recon(args, dev)
        if args.radius_sweep:
            line["radius_sweep"] = run_radius_sweep(args, dev)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()



# ---------------------------------------------------------------------------
# reconstruction time at equal PSNR (the second half of the metric)
# ---------------------------------------------------------------------------
RECON_FORMS = {
    "gaussians_fp32": {},
    "gaussians_fp32_ssim_loss": {"loss": "paper"},
    "nrf_grid_fp32": {"nrf": "grid", "nrf_precision": "fp32"},
    "nrf_grid_bf16": {"nrf": "grid", "nrf_precision": "bf16"},
}


def run_recon(args, dev):
    """Full reconstructions of the workload: ``--recon-iters`` Adam iterations
    of the L1+L2 slice loss (CUDA-graph replay of the whole iteration) plus
    inference sampling onto the phantom's isotropic grid; wall seconds and
    volume PSNR (FP64) against the phantom for the Gaussians alone (FP32) and
    with the hash-grid NRF (switched on at half of the iterations, 2^20-voxel
    batches) in FP32 and in BF16; the Gaussians alone are also fitted with the
    paper's smooth-L1 + 0.5 SSIM loss (Sec. 3.5.2). Each form runs with ``--recon-seeds`` seeds
    (batch order and NRF initialisation): the fit is a stochastic
    optimisation whose PSNR moves by a few tenths of a dB from run to run, so
    forms are compared on their means."""
    import torch

    from paper_2603_00145_b300 import recon
    from paper_2603_00145_b300.ops import NRF, mg_nrf_bwd, mg_nrf_fwd

    wl, G, target, vol = build_workload(args.workload, args.seed, dev, keep_volume=True)
    gd = vol.shape[0]
    half = wl.phantom.fov_mm / 2
    # untimed warm-up of every form (lazy module loading, first graph captures, allocator growth)
    for kw in RECON_FORMS.values():
        cfg = recon.FitConfig(iterations=40, nrf_start=20, nrf_batch=1 << 20, **kw)
        model, nrf, _ = recon.fit(wl.stacks, target, G, (0.0, 0.0, 0.0), half, cfg, device=dev)
        recon.sample(model, nrf, gd, wl.phantom.spacing)
        del model, nrf
    torch.cuda.synchronize()
    forms = {}
    for name, kw in RECON_FORMS.items():
        runs = []
        for seed in range(args.recon_seeds):
            cfg = recon.FitConfig(iterations=args.recon_iters, nrf_start=args.recon_iters // 2, nrf_batch=1 << 20,
                                  log_every=0, seed=seed, nrf_seed=seed, **kw)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            model, nrf, st = recon.fit(wl.stacks, target, G, (0.0, 0.0, 0.0), half, cfg, device=dev)
            V = recon.sample(model, nrf, gd, wl.phantom.spacing)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
            runs.append({"seed": seed, "seconds": sec, "fit_seconds": st["seconds"],
                         "replay_seconds": st["seconds_replay"], "psnr_db": recon.psnr(V, vol),
                         "final_loss": st["final_loss"], "iterations": st["iterations"],
                         "graph_captures": st["graph_captures"]})
            del model, nrf, V
            torch.cuda.empty_cache()
        ps = [r["psnr_db"] for r in runs]
        ts = [r["seconds"] for r in runs]
        forms[name] = {"seconds_mean": statistics.mean(ts), "psnr_db_mean": statistics.mean(ps),
                       "psnr_db_std": statistics.stdev(ps) if len(ps) > 1 else 0.0, "runs": runs}
    # the NRF pass alone: forward + backward of one 2^20-point batch, CUDA events
    import mg_synth as ms

    nrf_ms = {}
    xyz = torch.rand(1 << 20, 3, device=dev) * 2 - 1
    gout = torch.randn(1 << 20, device=dev)
    out = torch.empty(1 << 20, device=dev)
    for prec in ("fp32", "bf16"):
        W, b, t = ms.nrf_init("grid", 0, bf16=(prec == "bf16"), last_gain=0.1)
        net = NRF("grid", prec, W, b, t, device=dev)
        gp, gt = torch.empty_like(net.params), torch.empty_like(net.table)
        for _ in range(3):
            mg_nrf_fwd(net, xyz, out)
            mg_nrf_bwd(net, xyz, gout, gp, gt)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(20):
            mg_nrf_fwd(net, xyz, out)
            mg_nrf_bwd(net, xyz, gout, gp, gt)
        e1.record()
        torch.cuda.synchronize()
        nrf_ms[prec] = e0.elapsed_time(e1) / 20
    f32, b16, g32 = forms["nrf_grid_fp32"], forms["nrf_grid_bf16"], forms["gaussians_fp32"]
    return {"workload": wl.name, "iterations": args.recon_iters, "seeds": args.recon_seeds,
            "sampling": f"{gd}^3 at {wl.phantom.spacing} mm", "loss": "mean|r| + mean r^2 (FP64)",
            "nrf": "hash grid 16x2, 2x64 ReLU, on at half, 2^20 voxels/iter",
            "forms": forms,
            "bf16_minus_fp32_psnr_db": b16["psnr_db_mean"] - f32["psnr_db_mean"],
            # paired by seed (same NRF initialisation and batches); the standard
            # error says how far the mean difference is resolved
            "bf16_minus_fp32_psnr_db_sem": _paired_sem(b16["runs"], f32["runs"]),
            "bf16_speedup_vs_fp32": f32["seconds_mean"] / b16["seconds_mean"],
            "nrf_minus_gaussians_psnr_db": b16["psnr_db_mean"] - g32["psnr_db_mean"],
            "nrf_fwd_bwd_ms_per_2^20_points": nrf_ms}


def _paired_sem(runs_a, runs_b):
    d = [a["psnr_db"] - b["psnr_db"] for a, b in zip(runs_a, runs_b)]
    return statistics.stdev(d) / len(d) ** 0.5 if len(d) > 1 else None


def run_radius_sweep(args, dev):
    """The paper's local set (Eqs. E4-E6) at several block radii: the same
    FeTA-shaped fit (L1+L2, CUDA-graph replay) with the cell grid at the
    Gaussian spacing (one Gaussian per cell on average, the reading of the
    paper's grids), one seed per radius; seconds per fit + sampling, PSNR,
    and the evaluated pairs of one step, beside the K-sigma local set."""
    import torch

    from paper_2603_00145_b300 import recon

    wl, G, target, vol = build_workload(args.workload, args.seed, dev, keep_volume=True)
    gd = vol.shape[0]
    half = wl.phantom.fov_mm / 2
    spacing = float(np.median(np.asarray(G.scale)[:, 0]))  # the initial isotropic sigma = the Gaussian spacing
    res = max(1, int(round(2 * half / spacing)))
    out = {"grid_res": res, "cell_mm": 2 * half / res, "iterations": args.recon_iters, "runs": []}
    forms = [("ksigma", None)] + [("cells", r) for r in args.radius_sweep]
    for kind, r in forms:
        kw = {} if kind == "ksigma" else {"local_set": "cells", "grid_res": res, "block_radius": r}
        cfg = recon.FitConfig(iterations=40, **kw)
        recon.fit(wl.stacks, target, G, (0.0, 0.0, 0.0), half, cfg, device=dev)   # warm-up
        cfg = recon.FitConfig(iterations=args.recon_iters, **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        model, nrf, st = recon.fit(wl.stacks, target, G, (0.0, 0.0, 0.0), half, cfg, device=dev)
        V = recon.sample(model, nrf, gd, wl.phantom.spacing, cells=recon.cells_of(cfg, (0.0, 0.0, 0.0), half))
        torch.cuda.synchronize()
        out["runs"].append({"local_set": kind, "block_radius": r, "seconds": time.perf_counter() - t0,
                            "ms_per_iteration": 1e3 * st["seconds_replay"] / max(st["iterations"], 1),
                            "psnr_db": recon.psnr(V, vol)})
        del model, V
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# the CPU oracle (baseline leg and the reference arm)
# ---------------------------------------------------------------------------
def oracle_sample_step(G, wl, picks):
    """Oracle forward + adjoint (with the L1+L2 loss gradient) on the picked
    slices of the workload; returns the sub-stacks and their records."""
    import mg_synth as ms
    import oracle as orc
    from oracle import metrics

    sub, _ = ms.pick_slices(wl.stacks, picks)
    rec = orc.records(G, sub)
    S = orc.render(G, sub, rec)
    _, g = metrics.l1_l2(S, np.zeros_like(S))
    orc.grad(G, sub, rec, g)
    return sub, rec


def _sample_pairs(G, wl, picks):
    import mg_synth as ms
    import oracle as orc

    tot = 0
    for pk in picks:
        sub, _ = ms.pick_slices(wl.stacks, [pk])
        tot += orc.pair_counts(G, sub, orc.records(G, sub))[0]
    return tot


def cpu_baseline(G, wl, seconds: float):
    """The oracle as it stands, on whole slices of the same workload (one slice
    of each stack in turn) for about ``seconds`` of host time."""
    n_sl = [s.n_slices for s in wl.stacks]
    picks = []
    t0 = time.perf_counter()
    i = 0
    while time.perf_counter() - t0 < seconds or i == 0:
        pk = (i % len(n_sl), (i * 7 + 3) % n_sl[i % len(n_sl)])
        oracle_sample_step(G, wl, [pk])
        picks.append(pk)
        i += 1
    el = time.perf_counter() - t0
    pairs = _sample_pairs(G, wl, picks)
    return {"value": pairs / el, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{len(picks)} full slices (forward + adjoint, FP64, OpenMP) of the same workload in "
                      f"{el:.1f} s; pairs counted by the oracle"}


def run_reference(args, rank, world):
    """The reference arm: the CPU FP64 oracle on the same workload and metric,
    each step a bounded sample (one full slice, forward + adjoint)."""
    if rank != 0:
        return
    import torch  # noqa: F401

    import mg_synth as ms

    wl = {"feta": ms.feta_workload, "tiny": ms.tiny_workload, "motion": ms.motion_workload,
          "stress": ms.stress_workload}[args.workload](args.seed)
    G = ms.phantom_init_gaussians(wl, seed=args.seed) if args.workload != "tiny" else None
    if G is None:
        vol = wl.phantom.volume()
        data = [ms.simulate_stack(vol, 1.0, s, seed=i, noise_sigma=wl.noise_sigma).numpy()
                for i, s in enumerate(wl.stacks)]
        G = ms.devoxelised_gaussians(wl.stacks, data, wl.n_gaussians, seed=args.seed)
    n_sl = [s.n_slices for s in wl.stacks]
    picks = [(i % len(n_sl), (i * 7 + 3) % n_sl[i % len(n_sl)]) for i in range(args.warmup + args.steps)]
    tt = 0.0
    pairs = 0
    for i, pk in enumerate(picks):
        t0 = time.perf_counter()
        oracle_sample_step(G, wl, [pk])
        el = time.perf_counter() - t0
        if i >= args.warmup:
            tt += el
            pairs += _sample_pairs(G, wl, [pk])
    value = pairs / tt
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": wl.name, "gaussians": G.n, "sample_per_step": "one full slice, forward + adjoint"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{args.steps} slices of the workload, one per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["mgauss", "reference"], default="mgauss")
    ap.add_argument("--workload", default="feta", choices=["feta", "tiny", "motion", "stress"])
    ap.add_argument("--fitted", action="store_true",
                    help="time the step on the Gaussians after a 2000-iteration L1+L2 fit instead of the initial ones")
    ap.add_argument("--fit-iters", type=int, default=2000,
                    help="iterations of the fit whose Gaussians the 'fitted' sub-record times (0: skip it)")
    ap.add_argument("--nrf", type=int, default=1, help="time the NRF training pair (1) or not (0)")
    ap.add_argument("--sampler", type=int, default=1, help="time the volume sampler on the target grid (1) or not (0)")
    ap.add_argument("--only", choices=["nrf"], default=None,
                    help="nrf: time only the NRF training pair and print its line")
    ap.add_argument("--gaussians", default=None,
                    help="time the step on the Gaussians of this .npz (mean, quat, scale, alpha) instead")
    ap.add_argument("--save-gaussians", default=None,
                    help="write the Gaussians the step is timed on (initial, fitted or loaded) to this .npz")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--recon-iters", type=int, default=2000,
                    help="iterations of each timed full reconstruction (0: skip the reconstruction timing)")
    ap.add_argument("--recon-seeds", type=int, default=5, help="runs (seeds) per reconstruction form")
    ap.add_argument("--radius-sweep", type=lambda v: [int(x) for x in v.split(",")], default=[],
                    help="block radii of the paper's cell-grid local set to fit and time, e.g. 3,4,5,6,7")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if (args.fitted or args.gaussians or args.only) and args.impl == "reference":
        ap.error("--fitted, --gaussians and --only concern the GPU arm; the reference arm times the oracle on the "
                 "initial Gaussians only")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_mgauss(args, rank, world, local_rank)


if __name__ == "__main__":
    main()

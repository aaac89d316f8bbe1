#!/usr/bin/env python
"""Throughput of the checkpointed FWI gradient with lossy checkpoint
compression (Kukreja et al.) on GB300.

One step = one shot gradient on the Overthrust-shaped workload: 881 x 881 x 287
grid at 25 m, 40-cell absorbing layer, 2286 steps of 1.75 ms (4000 ms), 8 Hz
Ricker source near the surface centre, 441 x 441 receivers, full-history
checkpoints compressed at atol = 1e-4 and held in HBM.  Forward sweep with
compression of every state, misfit, adjoint sweep with decompression and
imaging -- the whole hot path.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

With N GPUs (torchrun) each rank models its own shot and the ranks' gradients
and misfits are summed (stacking, one all-reduce per step).  Prints one JSON
line (rank 0).  The default run finishes in a few minutes.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "shot-gradients/s at fixed gradient error"
UNIT = "shot-gradients/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="fwi", choices=["fwi", "reference"])
    p.add_argument("--atol", type=float, default=1e-4)
    p.add_argument("--nt", type=int, default=2286, help="time steps (2286 = 4000 ms)")
    p.add_argument("--grid", default="881,881,287")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-verify", action="store_true")
    p.add_argument("--arena-gb", type=float, default=0.0,
                   help="checkpoint arena size (0 = all free memory minus the working set)")
    p.add_argument("--workload", default="overthrust",
                   choices=["overthrust", "batch", "fwi", "codec", "tradeoff"],
                   help="batch: 32-shot survey, batched plan against one call per shot; "
                        "fwi: 16-shot inversion through autograd, batched against per shot; "
                        "codec: 512^3 shell snapshots, atol sweep; "
                        "tradeoff: gradient error vs memory for compression, subsampling, binomial")
    p.add_argument("--iters", type=int, default=10, help="fwi workload: descent iterations per path")
    p.add_argument("--shots", type=int, default=32)
    p.add_argument("--ckpt-k", type=int, default=10, help="batch workload: checkpoint pair every K steps")
    return p.parse_args()


# ---------------------------------------------------------------- distributed
def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return ws, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x: float) -> float:
    if pg is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def stack(pg, grad, phi: float) -> float:
    """Stacking across ranks (Sec. 2: the misfit and its gradient are sums
    over shots): every rank ends the step holding the sum of all ranks'
    shot gradients (in place) and returns the summed misfit."""
    if pg is None:
        return phi
    import torch
    pg.all_reduce(grad, op=pg.ReduceOp.SUM)
    t = torch.tensor([phi], dtype=torch.float64, device=grad.device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


# ---------------------------------------------------------------- workload
def workload(args, rank):
    import numpy as np
    from paper_2009_12623_gb300 import synth
    nx, ny, nz = (int(v) for v in args.grid.split(","))
    nbl = min(40, min(nx, ny, nz) // 6)
    # one shot per rank: sources 40 cells apart along x (wrapping inside the
    # absorbing layer), just under the water surface
    lo, hi = nbl + 1, nx - nbl - 2
    sx = lo + (nx // 2 - lo + 40 * rank) % max(1, hi - lo + 1)
    shot = synth.overthrust_like_shot(nx=nx, ny=ny, nz=nz, nt=args.nt, nbl=nbl, src_xy=(sx, ny // 2))
    return shot, np.float32


def config_dict(args, shot, policy):
    g = shot.geom
    return {"workload": f"overthrust-like single-shot gradient {g.nx}x{g.ny}x{g.nz} at {g.h:.0f} m, "
                        f"nt={g.nt} (dt={g.dt * 1e3:.2f} ms), 8 Hz Ricker, {len(shot.rec)} receivers, "
                        f"{policy}",
            "grid": [g.nx, g.ny, g.nz], "nt": g.nt, "atol": args.atol, "checkpoints": policy,
            "l2_flush": "inputs larger than L2 (0.9 GB fields)", "parallelism": "shot per GPU"}


# kernel classes of the gradient that run alone on the sweep's stream
IN_ORDER = ("stencil_forward", "stencil_adjoint", "zfp_decode")


def kernel_bytes(cells, enc_bytes_per_launch, live=1.0, image_in_decoder=False):
    """Algorithmic bytes per launch (halos and scratch excluded).  `live` is
    the mean fraction of each stored state's blocks that are not coded as
    zero.  Full-history compressed sweeps (image_in_decoder) run the adjoint
    step as a plain step (16 B/cell) and image in the decoder, which reads
    the stream and, for live blocks only, lambda_{k-1}, lambda_k,
    lambda_{k+1} and g and writes g (20 B/value); otherwise the adjoint
    stencil images (16 + 12 B/cell: u^k and g) after a decoder that writes
    u^k (4 B/value)."""
    if image_in_decoder:
        adj, dec = 16.0 * cells, 20.0 * live * cells + enc_bytes_per_launch
    else:
        adj, dec = (16.0 + 12.0 * live) * cells, 4.0 * live * cells + enc_bytes_per_launch
    return {
        "stencil_forward": 16.0 * cells,                 # read u^n, u^{n-1}, m; write u^{n+1}
        "stencil_adjoint": adj,
        "zfp_encode": 4.0 * cells + enc_bytes_per_launch,
        "zfp_decode": dec,
    }


def source_hash(kernel: str) -> str:
    """Hash of the sources the kernel's translation unit compiles: its .cu
    file and the project headers it includes."""
    csrc = os.path.join("paper_2009_12623_gb300", "csrc")
    common = [os.path.join(csrc, "common.cuh"), os.path.join("include", "fwi.h")]
    files = {"stencil_forward": [os.path.join(csrc, "stencil.cu")],
             "stencil_adjoint": [os.path.join(csrc, "stencil.cu")],
             "zfp_encode": [os.path.join(csrc, "codec.cu"), os.path.join(csrc, "codec_block.cuh")],
             "zfp_decode": [os.path.join(csrc, "codec.cu"), os.path.join(csrc, "codec_block.cuh")]}
    h = hashlib.sha256()
    for f in files[kernel] + common:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, cells: int):
    """DRAM bytes per launch from the committed ncu summary (scaled from the
    captured case by cells), if it was taken on the current source of that
    kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    e = d.get(kernel)
    if not e or e.get("source_hash") != source_hash(kernel):
        return None
    return round(e["dram_bytes_per_launch"] * cells / e["cells"])


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------- CPU oracle sample
SAMPLE_STEP = 1200          # the codec sample is the state at this step (2.1 s of 4 s)
SAMPLE_SLAB = 16            # planes per slab
_snapshot_cache = {}


def sample_planes(g):
    """Four 16-plane slabs: at the source depth and at 1/3, 1/2 and 2/3 of the
    depth (never the absorbing layer alone)."""
    zs = min(g.nbl + 2, g.nz - SAMPLE_SLAB)
    starts = [zs] + [min(g.nz - SAMPLE_SLAB, max(zs + SAMPLE_SLAB, int(g.nz * q))) for q in (1 / 3, 1 / 2, 2 / 3)]
    return [list(range(z0, z0 + SAMPLE_SLAB)) for z0 in starts]


def oracle_sample(shot, atol):
    """Time the oracle (as it stands) on a bounded sample of the workload and
    extrapolate to one shot gradient.  The same function, on the same inputs,
    serves both the GPU arm's cpu_baseline and the reference arm:
    * forward and adjoint steps on the full grid, per-step cost from nt = 2
      minus nt = 1 runs, after one untimed run of each (first touch of the
      oracle's FP64 fields);
    * encode + decode at atol of four 16-plane slabs (source depth, 1/3, 1/2
      and 2/3 of the depth) of the shot's wavefield at step 1200, the seeded
      analytic snapshot of synth.wavefield_snapshot (direct wave and layer
      reflections), scaled to the full depth."""
    import numpy as np
    import oracle
    from paper_2009_12623_gb300 import synth
    g = shot.geom
    og = oracle.geometry(g.nx, g.ny, g.nz, g.h, g.dt, 1, g.nbl, g.sponge_R, g.vmax)
    m = synth.slowness2(shot.v0).astype(np.float64)
    w = shot.wavelet.astype(np.float64)
    rec = shot.rec[:64]
    key = (g.nx, g.ny, g.nz, shot.src)
    if key not in _snapshot_cache:
        slabs = sample_planes(g)
        snap = synth.wavefield_snapshot(shot, SAMPLE_STEP * g.dt, [z for sl in slabs for z in sl])
        _snapshot_cache[key] = (slabs, [np.ascontiguousarray(snap[i * SAMPLE_SLAB:(i + 1) * SAMPLE_SLAB])
                                        for i in range(len(slabs))])
    slabs, fields = _snapshot_cache[key]

    def fwd(nt):
        og.nt = nt
        t = time.perf_counter()
        oracle.forward(og, m, w[:nt], shot.src, rec)
        return time.perf_counter() - t

    def adj(nt):
        og.nt = nt
        r = np.ones((nt, len(rec)))
        t = time.perf_counter()
        oracle.adjoint_trace(og, m, r, rec, shot.src)
        return time.perf_counter() - t

    fwd(1)
    adj(1)
    t_fwd = max(1e-9, fwd(2) - fwd(1))
    t_adj = max(1e-9, adj(2) - adj(1))
    t_codec = 0.0
    for f in fields:
        t = time.perf_counter()
        st = oracle.zfp_compress(f, atol)
        oracle.zfp_decompress(st, f.shape)
        t_codec += time.perf_counter() - t
    scale = g.nz / (SAMPLE_SLAB * len(fields))
    per_step = t_fwd + t_adj + t_codec * scale
    sec_per_gradient = per_step * g.nt
    sample = (f"oracle forward+adjoint step on the full {g.nx}x{g.ny}x{g.nz} grid (per-step time from "
              f"nt=2 minus nt=1 runs after a warm-up run: {t_fwd:.2f} s + {t_adj:.2f} s) and codec "
              f"encode+decode at atol={atol:g} of four {SAMPLE_SLAB}-plane slabs starting at z = "
              f"{', '.join(str(sl[0]) for sl in slabs)} (source depth, 1/3, 1/2, 2/3 of the depth) of the "
              f"shot's wavefield at step {SAMPLE_STEP} (seeded analytic snapshot: direct wave and layer "
              f"reflections), {t_codec:.2f} s, x{scale:.2f} to the full depth; extrapolated to {g.nt} steps")
    return 1.0 / sec_per_gradient, oracle.num_threads(), sample, per_step


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, local, pg = dist_setup(args)
    if rank != 0:
        return
    shot, _ = workload(args, 0)
    for _ in range(args.warmup):
        oracle_sample(shot, args.atol)
    vals = []
    t0 = time.perf_counter()
    cores = None
    sample = None
    for _ in range(args.steps):
        v, cores, sample, _ = oracle_sample(shot, args.atol)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = statistics.mean(vals)
    policy = f"full-history compressed checkpoints (atol={args.atol:g})"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(args, shot, policy),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "sample_wall_s": wall}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def run_fwi(args):
    import numpy as np
    import torch
    ws, rank, local, pg = dist_setup(args)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the product path has no CPU fallback)")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_12623_gb300 import api, synth

    shot, _ = workload(args, rank)
    g = shot.geom
    m0 = torch.from_numpy(synth.slowness2(shot.v0)).to(dev)
    mt = torch.from_numpy(synth.slowness2(shot.v_true)).to(dev)
    rec = torch.from_numpy(shot.rec).to(dev)
    w = shot.wavelet
    d_obs = api.forward(g, mt, w, shot.src, rec)
    del mt
    torch.cuda.synchronize()
    cells = g.nx * g.ny * g.nz

    free, total = torch.cuda.mem_get_info()
    reserve = 26 * (1 << 30) + 6 * cells * 4
    cap = max(1 << 30, free - reserve)
    if args.arena_gb > 0:
        cap = min(cap, int(args.arena_gb * (1 << 30)))
    store = api.CheckpointStore(cap)
    policy_mode, policy_k = api.FWI_CKPT_FULL, 1
    policy = f"full-history compressed checkpoints (atol={args.atol:g})"
    grad = torch.zeros(g.shape, dtype=torch.float32, device=dev)

    def step():
        grad.zero_()
        _, phi = api.gradient(g, m0, w, shot.src, rec, d_obs, store, mode=policy_mode, k=policy_k,
                              atol=args.atol, grad=grad)
        return grad, stack(pg, grad, phi)

    try:
        step()
    except api.FwiError as e:
        if e.status != -2:
            raise
        # the arena cannot hold every compressed state: keep pairs every K steps
        need = store.stats()["used_bytes"]
        policy_mode, policy_k = api.FWI_CKPT_EVERY_K, max(2, int(np.ceil(2 * need / cap)) + 1)
        policy = (f"every-{policy_k} compressed checkpoint pairs (atol={args.atol:g}; full history "
                  f"needs {need / 2**30:.0f} GiB > arena {cap / 2**30:.0f} GiB)")
        step()
    torch.cuda.synchronize()
    stats = store.stats()

    for _ in range(max(0, args.warmup - 1)):
        step()
    torch.cuda.synchronize()

    # ---- timed region --------------------------------------------------------
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    api.profile_reset()
    api.profile_enable(True)
    launches0 = api.kernel_launch_count()
    barrier(pg)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    phi = None
    for _ in range(args.steps):
        _, phi = step()
    ev1.record()
    torch.cuda.synchronize()
    barrier(pg)
    ms = ev0.elapsed_time(ev1)
    launches = api.kernel_launch_count() - launches0
    api.profile_enable(False)
    prof = api.profile_read()
    clk = clocks.stop()
    ms_max = max_over_ranks(pg, ms)
    value = ws * args.steps / (ms_max / 1e3)

    # ---- roofline of the dominant kernel ---------------------------------------
    pk, peak_kind = peaks()
    enc_bytes = stats["used_bytes"] / max(1, stats["n_checkpoints"])
    nblocks = -(-g.nx // 4) * -(-g.ny // 4) * -(-g.nz // 4)
    zero_blocks = store.slot_zero_blocks().astype(np.float64)
    full_lossy = policy_mode == api.FWI_CKPT_FULL and args.atol > 0
    live = float(1.0 - zero_blocks.mean() / nblocks) if full_lossy else 1.0
    kb = kernel_bytes(cells, enc_bytes, live, image_in_decoder=full_lossy)
    timed = {k: v for k, v in prof.items() if k in kb and v[1] > 0}
    # The dominant kernel is the one with the most device time among those that run alone, in
    # order, on the sweep's stream.  The encoder runs on a second stream beside the next forward
    # step, so its event-timed duration includes the time it waits for SMs held by that step.
    alone = [k for k in timed if k in IN_ORDER] or list(timed)
    dom = max(alone, key=lambda k: timed[k][0])
    dom_ms, dom_n = timed[dom]
    achieved = kb[dom] / (dom_ms / dom_n / 1e3) / 1e9
    kernels = {k: {"launches": n, "total_ms": round(t, 3), "avg_us": round(1e3 * t / n, 2),
                   "GB/s": round(kb[k] / (t / n / 1e3) / 1e9, 1),
                   "frac_of_hbm": round(kb[k] / (t / n / 1e3) / 1e9 / pk["hbm_gbs"], 3),
                   "share_of_step": round(t / ms, 3)}
               for k, (t, n) in timed.items()}
    traffic = measured_traffic(dom, cells)
    roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": pk["hbm_gbs"],
            "unit": "GB/s", "frac": round(achieved / pk["hbm_gbs"], 4), "traffic": traffic,
            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)",
            "dominant_rule": "most device time among kernels that run alone on the sweep's stream "
                             "(the encoder overlaps the next forward step on a second stream)",
            "algorithmic_bytes_per_launch": kb[dom]}

    # compressibility over the simulation (Sec. 4.1): CF of each tenth of the stored states
    sb = store.slot_bytes().astype(np.float64)
    cf_tenths = [round(float(cells * 4 * len(c) / c.sum()), 1) for c in np.array_split(sb, 10) if c.size]

    # ---- end to end through the host-memory entry point --------------------------
    d_obs_v = d_obs
    e2e = None
    if not args.no_e2e:
        h_m = torch.from_numpy(synth.slowness2(shot.v0)).pin_memory()
        h_obs = d_obs.cpu().pin_memory()
        h_rec = torch.from_numpy(shot.rec).pin_memory()
        h_grad = torch.zeros(g.shape, dtype=torch.float32).pin_memory()

        def hstep():
            h_grad.zero_()
            _, phi = api.gradient_host(g, h_m, w, shot.src, h_rec, h_obs, store, mode=policy_mode,
                                       k=policy_k, atol=args.atol, grad=h_grad)
            if pg is not None:  # stack the host gradients through the device
                dg = h_grad.to(dev, non_blocking=True)
                phi = stack(pg, dg, phi)
                h_grad.copy_(dg)
            return h_grad, phi
        hstep()
        barrier(pg)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            hstep()
        torch.cuda.synchronize()
        barrier(pg)
        t_e2e = max_over_ranks(pg, time.perf_counter() - t0)
        e2e = {"value": ws * args.steps / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": int(h_m.numel() * 4 + h_obs.numel() * 4 + h_rec.numel() * 4 +
                                         h_grad.numel() * 4 * (2 if ws > 1 else 1) + g.nt * 4),
               "d2h_bytes_per_step": int(h_grad.numel() * 4 * (2 if ws > 1 else 1) + 8),
               "entry_point": "fwi_gradient_host (pinned host buffers)"}

    # ---- gradient error at this tolerance vs raw (uncompressed) checkpoints ----
    # (after the timed region; the compressed store is released first so the
    # raw pairs and the recompute ring fit)
    verify = None
    plain_k = None
    if not args.no_verify:
        g_lossy = grad.clone()
        store.close()
        torch.cuda.empty_cache()
        K = 48
        free, _ = torch.cuda.mem_get_info()
        vstore = api.CheckpointStore(max(1 << 30, free - K * cells * 4 - 24 * (1 << 30)))
        grad.zero_()
        try:
            ev_a = torch.cuda.Event(enable_timing=True)
            ev_b = torch.cuda.Event(enable_timing=True)
            for rep in range(2):   # the first run sets up the recompute ring
                grad.zero_()
                ev_a.record()
                api.gradient(g, m0, w, shot.src, rec, d_obs_v, vstore, mode=api.FWI_CKPT_EVERY_K, k=K,
                             atol=0.0, grad=grad)
                ev_b.record()
            torch.cuda.synchronize()
            num = api.dot_f64(g_lossy - grad, g_lossy - grad)
            den = api.dot_f64(grad, grad)
            cos = api.dot_f64(g_lossy, grad) / np.sqrt(api.dot_f64(g_lossy, g_lossy) * den)
            verify = {"rel_l2_vs_raw_checkpoints": float(np.sqrt(num / den)),
                      "angle_rad": float(np.arccos(min(1.0, cos))),
                      "reference": f"same sweeps with raw FP32 checkpoint pairs every {K} steps"}
            # The paper's trade-off (Sec. 5): compression pays only where it beats recomputation.
            # The exact alternative: raw pairs every K steps, segments recomputed into a K-field ring.
            pairs = vstore.stats()["used_bytes"]
            ring = K * 4 * g.ny * g.nz * (-(-g.nx // 4) * 4)
            plain_k = {"k": K, "s_per_gradient": round(ev_a.elapsed_time(ev_b) / 1e3, 3),
                       "GiB_held": round((pairs + ring) / 2**30, 1),
                       "note": "second of two runs after the timed region (CUDA events); GiB = raw pairs + "
                               "recompute ring"}
        except api.FwiError as e:
            verify = {"error": str(e)}
        vstore.close()

    # ---- CPU oracle baseline (rank 0, N=1) ------------------------------------------
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, cores, sample, _ = oracle_sample(shot, args.atol)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_dict(args, shot, policy), "e2e": e2e, "gpu_launches": launches,
                "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
                "kernels": kernels,
                "checkpoint_store": {"live_block_fraction": round(live, 4),
                                     "used_GiB": round(stats["used_bytes"] / 2**30, 2),
                                     "compression_factor": round(stats["raw_bytes"] / max(1, stats["used_bytes"]), 2),
                                     "checkpoints": stats["n_checkpoints"],
                                     "cf_by_tenth_of_run": cf_tenths},
                "misfit": phi, "gradient_error": verify,
                "lossy_full_history": {"s_per_gradient": round(ms_max / args.steps / 1e3, 3),
                                       "GiB_held": round(stats["used_bytes"] / 2**30, 1)},
                "plain_every_k_raw": plain_k}
        print(json.dumps(line), flush=True)
    store.close()
    if pg is not None:
        pg.destroy_process_group()


def run_batch(args):
    """Survey of `shots` shots on a 600 x 600 x 200 layered model at 20 m
    (apertures 200-600 cells per side, records 1500-3000 ms at dt = 1.5 ms,
    10 Hz, 40-cell absorbing layer, receivers every 4th node), every-K
    compressed checkpoint pairs: one stacked gradient per step, through the
    batch plan (graph + autotuner) and through one fwi_gradient call per shot."""
    import numpy as np
    import torch
    ws, rank, local, pg = dist_setup(args)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the product path has no CPU fallback)")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_12623_gb300 import api, synth

    t_setup = time.perf_counter()
    sv = synth.batch_survey(nshots=args.shots, seed=rank)
    g = sv.geom
    m = torch.from_numpy(synth.slowness2(sv.v0)).to(dev)
    mt = torch.from_numpy(synth.slowness2(sv.v_true)).to(dev)
    w = sv.wavelets()
    d_obs = []
    for s, wi in zip(sv.shots, w):
        origin = torch.tensor([s.x0, s.y0, s.z0], dtype=torch.int32, device=dev)
        rec = (torch.from_numpy(np.asarray(s.rec, np.int32)).to(dev) - origin).contiguous()
        d_obs.append(api.forward(s.local_geometry(g), mt[s.window].contiguous(), wi,
                                 (s.src[0] - s.x0, s.src[1] - s.y0, s.src[2] - s.z0), rec))
    del mt
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    K, atol = args.ckpt_k, args.atol
    cell_steps = sum(s.nx * s.ny * s.nz * s.nt for s in sv.shots)

    def timed(fn, steps):
        barrier(pg)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = None
        for _ in range(steps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        barrier(pg)
        return max_over_ranks(pg, e0.elapsed_time(e1)), out

    # ---- plain path: one fwi_gradient call per shot ----------------------------
    store = api.CheckpointStore(int((args.arena_gb or 24) * (1 << 30)))
    g_plain = torch.zeros(g.shape, dtype=torch.float32, device=dev)

    def plain():
        g_plain.zero_()
        return api.gradient_per_shot(g, m, sv.shots, w, d_obs, store, mode=api.FWI_CKPT_EVERY_K, k=K,
                                     atol=atol, grad=g_plain)
    for _ in range(args.warmup):
        plain()
    l0 = api.kernel_launch_count()
    ms_plain, (_, phi_plain) = timed(plain, args.steps)
    launches_plain = (api.kernel_launch_count() - l0) // args.steps
    store.close()
    torch.cuda.empty_cache()

    # ---- batched plan (persistent multi-shot launches, CUDA graph, autotuner) ----
    free, _ = torch.cuda.mem_get_info()
    with api.Batch(g, sv.shots, mode=api.FWI_CKPT_EVERY_K, k=K, atol=atol, arena_bytes=1 << 30) as probe:
        need = probe.stats()["device_bytes"] - (1 << 30)
    arena = int(min(free - need - 8 * (1 << 30), 160 * (1 << 30)))
    b = api.Batch(g, sv.shots, mode=api.FWI_CKPT_EVERY_K, k=K, atol=atol, arena_bytes=arena, graph=True,
                  tune=True)
    obs = b.concat(d_obs)
    g_batch = torch.zeros(g.shape, dtype=torch.float32, device=dev)

    def batched():
        g_batch.zero_()
        return b.gradient(m, w, obs, grad=g_batch)
    t0 = time.perf_counter()
    batched()  # tunes, captures
    torch.cuda.synchronize()
    t_first = time.perf_counter() - t0
    for _ in range(max(0, args.warmup - 1)):
        batched()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    l0 = api.kernel_launch_count()
    ms_batch, (_, phi_batch) = timed(batched, args.steps)
    launches_batch = (api.kernel_launch_count() - l0) // args.steps
    clk = clocks.stop()
    st = b.stats()
    same = bool(torch.equal(g_batch, g_plain)) and bool(np.array_equal(phi_batch, phi_plain))
    b.close()

    value = ws * args.shots * args.steps / (ms_batch / 1e3)
    plain_value = ws * args.shots * args.steps / (ms_plain / 1e3)
    if rank == 0:
        line = {"metric": "shot-gradients/s at fixed gradient error vs plain path", "value": value,
                "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_batch / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"batched survey: {args.shots} shots on 600x600x200 at 20 m, apertures "
                                       f"200-600 cells, records 1500-3000 ms at 1.5 ms, 10 Hz, every-{K} "
                                       f"compressed checkpoint pairs (atol={atol:g})",
                           "shots": args.shots, "cell_steps_per_gradient": cell_steps,
                           "l2_flush": "inputs larger than L2 (>= 32 MB fields per shot, GBs per step)"},
                "plain": {"value": plain_value, "unit": UNIT, "ms_per_step": ms_plain / args.steps,
                          "gpu_launches_per_step": launches_plain,
                          "path": "one fwi_gradient call per shot on its window"},
                "speedup_vs_plain": ms_plain / ms_batch,
                "same_gradient_bitwise": same,
                "gpu_launches": launches_batch * args.steps,
                "plan": {k: st[k] for k in ("zc", "ctas", "zc_adjoint", "ctas_adjoint", "graph_nodes",
                                            "launches_per_call", "used_bytes", "raw_bytes", "device_bytes")},
                "first_call_s": t_first, "setup_s": t_setup, "clocks": clk}
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def run_fwi_inversion(args):
    """Differentiable FWI: 300 x 300 x 150 at 20 m, layered model with three
    +-8% Gaussian anomalies, 16 shots on a 4 x 4 grid, 2000 ms at 10 Hz,
    full-history checkpoints compressed at atol; `iters` steepest-descent
    iterations through autograd, once with one gradient call per shot and once
    through a batch plan (graph + autotuner).  value = shot-gradients/s of the
    batched path."""
    import math
    import numpy as np
    import torch
    ws, rank, local, pg = dist_setup(args)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the product path has no CPU fallback)")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_12623_gb300 import api, invert, synth

    nx, ny, nz, h, nshots = 300, 300, 150, 20.0, 16
    nbl = min(20, nz // 6)
    v = synth.layered_velocity(nx, ny, nz, seed=1, water=nbl + 5)
    v_true = synth.add_anomalies(v, seed=2, amplitude=0.08)
    v0 = synth.smooth(v_true, 4.0)
    vmax = float(v_true.max())
    dt = 0.4 * h / vmax
    nt = int(round(2.0 / dt))
    geom = api.Geometry(nx=nx, ny=ny, nz=nz, h=h, dt=dt, nt=nt, nbl=nbl, vmax=vmax)
    w = synth.wavelet(nt, dt, 10.0)
    zr = nbl + 2
    X, Y = np.meshgrid(np.arange(nbl, nx - nbl, 2), np.arange(nbl, ny - nbl, 2))
    rec_np = np.stack([X.ravel(), Y.ravel(), np.full(X.size, zr)], 1).astype(np.int32)
    rec = torch.from_numpy(rec_np).to(dev)
    side = int(math.ceil(math.sqrt(nshots)))
    sxs = np.linspace(nbl + 10, nx - nbl - 10, side).astype(int)
    srcs = [(int(sxs[i % side]), int(sxs[i // side]), zr) for i in range(nshots)]
    mt = torch.from_numpy(synth.slowness2(v_true)).to(dev)
    d_obs = [api.forward(geom, mt, w, s, rec) for s in srcs]
    del mt
    c0 = torch.from_numpy(v0).to(dev)
    ct = torch.from_numpy(v_true).to(dev)
    interior = torch.zeros_like(c0)
    interior[nbl:nz - nbl, nbl:ny - nbl, nbl:nx - nbl] = 1.0
    atol = args.atol

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    shots = [(geom, w, s, rec) for s in srcs]
    invert.invert(c0, shots, d_obs, iters=1, atol=atol, mask=interior)  # warm-up
    ms_plain, (c_plain, h_plain) = timed(lambda: invert.invert(c0, shots, d_obs, iters=args.iters, atol=atol,
                                                               mask=interior))
    torch.cuda.empty_cache()
    specs = [api.ShotSpec(0, 0, 0, nx, ny, nz, nt, s, rec_np) for s in srcs]
    with api.Batch(geom, specs, mode=api.FWI_CKPT_FULL, atol=atol, arena_bytes=96 << 30, graph=True,
                   tune=True) as plan:
        obs = plan.concat(d_obs)
        invert.invert_batched(c0, plan, [w] * nshots, obs, iters=1, mask=interior)  # tunes, captures
        ms_batch, (c_batch, h_batch) = timed(lambda: invert.invert_batched(c0, plan, [w] * nshots, obs,
                                                                           iters=args.iters, mask=interior))
        st = plan.stats()
    err = lambda c: float(torch.linalg.vector_norm(c - ct))
    value = nshots * args.iters / (ms_batch / 1e3)
    line = {"metric": "shot-gradients/s at fixed gradient error vs plain path (autograd inversion)",
            "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.iters, "warmup": 1,
            "ms_per_step": ms_batch / args.iters, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"differentiable FWI: {nx}x{ny}x{nz} at {h:.0f} m, layered + 3 anomalies (+-8%), "
                                   f"{nshots} shots, nt={nt} (dt={dt * 1e3:.3f} ms, 2000 ms), 10 Hz, "
                                   f"full-history checkpoints at atol={atol:g}, steepest descent",
                       "iterations": args.iters},
            "plain": {"value": nshots * args.iters / (ms_plain / 1e3), "unit": UNIT,
                      "ms_per_step": ms_plain / args.iters, "path": "autograd, one gradient call per shot"},
            "speedup_vs_plain": ms_plain / ms_batch,
            "misfit_batched": h_batch, "misfit_plain": h_plain,
            "model_error": {"start": err(c0), "batched": err(c_batch), "plain": err(c_plain)},
            "plan": {k: st[k] for k in ("zc", "ctas", "zc_adjoint", "ctas_adjoint", "graph_nodes",
                                        "used_bytes", "raw_bytes")}}
    print(json.dumps(line), flush=True)


def run_codec(args):
    """Codec microbenchmark: 512^3 FP32 snapshots (seeded sums of 8 spherical
    Ricker shells plus 1e-7 noise), compress + decompress at atol in
    {1e-1 .. 1e-6}: compression factor, max error, PSNR and GB/s (uncompressed
    bytes / kernel time, CUDA events).  value = compress GB/s at atol = 1e-4."""
    import numpy as np
    import torch
    ws, rank, local, pg = dist_setup(args)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the product path has no CPU fallback)")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_12623_gb300 import api, synth
    n = 512
    fields = [torch.from_numpy(synth.shells_field(n, seed=s)).to(dev) for s in range(max(1, args.steps))]
    nbytes = n ** 3 * 4
    out = torch.empty(api.zfp_max_compressed_bytes(n, n, n), dtype=torch.uint8, device=dev)
    dec = torch.empty((n, n, n), dtype=torch.float32, device=dev)
    pk, peak_kind = peaks()
    rows = []
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for atol in (1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6):
        for f in fields:  # warm-up
            s = api.zfp_compress(f, atol, out=out)
            api.zfp_decompress(s, f.shape, out=dec)
        torch.cuda.synchronize()
        api.profile_reset()
        api.profile_enable(True)
        cf, err, psnr = [], 0.0, []
        for f in fields:
            for _ in range(max(1, args.warmup)):
                s = api.zfp_compress(f, atol, out=out)
                api.zfp_decompress(s, f.shape, out=dec)
            torch.cuda.synchronize()
            cf.append(nbytes / s.numel())
            d = (dec - f).abs()
            err = max(err, float(d.max()))
            rng = float(f.max() - f.min())
            mse = float((d.double() ** 2).mean())
            psnr.append(20 * np.log10(rng) - 10 * np.log10(mse) if mse > 0 else float("inf"))
        api.profile_enable(False)
        prof = api.profile_read()
        e_ms, e_n = prof["zfp_encode"]
        d_ms, d_n = prof["zfp_decode"]
        enc = nbytes / (e_ms / e_n / 1e3) / 1e9
        dcd = nbytes / (d_ms / d_n / 1e3) / 1e9
        rows.append({"atol": atol, "compression_factor": float(np.mean(cf)), "max_error": err,
                     "max_error_below_atol": err <= atol, "psnr_db": float(np.mean(psnr)),
                     "compress_GBps": enc, "decompress_GBps": dcd,
                     "compress_frac_of_hbm": (nbytes + nbytes / np.mean(cf)) / (e_ms / e_n / 1e3) / 1e9 / pk["hbm_gbs"],
                     "decompress_frac_of_hbm": (nbytes + nbytes / np.mean(cf)) / (d_ms / d_n / 1e3) / 1e9 / pk["hbm_gbs"]})
    clk = clocks.stop()
    r4 = [r for r in rows if r["atol"] == 1e-4][0]
    line = {"metric": "codec compress GB/s (uncompressed bytes / kernel time)", "value": r4["compress_GBps"],
            "unit": "GB/s", "n_gpus": ws, "steps": len(fields), "warmup": 1, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"codec microbenchmark: {n}^3 FP32 shell snapshots (8 spherical 15 Hz Ricker shells, "
                                   f"radii 50-200 cells, N(0,1) amplitudes, 1e-7 noise), seeds 0..{len(fields) - 1}",
                       "l2_flush": "inputs larger than L2 (512 MB fields)"},
            "sweep": rows, "peak": {"hbm_gbs": pk["hbm_gbs"], "source": peak_kind}, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_tradeoff(args):
    """Memory / error / time trade-off of the checkpointing options on an
    Overthrust-shaped shot (440 x 440 x 200 at 25 m, 1200 steps of 1.75 ms,
    8 Hz): every gradient against the exact one from raw checkpoint pairs
    every 40 steps -- full-history lossy compression over atol (Sec. 4.4),
    subsampling of the imaging condition over f (Sec. 4.7), binomial
    checkpointing over the number of snapshot pairs (raw and compressed).
    Memory reduction = bytes of full raw history / bytes held; error = relative
    L2 and angle of the gradient (FP64 reductions on the GPU)."""
    import numpy as np
    import torch
    ws, rank, local, pg = dist_setup(args)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the product path has no CPU fallback)")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_12623_gb300 import api, synth

    shot = synth.overthrust_like_shot(nx=440, ny=440, nz=200, nt=1200, nbl=40, rec_stride=2)
    g = shot.geom
    m0 = torch.from_numpy(synth.slowness2(shot.v0)).to(dev)
    rec = torch.from_numpy(shot.rec).to(dev)
    w = shot.wavelet
    d_obs = api.forward(g, torch.from_numpy(synth.slowness2(shot.v_true)).to(dev), w, shot.src, rec)
    cells = g.nx * g.ny * g.nz
    full_raw = g.nt * cells * 4
    store = api.CheckpointStore(128 << 30)  # subsampling at f = 2 holds 600 raw states (93 GB)

    def grad(mode, k=1, atol=0.0):
        out = torch.zeros(g.shape, dtype=torch.float32, device=dev)
        api.gradient(g, m0, w, shot.src, rec, d_obs, store, mode=mode, k=k, atol=atol, grad=out)  # warm-up
        torch.cuda.synchronize()
        out.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        api.gradient(g, m0, w, shot.src, rec, d_obs, store, mode=mode, k=k, atol=atol, grad=out)
        e1.record()
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1), store.stats()

    ref, t_ref, _ = grad(api.FWI_CKPT_EVERY_K, 40)
    rr = api.dot_f64(ref, ref)

    def err(gr):
        d = gr - ref
        cos = api.dot_f64(gr, ref) / np.sqrt(api.dot_f64(gr, gr) * rr)
        return float(np.sqrt(api.dot_f64(d, d) / rr)), float(np.arccos(min(1.0, max(-1.0, cos))))

    def forward_steps(mode, k):
        return sum(1 for a in api.ckpt_schedule(g.nt, mode, k) if a[0] in (1, 4))

    rows = {"compression": [], "subsampling": [], "binomial": []}
    for atol in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6):
        gr, ms, st = grad(api.FWI_CKPT_FULL, 1, atol)
        e, ang = err(gr)
        rows["compression"].append({"atol": atol, "memory_reduction": full_raw / st["used_bytes"],
                                    "held_GiB": st["used_bytes"] / 2**30, "rel_l2": e, "angle_rad": ang, "ms": ms})
    for f in (2, 4, 8, 16, 32):
        gr, ms, st = grad(api.FWI_CKPT_SUBSAMPLE, f)
        e, ang = err(gr)
        rows["subsampling"].append({"f": f, "memory_reduction": full_raw / max(1, st["used_bytes"]),
                                    "held_GiB": st["used_bytes"] / 2**30, "rel_l2": e, "angle_rad": ang, "ms": ms})
    for snaps in (4, 8, 16, 32, 64):
        for atol in (0.0, 1e-4):
            gr, ms, st = grad(api.FWI_CKPT_BINOMIAL, snaps, atol)
            e, ang = err(gr)
            rows["binomial"].append({"snapshot_pairs": snaps, "atol": atol,
                                     "forward_steps": forward_steps(api.FWI_CKPT_BINOMIAL, snaps),
                                     "memory_reduction": full_raw / max(1, st["used_bytes"]),
                                     "held_GiB": st["used_bytes"] / 2**30, "rel_l2": e, "angle_rad": ang, "ms": ms})
    store.close()
    line = {"metric": "gradient error vs checkpoint memory (compression, subsampling, binomial)",
            "value": None, "unit": None, "n_gpus": ws, "steps": 1, "warmup": 1, "ms_per_step": None,
            "higher_is_better": None, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"overthrust-like single shot {g.nx}x{g.ny}x{g.nz} at {g.h:.0f} m, nt={g.nt} "
                                   f"(dt={g.dt * 1e3:.2f} ms), 8 Hz, {len(shot.rec)} receivers; reference: raw "
                                   f"checkpoint pairs every 40 steps ({t_ref:.0f} ms)",
                       "full_raw_history_GiB": full_raw / 2**30},
            "tradeoff": rows}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "fwi":
        run_fwi_inversion(args)
    elif args.workload == "codec":
        run_codec(args)
    elif args.workload == "tradeoff":
        run_tradeoff(args)
    else:
        run_fwi(args)


if __name__ == "__main__":
    main()

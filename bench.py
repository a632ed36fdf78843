"""Benchmark of the multi-resolution projection hot path on GB300.

One step = the whole hot path on one 512 x 512 microscopy-like residual
(400 Poisson emitters, PSF sigma 2 px, high-pass residual normalised by
sqrt(mean)), window sides 1..8, alpha = 0.9 (per-window fourth-root bounds):
  1. standard Dykstra projection to a relative step < 1e-6 (Algorithm 2);
  2. incomplete Dykstra with K = 3 (sides 1, 2, 4, 8) at the paper's tol 1e-3.
Metric: window projections per second over both (one unit = one window's
update), whole-job (all ranks).  Inputs are resident in HBM when the timed
region starts; the increment store (214 MB) is larger than L2 and L2 is also
flushed between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on this host's cores on a bounded
sample of the same workload (the reference arm of this benchmark).

On one GPU the line also carries "extras" (skip with --no-extras): the uneven
batch of 256 images (BF16 and FP32 increments against one projection per
image), mixed-precision increments on a 2048 x 2048 image (throughput and
error against the FP64 oracle), and the continuous-batching request loop on a
Poisson request stream (p50 / p99 latency and images/s against the plain
single-image API).
Multi-GPU: independent replicas (one image per rank, no collective on the
data path); weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H = W = 512
SIDES = list(range(1, 9))
ALPHA = 0.9
TOL = 1e-6
MAX_CYCLES = 20000
ICD_K = 3
ICD_TOL = 1e-3
WORKLOAD = "emitters512_sides1-8_std_rel1e-6+icd_K3_tol1e-3"


def rank_env():
    r = int(os.environ.get("RANK", "0"))
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return r, ws, lr


def replica_totals(dist, device, seconds, units):
    """Whole-job figures of N replicas (one image per rank, no data exchange
    between ranks): the time is the slowest rank's, the work the sum over the
    ranks.  Returns (seconds, units)."""
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    w = torch.tensor([float(units)], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


def make_input(seed):
    from synthetic import emitter_residual
    return np.ascontiguousarray(emitter_residual(H, W, n_emitters=400, seed=seed), np.float32)


def algorithmic_bytes_per_cycle(first=False):
    """q read + write (FP32) of every window of the cycle plus the x_prev read
    and write of the cycle-end norm; the first cycle only writes q."""
    qb = sum((H - L + 1) * (W - L + 1) * L * L for L in SIDES) * 4
    return (qb if first else 2 * qb) + 8 * H * W


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_index):
        self.dev = dev_index
        self.p = None
        # the raw samples (the JSON line carries their summary); SMRE_CLOCKS_DIR
        # chooses where they are kept
        out_dir = os.environ.get("SMRE_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"smre_clocks_rank{dev_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        if self.p is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]) if parts[3] not in
                             ("[N/A]", "N/A") else 0.0, parts[4:]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        pmax = max(r[2] for r in rows)
        load = [r for r in rows if r[2] >= 0.5 * pmax] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in load:
            for nm, v in zip(names, r[3][1:]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows), "samples_under_load": len(load),
                "power_w_max": pmax}


# DRAM traffic of the dominant kernel from one ncu capture (20 cycles of this
# workload, profiles/persist_reg_kernel_emitters512_20cycles.md), per library
# version: (first-cycle bytes, bytes per later cycle), the capture's total
# split like the algorithmic bytes.  A version without an entry reports
# traffic as null until it is captured again.
MEASURED_TRAFFIC = {
    "smre-gb300 0.8 (sm_103a)": (217.6e6, 433.1e6),
    "smre-gb300 0.9 (sm_103a)": (217.6e6, 433.1e6),
    "smre-gb300 0.10 (sm_103a)": (217.6e6, 433.0e6),
    "smre-gb300 0.11 (sm_103a)": (217.6e6, 433.1e6),
    "smre-gb300 0.12 (sm_103a)": (217.6e6, 433.1e6),
    "smre-gb300 0.13 (sm_103a)": (217.6e6, 433.2e6),
}

# Warp instructions one incomplete projection of this workload executes
# (icd_pass_kernel, passes i = 0..3, from one ncu capture:
# profiles/icd_pass_kernel_emitters512_K3.md), per library version.  The
# incomplete method is bound on chip (per-tile sweep chains in registers and
# shuffles, about 8 B of HBM traffic per pixel and pass): its roofline is the
# issue-slot ceiling, windows per second if every SM issued four warp
# instructions per cycle at the measured clock.
ICD_WARP_INSTRUCTIONS = {
    "smre-gb300 0.8 (sm_103a)": 21737554,
    "smre-gb300 0.9 (sm_103a)": 21737554,
    "smre-gb300 0.10 (sm_103a)": 21737554,
    "smre-gb300 0.11 (sm_103a)": 21737554,
    "smre-gb300 0.12 (sm_103a)": 24523220,   # K = 3 at 4 pixels a thread
    "smre-gb300 0.13 (sm_103a)": 24523220,
}


# DRAM traffic per cycle of the batched step kernels (all step launches of
# one later cycle, one ncu capture each: profiles/bstep_kernel_uneven_batch.md),
# per library version and workload: (bytes read, bytes written, launches the
# capture used).  The writes miss what each launch leaves dirty in L2 (ncu
# flushes caches between the serialised launches), so the reads are the check
# against the algorithmic bytes; both are reported.
BATCH_TRAFFIC = {
    "smre-gb300 0.9 (sm_103a)": {
        ("uneven256", 0): (135.795e9, 133.457e9, "per group"),
        ("uneven256", 1): (82.654e9, 80.306e9, "per group"),
        ("img2048", 0): (12.176e9, 7.194e9, "per group"), ("img2048", 1): (6.949e9, 2.154e9, "per group"),
    },
    "smre-gb300 0.10 (sm_103a)": {
        ("uneven256", 0): (135.798e9, 133.456e9, "per group"),
        ("uneven256", 1): (82.652e9, 80.354e9, "per group"),
        ("img2048", 0): (11.325e9, 11.312e9, "per side"), ("img2048", 1): (5.903e9, 5.797e9, "per side"),
    },
    "smre-gb300 0.11 (sm_103a)": {
        ("uneven256", 0): (135.797e9, 133.457e9, "per group"),
        ("uneven256", 1): (82.651e9, 80.306e9, "per group"),
        ("img2048", 0): (11.321e9, 11.288e9, "per side"), ("img2048", 1): (5.899e9, 5.763e9, "per side"),
    },
    "smre-gb300 0.12 (sm_103a)": {
        ("uneven256", 0): (135.797e9, 133.456e9, "per group"),
        ("uneven256", 1): (82.652e9, 80.306e9, "per group"),
        ("img2048", 0): (11.322e9, 11.287e9, "per side"), ("img2048", 1): (5.899e9, 5.762e9, "per side"),
    },
    "smre-gb300 0.13 (sm_103a)": {
        ("uneven256", 0): (135.797e9, 133.457e9, "per group"),
        ("uneven256", 1): (82.652e9, 80.306e9, "per group"),
        ("img2048", 0): (11.326e9, 11.290e9, "per side"), ("img2048", 1): (5.901e9, 5.767e9, "per side"),
    },
}


def x_row_bytes_per_cycle(shapes, sides):
    """x rows a cycle's step launches read and write: every group launch
    (L, a) stages the rows of its window-rows, 8 bytes a pixel."""
    return sum(8 * h * w * L for (h, w) in shapes for L in sides)


def batch_traffic(smre, case, qdt, shapes, sides):
    t = BATCH_TRAFFIC.get(smre.smre_version(), {}).get((case, qdt))
    if t is None:
        return None
    inc = q_bytes_per_cycle(shapes, sides, qdt) - 8 * sum(h * w for h, w in shapes)
    xr = x_row_bytes_per_cycle(shapes, sides)
    return {"read": t[0], "write": t[1], "launches": t[2],
            "algorithmic_increments": inc, "algorithmic_x_rows": xr,
            "read_over_algorithmic_read": t[0] / ((inc + xr) / 2),
            "note": "all step launches of one later cycle; writes miss what stays dirty in L2 "
                    "between the serialised launches"}


def icd_critical_path(sweeps, H, W, K, seconds):
    """The incomplete projection's passes run their tiles side by side, each
    tile's sweeps one after another: a pass lasts as long as its tile with the
    most sweeps.  sweeps: per-tile counts of the last call, pass by pass
    (i = 0..K), tiles row-major; pass i covers the B x B tiles (B = 2^K) at
    offset (1 << i) mod B that lie inside the image."""
    B = 1 << K
    counts = [((H - (1 << i) % B) // B) * ((W - (1 << i) % B) // B) for i in range(K + 1)]
    if len(sweeps) != sum(counts):
        return None
    o, longest = 0, []
    for i in range(K + 1):
        n = counts[i]
        longest.append(int(max(sweeps[o:o + n])) if n else 0)
        o += n
    crit = sum(longest)
    return {"longest_tile_sweeps_per_pass": longest, "sweeps": crit,
            "us_per_sweep_on_it": 1e6 * seconds / crit if crit else None,
            "tiles_total_sweeps": int(sum(sweeps)),
            "note": "a call takes at least its passes' longest tile chains of sweeps"}


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return float(json.load(open(p))["hbm_gbs"]), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


def cpu_sample(x0, threads, cycles):
    """The oracle as it stands on a bounded sample: `cycles` standard cycles
    plus one full incomplete projection.  Returns (windows, seconds)."""
    import oracle
    x = x0.astype(np.float64)
    cS = oracle.bounds(SIDES, ALPHA)
    t0 = time.perf_counter()
    oracle.dykstra(x, SIDES, cS, max_cycles=cycles, tol=-1, n_threads=threads)
    t1 = time.perf_counter()
    r = oracle.icd(x, ICD_K, [cS[0], cS[1], cS[3], cS[7]], tol=ICD_TOL)
    t2 = time.perf_counter()
    B = 1 << ICD_K
    w_icd = 0
    for i, sw in enumerate(r.sweeps):
        per = sum((B >> k) ** 2 for k in range(i, ICD_K + 1))
        w_icd += per * int(sw.sum())
    w_std = cycles * oracle.n_windows(H, W, SIDES)
    return w_std + w_icd, (t1 - t0) + (t2 - t1)


def run_reference(args):
    rank, world, _ = rank_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    x0 = make_input(1002)
    cycles = 20
    for _ in range(args.warmup):
        cpu_sample(x0, threads, 2)
    tot_w, tot_s = 0, 0.0
    for _ in range(args.steps):
        w, s = cpu_sample(x0, threads, cycles)
        tot_w += w
        tot_s += s
    v = tot_w / tot_s
    line = {
        "impl": "reference", "metric": "window-projections/s", "value": v,
        "unit": "window-projections/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "H": H, "W": W, "sides": "1..8",
                   "sample": f"{cycles} standard cycles + 1 full incomplete projection per step"},
        "cpu_baseline": {"value": v, "unit": "window-projections/s", "cores": threads,
                         "kind": "oracle",
                         "sample": f"{cycles} of the standard cycles + the full incomplete "
                                   f"projection, FP64 C oracle, {threads} OpenMP threads"},
        "e2e": {"value": v, "unit": "window-projections/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ extras
# The other workloads of the method, reported beside the main line (rank 0 of
# a one-GPU run): the uneven batch, mixed-precision increments on a large
# image, and the continuous-batching request loop.

def q_bytes_per_cycle(shapes, sides, qdt):
    """Algorithmic bytes of one cycle: every window's increments read and
    written (FP32: 8 L^2 bytes; 16-bit: 4 L^2 + 8 with the window scale), plus
    the x_prev read and write of the norm (8 bytes a pixel)."""
    tot = 0
    for (h, w) in shapes:
        for L in sides:
            nw = (h - L + 1) * (w - L + 1)
            tot += nw * (8 * L * L if qdt == 0 else 4 * L * L + 8)
        tot += 8 * h * w
    return tot


def windows_per_cycle(shapes, sides):
    return sum((h - L + 1) * (w - L + 1) for (h, w) in shapes for L in sides)


def timed_batch_cycles(smre, torch, xs, sides, cS, qdt, cycles, stream, tune=False, flags=0):
    """Per-cycle device time of a batch over xs (device tensors): the first
    cycle (no increments to read) runs untimed -- with tune, the autotuner's
    cycles too (one untimed, one per candidate schedule) -- then `cycles`
    timed.  Returns (seconds per cycle, launches, (spread, tuned, per_side))."""
    warm = 5 if tune else 1
    need = sum(smre.smre_batch_image_bytes(smre.make_batch_params(sides, q_dtype=qdt,
                                                                  max_cycles=cycles + warm), *x.shape)
               for x in xs)
    with smre.Batch(sides, stream=stream, cmode=smre.SMRE_C_EXPLICIT, c_explicit=cS, q_dtype=qdt,
                    max_cycles=cycles + warm, tol=-1.0, max_images=len(xs),
                    device_bytes=need + (64 << 20),
                    flags=(smre.SMRE_BF_AUTOTUNE if tune else 0) | flags) as B:
        for x in xs:
            assert B.submit(x) >= 0
        B.run(warm)
        spread = B.item_spread() + (B.per_side(),)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.run(cycles)
        e1.record(stream)
        torch.cuda.synchronize()
        done = B.poll()
        outs = {}
        for s in done:
            outs[s] = B.retrieve(s)
        launches = B.kernel_launches()
    return e0.elapsed_time(e1) / 1e3 / cycles, launches, spread


def bench_batched(smre, torch, stream, peak):
    """256 residual images, sides s in {128..1024}, half of them s x 2s, window
    sides 1..8: batched launches (BF16 and FP32 increments) against one
    projection per image through the single-image API (FP32)."""
    from synthetic import batch_images
    xs_h = [np.ascontiguousarray(a, np.float32) for a in batch_images(256)]
    xs = [torch.from_numpy(a).cuda() for a in xs_h]
    shapes = [x.shape for x in xs_h]
    cS = smre.smre_bounds(smre.make_params(64, 64, SIDES, alpha=ALPHA))
    wpc = windows_per_cycle(shapes, SIDES)
    out = {"images": len(xs), "pixels": int(sum(h * w for h, w in shapes)), "sides": "1..8",
           "windows_per_cycle": wpc}
    cycles = 4
    for name, qdt in (("bf16", smre.SMRE_Q_BF16), ("fp32", smre.SMRE_Q_FP32)):
        sec, _, (spread, tuned, per_side) = timed_batch_cycles(smre, torch, xs, SIDES, cS, qdt, cycles,
                                                               stream, tune=True)
        gbs = q_bytes_per_cycle(shapes, SIDES, qdt) / sec / 1e9
        out[name] = {"ms_per_cycle": 1e3 * sec, "window_projections_per_s": wpc / sec,
                     "achieved_gbs": gbs, "frac_of_measured_hbm": gbs / peak,
                     "item_spread": spread, "launches": "per side" if per_side else "per group",
                     "schedule_autotuned": {1: "measured", 2: "cached"}.get(tuned, "no"),
                     "step_kernel_dram_traffic_per_cycle": batch_traffic(smre, "uneven256", qdt, shapes, SIDES)}
        # the untuned schedules (spread 1) beside the tuned one
        sec1, _, _ = timed_batch_cycles(smre, torch, xs, SIDES, cS, qdt, cycles, stream)
        secs, _, _ = timed_batch_cycles(smre, torch, xs, SIDES, cS, qdt, cycles, stream,
                                        flags=smre.SMRE_BF_PER_SIDE)
        out[name]["ms_per_cycle_per_group_spread1"] = 1e3 * sec1
        out[name]["ms_per_cycle_per_side_spread1"] = 1e3 * secs
    # one launch per image (FP32 single-image API), on the first 24 images
    tot_w, tot_s = 0, 0.0
    for x in xs[:24]:
        h, w = x.shape
        with smre.Projector(h, w, SIDES, stream=stream, cmode=smre.SMRE_C_EXPLICIT, c_explicit=cS,
                            max_cycles=3, tol=-1.0) as P:
            o = torch.empty_like(x)
            P.project(x, o)                       # first cycles and allocation untimed
            r = P.project(x, o)
            tot_w += r.windows
            tot_s += r.seconds
    out["one_launch_per_image_fp32"] = {"window_projections_per_s": tot_w / tot_s,
                                        "sample": "first 24 images, 3 cycles each"}
    # at equal precision (FP32 increments on both sides), and BF16 beside it
    out["speedup_fp32_vs_one_launch_per_image"] = (out["fp32"]["window_projections_per_s"] /
                                                   (tot_w / tot_s))
    out["speedup_bf16_vs_one_launch_per_image"] = (out["bf16"]["window_projections_per_s"] /
                                                   (tot_w / tot_s))
    out["bf16_over_fp32_ms_per_cycle"] = out["bf16"]["ms_per_cycle"] / out["fp32"]["ms_per_cycle"]
    return out


def bench_mixed(smre, torch, stream, peak, threads):
    """One 2048 x 2048 residual (1600 emitters), window sides 1..12: FP32 vs
    BF16 vs FP16 increments with per-window scales; error against the FP64
    oracle measured on the whole image after 3 cycles."""
    import oracle
    from synthetic import emitter_residual_2048
    sides = list(range(1, 13))
    x_h = np.ascontiguousarray(emitter_residual_2048(), np.float32)
    x = torch.from_numpy(x_h).cuda()
    cS = smre.smre_bounds(smre.make_params(64, 64, sides, alpha=ALPHA))
    shapes = [x_h.shape]
    wpc = windows_per_cycle(shapes, sides)
    out = {"image": "2048x2048", "sides": "1..12", "windows_per_cycle": wpc}
    cycles = 3
    res = {}
    for name, qdt in (("fp32", 0), ("bf16", 1), ("fp16", 2)):
        sec, _, (spread, tuned, per_side) = timed_batch_cycles(smre, torch, [x], sides, cS, qdt, cycles,
                                                               stream, tune=True)
        secg, _, _ = timed_batch_cycles(smre, torch, [x], sides, cS, qdt, cycles, stream)
        secs, _, _ = timed_batch_cycles(smre, torch, [x], sides, cS, qdt, cycles, stream,
                                        flags=smre.SMRE_BF_PER_SIDE)
        gbs = q_bytes_per_cycle(shapes, sides, qdt) / sec / 1e9
        out[name] = {"ms_per_cycle": 1e3 * sec, "item_spread": spread,
                     "launches": "per side" if per_side else "per group",
                     "ms_per_cycle_per_group_spread1": 1e3 * secg,
                     "ms_per_cycle_per_side_spread1": 1e3 * secs,
                     "window_projections_per_s": wpc / sec,
                     "achieved_gbs": gbs, "frac_of_measured_hbm": gbs / peak,
                     "step_kernel_dram_traffic_per_cycle": batch_traffic(smre, "img2048", qdt, shapes, sides)}
    out["bf16_over_fp32_ms_per_cycle"] = out["bf16"]["ms_per_cycle"] / out["fp32"]["ms_per_cycle"]
    # accuracy: the whole image, 3 cycles, each storage type against the FP64 oracle
    ref = oracle.dykstra(x_h.astype(np.float64), sides, cS, max_cycles=3, tol=-1,
                         n_threads=threads).x
    scale = np.abs(ref).max()
    for name, qdt in (("fp32", 0), ("bf16", 1), ("fp16", 2)):
        with smre.Projector(2048, 2048, sides, stream=stream, cmode=smre.SMRE_C_EXPLICIT,
                            c_explicit=cS, max_cycles=3, tol=-1.0, q_dtype=qdt) as P:
            o = np.empty_like(x_h)
            P.project(x_h, o)
        res[name] = float(np.abs(o.astype(np.float64) - ref).max() / scale)
        out[name]["err_vs_fp64_oracle"] = res[name]
    out["accuracy_sample"] = "the whole 2048x2048 image, sides 1..12, 3 cycles, max-abs relative"
    return out


def _quantiles(lat):
    lat = sorted(lat)
    return lat[len(lat) // 2], lat[min(len(lat) - 1, int(round(0.99 * (len(lat) - 1))))]


def _serve(smre, stream, imgs, arrivals, kw, slots, qdt):
    """The request loop on one arrival stream with increments of type qdt:
    images/s and latency quantiles (submission to result, queueing included),
    plus every request's result and cycle count."""
    outs = [np.empty_like(a) for a in imgs]
    with smre.Server(SIDES, cycles_per_round=4, stream=stream, q_dtype=qdt,
                     max_images=slots, device_bytes=48 << 30, **kw) as S:
        t0 = time.perf_counter()
        tickets = []
        for a, img, o in zip(arrivals, imgs, outs):
            d = t0 + a - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tickets.append(S.submit(img, o))
        cycles = [S.wait(t).cycles for t in tickets]
        st = S.stats()
    return ({"images_per_s": st.images_per_s, "p50_s": st.p50_s, "p99_s": st.p99_s,
             "max_s": st.max_s, "peak_active": st.peak_active, "rounds": st.rounds}, outs, cycles)


def _plain(smre, stream, imgs, arrivals, kw):
    """The plain single-image API (FP32) on the same stream, one request at a
    time in arrival order.  A handle is created for each request but its
    creation (device allocation of up to 3.4 GB of increments) is left out of
    the timeline: the clock stops while it runs, so the latencies are those of
    a plain server that had its handles ready.  The creation time is reported
    beside them."""
    lat, outs, cycles = [], [], []
    t0 = time.perf_counter()
    t_create = 0.0
    for a, img in zip(arrivals, imgs):
        d = t0 + t_create + a - time.perf_counter()
        if d > 0:
            time.sleep(d)
        h, w = img.shape
        c = time.perf_counter()
        P = smre.Projector(h, w, SIDES, stream=stream, **kw)
        t_create += time.perf_counter() - c
        o = np.empty_like(img)
        r = P.project(img, o)
        lat.append(time.perf_counter() - t0 - t_create - a)
        c = time.perf_counter()
        P.close()
        t_create += time.perf_counter() - c
        outs.append(o)
        cycles.append(r.cycles)
    t_all = time.perf_counter() - t0 - t_create
    p50, p99 = _quantiles(lat)
    return ({"images_per_s": len(imgs) / t_all, "p50_s": p50, "p99_s": p99,
             "handle_create_destroy_s_excluded": t_create}, outs, cycles)


def bench_serving(smre, torch, stream, threads, n_req=None, rate=500.0, slots=16,
                  sweep=((5.0, 24), (15.0, 24))):
    """Poisson arrivals (mean `rate` per second) of square SOFI-like requests,
    side uniform in 64..2048, window sides 1..8, at most 100 cycles or a
    relative step of 1e-6: the request loop with FP32 increments and with
    BF16 increments against the plain single-image API (FP32, one request at
    a time, in arrival order, handle creation left out of its timeline) -- at
    the overloading rate (saturation throughput) and at rates below it.  Each
    arm's error against the FP64 oracle is measured on the smallest requests
    of the stream (the oracle run to each request's own cycle count).
    n_req: SMRE_SERVING_REQUESTS, default 256."""
    from synthetic import request_stream, request_image, sofi_canvas
    import oracle
    if n_req is None:
        n_req = int(os.environ.get("SMRE_SERVING_REQUESTS", "256"))
    canvas = sofi_canvas()
    cS = smre.smre_bounds(smre.make_params(64, 64, SIDES, alpha=ALPHA))
    kw = dict(cmode=smre.SMRE_C_EXPLICIT, c_explicit=cS, max_cycles=100, tol=1e-6,
              tol_relative=True)

    def stream_of(n, r):
        reqs = request_stream(n=n, rate=r)
        imgs = [np.ascontiguousarray(request_image(canvas, side, sd), np.float32)
                for (_, side, sd) in reqs]
        return imgs, [a for (a, _, _) in reqs]

    imgs, arrivals = stream_of(n_req, rate)
    arms = {}
    results = {}
    for name, fn in (("served_fp32", lambda: _serve(smre, stream, imgs, arrivals, kw, slots, 0)),
                     ("served_bf16", lambda: _serve(smre, stream, imgs, arrivals, kw, slots, 1)),
                     ("plain_single_image_fp32", lambda: _plain(smre, stream, imgs, arrivals, kw))):
        arms[name], outs, cyc = fn()
        results[name] = (outs, cyc)
    # accuracy: the oracle on the smallest requests, to each arm's cycle count
    sample = sorted(range(len(imgs)), key=lambda i: imgs[i].size)[:4]
    for name, (outs, cyc) in results.items():
        worst = 0.0
        for i in sample:
            ref = oracle.dykstra(imgs[i].astype(np.float64), SIDES, cS, max_cycles=cyc[i], tol=-1,
                                 n_threads=threads).x
            worst = max(worst, float(np.abs(outs[i].astype(np.float64) - ref).max() / np.abs(ref).max()))
        arms[name]["err_vs_fp64_oracle"] = worst
    arms["accuracy_sample"] = ("the 4 smallest requests (sides %s), max-abs relative, oracle run to "
                               "the same cycle count" % [int(imgs[i].shape[0]) for i in sample])
    below = []
    for r, n in sweep:
        im, ar = stream_of(n, r)
        below.append({"rate_per_s": r, "requests": n,
                      "served_fp32": _serve(smre, stream, im, ar, kw, slots, 0)[0],
                      "served_bf16": _serve(smre, stream, im, ar, kw, slots, 1)[0],
                      "plain_single_image_fp32": _plain(smre, stream, im, ar, kw)[0]})
    plain_ips = arms["plain_single_image_fp32"]["images_per_s"]
    return {"requests": n_req, "rate_per_s": rate, "sides": "1..8", "slots": slots,
            "stop": "rel step < 1e-6 or 100 cycles", **arms,
            "images_per_s_ratio_fp32_served_vs_plain": arms["served_fp32"]["images_per_s"] / plain_ips,
            "images_per_s_ratio_bf16_served_vs_plain": arms["served_bf16"]["images_per_s"] / plain_ips,
            "below_saturation": below}


def bench_admm(smre, torch, stream, threads, iters=10):
    """The full estimator (ADMM, Algorithm 1) on the 512 x 512 emitter residual
    with its generator's PSF (Gaussian, sigma 2), sides 1..8: each eps-step
    runs Dykstra to a relative step of 1e-3 (at most 200 cycles), 20 TV dual
    steps per iteration; then the same with the incomplete Dykstra as the
    eps-step (the paper's fast estimator).  Error against the FP64 oracle on
    the same image with fixed counts (3 iterations of 20 cycles)."""
    import oracle
    from oracle import admm as oadmm
    x_h = make_input(1002)
    H, W = x_h.shape
    cS = smre.smre_bounds(smre.make_params(64, 64, SIDES, alpha=ALPHA))
    I = torch.from_numpy(x_h).cuda()
    x = torch.empty_like(I)
    kw = dict(cmode=smre.SMRE_C_EXPLICIT, c_explicit=cS, stream=stream)
    with smre.Admm(H, W, SIDES, 2.0, tv_iters=20, max_iters=iters, delta=-1.0, max_cycles=200,
                   tol=1e-3, tol_relative=True, **kw) as A:
        A.solve(I, x)                                   # warm-up
        l0, p0 = A.kernel_launches(), A.projection_launches()
        r = A.solve(I, x)
        launches = A.kernel_launches() - l0 + A.projection_launches() - p0
    wpc = windows_per_cycle([(H, W)], SIDES)
    out = {"image": "512x512 emitters", "psf_sigma": 2.0, "sides": "1..8", "iterations": r.iters,
           "eps_step": "Dykstra to rel step 1e-3 (<= 200 cycles)", "tv_iters": 20,
           "ms_per_iteration": 1e3 * r.seconds / r.iters,
           "projection_share": r.projection_seconds / r.seconds,
           "dykstra_cycles_per_iteration": r.dykstra_cycles / r.iters,
           "eps_step_window_projections_per_s": r.dykstra_cycles * wpc / max(r.projection_seconds, 1e-12),
           "gpu_launches": launches, "final_dx": r.dx, "final_residual": r.residual}
    # the paper's faster estimator: the eps-step by the incomplete Dykstra
    # (K = 3, tol 1e-3), the same number of iterations
    with smre.Admm(H, W, SIDES, 2.0, tv_iters=20, max_iters=iters, delta=-1.0, eps_incomplete=True,
                   icd_K=ICD_K, icd_tol=ICD_TOL, **kw) as A:
        A.solve(I, x)
        ri = A.solve(I, x)
    out["incomplete_eps_step"] = {
        "eps_step": f"incomplete Dykstra K={ICD_K}, tol {ICD_TOL}",
        "ms_per_iteration": 1e3 * ri.seconds / ri.iters,
        "projection_share": ri.projection_seconds / ri.seconds,
        "speedup_vs_standard_eps_step": r.seconds / ri.seconds}
    # the FP64 oracle beside it: two iterations with each eps-step, same settings
    t = time.perf_counter()
    ro = oadmm.admm(x_h.astype(np.float64), SIDES, cS, sigma=2.0, tv_iters=20, max_iters=2,
                    dyk_cycles=200, dyk_tol=1e-3, dyk_relative=True, n_threads=threads)
    t_std = (time.perf_counter() - t) / ro.iters
    t = time.perf_counter()
    ri_o = oadmm.admm(x_h.astype(np.float64), SIDES, cS, sigma=2.0, tv_iters=20, max_iters=2,
                      eps_incomplete=True, icd_K=ICD_K, icd_tol=ICD_TOL)
    t_icd = (time.perf_counter() - t) / ri_o.iters
    out["oracle"] = {"kind": "oracle", "cores": threads,
                     "ms_per_iteration_standard_eps_step": 1e3 * t_std,
                     "ms_per_iteration_incomplete_eps_step": 1e3 * t_icd,
                     "sample": "2 iterations each (FP64 numpy + C; Dykstra on all cores, the incomplete "
                               "step single-threaded)"}
    xs, es = torch.empty_like(I), torch.empty_like(I)
    with smre.Admm(H, W, SIDES, 2.0, tv_iters=20, max_iters=3, delta=-1.0, max_cycles=20,
                   tol=-1.0, **kw) as A:
        A.solve(I, xs, None, es)
    ref = oadmm.admm(x_h.astype(np.float64), SIDES, cS, sigma=2.0, tv_iters=20, max_iters=3,
                     dyk_cycles=20, n_threads=threads)
    out["err_vs_fp64_oracle"] = {
        "x": float(np.abs(xs.cpu().numpy() - ref.x).max() / np.abs(ref.x).max()),
        "eps": float(np.abs(es.cpu().numpy() - ref.eps).max() / np.abs(ref.eps).max()),
        "sample": "3 iterations x 20 cycles, max-abs relative"}
    return out


def run_extras(smre, torch, stream, peak, threads):
    out = {}
    for name, fn in (("batched_256_uneven", lambda: bench_batched(smre, torch, stream, peak)),
                     ("mixed_precision_2048", lambda: bench_mixed(smre, torch, stream, peak, threads)),
                     ("serving_poisson", lambda: bench_serving(smre, torch, stream, threads)),
                     ("admm_512", lambda: bench_admm(smre, torch, stream, threads))):
        t = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as e:   # a failed extra is reported, the main line stands
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = time.perf_counter() - t
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched, mixed-precision, serving and ADMM workloads")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_1503_03492_gb300 as smre

    rank, world, lrank = rank_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(lrank)
    dev = torch.device("cuda", lrank)
    stream = torch.cuda.current_stream(dev)

    x0 = make_input(1002 + rank)
    cS = smre.smre_bounds(smre.make_params(H, W, SIDES, alpha=ALPHA))
    # the handle's schedule autotuner times every schedule that can run the
    # shape (persistent launch, one-image batch, group launches) at create
    P = smre.Projector(H, W, SIDES, stream=stream, cmode=smre.SMRE_C_EXPLICIT, c_explicit=cS,
                       max_cycles=MAX_CYCLES, tol=TOL, tol_relative=True, flags=smre.SMRE_F_AUTOTUNE)
    schedule = {smre.SMRE_SCHED_PERSISTENT: "persistent", smre.SMRE_SCHED_BATCHED: "one-image batch",
                smre.SMRE_SCHED_GROUPS: "group launches"}.get(P.schedule(), "unknown")
    xd = torch.from_numpy(x0).to(dev)
    out_std = torch.empty_like(xd)
    out_icd = torch.empty_like(xd)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (126 MB)

    def step():
        r1 = P.project(xd, out_std)
        r2 = P.project_incomplete(xd, out_icd, K=ICD_K, tol=ICD_TOL)
        return r1, r2

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = P.kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    std_s, std_bytes, std_windows, icd_windows, cycles, icd_s = [], [], 0, 0, [], []
    with Clocks(lrank) as clk:
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            r1, r2 = step()
            ev[i][1].record(stream)
            std_s.append(r1.seconds)
            cycles.append(r1.cycles)
            std_bytes.append(algorithmic_bytes_per_cycle(True) +
                             (r1.cycles - 1) * algorithmic_bytes_per_cycle(False))
            std_windows += r1.windows
            icd_windows += r2.windows
            icd_s.append(r2.seconds)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    launches = P.kernel_launches() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_max, w_all = replica_totals(dist, dev, sum(step_ms) / 1e3, std_windows + icd_windows)
    value = w_all / t_max

    # end to end through the public API with host buffers (pinned), copies inside
    x_host = torch.from_numpy(x0.copy()).pin_memory()
    o1 = torch.empty_like(x_host).pin_memory()
    o2 = torch.empty_like(x_host).pin_memory()
    e2e_w, e2e_t = 0, 0.0
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        a = P.project(x_host.numpy(), o1.numpy())
        b = P.project_incomplete(x_host.numpy(), o2.numpy(), K=ICD_K, tol=ICD_TOL)
        e2e_t += time.perf_counter() - t0
        e2e_w += a.windows + b.windows
    e2e_t, e2e_w = replica_totals(dist, dev, e2e_t, e2e_w)
    e2e_val = e2e_w / e2e_t

    peak, peak_src = measured_peak_hbm()
    avg_std = sum(std_s) / len(std_s)
    achieved = (sum(std_bytes) / len(std_bytes)) / avg_std / 1e9
    clocks = clk.summary()
    tr = MEASURED_TRAFFIC.get(smre.smre_version()) if schedule == "persistent" else None
    cyc_med = int(np.median(cycles))
    traffic = None if tr is None else tr[0] + (cyc_med - 1) * tr[1]
    # the incomplete projection against its on-chip (issue-slot) ceiling
    icd_sec = sum(icd_s) / len(icd_s)
    icd_w = icd_windows / args.steps
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_mhz = clocks.get("sm_mhz") or 2070.0
    ins = ICD_WARP_INSTRUCTIONS.get(smre.smre_version())
    icd_ceiling = None if ins is None else icd_w / (ins / (n_sm * 4 * clk_mhz * 1e6))
    roofline_icd = {"bound": "issue", "achieved": icd_w / icd_sec, "peak": icd_ceiling,
                    "unit": "window-projections/s",
                    "frac": None if icd_ceiling is None else (icd_w / icd_sec) / icd_ceiling,
                    "kernel": "icd_pass_kernel<3> (passes i = 0..3 of one incomplete projection)",
                    "peak_source": "warp instructions per call from ncu x (SMs x 4 issue slots x "
                                   "median SM clock)",
                    "warp_instructions_per_call": ins, "seconds_per_call": icd_sec,
                    "hbm_bytes_per_call": 8 * H * W * (ICD_K + 1),
                    "critical_path": icd_critical_path(P.icd_sweeps(), H, W, ICD_K, icd_sec)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        threads = os.cpu_count() or 1
        cyc = int(os.environ.get("SMRE_CPU_SAMPLE_CYCLES", "800"))
        wv, sv = cpu_sample(x0, threads, cyc)
        cpu = {"value": wv / sv, "unit": "window-projections/s", "cores": threads, "kind": "oracle",
               "sample": f"{cyc} of the {int(np.median(cycles))} standard cycles + the full "
                         f"incomplete projection of the same image, FP64 C oracle, "
                         f"{threads} OpenMP threads ({sv:.1f} s)"}

    extras = None
    if rank == 0 and world == 1 and not args.no_extras:
        P.close()
        extras = run_extras(smre, torch, stream, peak, os.cpu_count() or 1)

    if rank == 0:
        line = {
            "metric": "window-projections/s", "value": value, "unit": "window-projections/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "H": H, "W": W, "sides": "1..8", "alpha": ALPHA,
                       "bounds": "per-window fourth-root (Sec. 2.1)",
                       "standard_cycles_per_step": int(np.median(cycles)),
                       "standard_windows_per_step": std_windows // args.steps,
                       "icd_windows_per_step": icd_windows // args.steps,
                       "l2": "flushed between timed steps (256 MB write); q store 214 MB > L2",
                       "schedule": schedule + " (SMRE_F_AUTOTUNE)",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": ("persist_reg_kernel<8> (one launch = one standard projection)"
                                    if schedule == "persistent" else schedule),
                         "peak_source": peak_src,
                         "bytes_per_launch": sum(std_bytes) / len(std_bytes),
                         "seconds_per_launch": avg_std},
            "roofline_icd": roofline_icd,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "window-projections/s",
                    "h2d_bytes_per_step": 2 * H * W * 4, "d2h_bytes_per_step": 2 * H * W * 4},
            "gpu_launches": launches,
            "clocks": clocks,
            "extras": extras,
        }
        print(json.dumps(line), flush=True)
    P.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

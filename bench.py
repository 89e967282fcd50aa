#!/usr/bin/env python
"""Benchmark: track-solid queries per second on the precision-form workload.

One step = all five queries (Inside, DistanceToIn, DistanceToOut, SafetyToIn,
SafetyToOut) for 2^24 tracks against each of five solids (box 10x20x30, trd
(10,20,15,5,30), tube segment (5,20,30, phi 0-270 deg), cone segment
(0,10,5,25,40), an 8-plane polycone), i.e. 5 * 2^24 tracks and 25 * 2^24
queries, inputs resident in HBM.  Synthetic, seeded inputs (half inside each
solid, 10% within 1e-8 mm of a surface, isotropic directions).

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead, on a bounded sample of the same workload, on the host cores.

Multi-GPU (torchrun): every rank runs its own copy of the workload (the tracks
are independent; no data-path collective) -> weak scaling; the time is the max
over ranks.
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

N_QUERIES = 5
BYTES_PER_TRACK = 6 * 8 + 1 + 4 * 8  # SoA point + direction in, code + 4 doubles out
# DRAM bytes per track of each binary32 pass, from one ncu capture per pass at 2^22 tracks
# (dram__bytes_read.sum + dram__bytes_write.sum of one launch; results still in L2 at the end of a
# launch are not counted, at most 129 MB); valid only while the kernel sources hash to the value
# recorded with them, else the bench reports traffic = null.
DRAM_CAPTURE = {
    "sources_sha256": "76e9d0d63b2268d4487bf17bc51db7e11e496f00247adc8c5ffbb5284f2e4c3a",
    "bytes_per_track": {'box': 71.89, 'trd': 72.45, 'tube': 73.43, 'cone': 73.60, 'polycone': 72.30},
    "profile": "profiles/query_fp32_passes_4M_counters.md",
}
# Warp instructions per track of each binary32 pass (smsp__inst_executed.sum of one launch ÷
# its tracks, from the same captures; the counts do not depend on the basket size), valid while
# the kernel sources hash to the recorded value.
ISSUE_CAPTURE = {
    "sources_sha256": "76e9d0d63b2268d4487bf17bc51db7e11e496f00247adc8c5ffbb5284f2e4c3a",
    "warp_inst_per_track": {'box': 18.61, 'trd': 34.34, 'tube': 62.04, 'cone': 57.16, 'polycone': 116.11},
    "profile": "profiles/query_fp32_passes_4M_counters.md",
}
KERNEL_SOURCES = ("solid_fp32.cuh", "query_fp32.cu", "gv_desc.h")
# FP64-pipe warp instructions per track of the binary64 pass on the 2^20-track tube and cone
# (sm__inst_executed_pipe_fp64.sum of one launch / its tracks), valid while the binary64 sources
# hash to the recorded value.
FP64_CAPTURE = {
    "sources_sha256": "a07399a0b4f95abb2a949a3ac5e9237dcdb23b0aab450eaf2b66597fbf4d00c7",
    "fp64_warp_inst_per_track": {'tube': 10.47, 'cone': 7.29},
    "profile": "profiles/query_fp64_tube_cone_1M_pipe.md",
}
FP64_KERNEL_SOURCES = ("solid_fp64.cuh", "query_fp64.cu", "gv_desc.h", "work_class.cuh")
E2E_CHUNK = 1 << 22  # tracks per host-streaming chunk (2^19-2^22 measured: larger is faster)
E2E_SLOTS = 3


def specs():
    return [("box", W.BOX_M1), ("trd", W.TRD_M3), ("tube", W.TUBE_M2), ("cone", W.CONE_M2),
            ("polycone", W.polycone_m3())]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "fp64", "fp32_refine"])
    ap.add_argument("--tracks", type=int, default=1 << 24, help="tracks per solid")
    ap.add_argument("--cpu-sample", type=int, default=40000, help="tracks per solid for the oracle")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched, navigation and serving forms")
    ap.add_argument("--form", default="all", choices=["all", "batched", "transport", "peaks", "fp64"],
                    help="batched / transport / fp64 (the binary64 tube and cone): only that form (for "
                         "profiling); peaks: the probe rates")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock/throttle samples taken while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- CPU oracle

def cpu_baseline(tracks_per_solid: dict, sample: int):
    """The oracle as it stands, on a bounded sample of each solid's tracks, all host cores."""
    import oracle
    threads = os.cpu_count() or 1
    total_tracks = 0
    t0 = time.perf_counter()
    for name, spec in specs():
        tr = {k: v[:sample] for k, v in tracks_per_solid[name].items()}
        oracle.Solid.from_spec(spec).query(**tr, threads=threads)
        total_tracks += len(tr["x"])
    dt = time.perf_counter() - t0
    return {"value": total_tracks * N_QUERIES / dt, "unit": "queries/s", "cores": threads,
            "kind": "oracle",
            "sample": f"first {sample} tracks of each of the 5 solids' 2^24-track baskets, all five queries"}


def cpu_closed_form(tracks_per_solid: dict, oracle_sample: int, sample: int = 1 << 20):
    """The fair CPU baseline (cpu_baseline/: the binary64 closed forms compiled for the host),
    on all host cores over the first `sample` tracks of each solid and on one core over a
    sixteenth of that, all five queries; checked against the oracle on the oracle's sample."""
    import cpu_baseline
    import oracle
    threads = os.cpu_count() or 1
    res = {"kind": "closed-form binary64 loop (the library's binary64 solid code on the host)",
           "cores": threads, "unit": "queries/s"}
    for label, th, m in (("allcores", threads, sample), ("1core", 1, sample // 16)):
        total, t = 0, 0.0
        for name, spec in specs():
            tr = {k: v[:m] for k, v in tracks_per_solid[name].items()}
            c = cpu_baseline.Solid(spec)
            t0 = time.perf_counter()
            c.query(**tr, threads=th)
            t += time.perf_counter() - t0
            total += m
        res[f"{label}_value"] = total * N_QUERIES / t
        res[f"{label}_sample"] = f"first {m} tracks of each of the 5 solids' baskets"
    # parity with the oracle on its sample: codes equal; zeros, -1 and +inf equal; others within 1e-9 mm
    bad = 0
    for name, spec in specs():
        tr = {k: v[:oracle_sample] for k, v in tracks_per_solid[name].items()}
        got = cpu_baseline.Solid(spec).query(**tr, threads=threads)
        want = oracle.Solid.from_spec(spec).query(**tr, threads=threads)
        bad += int((got["inside"] != want["inside"]).sum())
        for k in ("dist_in", "dist_out", "safety_in", "safety_out"):
            g, w = got[k], want[k]
            special = ~np.isfinite(w) | (w <= 0)
            with np.errstate(invalid="ignore"):
                ok = np.where(special, (g == w) | (np.isinf(g) & np.isinf(w)), np.abs(g - w) <= 1e-9)
            bad += int((~ok).sum())
    res["parity_vs_oracle"] = {"mismatches": bad, "tracks": 5 * oracle_sample, "tolerance_mm": 1e-9}
    return res


def cpu_baseline_extras():
    """The oracle beside the other forms, all host cores, on bounded samples of their
    workloads: the transport loop (nested detector, 16384 tracks, kmax 64), boolean solids
    (the bench's three, 100000 tracks each, all five queries), the navigation step in the
    nested detector (100000 tracks) and in the crowded lattice (20000 tracks, every daughter
    scanned)."""
    import oracle
    threads = os.cpu_count() or 1
    res = {"cores": threads}
    geo = W.nested_geometry()
    O = oracle.Geometry(geo["solids"], geo["nodes"])
    n, kmax = 16384, 64
    tr = W.nested_tracks(n, seed=11, geom=geo)
    node0 = O.locate(tr["x"], tr["y"], tr["z"], threads=threads)
    m = W.transport_materials(geo)
    xi = W.transport_xi(n, kmax, seed=1)
    t0 = time.perf_counter()
    out = O.transport(tr["x"], tr["y"], tr["z"], tr["dx"], tr["dy"], tr["dz"], node0, m["node_material"],
                      m["sigma_n"], xi, kmax, threads=threads)
    dt = time.perf_counter() - t0
    res["transport"] = {"tracks_per_s": n / dt, "steps_per_s": float(out["steps"].sum()) / dt, "sample": n}
    res["boolean"] = {}
    for spec in W.boolean_table(3, seed=13):
        tb = W.tracks_for_solid(spec, 100000, seed=21)
        t0 = time.perf_counter()
        oracle.Solid.from_spec(spec).query(**tb, threads=threads)
        res["boolean"][spec["params"][0]] = {"queries_per_s": 100000 * N_QUERIES / (time.perf_counter() - t0)}
    for label, g, k, mk in (("nav_nested", geo, 100000, lambda: W.nested_tracks(100000, seed=1, geom=geo)),
                            ("nav_crowded", W.crowded_geometry(), 20000, None)):
        Og = oracle.Geometry(g["solids"], g["nodes"])
        tn = mk() if mk else W.crowded_tracks(g, k, seed=2, surf_frac=0.0)
        nd = Og.locate(tn["x"], tn["y"], tn["z"], threads=threads)
        t0 = time.perf_counter()
        Og.nav_step(tn["x"], tn["y"], tn["z"], tn["dx"], tn["dy"], tn["dz"], nd, threads=threads)
        res[label] = {"steps_per_s": k / (time.perf_counter() - t0), "sample": k}
    return res


def cpu_baseline_sweep(max_exp: int = 16):
    """The oracle and the closed-form CPU loop on the sweep's tracks for N <= 2^max_exp, one
    core and all cores (DistanceToOut only), for the GPU-over-CPU ratio of the paper's figure."""
    import cpu_baseline
    import oracle
    threads = os.cpu_count() or 1
    res = {}
    for name, spec in SWEEP_SPECS:
        o = oracle.Solid.from_spec(spec)
        c = cpu_baseline.Solid(spec)
        rows = []
        for e in SWEEP_EXPONENTS:
            if e > max_exp:
                break
            n = 1 << e
            tr = sweep_tracks(spec, n)
            row = {"n": n}
            for label, th in (("1core", 1), ("allcores", threads)):
                reps = max(1, min(200, (1 << 14) // n))
                t0 = time.perf_counter()
                for _ in range(reps):
                    o.query(**tr, threads=th, want=("dist_out",))
                row[f"oracle_{label}_tracks_per_s"] = n * reps / (time.perf_counter() - t0)
                reps = max(1, min(2000, (1 << 18) // n))
                t0 = time.perf_counter()
                for _ in range(reps):
                    c.query(**tr, threads=th, want=("dist_out",))
                row[f"closed_form_{label}_tracks_per_s"] = n * reps / (time.perf_counter() - t0)
            rows.append(row)
        res[name] = rows
    return {"cores": threads, "rows": res}


def tracks_label(n: int) -> str:
    """2^k when n is a power of two, else the number."""
    return f"2^{n.bit_length() - 1}" if n > 0 and n & (n - 1) == 0 else str(n)


def kernel_sources_sha256(files=KERNEL_SOURCES) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1512_06637_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def gen_inputs(n: int):
    return {name: W.tracks_for_solid(spec, n, seed=2) for name, spec in specs()}


# ------------------------------------------------------------- reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sample = args.cpu_sample
    inputs = {name: W.tracks_for_solid(spec, sample, seed=2) for name, spec in specs()}
    for _ in range(args.warmup):
        cpu_baseline(inputs, sample)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cb = cpu_baseline(inputs, sample)
    dt = time.perf_counter() - t0
    value = args.steps * 5 * sample * N_QUERIES / dt
    line = {"metric": "track-solid queries/s", "value": value, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "precision form: box, trd, tube, cone, polycone; 2^24 tracks per solid "
                                   "(oracle step = bounded sample)", "tracks_per_solid_sampled": sample},
            "cpu_baseline": {**cb, "value": value},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def run_ours(args):
    import torch

    import paper_1512_06637_gb300 as gv
    from paper_1512_06637_gb300 import build

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    n = args.tracks
    # host inputs are generated before the first CUDA call
    inputs = gen_inputs(n)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    precision = args.precision
    if precision == "auto":
        precision = "fp32_refine" if gv_supports_fp32(gv) else "fp64"
    dev = {name: {k: torch.from_numpy(v).cuda() for k, v in tr.items()} for name, tr in inputs.items()}
    solids = {name: gv.Solid.from_spec(spec) for name, spec in specs()}
    outs = {name: gv.alloc_results(n, "cuda") for name in solids}
    ws = gv.Workspace(n) if precision == "fp32_refine" else None
    stream = torch.cuda.current_stream()
    names = list(solids)
    launches_per_query = 2 if precision == "fp32_refine" else 1

    def step(events=None):
        for i, name in enumerate(names):
            if events is not None:
                events[i][0].record(stream)
            gv.query(solids[name], dev[name], precision=precision, out=outs[name], workspace=ws,
                     stream=stream)
            if events is not None:
                events[i][1].record(stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # timed region: K steps, barrier + synchronize on both sides, clocks sampled
    ev = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in names]
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        step(ev[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ck = clocks.stop()
    ms = t_start.elapsed_time(t_end)
    per_solid_ms = {name: statistics.mean(ev[k][i][0].elapsed_time(ev[k][i][1]) for k in range(args.steps))
                    for i, name in enumerate(names)}
    ms = reduce_max(ms, world)
    value = aggregate(args.steps * len(names) * n * N_QUERIES, world, ms)

    # dominant kernel: the query pass with the largest mean time per launch
    dom = max(per_solid_ms, key=per_solid_ms.get)
    dom_ms = per_solid_ms[dom]
    peaks = load_peaks()
    achieved = n * BYTES_PER_TRACK / (dom_ms * 1e-3) / 1e9
    traffic = None
    sha = kernel_sources_sha256()
    if precision == "fp32_refine" and sha == DRAM_CAPTURE["sources_sha256"]:
        per_track = DRAM_CAPTURE["bytes_per_track"].get(dom)
        traffic = None if per_track is None else per_track * n
    hbm = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
           "kernel": f"query pass ({precision}) on {dom}", "peak_source": peaks["source"],
           "traffic_source": DRAM_CAPTURE["profile"] if traffic is not None else
           "none: the kernel sources changed since the last DRAM capture"}
    # the same launch against the measured warp-instruction issue peak (these passes are
    # issue-bound: the one whose fraction is larger binds)
    alu = bench_alu_peaks(torch, local)
    issue = None
    if precision == "fp32_refine" and sha == ISSUE_CAPTURE["sources_sha256"] and dom in ISSUE_CAPTURE["warp_inst_per_track"]:
        inst_rate = ISSUE_CAPTURE["warp_inst_per_track"][dom] * n / (dom_ms * 1e-3)
        mhz = ck.get("sm_mhz") or alu["sm_mhz"]
        ipeak = alu["issue_warp_inst_per_clk_per_sm"] * alu["sms"] * mhz * 1e6
        issue = {"bound": "alu", "achieved": inst_rate, "peak": ipeak, "unit": "warp instructions/s",
                 "frac": inst_rate / ipeak, "traffic": traffic, "kernel": hbm["kernel"],
                 "peak_source": "measured (probe: binary32 multiply-add issue rate x SMs x sampled clock)",
                 "instructions_source": ISSUE_CAPTURE["profile"]}
    roofline = dict(issue if issue is not None and issue["frac"] > hbm["frac"] else hbm)
    roofline["hbm_frac"] = hbm["frac"]
    roofline["issue_frac"] = None if issue is None else issue["frac"]

    refined = None
    if precision == "fp32_refine":
        refined = {}
        for name in names:
            gv.query(solids[name], dev[name], precision=precision, out=outs[name], workspace=ws, stream=stream)
            refined[name] = ws.refined(stream) / n

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(gv, torch, inputs, solids, precision, n, max(1, min(args.steps, 3)), world)

    line = {
        "metric": "track-solid queries/s", "value": value, "unit": "queries/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if precision == "fp32_refine" else "f64", "data": "synthetic",
        "config": {"workload": f"precision form: box, trd, tube, cone, polycone; {tracks_label(n)} tracks per "
                               "solid; all five queries", "tracks_per_solid": n, "precision": precision,
                   "l2": f"inputs {'larger' if 5 * n * 48 > 129e6 else 'smaller'} than L2 "
                         f"({5 * n * 48 / 1e9:.2f} GB per step)",
                   "parallelism": f"replicas x{world}"},
        "per_solid_ms": per_solid_ms,
        "roofline": roofline,
        "alu_peaks": alu,
        "clocks": ck,
        "gpu_launches": args.steps * len(names) * launches_per_query,
        "e2e": e2e,
    }
    if refined is not None:
        line["refined_fraction"] = refined
    if not args.no_extra:
        if precision == "fp32_refine":
            line["fp64_form"] = bench_fp64_form(gv, torch, solids, dev, outs, names, n)
        # release the precision-form buffers before the other forms
        del dev, outs
        torch.cuda.empty_cache()
        line["box1024"] = bench_box1024(gv, torch)
        line["fp64_tube_cone_2e20"] = bench_fp64_m2(gv, torch, peaks, line.get("alu_peaks"))
        line["sweep_dist_out"] = bench_sweep(gv, torch)
        line["batched"] = bench_batched(gv, torch, max(3, args.steps), peaks)
        line["nav"] = bench_nav(gv, torch, max(3, args.steps))
        line["transport"] = bench_transport(gv, torch)
        line["boolean"] = bench_boolean(gv, torch)
        line["voxels"] = bench_voxels(gv, torch)
        if rank == 0:
            line["serving"] = bench_serving(gv, torch)
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(inputs, args.cpu_sample)
        line["cpu_closed_form"] = cpu_closed_form(inputs, args.cpu_sample)
        if not args.no_extra:
            line["sweep_dist_out_oracle"] = cpu_baseline_sweep()
            line["oracle_extras"] = cpu_baseline_extras()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_e2e(gv, torch, inputs, solids, precision, n, steps, world):
    """Same metric through the public host-buffer call (gv_query_host): pinned host inputs
    streamed in, queries, results streamed back into pinned host arrays, all inside the
    timed region; the five solids go back to back through one pipeline."""
    host_in = {name: {k: torch.from_numpy(v).pin_memory() for k, v in tr.items()} for name, tr in inputs.items()}
    host_out = {name: {k: torch.empty(n, dtype=torch.int8 if k == "inside" else torch.float64).pin_memory()
                       for k in gv.QUERIES} for name in solids}
    pipe = gv.Pipeline(E2E_CHUNK, E2E_SLOTS)
    stream = torch.cuda.current_stream()

    def step():
        for name in solids:
            gv.query_host(solids[name], host_in[name], host_out[name], pipe, precision=precision, stream=stream)
        pipe.join(stream)

    step()
    torch.cuda.synchronize()
    # The host link is shared with the machine's other GPUs and their jobs: time five
    # separate windows and report the median one (all five are listed).
    windows = []
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            step()
        b.record(stream)
        torch.cuda.synchronize()
        windows.append(reduce_max(a.elapsed_time(b), world))
    ms = sorted(windows)[2]
    h2d = sum(t.numel() * t.element_size() for tr in host_in.values() for t in tr.values())
    d2h = sum(t.numel() * t.element_size() for tr in host_out.values() for t in tr.values())
    link = host_link(torch)
    # the fewest milliseconds the step's copies can take on this link (directions overlap)
    bound_ms = 1e3 * max(h2d / (link["h2d_gbs"] * 1e9), d2h / (link["d2h_gbs"] * 1e9),
                         (h2d + d2h) / (link["both_gbs"] * 1e9))
    return {"value": aggregate(steps * len(solids) * n * N_QUERIES, world, ms), "unit": "queries/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "windows_ms_per_step": [w / steps for w in windows], "statistic": "median of 5 windows",
            "path": f"gv_query_host, chunks of {E2E_CHUNK} tracks, {E2E_SLOTS} staging slots",
            "link": link, "link_bound_ms_per_step": bound_ms, "link_frac": bound_ms / (ms / steps)}


def host_link(torch, copies: int = 16, mib: int = 32) -> dict:
    """Copy bandwidth between pinned host memory and this GPU (GB/s): host to device,
    device to host, and both directions at once on two streams; `copies` copies of `mib` MiB
    each way, timed with CUDA events.  More streams per direction measured no faster."""
    n = mib * (1 << 20) // 8
    h_in = [torch.ones(n, dtype=torch.float64).pin_memory() for _ in range(copies)]
    h_out = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(copies)]
    d = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(copies)]
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def run(up: bool, down: bool) -> float:
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        a.record()
        s_in.wait_event(a)
        s_out.wait_event(a)
        for j in range(copies):
            if up:
                with torch.cuda.stream(s_in):
                    d[j].copy_(h_in[j], non_blocking=True)
            if down:
                with torch.cuda.stream(s_out):
                    h_out[j].copy_(d[(j + 1) % copies], non_blocking=True)
        ends = []
        for st in (s_in, s_out):
            e = torch.cuda.Event(enable_timing=True)
            e.record(st)
            ends.append(e)
        torch.cuda.synchronize()
        sec = max(a.elapsed_time(e) for e in ends) / 1e3
        return (int(up) + int(down)) * copies * n * 8 / sec / 1e9

    run(True, True)  # warm-up
    return {"h2d_gbs": run(True, False), "d2h_gbs": run(False, True), "both_gbs": run(True, True)}


def reduce_max(value: float, world: int, device: str = "cuda") -> float:
    """Max of a per-rank time over all ranks (the only collective of a replicated run)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput: units processed by all ranks over the slowest rank's time."""
    return world * units_per_rank / (ms_max * 1e-3)


def _timed(torch, fn, reps):
    """Mean device time (ms) of fn() over reps calls, CUDA events on the current stream."""
    stream = torch.cuda.current_stream()
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


SWEEP_EXPONENTS = tuple(range(4, 25, 2))  # N = 2^4 ... 2^24
SWEEP_SPECS = (("box", W.BOX_M1), ("tube", W.TUBE_M2))


def sweep_tracks(spec, n):
    """The paper's experiment: points inside the solid, isotropic directions."""
    return W.tracks_for_solid(spec, n, seed=6637, near_frac=0.0, inside_frac=1.0)


def bench_sweep(gv, torch):
    """The paper's measurement (its one figure): Box and Tube DistanceToOut throughput
    against the number of tracks N, for points inside with isotropic directions.  Per N
    the mean device time of one gv_query call over many repetitions (about 2^26 tracks
    per N in total, at least 8 calls; for small N that is the host's submission rate),
    and for N <= 2^16 one call replayed from a CUDA graph (the device's own rate)."""
    res = {}
    nmax = 1 << max(SWEEP_EXPONENTS)
    for name, spec in SWEEP_SPECS:
        dev = {k: torch.from_numpy(v).cuda() for k, v in sweep_tracks(spec, nmax).items()}
        s = gv.Solid.from_spec(spec)
        ws = gv.Workspace(nmax)
        dout = torch.empty(nmax, dtype=torch.float64, device="cuda")
        rows = []
        for e in SWEEP_EXPONENTS:
            n = 1 << e
            sub = {k: v[:n] for k, v in dev.items()}
            out = {"dist_out": dout[:n]}
            reps = max(8, min(5000, (1 << 26) // n))
            row = {"n": n}
            for prec in ("fp32_refine", "fp64"):
                ms = _timed(torch, lambda: gv.query(s, sub, precision=prec, out=out, workspace=ws), reps)
                row[prec + "_tracks_per_s"] = n / (ms * 1e-3)
                row[prec + "_us_per_call"] = ms * 1e3
            if n <= 1 << 16:  # small baskets: one captured call replayed (no host submission cost)
                for prec in ("fp32_refine", "fp64"):
                    stream = torch.cuda.Stream()
                    g = torch.cuda.CUDAGraph()
                    with torch.cuda.stream(stream):
                        gv.query(s, sub, precision=prec, out=out, workspace=ws, stream=stream)
                        torch.cuda.synchronize()
                        with torch.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
                            gv.query(s, sub, precision=prec, out=out, workspace=ws, stream=stream)
                    ms = _timed(torch, g.replay, reps)
                    row[prec + "_graph_us_per_call"] = ms * 1e3
                    row[prec + "_graph_tracks_per_s"] = n / (ms * 1e-3)
            rows.append(row)
        res[name] = rows
    return res


def bench_box1024(gv, torch, reps=5000):
    """1024 tracks against the (10,20,30) box, all five queries: a launch-latency bound
    basket; mean time per gv_query call and per replay of a captured call."""
    tr = W.box1024()
    dev = {k: torch.from_numpy(v).cuda() for k, v in tr.items()}
    s = gv.Solid.from_spec(W.BOX_M1)
    ws = gv.Workspace(1024)
    out = gv.alloc_results(1024, "cuda")
    res = {"workload": "box (10,20,30), 1024 tracks, 5% within 1e-10 mm of a face, all five queries"}
    for prec in ("fp32_refine", "fp64"):
        res[prec + "_us_per_call"] = 1e3 * _timed(
            torch, lambda: gv.query(s, dev, precision=prec, out=out, workspace=ws), reps)
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        gv.query(s, dev, precision="fp32_refine", out=out, workspace=ws, stream=stream)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
            gv.query(s, dev, precision="fp32_refine", out=out, workspace=ws, stream=stream)
    res["fp32_refine_graph_us_per_call"] = 1e3 * _timed(torch, g.replay, reps)
    return res


def bench_fp64_form(gv, torch, solids, dev, outs, names, n, reps=2):
    """The same workload in plain binary64 (all five queries, the inputs already on the device):
    per-solid CUDA-event times and the step's rate.  Baskets this large are evaluated in tiles
    ordered by work class."""
    per = {}
    for name in names:
        per[name] = _timed(torch, lambda: gv.query(solids[name], dev[name], precision="fp64", out=outs[name]), reps)
    ms = sum(per.values())
    return {"ms_per_step": ms, "queries_per_s": len(names) * n * N_QUERIES / (ms * 1e-3), "per_solid_ms": per}


def bench_fp64_m2(gv, torch, peaks, alu=None, reps=20):
    """Tube (5,20,30,0,270 deg) and cone (0,10,5,25,40,0,360 deg), 2^20 tracks each, plain
    binary64, all five queries (the binary64 kernels alone), against the HBM roof and, while the
    binary64 sources match the recorded capture, against the FP64 pipe: the captured FP64-pipe
    warp instructions per track x tracks / time, over the probe's binary64 multiply-add rate in
    warp instructions (its per-SM rate / 32 lanes x SMs x clock)."""
    res = {}
    n = 1 << 20
    fp64_ok = FP64_CAPTURE["sources_sha256"] == kernel_sources_sha256(FP64_KERNEL_SOURCES)
    for name, spec in (("tube", W.TUBE_M2), ("cone", W.CONE_M2)):
        dev = {k: torch.from_numpy(v).cuda() for k, v in W.tracks_for_solid(spec, n, seed=8).items()}
        s = gv.Solid.from_spec(spec)
        out = gv.alloc_results(n, "cuda")
        ms = _timed(torch, lambda: gv.query(s, dev, precision="fp64", out=out), reps)
        gbs = n * BYTES_PER_TRACK / (ms * 1e-3) / 1e9
        r = {"queries_per_s": n * N_QUERIES / (ms * 1e-3), "us": ms * 1e3, "hbm_gbs": gbs,
             "hbm_frac": gbs / peaks["hbm_gbs"], "fp64_pipe_frac": None}
        per_track = FP64_CAPTURE["fp64_warp_inst_per_track"].get(name)
        if alu is not None and fp64_ok and per_track is not None:
            peak = alu["fp64_fma"]["per_clk_per_sm"] / 32.0 * alu["sms"] * alu["sm_mhz"] * 1e6
            r["fp64_pipe_frac"] = per_track * n / (ms * 1e-3) / peak
            r["fp64_pipe_source"] = FP64_CAPTURE["profile"]
        res[name] = r
    return res


def bench_transport(gv, torch, reps=3, n=1 << 20, kmax=64):
    """The transport loop (binary64): 2^20 tracks uniform in the nested detector, vacuum world,
    light shells and dense cells, random numbers given; tracks and steps per second."""
    geo = W.nested_geometry()
    G = gv.Geometry(geo["solids"], geo["nodes"])
    tr = W.nested_tracks(n, seed=11, geom=geo)
    dev = {k: torch.from_numpy(v).cuda() for k, v in tr.items()}
    node0 = G.locate(dev)
    m = W.transport_materials(geo)
    mat = torch.from_numpy(m["node_material"]).cuda()
    sig = torch.from_numpy(m["sigma_n"]).cuda()
    xi = torch.from_numpy(W.transport_xi(n, kmax, seed=1)).cuda()
    out = G.transport(dev, node0, mat, sig, xi, kmax)
    ms = _timed(torch, lambda: G.transport(dev, node0, mat, sig, xi, kmax, out=out), reps)
    steps = int(out["steps"].sum().item())
    res = {"workload": "nested detector, 2^20 tracks, kmax 64, binary64", "tracks_per_s": n / (ms * 1e-3),
           "steps_per_s": steps / (ms * 1e-3), "mean_steps": steps / n, "ms": ms,
           "reasons": torch.bincount(out["reason"].long(), minlength=4).tolist()}
    # candidates and codes ranked in binary32 first (the same results)
    ms32 = _timed(torch, lambda: G.transport(dev, node0, mat, sig, xi, kmax, out=out, precision="fp32_refine"), reps)
    res["rank32"] = {"tracks_per_s": n / (ms32 * 1e-3), "steps_per_s": steps / (ms32 * 1e-3), "ms": ms32}
    return res


def bench_boolean(gv, torch, reps=5, n=1 << 20):
    """Boolean solids (binary64): a union, a subtraction and an intersection of random
    primitives, 2^20 tracks each, all five queries."""
    res = {}
    for spec in W.boolean_table(3, seed=13):
        op = spec["params"][0]
        dev = {k: torch.from_numpy(v).cuda() for k, v in W.tracks_for_solid(spec, n, seed=21).items()}
        s = gv.Solid.from_spec(spec)
        out = gv.alloc_results(n, "cuda")
        ms = _timed(torch, lambda: gv.query(s, dev, precision="fp64", out=out), reps)
        res[op] = {"components": [spec["params"][1]["kind"], spec["params"][2]["kind"]],
                   "queries_per_s": n * N_QUERIES / (ms * 1e-3), "us": ms * 1e3}
    return res


def bench_batched(gv, torch, reps, peaks):
    """Mixed baskets: 4096 baskets of 16-4096 tracks over 64 solids of the six types,
    one persistent launch replayed from a CUDA graph, launch shape from the autotuner."""
    work = W.batched()
    n = len(work["tracks"]["x"])
    dev = {k: torch.from_numpy(v).cuda() for k, v in work["tracks"].items()}
    solids = [gv.Solid.from_spec(sp) for sp in work["solids"]]
    res = {"workload": "4096 baskets, log-uniform 16-4096 tracks, 64 solids of 6 types", "tracks": n}
    for prec in ("fp32_refine", "fp64"):
        b = gv.Batch(solids, work["offset"], work["n"], work["solid"])
        out = gv.alloc_results(n, "cuda")
        cfg = b.autotune(dev, out, precision=prec)
        ms = _timed(torch, lambda: b.run(dev, out, precision=prec), reps)
        gbs = n * BYTES_PER_TRACK / (ms * 1e-3) / 1e9
        res[prec] = {"queries_per_s": n * N_QUERIES / (ms * 1e-3), "ms": ms, "config": cfg,
                     "hbm_gbs": gbs, "hbm_frac": gbs / peaks["hbm_gbs"]}
        if prec == "fp32_refine":
            res[prec]["refined_fraction"] = b.refined() / n
    res["fp32_over_fp64"] = res["fp32_refine"]["queries_per_s"] / res["fp64"]["queries_per_s"]
    return res


def bench_nav(gv, torch, reps, n=1 << 22):
    """Navigation step in the nested detector (world box, 10 tube shells, 32 box cells
    each): tracks uniform in the world, located once, one step timed."""
    geo = W.nested_geometry()
    G = gv.Geometry(geo["solids"], geo["nodes"])
    tr = W.nested_tracks(n, seed=1, geom=geo)
    dev = {k: torch.from_numpy(v).cuda() for k, v in tr.items()}
    node = G.locate(dev)
    torch.cuda.synchronize()
    # queries per track-step: mother DistanceToOut + SafetyToOut, each daughter DistanceToIn + SafetyIn
    ndaughters = np.zeros(len(geo["nodes"]) + 1, np.int64)
    for nd in geo["nodes"][1:]:
        ndaughters[nd["parent"]] += 1
    nn = node.cpu().numpy()
    q_per_step = float(np.mean(2 * (1 + ndaughters[np.where(nn >= 0, nn, len(geo["nodes"]))])))
    res = {"workload": "nested detector, 2^22 tracks uniform in the world", "queries_per_track_step": q_per_step}
    ws = gv.Workspace(n)
    out = None
    for prec in ("fp32_refine", "fp64"):
        out = G.step(dev, node, precision=prec, workspace=ws, out=out)
        ms = _timed(torch, lambda: G.step(dev, node, precision=prec, workspace=ws, out=out), reps)
        res[prec] = {"steps_per_s": n / (ms * 1e-3), "queries_per_s": n * q_per_step / (ms * 1e-3), "ms": ms}
        if prec == "fp32_refine":
            res[prec]["refined_fraction"] = ws.refined() / n
    res["locate_ms"] = _timed(torch, lambda: G.locate(dev, out=node), max(1, reps // 2))
    return res


def bench_voxels(gv, torch, reps=3, n=1 << 20, n_transport=1 << 18, kmax=32):
    """Voxelised navigation: the crowded lattice (1728 daughters of the world, one holding 27
    more), 2^20 tracks uniform in the world (10% along an axis), located once; locate, one
    binary64 step, one binary32 + refinement step (each with and without the safety, which
    is a minimum over every daughter), and the transport loop (2^18 tracks, kmax 32,
    binary64) with the daughters' grids on and off."""
    geo = W.crowded_geometry()
    G = gv.Geometry(geo["solids"], geo["nodes"])
    dev = {k: torch.from_numpy(v).cuda() for k, v in W.crowded_tracks(geo, n, seed=2, surf_frac=0.0).items()}
    node = G.locate(dev)
    ws = gv.Workspace(n)
    out = G.step(dev, node, precision="fp64", workspace=ws)
    tdev = {k: v[:n_transport].contiguous() for k, v in dev.items()}
    node0 = node[:n_transport].contiguous()
    m = W.crowded_materials(geo)
    mat = torch.from_numpy(m["node_material"]).cuda()
    sig = torch.from_numpy(m["sigma_n"]).cuda()
    xi = torch.from_numpy(W.transport_xi(n_transport, kmax, seed=2)).cuda()
    tout = G.transport(tdev, node0, mat, sig, xi, kmax)
    res = {"workload": "crowded lattice, 1728 + 27 daughters, 2^20 tracks; transport 2^18 tracks, kmax 32",
           "grids": G.voxel_count}
    for on in (True, False):
        G.set_voxels(on)
        r = max(1, reps if on else 1)
        key = "grids" if on else "brute_force"
        res[key] = {
            "locate_ms": _timed(torch, lambda: G.locate(dev, out=node), r),
            "fp64_step_ms": _timed(torch, lambda: G.step(dev, node, precision="fp64", workspace=ws, out=out), r),
            "fp32_refine_step_ms": _timed(torch, lambda: G.step(dev, node, precision="fp32_refine", workspace=ws,
                                                                out=out), r),
            "fp64_step_nosafety_ms": _timed(torch, lambda: G.step(dev, node, precision="fp64", workspace=ws, out=out,
                                                                  safety=False), r),
            "fp32_refine_step_nosafety_ms": _timed(torch, lambda: G.step(dev, node, precision="fp32_refine",
                                                                         workspace=ws, out=out, safety=False), r),
            "transport_ms": _timed(torch, lambda: G.transport(tdev, node0, mat, sig, xi, kmax, out=tout), r),
            "transport_rank32_ms": _timed(torch, lambda: G.transport(tdev, node0, mat, sig, xi, kmax, out=tout,
                                                                     precision="fp32_refine"), r)}
        res[key]["fp64_steps_per_s"] = n / (res[key]["fp64_step_ms"] * 1e-3)
        res[key]["transport_steps_per_s"] = int(tout["steps"].sum().item()) / (res[key]["transport_ms"] * 1e-3)
    G.set_voxels(True)
    res["fp64_step_speedup"] = res["brute_force"]["fp64_step_ms"] / res["grids"]["fp64_step_ms"]
    res["fp64_step_nosafety_speedup"] = (res["brute_force"]["fp64_step_nosafety_ms"] /
                                         res["grids"]["fp64_step_nosafety_ms"])
    res["transport_speedup"] = res["brute_force"]["transport_ms"] / res["grids"]["transport_ms"]
    return res


def bench_serving(gv, torch, seconds=1.5):
    """Continuous batching: Poisson arrivals of navigation requests with sizes
    log-uniform in 1-65536 tracks; saturated throughput first, then p50/p99 latency at
    50%, 80% and 95% of it."""
    import time as _t
    geo = W.nested_geometry()
    G = gv.Geometry(geo["solids"], geo["nodes"])
    srv = gv.Server(G, arena_bytes=2 << 30, max_slots=4096, streams=4, precision="fp32_refine")
    # 256 requests of log-uniform sizes, packed once into pinned host buffers and
    # submitted in turn (a buffer may be in flight twice; only timing is read here)
    sizes = W.request_sizes(256, seed=3)
    pool = []
    for k, n in enumerate(sizes):
        inp, out = gv.Server.buffers(int(n))
        tr = W.nested_tracks(int(n), seed=900 + k, geom=geo)
        for c, key in enumerate(("x", "y", "z", "dx", "dy", "dz")):
            inp[c].copy_(torch.from_numpy(tr[key]))
        pool.append((inp, out, int(n)))

    def submit(k):
        inp, out, n = pool[k % len(pool)]
        return srv.submit(inp, out), n

    # saturated: a burst of requests, all waited
    burst = 400
    t0 = _t.perf_counter()
    tickets = [submit(k) for k in range(burst)]
    for t, _ in tickets:
        srv.wait(t, 120)
    sat_rate = burst / (_t.perf_counter() - t0)
    res = {"workload": "nested detector, requests log-uniform 1-65536 tracks, Poisson arrivals",
           "saturated_requests_per_s": sat_rate,
           "saturated_tracks_per_s": sum(n for _, n in tickets) / (_t.perf_counter() - t0)}
    g = np.random.default_rng(11)
    for rho in (0.5, 0.8, 0.95):
        srv.reset_stats()
        rate = rho * sat_rate
        t_next = _t.perf_counter()
        live, k = [], burst
        t_end = t_next + seconds
        while t_next < t_end:
            now = _t.perf_counter()
            if now < t_next:
                if t_next - now > 2e-4:
                    _t.sleep((t_next - now) * 0.5)
                continue
            live.append(submit(k)[0])
            k += 1
            t_next += g.exponential(1.0 / rate)
        for t in live:
            srv.wait(t, 120)
        st = srv.stats()
        res[f"load_{rho}"] = {"offered_requests_per_s": rate, "completed": st["completed"],
                              "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
                              "launch_groups": st["launches"]}
    srv.close()
    return res


def gv_supports_fp32(gv) -> bool:
    return getattr(gv, "HAS_FP32_REFINE", False)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured (MEASURED_PEAKS.json, copy)"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "source": "fallback 6.8 TB/s"}


def bench_alu_peaks(torch, index: int, reps: int = 5):
    """Measured ALU-side peaks (probe/gvprobe.cu): binary32 and binary64 multiply-adds, an
    integer-pipe step (a funnel shift and an xor), and the warp-instruction issue rate (binary32
    multiply-adds and integer steps on separate chains), each as the best of `reps` CUDA-event
    timed launches of 8 blocks of 256 threads per SM, with the SM clock sampled meanwhile.
    Rates per clock and SM use the sampled median clock."""
    import ctypes
    from paper_1512_06637_gb300 import build
    lib = ctypes.CDLL(build.build_probe())
    props = torch.cuda.get_device_properties(index)
    sms = props.multi_processor_count
    threads, blocks = 256, sms * 8
    sink = torch.zeros(blocks, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # (name, function, iterations, operations per thread per iteration, warp instructions per op)
    probes = [("fp32_fma", lib.gvp_fma32, 4096, 16 * 8), ("fp64_fma", lib.gvp_fma64, 128, 16 * 8),
              ("alu_step", lib.gvp_alu, 2048, 16 * 8), ("issue_mix", lib.gvp_issue, 4096, 16 * 8)]
    clocks = ClockSampler(index)
    clocks.start()
    time.sleep(0.3)
    best = {}
    for name, fn, iters, per_iter in probes:
        ms = ctypes.c_float(0.0)
        times = []
        for _ in range(reps + 1):
            rc = fn(blocks, threads, iters, ctypes.c_void_p(sink.data_ptr()), stream, ctypes.byref(ms))
            if rc != 0:
                raise RuntimeError(f"probe {name} failed")
            times.append(ms.value)
        best[name] = (min(times[1:]), iters * per_iter * threads * blocks)
    ck = clocks.stop()
    mhz = ck["sm_mhz"] or ck["sm_max_mhz"] or 2070.0
    out = {"sms": sms, "sm_mhz": mhz, "clocks": ck}
    for name, (ms, ops) in best.items():
        per_s = ops / (ms * 1e-3)
        out[name] = {"ms": ms, "ops_per_s": per_s, "per_clk_per_sm": per_s / (sms * mhz * 1e6)}
    # warp instructions per clock per SM: a binary32 multiply-add is one instruction per thread,
    # so the multiply-add probe's rate / 32 is the issue rate it reached (the mixed probe shows
    # whether two pipes together get past it)
    out["issue_warp_inst_per_clk_per_sm"] = out["fp32_fma"]["per_clk_per_sm"] / 32.0
    out["fp32_flops"] = 2 * out["fp32_fma"]["ops_per_s"]
    out["fp64_flops"] = 2 * out["fp64_fma"]["ops_per_s"]
    return out


def run_batched_only(args):
    """The batched form alone (for profiling): launch shape 256 threads x 2 tracks, as many
    CTAs as fit, W warm-up and K timed graph replays, FP32 + refinement (--precision fp64:
    binary64)."""
    import torch
    import paper_1512_06637_gb300 as gv
    work = W.batched()
    n = len(work["tracks"]["x"])
    dev = {k: torch.from_numpy(v).cuda() for k, v in work["tracks"].items()}
    b = gv.Batch([gv.Solid.from_spec(sp) for sp in work["solids"]], work["offset"], work["n"], work["solid"])
    b.set_config(256, 2, 0)
    out = gv.alloc_results(n, "cuda")
    prec = "fp64" if args.precision == "fp64" else "fp32_refine"
    for _ in range(args.warmup):
        b.run(dev, out, precision=prec)
    ms = _timed(torch, lambda: b.run(dev, out, precision=prec), max(1, args.steps))
    print(json.dumps({"form": "batched", "precision": prec, "tracks": n, "ms": ms,
                      "queries_per_s": n * N_QUERIES / (ms * 1e-3),
                      "refined": b.refined() if prec == "fp32_refine" else None}), flush=True)


def run_transport_only(args, n=1 << 17, kmax=64):
    """The transport loop alone (for profiling): nested detector, 2^17 tracks, kmax 64;
    --precision fp32_refine ranks the candidates in binary32 first (auto: binary64)."""
    import torch
    import paper_1512_06637_gb300 as gv
    geo = W.nested_geometry()
    G = gv.Geometry(geo["solids"], geo["nodes"])
    dev = {k: torch.from_numpy(v).cuda() for k, v in W.nested_tracks(n, seed=11, geom=geo).items()}
    node0 = G.locate(dev)
    m = W.transport_materials(geo)
    mat = torch.from_numpy(m["node_material"]).cuda()
    sig = torch.from_numpy(m["sigma_n"]).cuda()
    xi = torch.from_numpy(W.transport_xi(n, kmax, seed=1)).cuda()
    prec = "fp32_refine" if args.precision == "fp32_refine" else "fp64"
    out = G.transport(dev, node0, mat, sig, xi, kmax, precision=prec)
    for _ in range(args.warmup):
        G.transport(dev, node0, mat, sig, xi, kmax, out=out, precision=prec)
    ms = _timed(torch, lambda: G.transport(dev, node0, mat, sig, xi, kmax, out=out, precision=prec), max(1, args.steps))
    steps = int(out["steps"].sum().item())
    print(json.dumps({"form": "transport", "precision": prec, "tracks": n, "ms": ms,
                      "steps_per_s": steps / (ms * 1e-3)}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.form == "batched":
        run_batched_only(args)
    elif args.form == "transport":
        run_transport_only(args)
    elif args.form == "fp64":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        import paper_1512_06637_gb300 as gv
        from paper_1512_06637_gb300 import build
        build.build()
        alu = bench_alu_peaks(torch, torch.cuda.current_device())
        res = bench_fp64_m2(gv, torch, load_peaks(), alu, reps=max(1, args.steps))
        print(json.dumps({"form": "fp64", **res}), flush=True)
    elif args.form == "peaks":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        from paper_1512_06637_gb300 import build
        build.build()
        print(json.dumps({"form": "peaks", **bench_alu_peaks(torch, torch.cuda.current_device())}), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

"""Benchmark of the DG-SWEM hot path on one GB300 (or N independent replicas under torchrun).

Headline: element-stage updates/s of the FP64 form on the 199,712-element shelf workload
(100 km x 50 km, 316x316 cells split by seeded diagonals, jittered, M2 tide on x = 0, wetting/
drying with h0 = 0.01 m, quadratic friction, slope limiter; synthetic data).  One benchmark step
= one SSP-RK2 time step (two stages) over the whole mesh.  The working set (~60 MB) is smaller
than L2, so a 256 MB buffer is written between timed steps (outside the timed region).

Also reported on one GPU: the FP32-mixed form at p = 1 and p = 2 on the same mesh, the FP64 form
on the 3.2M-element storm domain, and the batched storm ensemble (64 scenarios on 4 meshes).

--impl reference times the CPU oracle (tests' reference implementation, plain C, OpenMP build
on all host cores) on the same workload and metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "element-stage updates/s (FP64, 199,712-element shelf)"
UNIT = "element-stage updates/s"
NE_SHELF = 199712
L2_FLUSH_BYTES = 256 << 20


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# FP64 arithmetic peak from unit counts and clocks: 152 SMs x 2 FP64 FMA lanes/clock/SM x 2 flop x
# 2.07 GHz (consistent with GB300's 1.25 TFLOP/s nominal dense FP64).
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070


class ClockSampler:
    """nvidia-smi clocks / throttle reasons, sampled every 200 ms while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) > 8 for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def kernel_source_sha():
    """Hash of the device code and of what shapes its data (kernel sources and instantiations,
    the structs passed to kernels, the mesh preprocessing that builds tables and tile lists)."""
    h = hashlib.sha256()
    for f in ("kernels.cuh", "kernels_f64.cu", "kernels_f32.cu", "common_kernels.cu", "internal.h", "mesh.cu"):
        h.update(open(os.path.join(ROOT, "paper_2508_21208_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, form: str, elements: int, variant, p: int = 1, scale: bool = False):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the current kernels
    (same kernel, form, variant and degree p) and on a mesh of the same size; with scale, on any
    mesh, scaled per element (the ensemble: its capture is a smaller batch of the same meshes)."""
    path = os.path.join(ROOT, "profiles", "traffic_per_launch.txt")
    if not os.path.exists(path):
        return None
    sha = kernel_source_sha()
    for line in open(path):
        kv = dict(re.findall(r"(\w+)=(\S+)", line))
        if (kv.get("kernel") == kernel and kv.get("form") == form and kv.get("src_sha") == sha
                and kv.get("variant") in ("*", str(variant)) and kv.get("p", "1") == str(p)
                and (scale or int(kv["elements"]) == elements)):
            return float(kv["bytes"]) / float(kv["elements"]) * elements
    return None


# ---------------------------------------------------------------- algorithmic cost per element-stage
# Bytes the method must move per element-stage (neighbour traces assumed to come from L2):
# state u^s read (9 x 8), u^n read on stage 2 (9 x 8 / 2), u^(s+1) written (9 x 8), element
# statics (inverse Jacobian + det J + 3 vertex depths; 3 neighbour ids, 1 byte of local edges,
# 1 wet/dry flag) and the edge statics x 1.5 edges per element (normal, length, 2 element ids,
# 2 local ids).  FP64: 72 + 36 + 72 + 64 + 14 + 51 = 309 B.  Mixed: statics in float:
# 72 + 36 + 72 + 32 + 14 + 33 = 259 B.  p = 2 adds 3 x 3 modes: FP64 453 B, mixed 403 B.
ALG_BYTES = {("fp64", 1): 309, ("mixed", 1): 259, ("fp64", 2): 453, ("mixed", 2): 403}
# FP64 flops per element-stage of the element-update kernel, counting each add, multiply, divide
# and square root as one flop and an FMA as two (the paper's convention, Sec. 6.2), for the split
# variant at p = 1: area integrals 6 points x 46 + 40, 3 local edges x (2 points x 18 + 12) and
# update 9 x 6 (the edge kernel's share is counted on the edge kernel: 2 points x 86 per edge).
ALG_FLOPS_ELEMENT_P1 = 6 * 46 + 40 + 3 * (2 * 18 + 12) + 9 * 6
ALG_FLOPS_EDGE_P1 = 2 * 86


def aggregate(seconds, units, dist=None, device="cpu"):
    """Replica aggregation: the job's time is the slowest rank's, its work the sum over ranks."""
    if dist is None:
        return seconds, units
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())


def make_model(case, stream, **kw):
    from paper_2508_21208_gb300 import Model
    return Model(case.mesh, case.bathy, case.params, init_nodal=case.init_nodal, stream=stream, **kw)


KERNEL_TIMING_EVERY = 10


def kernel_timed_steps(steps):
    return (steps + KERNEL_TIMING_EVERY - 1) // KERNEL_TIMING_EVERY


def time_steps(model, steps, warmup, stream, flush, per_kernel=False, dist=None):
    """Per-step CUDA-event timing on the library's stream, L2 flushed between steps.

    With per_kernel, every KERNEL_TIMING_EVERY-th timed step replays the graph variant with
    event-record nodes between its kernels, whose per-kernel durations are collected; the
    other steps replay the plain graph (the event nodes lengthen a step by a few microseconds)."""
    import torch
    for _ in range(warmup):
        model.step(1)
    model.sync()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    kt = {}
    if per_kernel:  # capture both graphs before the timed region
        model.set_kernel_timing(True)
        model.set_kernel_timing(False)
    torch.cuda.synchronize()
    if dist:  # every rank starts its timed steps together
        dist.barrier()
    torch.cuda.synchronize()
    torch.cuda.profiler.start()  # an ncu run with --profile-from-start off sees only these steps
    for i in range(steps):
        timed = per_kernel and i % KERNEL_TIMING_EVERY == 0
        if per_kernel:
            model.set_kernel_timing(timed)
        with torch.cuda.stream(stream):
            flush.zero_()
        ev[i][0].record(stream)
        model.step(1)
        ev[i][1].record(stream)
        if timed:
            stream.synchronize()
            for name, ms in model.kernel_times():
                kt.setdefault(name, []).append(ms)
    stream.synchronize()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.profiler.stop()
    model.sync()
    ms = [a.elapsed_time(b) for a, b in ev]
    return ms, kt


def run_form(case, steps, warmup, stream, flush, per_kernel=True, dist=None, **kw):
    m = make_model(case, stream, **kw)
    if per_kernel:
        m.set_kernel_timing(True)
    ms, kt = time_steps(m, steps, warmup, stream, flush, per_kernel, dist)
    kps, variant, block = m.graph_info()
    return m, ms, kt, (kps, variant, block)


def run_stats(ms, units_per_step, runs=5):
    """The timed steps split into `runs` consecutive runs of equal length: each run's rate, their
    median and spread (the value reported stays the whole timed region's)."""
    k = len(ms) // runs
    if k < 1:
        return None
    rates = [units_per_step * k / (sum(ms[i * k:(i + 1) * k]) * 1e-3) for i in range(runs)]
    return {"runs": runs, "steps_per_run": k, "rates": rates, "median": statistics.median(rates),
            "min": min(rates), "max": max(rates)}


def hbm_roofline(name, kt, steps, bytes_per_elem_stage, elements, hbm, hbm_kind, traffic=None):
    """Roofline of an HBM-bound kernel: algorithmic bytes of one launch (bytes per element-stage x
    elements) over its average CUDA-event duration, against the measured copy bandwidth."""
    avg_s = statistics.mean(kt[name]) * 1e-3
    ach = bytes_per_elem_stage * elements / avg_s / 1e9
    tot = {k: sum(v) for k, v in kt.items()}
    return {"kernel": name, "bound": "hbm", "unit": "GB/s", "achieved": ach, "peak": hbm,
            "peak_kind": hbm_kind, "frac": ach / hbm, "traffic": traffic, "avg_launch_ms": avg_s * 1e3,
            "launches_per_step": len(kt[name]) // kernel_timed_steps(steps),
            "share_of_step": tot[name] / sum(tot.values())}


def alu_roofline(name, kt, steps, variant, elements, traffic=None):
    """Roofline of an FP64-pipe-bound element kernel (algorithmic flops, Sec. 6.2 counting)."""
    avg_s = statistics.mean(kt[name]) * 1e-3
    if name == "element_update" and variant == 1:
        flops = ALG_FLOPS_ELEMENT_P1 * elements
    elif name == "element_update":
        # fused and tiled variants evaluate the edge fluxes inside the element kernel
        flops = (ALG_FLOPS_ELEMENT_P1 + 1.5 * ALG_FLOPS_EDGE_P1) * elements
    elif name == "edge_flux":
        flops = ALG_FLOPS_EDGE_P1 * 1.5 * elements
    else:
        flops = None
    tot = {k: sum(v) for k, v in kt.items()}
    ach = flops / avg_s / 1e9 if flops else None
    return {"kernel": name, "bound": "alu", "unit": "GFLOP/s", "achieved": ach, "peak": FP64_PEAK_GFLOPS,
            "peak_kind": "derived from unit counts and clocks (FP64); the FMA probe measured 1,054 GFLOP/s",
            "frac": ach / FP64_PEAK_GFLOPS if ach else None, "traffic": traffic, "avg_launch_ms": avg_s * 1e3,
            "launches_per_step": len(kt[name]) // kernel_timed_steps(steps),
            "share_of_step": tot[name] / sum(tot.values())}


def dominant(kt):
    tot = {k: sum(v) for k, v in kt.items()}
    name = max(tot, key=tot.get)
    return name, statistics.mean(kt[name]) * 1e-3, tot


def cpu_baseline(case, budget_s=12.0):
    """The oracle as it stands (OpenMP build, all host cores), a bounded number of steps."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    o = oracle.Oracle(case.mesh, case.bathy, case.params, init_nodal=case.init_nodal, omp=True)
    o.step(1)
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s and n < 400:
        o.step(1)
        n += 1
    el = time.perf_counter() - t0
    out = {"value": case.mesh.n_elems * 2 * n / el, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{n} SSP-RK2 steps of the full 199,712-element shelf workload ({el:.1f} s, OpenMP build)"}
    # the plain single-thread build of the same source, on a shorter sample
    o1 = oracle.Oracle(case.mesh, case.bathy, case.params, init_nodal=case.init_nodal, omp=False)
    n1, t1 = 0, time.perf_counter()
    while time.perf_counter() - t1 < budget_s / 3 and n1 < 100:
        o1.step(1)
        n1 += 1
    el1 = time.perf_counter() - t1
    out["single_thread"] = {"value": case.mesh.n_elems * 2 * n1 / el1, "unit": UNIT, "cores": 1,
                            "sample": f"{n1} steps of the same workload ({el1:.1f} s, serial build)"}
    out["other_workloads"] = oracle_other_workloads()
    return out


def oracle_other_workloads(budget_s=2.5):
    """The OpenMP oracle on the other workloads, a bounded number of steps each (at least one)."""
    import oracle
    from paper_2508_21208_gb300 import synth
    cases = [("800-triangle basin (Manning)", synth.config1()),
             ("storm 3,200,450 elements (FP64, hurricane, Coriolis)", synth.config3())]
    meshes, bathys, members = synth.ensemble(members_per_mesh=1, precision=synth.FP64)
    for mi, (mesh, hb) in enumerate(zip(meshes, bathys)):
        cases.append((f"ensemble mesh {mesh.n_elems} elements (one storm)",
                      synth.Case("ens", mesh, hb, np.zeros((3, mesh.n_nodes)), members[mi][1], 1)))
    res = {}
    for name, c in cases:
        o = oracle.Oracle(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal, omp=True)
        n, t0 = 0, time.perf_counter()
        while n == 0 or (time.perf_counter() - t0 < budget_s and n < 200):
            o.step(1)
            n += 1
        el = time.perf_counter() - t0
        res[name] = {"value": c.mesh.n_elems * 2 * n / el, "unit": UNIT, "steps": n, "seconds": round(el, 2)}
        del o
    return res


def e2e(case, steps, stream):
    """Same metric through the C ABI with pinned host buffers: per step the state is copied host ->
    device (dgswem_set_state), one step runs, and the state is copied back (dgswem_get_state)."""
    import torch
    m = make_model(case, stream)
    u = m.state()
    host = [torch.from_numpy(np.ascontiguousarray(u[v])).pin_memory() for v in range(3)]
    outs = [torch.empty_like(h).pin_memory() for h in host]
    hp = [h.numpy() for h in host]
    op = [o.numpy() for o in outs]
    for _ in range(3):
        m.set_state_from(hp[0], hp[1], hp[2], 0.0)
        m.step(1)
        m.get_state_into(op[0], op[1], op[2])
    t0 = time.perf_counter()
    for _ in range(steps):
        m.set_state_from(hp[0], hp[1], hp[2], 0.0)
        m.step(1)
        m.get_state_into(op[0], op[1], op[2])
    el = time.perf_counter() - t0
    nbytes = 3 * u.shape[1] * u.shape[2] * 8
    return {"value": case.mesh.n_elems * 2 * steps / el, "unit": UNIT, "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes}


def reference_arm(args, rank):
    """--impl reference: the CPU oracle on the same workload, K timed steps after W warm-up."""
    if rank != 0:
        return
    import oracle
    from paper_2508_21208_gb300 import synth
    case = synth.config2()
    cores = len(os.sched_getaffinity(0))
    o = oracle.Oracle(case.mesh, case.bathy, case.params, init_nodal=case.init_nodal, omp=True)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    el = time.perf_counter() - t0
    v = NE_SHELF * 2 * args.steps / el
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "shelf-199712 (316x316 cells, tide, wet/dry, limiter, FP64, p=1)",
                       "global_batch": NE_SHELF, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} SSP-RK2 steps of the full workload, OpenMP build"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--profile", choices=["storm", "storm-mixed", "shelf", "shelf-mixed", "shelf-mixed-p2",
                                          "ensemble-small"],
                    help="run 3 steps of one workload in a fixed launch configuration (for ncu)")
    ap.add_argument("--variant", type=int, default=1, help="with --profile: 1 split, 2 fused, 3 tiled")
    ap.add_argument("--block", type=int, default=64, help="with --profile: threads per block / tile size")
    ap.add_argument("--profile-steps", type=int, default=3, help="with --profile: steps to run")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank)

    import torch
    from paper_2508_21208_gb300 import synth
    from paper_2508_21208_gb300.build import build_library
    build_library()
    torch.cuda.set_device(local)
    if args.profile == "ensemble-small":
        # 8 storms on the 199,712- and 399,618-element meshes (~2.4M elements per stage)
        from paper_2508_21208_gb300 import Ensemble
        meshes, bathys, members = synth.ensemble(members_per_mesh=4, mesh_n=(316, 447))
        mode = 2 if args.variant == 2 else 1  # --variant 2: one launch per phase, else persistent
        ens = Ensemble(meshes, bathys, members, block=args.block, mode=mode, stream=torch.cuda.Stream())
        ens.step(3)
        ens.sync()
        print(json.dumps({"profile": args.profile, "members": len(members), "steps": 3, "mode": mode}))
        return
    if args.profile:
        mixed = synth.FP32_MIXED if "mixed" in args.profile else synth.FP64
        p = 2 if args.profile.endswith("p2") else 1
        case = synth.config3(precision=mixed) if args.profile.startswith("storm") else synth.config2(p=p, precision=mixed)
        m = make_model(case, torch.cuda.Stream(), variant=args.variant, block=args.block)
        m.step(args.profile_steps)
        m.sync()
        print(json.dumps({"profile": args.profile, "elements": case.mesh.n_elems, "steps": args.profile_steps,
                          "variant": args.variant, "block": args.block}))
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    case = synth.config2()
    with ClockSampler(local) as clk:
        model, ms, kt, (kps, variant, block) = run_form(case, args.steps, args.warmup, stream, flush, dist=dist)
    total_s, units = aggregate(sum(ms) * 1e-3, case.mesh.n_elems * 2 * args.steps, dist, "cuda")
    value = units / total_s
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    hbm, hbm_kind = peaks()
    name, avg_s, tot = dominant(kt)
    ne = case.mesh.n_elems
    roof = alu_roofline(name, kt, args.steps, variant, ne, recorded_traffic(name, "fp64", ne, variant))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "shelf-199712 (316x316 cells, tide, wet/dry, limiter, FP64, p=1)",
                       "global_batch": ne * world, "parallelism": f"replicas x{world}",
                       "l2": "256 MB buffer written between timed steps", "variant": variant,
                       "block": block, "autotune_ms_per_step": model.tune_log()},
            "gpu_launches": kps * args.steps,
            "hbm_gbs_algorithmic": ALG_BYTES[("fp64", 1)] * value / world / 1e9,
            "hbm_peak_gbs": hbm, "hbm_peak_kind": hbm_kind,
            "roofline": roof,
            "runs": run_stats(ms, case.mesh.n_elems * 2),
            "kernel_ms_per_step": {k: sum(v) / kernel_timed_steps(args.steps) for k, v in kt.items()},
            "clocks": clk.summary()}
    if world == 1:
        line["e2e"] = e2e(case, max(10, args.steps // 4), stream)
        if not args.no_extras:
            line["forms"] = extras(stream, flush, hbm)
        line["cpu_baseline"] = cpu_baseline(case)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def extras(stream, flush, hbm):
    """FP32-mixed (p = 1, 2), FP64 on the 3.2M-element storm domain; 20 timed steps each."""
    from paper_2508_21208_gb300 import synth
    out = {}
    for key, case, form, p in (("fp32_mixed_p1", synth.config2(precision=synth.FP32_MIXED), "mixed", 1),
                               ("fp32_mixed_p2", synth.config2(p=2, precision=synth.FP32_MIXED), "mixed", 2),
                               ("fp64_storm_3.2M", synth.config3(), "fp64", 1),
                               ("fp32_mixed_storm_3.2M", synth.config3(precision=synth.FP32_MIXED), "mixed", 1)):
        steps = 20
        m, ms, kt, (kps, variant, block) = run_form(case, steps, 3, stream, flush)
        ne = case.mesh.n_elems
        rate = ne * 2 * steps / (sum(ms) * 1e-3)
        name, avg_s, tot = dominant(kt)
        gbs = ALG_BYTES[(form, p)] * rate / 1e9
        hbm_kind = peaks()[1]
        if form == "fp64":
            roof = alu_roofline(name, kt, steps, variant, ne, recorded_traffic(name, form, ne, variant, p))
        else:
            roof = hbm_roofline("element_update", kt, steps, ALG_BYTES[(form, p)], ne, hbm, hbm_kind,
                                recorded_traffic("element_update", form, ne, variant, p))
        out[key] = {"value": rate, "unit": UNIT, "elements": ne, "ms_per_step": sum(ms) / steps,
                    "variant": variant, "block": block, "hbm_gbs_algorithmic": gbs, "hbm_frac": gbs / hbm,
                    "dominant_kernel": name, "roofline": roof, "runs": run_stats(ms, ne * 2),
                    "kernel_ms_per_step": {k: sum(v) / kernel_timed_steps(steps) for k, v in kt.items()}}
        del m
    out["ensemble_64_storms"] = ensemble_form(stream)
    return out


def ensemble_form(stream, steps=10):
    """64 storm scenarios on 4 basin meshes (49,928 / 199,712 / 399,618 / 798,848 elements, 16 each),
    FP32-mixed, one graph replay per step; compared with 64 sequential FP64 single-model runs,
    whose time is estimated from timed FP64 steps on each mesh."""
    import torch
    from paper_2508_21208_gb300 import Ensemble, Model, synth
    meshes, bathys, members = synth.ensemble()
    ens = Ensemble(meshes, bathys, members, stream=stream)
    kps, mode, block = ens.graph_info()
    tune = ens.tune_log()
    ens.step(3)
    ens.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    run_ms = []
    for _ in range(5):  # five runs of `steps` steps; the median is reported
        e0.record(stream)
        ens.step(steps)
        e1.record(stream)
        ens.sync()
        run_ms.append(e0.elapsed_time(e1) / steps)
    ms = statistics.median(run_ms)
    units = sum(meshes[mi].n_elems for mi, _, _ in members) * 2
    # per-kernel times of one step (event nodes between the ensemble's launches)
    ens.set_kernel_timing(True)
    ens.step(1)
    ens.sync()
    kt = {}
    for name, t in ens.kernel_times():
        kt.setdefault(name, []).append(t)
    ens.set_kernel_timing(False)
    del ens
    seq_ms = 0.0
    per_mesh = {}
    for mi, mesh in enumerate(meshes):
        prm = dict(next(p for j, p, _ in members if j == mi))
        prm["precision"] = synth.FP64
        m = Model(mesh, bathys[mi], prm, stream=stream)
        m.step(2)
        m.sync()
        e0.record(stream)
        m.step(5)
        e1.record(stream)
        m.sync()
        t = e0.elapsed_time(e1) / 5
        per_mesh[mesh.n_elems] = t
        seq_ms += t * sum(1 for j, _, _ in members if j == mi)
        del m
    hbm, hbm_kind = peaks()
    ach = ALG_BYTES[("mixed", 1)] * units / (ms * 1e-3) / 1e9
    roof = {"kernel": "the whole ensemble step (" + ("one persistent launch" if mode == 1 else "all phase launches") + ")",
            "bound": "hbm", "unit": "GB/s", "achieved": ach, "peak": hbm, "peak_kind": hbm_kind, "frac": ach / hbm,
            "traffic": recorded_traffic("ensemble_step", "mixed", units // 2, "persistent" if mode == 1 else "phased",
                                        scale=True),
            "avg_launch_ms": ms, "launches_per_step": kps}
    return {"value": units / (ms * 1e-3), "unit": UNIT, "members": len(members),
            "elements_per_stage": units // 2, "ms_per_step": ms, "ms_per_step_runs": run_ms,
            "roofline": roof, "kernel_ms_one_step": {k: sum(v) for k, v in kt.items()},
            "mode": "persistent" if mode == 1 else "phased",
            "block": block, "gpu_launches_per_step": kps, "l2": "working set ~4 GB > L2, no flush",
            "autotune_ms_per_step": tune,
            "fp64_sequential_ms_per_step": seq_ms, "fp64_single_ms_per_step_by_mesh": per_mesh,
            "speedup_vs_64_sequential_fp64": seq_ms / ms,
            "hbm_gbs_algorithmic": ALG_BYTES[("mixed", 1)] * units / (ms * 1e-3) / 1e9}


if __name__ == "__main__":
    main()

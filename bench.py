"""Benchmark of the DMS hot path on GB300: grid vertices/s from a float32
field to its D0/D2 persistence pairs.

A step is one pass of the whole path over one field resident in HBM:
dms_order -> dms_gradient -> dms_critical -> dms_diagram_d0d2.  The default
workload is the 1024^3 field (sum of 256 Gaussians, sigma in [0.01, 0.1], plus
U[0, 1e-2) noise), synthetic and seeded.  Every step re-reads inputs of 4 GiB
and more, far larger than the 129 MB L2, so no flush is needed between steps.

Under torchrun (N > 1) every rank runs an independent replica of the workload
on its own GPU (the path has no exchange step); the timed region is bracketed
by barriers and the maximum time over ranks is used.

--impl reference times the CPU oracle (the plain single-threaded restatement
the tests check the GPU against) on bounded crops of the same workload.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "c3": dict(desc="1024^3 float32, 256 Gaussians (sigma U[0.01,0.1], amplitude U[-1,1]) "
                    "+ U[0,1e-2) noise", n=1024),
    "c2": dict(desc="512^3 float32, U[0,1) quantised to 256 levels", n=512),
    "c1": dict(desc="64^3 float32, 16 Gaussians (sigma U[0.05,0.2]) + U[0,1e-3) noise", n=64),
}
METRIC = "grid vertices/s to D0/D2 diagrams"


def make_field(workload: str, n: int, device, seed=0):
    from paper_2505_21266_gb300 import fields
    if workload == "c3":
        return fields.config3(seed, device, n=n)
    if workload == "c2":
        return fields.config2(seed, device, n=n)
    return fields.config1(seed, device, n=n)


def load_peaks():
    """(HBM GB/s, max SM MHz, which): the measured copy bandwidth and SM clock
    from MEASURED_PEAKS.json, else the fallback figures."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    return 6800.0, 2070.0, "fallback"


# The gradient kernel's roofline is HBM: per vertex it reads the 4-byte order
# and writes the 8-byte record and the 1-byte desc (13 B; the 4-byte critical
# mask of the plan is not written, the critical bits live in the record).  It
# is in fact bound by integer instruction issue, so the line also reports the
# issue rate it fills.  Its per-vertex counters (warp instructions, DRAM
# bytes) come from the committed ncu summary of the kernel, and are used only
# when that summary was taken on the very sources being benchmarked (the
# summary records a hash of them); otherwise they are reported as null.
GRAD_ALGO_BYTES_PER_VERTEX = 4 + 8 + 1
GRAD_PROFILE = os.path.join(ROOT, "profiles", "gradient_kernel_c3.md")
GRAD_SOURCES = [os.path.join(ROOT, "paper_2505_21266_gb300", "csrc", n)
                for n in ("dms_gradient.cu", "dms_lowerstar.cuh", "dms_star.cuh", "dms_common.cuh")]


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for p in GRAD_SOURCES:
        with open(p, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_figures():
    """The gradient kernel's per-vertex ncu figures from its committed
    summary (a line 'figures: sources=<hash> warp_inst_per_vertex=<x>
    dram_bytes_per_vertex=<y> ...'), or None when the summary is missing or
    was taken on other sources."""
    try:
        with open(GRAD_PROFILE) as fh:
            text = fh.read()
    except OSError:
        return None
    for line in text.splitlines():
        line = line.strip().strip("`")
        if line.startswith("figures:"):
            kv = dict(item.split("=", 1) for item in line[len("figures:"):].split() if "=" in item)
            if kv.get("sources") != kernel_source_hash():
                return None
            try:
                return {k: (v if k == "sources" else float(v)) for k, v in kv.items()}
            except ValueError:
                return None
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
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def host_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_baseline(field_np: np.ndarray, crop: int):
    """The oracle, as it stands, on a crop of the workload: the whole path
    with the lower stars of its gradient step spread over all host cores by
    z-slabs (the paper's shared-memory parallel shape; the order and the D0/D2
    pairing stay sequential, as in DMS), and the same path on one core; plus
    the order + gradient steps alone on one core and on all cores."""
    import oracle
    oracle.build()
    sub = np.ascontiguousarray(field_np[:crop, :crop, :crop])
    nthr = host_threads()

    def timed(**kw):
        t0 = time.perf_counter()
        oracle.run(sub, **kw)
        return time.perf_counter() - t0

    t_all = timed(threads=nthr)
    t_one = timed(threads=1)
    g_one = timed(diagrams=False, threads=1)
    g_all = timed(diagrams=False, threads=nthr)
    return {"value": sub.size / t_all, "unit": "vertices/s", "cores": nthr, "kind": "oracle",
            "sample": f"full oracle path (order, gradient on {nthr} threads by z-slabs, critical, "
                      f"D0/D2) on a {crop}^3 crop of the workload field, {t_all:.1f} s",
            "one_core": {"value": sub.size / t_one, "unit": "vertices/s", "seconds": t_one},
            "order_gradient": {"one_core": sub.size / g_one, "all_cores": sub.size / g_all,
                               "unit": "vertices/s", "threads": nthr}}


def whole_job(ms_local: float, units_local: int, steps: int, device=None):
    """Whole-job throughput of N replicas: the units all ranks processed over
    the slowest rank's time (every rank calls this; N = 1 needs no process
    group).  Returns (units per second, the max time in ms)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return units_local * steps / (ms_local / 1e3), ms_local
    t = torch.tensor([ms_local, float(units_local)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    tsum = t.clone()
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    dist.barrier()
    ms = float(tmax[0].item())
    return float(tsum[1].item()) * steps / (ms / 1e3), ms


def bench_batched(dev, steps: int, warmup: int):
    """256 fields of uneven dims (each axis U{32..256}; even fields Gaussian
    mixtures, odd fields U[0,1)), all resident in HBM: one batched launch
    replayed from a CUDA graph against the same fields run one by one
    through the single-field calls."""
    import torch
    from paper_2505_21266_gb300 import batch as B
    from paper_2505_21266_gb300 import fields
    shapes = fields.batch_shapes(256, 32, 256, seed=0)
    xs = [fields.batch_field(i, s, seed=0, device=dev) for i, s in enumerate(shapes)]
    total = int(sum(a * b * c for a, b, c in shapes))
    variant = B.autotune(shapes, dev, fields=xs)
    b = B.Batch(shapes, dev, tile_variant=variant)
    b.set_fields(xs)
    b.capture()
    for _ in range(warmup):
        b.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        b.replay()
    e1.record()
    torch.cuda.synchronize()
    b.check()
    batched_ms = e0.elapsed_time(e1) / steps
    del b
    torch.cuda.empty_cache()
    B.per_field(xs)  # warm-up
    torch.cuda.synchronize()
    e0.record()
    reps = max(1, min(steps, 2))
    for _ in range(reps):
        B.per_field(xs)
    e1.record()
    torch.cuda.synchronize()
    per_ms = e0.elapsed_time(e1) / reps
    del xs
    torch.cuda.empty_cache()
    return {"workload": "256 fields, axes U{32..256}, half Gaussian mixtures (16, sigma "
                        "U[0.05,0.2]) + U[0,1e-3), half U[0,1)",
            "fields": 256, "vertices": total, "tile_variant": variant,
            "variant": B.variant_name(variant),
            "autotune_ms": {B.variant_name(i): round(t, 2)
                            for i, t in enumerate((B.autotune.last or {}).get("ms", []))},
            "batched_ms": batched_ms, "batched_fields_per_s": 256 / (batched_ms / 1e3),
            "batched_vertices_per_s": total / (batched_ms / 1e3),
            "per_field_ms": per_ms, "per_field_fields_per_s": 256 / (per_ms / 1e3),
            "speedup": per_ms / batched_ms, "graph": True}


def bench_differentiable(dev, steps: int, warmup: int):
    """128^3 field (32 Gaussians + U[0,1e-4)): one gradient-descent step on
    the topological loss (diagram, loss, backward kernel, update) against the
    forward-only diagram of the same field."""
    import torch
    import paper_2505_21266_gb300 as dms
    from paper_2505_21266_gb300 import fields
    f0 = fields.config4(0, dev)
    x = f0.clone().requires_grad_(True)

    def gd_step():
        loss = dms.topological_loss(x, 0.05)
        loss.backward()
        with torch.no_grad():
            x.sub_(1e-2 * x.grad)
            x.grad = None
        return loss

    def fwd():
        return dms.diagram(f0)

    out = {}
    for name, fn in (("forward_ms", fwd), ("gd_step_ms", gd_step)):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            fn()
        torch.cuda.synchronize()
        out[name] = (time.perf_counter() - t0) / steps * 1e3
    out["workload"] = "128^3, 32 Gaussians (sigma U[0.05,0.2]) + U[0,1e-4); loss = sum of " \
                      "(death - birth)^2 over pairs with persistence < 0.05, lr 1e-2"
    out["gd_over_forward"] = out["gd_step_ms"] / out["forward_ms"]
    return out


def bench_2d(dev, steps: int, warmup: int, n: int = 16384):
    """The 2D path on an n x n field (64 Gaussians, sigma U[0.01,0.1], plus
    U[0,1e-2)): order, gradient, critical simplices, D0 and D1 -- the whole
    diagram of a 2D field -- in vertices/s."""
    import torch
    import paper_2505_21266_gb300 as dms
    from paper_2505_21266_gb300 import fields
    f = fields.gaussian_mixture((1, n, n), 64, (0.01, 0.1), 1e-2, 0, dev)[0].contiguous()
    for _ in range(warmup):
        r = dms.diagram2d(f)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        r = dms.diagram2d(f)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    out = {"workload": f"{n}^2 float32, 64 Gaussians (sigma U[0.01,0.1]) + U[0,1e-2)",
           "vertices": n * n, "ms_per_step": ms, "vertices_per_s": n * n / (ms / 1e3),
           "critical": [int(c.numel()) for c in r.crit],
           "pairs_d0_d1": [int(r.diagrams.d0.shape[0]), int(r.diagrams.d1.shape[0])]}
    del f, r
    torch.cuda.empty_cache()
    return out


def bench_d1(dev, steps: int, warmup: int, n: int = 256):
    """D1 (the saddle-saddle pairs, after D0/D2) on the n^3 quantised-noise
    field (256 levels): the dms_diagram_d1 call alone, with its pool sized
    on the first call, in ms and vertices/s."""
    import torch
    import paper_2505_21266_gb300 as dms
    from paper_2505_21266_gb300 import fields
    f = fields.config2(0, dev, n=n)
    r = dms.diagram(f)
    d1 = dms.diagram_d1(f, r.order, r.grad, r.crit, r.diagrams)
    for _ in range(max(0, warmup - 1)):
        d1 = dms.diagram_d1(f, r.order, r.grad, r.crit, r.diagrams)
    torch.cuda.synchronize()
    reps = max(1, min(steps, 3))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        d1 = dms.diagram_d1(f, r.order, r.grad, r.crit, r.diagrams)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    out = {"workload": f"{n}^3 float32, U[0,1) quantised to 256 levels", "vertices": n ** 3,
           "d1_ms": ms, "vertices_per_s": n ** 3 / (ms / 1e3), "pairs_d1": int(d1.shape[0]),
           "critical": [int(c.numel()) for c in r.crit],
           "pairs_d0_d2": [int(r.diagrams.d0.shape[0]), int(r.diagrams.d2.shape[0])]}
    del f, r, d1
    torch.cuda.empty_cache()
    return out


def run_reference(args):
    """--impl reference: the oracle on bounded crops of the workload field."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch
    import oracle
    from paper_2505_21266_gb300 import fields
    oracle.build()
    wl = WORKLOADS[args.workload]
    n = args.size or wl["n"]
    crop = args.crop
    # a crop of the same field, generated directly on the host
    if args.workload == "c3":
        full = fields.mixture_crop(n, crop, 256, (0.01, 0.1), 1e-2, 0).numpy()
    elif args.workload == "c2":
        full = fields.config2(0, n=crop).numpy()
    else:
        full = fields.mixture_crop(n, crop, 16, (0.05, 0.2), 1e-3, 0).numpy()
    f = np.ascontiguousarray(full, dtype=np.float32)
    nthr = host_threads()
    for _ in range(args.warmup):
        oracle.run(f, threads=nthr)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run(f, threads=nthr)
    dt = time.perf_counter() - t0
    v = f.size * args.steps / dt
    line = {"metric": METRIC, "value": v, "unit": "vertices/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": wl["desc"], "sample": f"{crop}^3 crop per step"},
            "cpu_baseline": {"value": v, "unit": "vertices/s", "cores": nthr, "kind": "oracle",
                             "sample": f"{crop}^3 crop of the workload per step, gradient "
                                       f"on {nthr} threads by z-slabs"},
            "e2e": {"value": v, "unit": "vertices/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--size", type=int, default=0, help="override the grid edge length")
    ap.add_argument("--crop", type=int, default=64, help="oracle crop edge (CPU legs)")
    ap.add_argument("--source-hash", action="store_true",
                    help="print the hash of the gradient kernel's sources and exit")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-field batch leg")
    ap.add_argument("--no-diff", action="store_true", help="skip the differentiable leg")
    ap.add_argument("--no-2d", action="store_true", help="skip the 2D leg")
    ap.add_argument("--no-pairing-cmp", action="store_true",
                    help="skip the D0/D2 pairing comparison (rounds vs self-correcting)")
    ap.add_argument("--with-d1", action="store_true",
                    help="add the D1 leg (saddle-saddle pairs, 256^3 quantised noise)")
    ap.add_argument("--leg", choices=["batched", "diff", "2d", "d1"], default=None,
                    help="run one comparison leg alone (its own JSON line), e.g. to profile it")
    args = ap.parse_args()
    if args.source_hash:
        print(kernel_source_hash())
        return
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist
    import paper_2505_21266_gb300 as dms
    from paper_2505_21266_gb300 import _lib

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = _lib.load()
    if args.leg:
        legs = {"batched": bench_batched, "diff": bench_differentiable, "2d": bench_2d,
                "d1": bench_d1}
        if args.leg == "d1" and args.size:
            out = bench_d1(dev, args.steps, args.warmup, n=args.size)
        else:
            out = legs[args.leg](dev, args.steps, args.warmup)
        print(json.dumps({"leg": args.leg, **out}), flush=True)
        return

    wl = WORKLOADS[args.workload]
    n = args.size or wl["n"]
    f = make_field(args.workload, n, dev)
    torch.cuda.synchronize()
    nvert = f.numel()
    stream = torch.cuda.current_stream(dev)

    def step(field, ev=None):
        st = torch.zeros(1, dtype=torch.int32, device=dev)
        o = dms.order(field, status=st)
        if ev is not None:
            ev[0].record(stream)
        g = dms.gradient(o)
        if ev is not None:
            ev[1].record(stream)
        c = dms.critical(g)
        d = dms.diagram_d0d2(field, o, g, c, status=st)
        return d, st, c

    def staged(field):
        """One step with a synchronisation after every stage (stderr report)."""
        st = torch.zeros(1, dtype=torch.int32, device=dev)
        marks = [time.perf_counter()]
        o = dms.order(field, status=st)
        torch.cuda.synchronize()
        marks.append(time.perf_counter())
        g = dms.gradient(o)
        torch.cuda.synchronize()
        marks.append(time.perf_counter())
        c = dms.critical(g)
        torch.cuda.synchronize()
        marks.append(time.perf_counter())
        d = dms.diagram_d0d2(field, o, g, c, status=st)
        torch.cuda.synchronize()
        marks.append(time.perf_counter())
        names = ["order", "gradient", "critical", "d0d2"]
        print("stages ms: " + ", ".join(f"{nm} {1e3 * (b - a):.2f}"
                                        for nm, a, b in zip(names, marks, marks[1:])),
              file=sys.stderr, flush=True)
        return d, st, c

    print(f"field ready: {nvert} vertices", file=sys.stderr, flush=True)
    d, st, c = staged(f)  # the first pass also sizes the capacities
    for _ in range(args.warmup - 1):
        d, st, c = staged(f)
    torch.cuda.synchronize()
    if int(st.item()) != 0:
        raise RuntimeError(f"device status {int(st.item())}")
    crit_counts = [int(x.numel()) for x in c]
    n_pairs = [int(d.d0.shape[0]), int(d.d2.shape[0])]

    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    l0 = lib.dms_launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    sev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    t_start.record(stream)
    for k in range(args.steps):
        sev[k].record(stream)
        step(f, gev[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    launches = lib.dms_launch_count() - l0
    clocks = sampler.stop()
    ms = t_start.elapsed_time(t_end)
    grad_ms = statistics.mean(a.elapsed_time(b) for a, b in gev)
    # per-stage times of the timed steps (events between the stages, no
    # synchronisation): order, gradient, and critical + D0/D2 to the next step
    ends = sev[1:] + [t_end]
    stages = {"order": statistics.mean(sev[k].elapsed_time(gev[k][0]) for k in range(args.steps)),
              "gradient": grad_ms,
              "critical_d0d2": statistics.mean(gev[k][1].elapsed_time(ends[k])
                                               for k in range(args.steps))}
    value, ms = whole_job(ms, nvert, args.steps, dev)

    # the D0/D2 stage under the two parallel forms of Alg. 1: the default
    # (spanning forest, then exact rounds) and the paper's self-correcting
    # pairing (Alg. 4) as a fixpoint, on the same gradient
    pairing_cmp = None
    if world == 1 and not args.no_pairing_cmp:
        o_ = dms.order(f)
        g_ = dms.gradient(o_)
        c_ = dms.critical(g_)
        pairing_cmp = {}
        for mode in ("rounds", "selfcorrecting"):
            dms.diagram_d0d2(f, o_, g_, c_, pairing=mode)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            reps = max(1, min(args.steps, 3))
            for _ in range(reps):
                dms.diagram_d0d2(f, o_, g_, c_, pairing=mode)
            b.record(stream)
            torch.cuda.synchronize()
            pairing_cmp[f"{mode}_ms"] = a.elapsed_time(b) / reps
        pairing_cmp["note"] = "D0/D2 stage only (walks, pairing, pair lists) on the step's gradient"
        del o_, g_, c_

    # end to end through the public API, the fields coming from pinned host
    # memory: a stream of `steps` fields through diagrams_from_host (each
    # field copied in -- overlapped with the previous field's path -- and its
    # pairs copied out); the first field's copy is inside the timed region
    e2e = None
    if not args.no_e2e:
        host = f.cpu().pin_memory()
        h2d = host.numel() * 4
        # the other legs' buffers go back to the device first; the warm-up
        # runs the same two-buffer stream, so the timed region allocates nothing
        d = st = c = None
        torch.cuda.empty_cache()
        for _ in range(2):  # the timed stream's own pattern, twice: device and
            for d0, d2, ess in dms.diagrams_from_host([host] * max(2, args.steps), dev):
                pass        # page-locked host buffers are then all cached
        d0 = d2 = ess = None
        gc.collect()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d2h = 0
        marks = []
        for d0, d2, ess in dms.diagrams_from_host([host] * args.steps, dev):
            d2h = d0.nbytes + d2.nbytes + ess.nbytes
            marks.append(time.perf_counter())
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": nvert * world * args.steps / dt, "unit": "vertices/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "overlap": "next field's host-to-device copy on a second stream; pairs copied "
                          "back on a third stream while the next field's gradient kernel runs "
                          "(a field's arrays arrive one field later)",
               "field_ms": [round(1e3 * (b - a), 1) for a, b in zip([t0] + marks, marks)]}

    hbm_peak, sm_mhz, peak_kind = load_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    issue_peak = sms * 4 * 32 * sm_mhz * 1e6 / 1e12  # lane-instructions/s, in T
    grad_bytes = GRAD_ALGO_BYTES_PER_VERTEX * nvert
    grad_gbs = grad_bytes / (grad_ms / 1e3) / 1e9
    fig = profile_figures() if args.workload == "c3" else None
    issue = None
    if fig and "warp_inst_per_vertex" in fig:
        ach = fig["warp_inst_per_vertex"] * 32 * nvert / (grad_ms / 1e3) / 1e12
        issue = {"achieved": ach, "peak": issue_peak, "unit": "Tinst/s (lane-instructions)",
                 "frac": ach / issue_peak, "warp_inst_per_vertex": fig["warp_inst_per_vertex"],
                 "peak_kind": f"derived: {sms} SMs x 4 schedulers x 32 lanes x {sm_mhz:.0f} MHz"}
    line = {
        "metric": METRIC, "value": value, "unit": "vertices/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": wl["desc"], "n": n, "vertices": nvert,
                   "l2": "inputs (4 GiB field, 4 GiB order) larger than L2, no flush",
                   "critical": crit_counts, "pairs_d0_d2": n_pairs,
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "kernel": "gradient_kernel", "achieved": grad_gbs,
                     "peak": hbm_peak, "unit": "GB/s", "frac": grad_gbs / hbm_peak,
                     "peak_kind": peak_kind,
                     "algorithmic_bytes_per_vertex": GRAD_ALGO_BYTES_PER_VERTEX,
                     "kernel_ms": grad_ms,
                     # DRAM bytes per vertex of the committed ncu summary of
                     # these very sources, scaled to this launch (null if none)
                     "traffic": fig["dram_bytes_per_vertex"] * nvert
                     if fig and "dram_bytes_per_vertex" in fig else None,
                     "figures_from": os.path.relpath(GRAD_PROFILE, ROOT) if fig else None,
                     "sources": kernel_source_hash(),
                     "issue": issue},
        "stages_ms": stages,
        # the same steps without the order stage (a user that already holds
        # the order, or compares (key, vertex) pairs directly)
        "excluding_order": {"ms_per_step": ms / args.steps - stages["order"],
                            "value": nvert * world / ((ms / args.steps - stages["order"]) / 1e3),
                            "unit": "vertices/s"},
        "d0d2_pairing": pairing_cmp,
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": e2e,
    }
    # the CPU baseline and the single-GPU comparison legs belong to the N = 1 line
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(f.cpu().numpy(), args.crop)
    del f, d, c
    torch.cuda.empty_cache()
    if world == 1 and not args.no_batched:
        line["batched"] = bench_batched(dev, args.steps, args.warmup)
    if world == 1 and not args.no_diff:
        line["differentiable"] = bench_differentiable(dev, args.steps, args.warmup)
    if world == 1 and not args.no_2d:
        line["grid_2d"] = bench_2d(dev, args.steps, args.warmup)
    if world == 1 and args.with_d1:
        line["d1"] = bench_d1(dev, args.steps, args.warmup)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

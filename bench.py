"""Benchmark of the PW advection hot path on B300.

One STEP = one pass of the per-timestep hot path over the 1024 x 1024 x 128
synthetic domain (dx = dy = 25 m, stretched dz, anelastic density): periodic
halo fill of u, v, w followed by the PW stencil u, v, w -> su, sv, sw in FP64
(the paper's offloaded advection component, sections 2.1 and 3).  The headline
`value` is advected grid points per second with inputs resident in HBM; `e2e`
is the same metric through the public API with pinned host buffers (host to
device copy of u, v, w and device to host copy of su, sv, sw inside every
step).  Extra objects measure the FP32 and BF16 storage variants on the same
domain, the native-FP64 kernel, the FP64 conservation reductions, the batched
ensemble and the adjoint loop.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the workload
(weak scaling, no data-path collective); rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import os
import platform
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2009_12850_b300 import synthetic  # noqa: E402

WL = synthetic.LARGE   # replaced by --nx/--ny/--nz for profiling captures of a smaller case
METRIC = "advected grid points/s (u,v,w) & % HBM roofline; FP32 vs FP64 at stated error"
UNIT = "points/s"
BYTES_PER_POINT = {"f64": 48, "f32": 24, "bf16": 18, "bf16_out": 12}   # compulsory: read u,v,w + write su,sv,sw
PEAKS_FALLBACK = {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def kernel_source_hash(sources):
    """Hash of the code of the files that define one kernel and its launch
    (paths relative to the repository root); comments and white space do not
    count, so documentation edits keep a recorded measurement valid."""
    import re
    h = hashlib.sha256()
    for name in sources:
        text = open(os.path.join(ROOT, name)).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_key):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, or None when that kernel's sources changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(kernel_key)
    if not d or d.get("source_hash") != kernel_source_hash(d.get("sources", [])):
        return None
    return d.get("bytes_per_launch")


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        smax = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[4 + q].lower().startswith("active")})
        power = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(power) if power else None}


# ----------------------------------------------------------------------------
# the GPU arm
# ----------------------------------------------------------------------------
def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """Largest value over ranks (the slowest rank's time)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(points_per_rank, world, steps, seconds):
    """Weak scaling: every rank advects its own replica; the job's rate is all
    ranks' points over the slowest rank's time."""
    return world * points_per_rank * steps / seconds


def world_size():
    return int(os.environ.get("WORLD_SIZE", "1"))


def spin_up(fn, seconds=0.3):
    """Run fn until `seconds` of device work have passed, so that a short timed
    region does not start on a GPU whose clocks dropped while the host was
    preparing inputs."""
    import torch
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        fn()
        torch.cuda.synchronize()


def time_steps(step, steps, warmup, world, events_for=None):
    """W untimed steps, then exactly K timed steps between barriers and
    synchronisations; returns (total seconds of the slowest rank, per-launch ms
    of the kernel recorded by step())."""
    import torch
    spin_up(lambda: step(None), 0.25)  # clocks at their working level first
    for _ in range(warmup):
        step(None)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    rec = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step(rec)
    e1.record()
    torch.cuda.synchronize()
    barrier(world)
    total = e0.elapsed_time(e1) / 1e3
    kern = [a.elapsed_time(b) for a, b in rec]
    return max_over_ranks(total, world), (float(np.mean(kern)) if kern else None)


def run_gpu(args):
    import torch
    from paper_2009_12850_b300 import api

    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    peaks, peaks_kind = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    nx, ny, nz = WL.nx, WL.ny, WL.nz
    pts = WL.points
    u, v, w = synthetic.fields_for(WL)

    def build(dtype, algo="auto"):
        m = api.Mesh(nx, ny, nz, WL.dx, WL.dy, dtype=dtype, algo=algo, device=dev)
        U = [m.from_interior(a) for a in (u, v, w)]
        S = [m.empty_out() for _ in range(3)]
        return m, U, S

    def make_step(m, U, S):
        stream = torch.cuda.current_stream()

        def step(rec):
            m.halo(*U, stream=stream)
            if rec is None:
                m.advect(*U, *S, stream=stream)
            else:
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                m.advect(*U, *S, stream=stream)
                b.record(stream)
                rec.append((a, b))
        return step

    # ---------------- headline: FP64 on the device ----------------
    hd = args.dtype
    m64, U64, S64 = build(hd, args.algo)
    with ClockSampler(local) as clk:
        total, kern_ms = time_steps(make_step(m64, U64, S64), args.steps, args.warmup, world)
    clocks = clk.summary()
    assert m64.device_status() == 0, "device wait timed out"
    value = whole_job_rate(pts, world, args.steps, total)
    achieved = BYTES_PER_POINT[hd] * pts / (kern_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "traffic": recorded_traffic(f"pw_advect_{hd}_{args.algo}"),
            "kernel": f"pw_advect ({hd}, {args.algo})", "kernel_ms": round(kern_ms, 4),
            "algorithmic_bytes_per_point": BYTES_PER_POINT[hd], "points_per_launch": pts,
            "peak_kind": f"{peaks_kind} copy bandwidth"}
    s64 = [m64.interior(s) for s in S64]

    extras = {}
    rows = None if args.extras is None else set(args.extras.split(","))

    # extra rows run on single-GPU runs only: a multi-GPU run measures the
    # replicated headline step and its e2e
    def want(name):
        return not args.no_extras and hd == "f64" and world == 1 and (rows is None or name in rows)

    if not args.no_extras and hd == "f64" and world == 1:
        for dtype, algo_name in (("f32", "auto"), ("bf16", "auto"), ("bf16_out", "auto"), ("f64", "native")):
            key = dtype if algo_name == "auto" else "f64_native"
            if not want(key):
                continue
            m, U, S = build(dtype, algo_name)
            tot, kms = time_steps(make_step(m, U, S), max(3, args.steps // 2), 3, world)
            bpp = BYTES_PER_POINT[dtype]
            err = {}
            for q, nm in enumerate(("su", "sv", "sw")):
                ref = s64[q]
                d = (m.interior(S[q]).double() - ref).abs()
                err[nm] = {"max_abs": float(d.max()), "rms": float(d.pow(2).mean().sqrt()),
                           "rel_to_max": float(d.max() / ref.abs().max())}
            extras[key] = {"value": world * pts * max(3, args.steps // 2) / tot, "unit": UNIT,
                           "kernel_ms": round(kms, 4),
                           "hbm_frac": round(bpp * pts / (kms * 1e-3) / 1e9 / hbm, 4),
                           "bytes_per_point": bpp, "error_vs_f64_path": err}
            if key == "f32":
                extras[key]["speedup_vs_f64"] = round(extras[key]["value"] / value, 3)
            if key == "f64_native":
                extras[key]["dp_ops_per_point_est"] = 42
            del m, U, S
            torch.cuda.empty_cache()
    if want("residuals"):
        # conservation reductions (A5) on the FP64 fields: each call ends with the
        # 12 sums on the host, so a call is timed on the host clock (after two
        # untimed calls: the first one also loads the kernels); the device time
        # of the same calls (both passes and the copy of the sums) beside it
        for _ in range(2):
            m64.residual_sums(*U64, *S64)
        torch.cuda.synchronize()
        nres = 10
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        t0 = time.perf_counter()
        ev[0].record()
        for _ in range(nres):
            sums = m64.residual_sums(*U64, *S64)
        ev[1].record()
        dt = (time.perf_counter() - t0) / nres
        torch.cuda.synchronize()
        re, rm = m64.residuals(*U64, *S64)
        extras["residuals"] = {"ms_per_call": round(dt * 1e3, 3),
                               "device_ms_per_call": round(ev[0].elapsed_time(ev[1]) / nres, 3),
                               "R_E": list(re), "R_M": list(rm)}

    for name, fn in (("small_latency", lambda: bench_small_latency(args, world)),
                     ("scalars", lambda: bench_scalars(args, world, hbm)),
                     ("tvd", lambda: bench_tvd(args, world, hbm)),
                     ("paper_strong_f32", lambda: bench_paper_strong(args, world, hbm)),
                     ("fused_step", lambda: bench_fused_step(args, world, hbm)),
                     ("batched", lambda: bench_batched(args, world, hbm)),
                     ("adjoint_loop", lambda: bench_adjoint_loop(args)),
                     ("adjoint_kernel", lambda: bench_adjoint_kernel(args)),
                     ("precision", bench_precision)):
        if want(name):
            extras[name] = fn()
            torch.cuda.empty_cache()

    # ---------------- e2e: host arrays through the C-ABI (pw_advect_host) ----
    # pinned host arrays in, sources back in host arrays; the copies of each
    # x-slab overlap the halo fill and stencil of its neighbours
    pipe = api.Pipeline(m64)
    host_in = [pipe.empty_host() for _ in range(3)]
    host_out = [pipe.empty_host(out=True) for _ in range(3)]
    for h, a in zip(host_in, (u, v, w)):
        h[2:nx + 2, 2:ny + 2, :nz] = torch.from_numpy(a).to(h.dtype)
    stream = torch.cuda.current_stream()

    def e2e_step(rec):
        pipe.advect_host(*host_in, *host_out, stream=stream)

    e2e_steps = max(3, args.steps // 4)
    e2e_total, _ = time_steps(e2e_step, e2e_steps, 2, world)
    assert m64.device_status() == 0
    row_in = ny * m64.nzp * host_in[0].element_size()
    row_out = ny * m64.nzp * host_out[0].element_size()
    cols_in = nx + (1 if pipe.nslab > 1 else 0)   # column nx-1 travels first, once more
    e2e = {"value": world * pts * e2e_steps / e2e_total, "unit": UNIT,
           "h2d_bytes_per_step": 3 * cols_in * row_in, "d2h_bytes_per_step": 3 * nx * row_out,
           "api": "pw_advect_host (pinned host arrays, x-slabs of %d columns, %d slabs)" % (pipe.slab, pipe.nslab)}
    err = max(float((host_out[q][2:nx + 2, 2:ny + 2, :nz].to(s64[q].device) - s64[q]).abs().max()) for q in range(3))
    e2e["max_abs_diff_vs_device_path"] = err
    del pipe, host_in, host_out
    if want("e2e_theta_5q"):
        extras["e2e_theta_5q"] = bench_host_scalars(args, world)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": hd, "data": "synthetic",
        "config": {"workload": WL.name, "algo": args.algo, "nx": nx, "ny": ny, "nz": nz, "dx": WL.dx,
                   "fields": "u,v = 5 + N(0,1) m/s; w = N(0,0.3) m/s, lid 0; dz 10->40 m geometric; "
                             "rho = 1.2 exp(-z/8000)",
                   "step": f"halo fill of u,v,w + PW stencil -> su,sv,sw ({hd}, beta=0)",
                   "l2": "inputs larger than L2 (6.5 GB of fields per step vs 126 MB)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": 2 * args.steps,
        "clocks": clocks,
        "extras": extras,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        pv = precision_vs_oracle()
        if pv is not None and "precision" in extras:
            extras["precision"]["error_vs_oracle"] = pv
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


# ----------------------------------------------------------------------------
# extra rows: batched ensemble, adjoint loop, precision study
# ----------------------------------------------------------------------------
def bench_batched(args, world, hbm):
    """64 uneven FP32 subdomains in one persistent launch: autotuned tile shape,
    halo fill + advect captured in a CUDA graph, replayed K times."""
    import tempfile as tf

    import torch
    from paper_2009_12850_b300 import api
    members = synthetic.ensemble(64)
    meshes, fields, sources, pts = [], [], [], 0
    for mb in members:
        m = api.Mesh(mb.nx, mb.ny, mb.nz, mb.dx, mb.dx, dtype="f32")
        f = synthetic.wind_fields(mb.nx, mb.ny, mb.nz, mb.seed)
        meshes.append(m)
        fields.append([m.from_interior(a) for a in f])
        sources.append([m.empty_out() for _ in range(3)])
        pts += mb.nx * mb.ny * mb.nz
    b = api.Batch(meshes)
    b.bind(fields, sources)
    if args.batch_tune:  # a kept cache: a second run reuses the first run's choice
        tune_ms = b.autotune(args.batch_tune)
    else:
        with tf.TemporaryDirectory() as d:
            tune_ms = b.autotune(os.path.join(d, "tune.txt"))
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        b.halo(stream=side)
        b.advect(stream=side)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.halo()
        b.advect()
    steps = max(5, args.steps)
    total, _ = time_steps(lambda rec: graph.replay(), steps, 3, world)
    assert b.status() == 0
    # the same work as one launch per member (no batching, no graph)
    def loop_step(rec):
        for m, f, s in zip(meshes, fields, sources):
            m.halo(*f)
            m.advect(*f, *s)
    loop_total, _ = time_steps(loop_step, max(3, steps // 2), 2, world)
    per = total / steps
    per_loop = loop_total / max(3, steps // 2)
    return {"workload": "64 members, nx,ny in 32..384 (x8), nz in 64..160, dx in 25..100 m, FP32",
            "points_per_step": pts, "value": world * pts / per, "unit": UNIT, "ms_per_step": round(per * 1e3, 4),
            "hbm_frac": round(24 * pts / per / 1e9 / hbm, 4), "autotune_ms": round(tune_ms, 4),
            "per_member_launch_ms_per_step": round(per_loop * 1e3, 4),
            "speedup_vs_per_member_launches": round(per_loop / per, 3),
            "gpu_launches_per_step": 3}


SCALAR_BYTES = {"f64": (8, 8), "f32": (4, 4), "bf16": (2, 4)}


def bench_scalars(args, world, hbm):
    """theta + 5 moisture fields (the paper's tank experiment advects five q
    fields) on 1024 x 1024 x 128, advected by the same wind in one launch per
    step; every storage type.  Rate = scalar values produced per second."""
    import torch
    from paper_2009_12850_b300 import api
    wl, n = WL, 6
    wind = synthetic.fields_for(wl)
    phis = synthetic.scalar_fields(wl.nx, wl.ny, wl.nz, n, wl.seed + 100)
    pts = wl.points
    out = {"workload": f"{wl.name}, theta + 5 q", "scalars": n}
    for dtype, algo in (("f64", "auto"), ("f64", "native"), ("f32", "auto"), ("bf16", "auto")):
        m = api.Mesh(wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, dtype=dtype, algo=algo)
        U = [m.from_interior(a) for a in wind]
        P = [m.from_interior(a) for a in phis]
        S = [m.empty_out() for _ in range(n)]
        stream = torch.cuda.current_stream()

        def step(rec):
            if rec is None:
                m.advect_scalars(*U, P, S, stream=stream)
                return
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            m.advect_scalars(*U, P, S, stream=stream)
            b.record(stream)
            rec.append((a, b))
        steps = max(3, args.steps // 2)
        tot, kms = time_steps(step, steps, 3, world)
        assert m.device_status() == 0
        ei, eo = SCALAR_BYTES[dtype]
        bpp = 3 * ei + n * (ei + eo)
        key = dtype if algo == "auto" else "f64_native"
        out[key] = {"value": world * pts * n * steps / tot, "unit": "scalar values/s",
                    "kernel_ms": round(kms, 4), "bytes_per_point": bpp,
                    "hbm_frac": round(bpp * pts / (kms * 1e-3) / 1e9 / hbm, 4)}
        del m, U, P, S
        torch.cuda.empty_cache()
    return out


def bench_tvd(args, world, hbm):
    """The positivity-preserving ULTIMATE-QUICKEST scheme on theta + 5 q over
    1024 x 1024 x 128 (dt 2 s: Courant numbers around 0.4 at dx 25 m), one
    launch per step; FP64 (double-float and native), FP32 and BF16 storage.  Rate = scalar values
    produced per second; compulsory bytes count the wind once per launch."""
    import torch
    from paper_2009_12850_b300 import api
    wl, n, dt = WL, 6, 2.0
    wind = synthetic.fields_for(wl)
    phis = synthetic.scalar_fields(wl.nx, wl.ny, wl.nz, n, wl.seed + 100)
    pts = wl.points
    out = {"workload": f"{wl.name}, theta + 5 q, dt {dt} s", "scalars": n,
           "f64_note": "f64: double-float on the FP32 pipe (the FP64 default); f64_native: FP64 instructions"}
    for dtype, algo in (("f64", "auto"), ("f64", "native"), ("f32", "auto"), ("bf16", "auto")):
        m = api.Mesh(wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, dtype=dtype, algo=algo)
        U = [m.from_interior(a) for a in wind]
        P = [m.from_interior(a) for a in phis]
        S = [m.empty_out() for _ in range(n)]
        stream = torch.cuda.current_stream()

        def step(rec):
            if rec is None:
                m.advect_tvd(*U, P, dt, S, stream=stream)
                return
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            m.advect_tvd(*U, P, dt, S, stream=stream)
            b.record(stream)
            rec.append((a, b))
        steps = max(3, args.steps // 2)
        tot, kms = time_steps(step, steps, 3, world)
        assert m.device_status() == 0
        ei, eo = SCALAR_BYTES[dtype]
        bpp = 3 * ei + n * (ei + eo)
        out[dtype if algo == "auto" else dtype + "_native"] = {
            "value": world * pts * n * steps / tot, "unit": "scalar values/s", "kernel_ms": round(kms, 4),
            "bytes_per_point": bpp, "hbm_frac": round(bpp * pts / (kms * 1e-3) / 1e9 / hbm, 4)}
        del m, U, P, S
        torch.cuda.empty_cache()
    return out


def bench_host_scalars(args, world):
    """The paper's hybrid step with theta + 5 q on the device (they travel with
    the wind, section 3): host arrays of 512 x 512 x 128 FP64 through
    pw_advect_host_scalars, copies overlapped slab by slab."""
    import torch
    from paper_2009_12850_b300 import api
    nx, ny, nz, n = 512, 512, 128, 6
    m = api.Mesh(nx, ny, nz, WL.dx, WL.dy, dtype="f64")
    pipe = api.Pipeline(m)
    pipe.reserve_scalars(n)
    wind = synthetic.wind_fields(nx, ny, nz, WL.seed)
    phis = synthetic.scalar_fields(nx, ny, nz, n, WL.seed + 100)
    hin = [pipe.empty_host() for _ in range(3 + n)]
    hout = [pipe.empty_host(out=True) for _ in range(3 + n)]
    for h, a in zip(hin, list(wind) + list(phis)):
        h[2:nx + 2, 2:ny + 2, :nz] = torch.from_numpy(a)
    stream = torch.cuda.current_stream()

    def step(rec):
        pipe.advect_host(*hin[:3], *hout[:3], scalars=hin[3:], sources=hout[3:], stream=stream)
    steps = max(3, args.steps // 4)
    tot, _ = time_steps(step, steps, 2, world)
    assert m.device_status() == 0
    moved = (3 + n) * nx * ny * nz * 8 * 2 + (3 * nx * ny * nz * 8 if pipe.nslab > 1 else 0) // nx
    out = {"workload": f"pw_{nx}x{ny}x{nz}_dx25, wind + theta + 5 q, FP64", "value": world * nx * ny * nz * steps / tot,
           "unit": UNIT, "ms_per_step": round(tot / steps * 1e3, 3), "bytes_per_step": moved,
           "GBs": round(moved * steps / tot / 1e9, 1)}
    del pipe, hin, hout, m
    torch.cuda.empty_cache()
    return out


def bench_small_latency(args, world):
    """The paper's weak-scaling local domain, 64 x 64 x 64 (262,144 points,
    12.6 MB of FP64 fields: L2-resident), as latency per step: halo fill +
    stencil launched eagerly, and the same two launches captured in a CUDA
    graph and replayed."""
    import torch
    from paper_2009_12850_b300 import api
    wl = synthetic.SMALL
    f = synthetic.fields_for(wl)
    out = {"workload": wl.name, "points": wl.points, "note": "L2-resident: latency, not a roofline fraction"}
    for dtype in ("f64", "f32"):
        m = api.Mesh(wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, dtype=dtype)
        U = [m.from_interior(a) for a in f]
        S = [m.empty_out() for _ in range(3)]
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(3):
                m.halo(*U, stream=side)
                m.advect(*U, *S, stream=side)
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            m.halo(*U)
            m.advect(*U, *S)
        stream = torch.cuda.current_stream()

        def eager(rec):
            m.halo(*U, stream=stream)
            m.advect(*U, *S, stream=stream)
        steps = max(200, args.steps * 10)
        te, _ = time_steps(eager, steps, 5, world)
        tg, _ = time_steps(lambda rec: graph.replay(), steps, 5, world)
        assert m.device_status() == 0
        out[dtype] = {"us_per_step_eager": round(te / steps * 1e6, 2), "us_per_step_graph": round(tg / steps * 1e6, 2),
                      "points_per_s_graph": world * wl.points * steps / tg}
        del graph, m, U, S
    return out


def bench_fused_step(args, world, hbm):
    """One forward Euler timestep on 1024 x 1024 x 128: the fused stencil +
    update (pw_advect_step, halos of the new state written in the same pass)
    against halo fill + pw_advect + pw_euler; and the whole advection step of
    the wind with theta + 5 q (pw_advect_step + pw_advect_scalars_step against
    halos + both stencils + three pw_euler passes).  Every timed step starts
    from the same state (the new state goes to a second buffer), so the work
    per step is exactly one step of the initial fields: hundreds of chained
    advection-only Euler steps would let the state grow without bound."""
    import torch
    from paper_2009_12850_b300 import api
    out = {"workload": WL.name, "dt": 0.5}
    f = synthetic.fields_for(WL)
    phis = synthetic.scalar_fields(WL.nx, WL.ny, WL.nz, 6, WL.seed + 100)
    pts = WL.points
    for dtype in ("f64", "f32"):
        m = api.Mesh(WL.nx, WL.ny, WL.nz, WL.dx, WL.dy, dtype=dtype)
        A = [m.from_interior(a) for a in f]
        B = [m.empty() for _ in range(3)]

        def fused(rec):
            m.step(*A, *B, dt=0.5)
        steps = max(3, args.steps // 2)
        tf, _ = time_steps(fused, steps, 3, world)
        S = [m.empty_out() for _ in range(3)]
        E = [t.clone() for t in A]   # the update target of the unfused sequence

        def unfused(rec):
            m.halo(*A)
            m.advect(*A, *S)
            m.euler(*E, *S, 0.5)
        tu, _ = time_steps(unfused, steps, 3, world)
        assert m.device_status() == 0
        es = {"f64": 8, "f32": 4}[dtype]
        out[dtype] = {"fused_value": world * pts * steps / tf, "unfused_value": world * pts * steps / tu,
                      "unit": UNIT, "fused_ms": round(tf / steps * 1e3, 4), "unfused_ms": round(tu / steps * 1e3, 4),
                      "speedup": round(tu / tf, 3), "fused_bytes_per_point": 6 * es,
                      "unfused_bytes_per_point": 15 * es}
        # the whole advection step of the wind and theta + 5 q (old wind for all)
        P = [m.from_interior(a) for a in phis]
        Q = [m.empty() for _ in range(6)]

        def fused_all(rec):
            m.step(*A, *B, dt=0.5)
            m.step_scalars(*A, P, Q, dt=0.5)
        tfa, _ = time_steps(fused_all, steps, 3, world)
        SP = [m.empty_out() for _ in range(6)]
        EP = [t.clone() for t in P]

        def unfused_all(rec):
            m.halo(*A)
            m.halo(*P[:3])
            m.halo(*P[3:])
            m.advect(*A, *S)
            m.advect_scalars(*A, P, SP)
            m.euler(*E, *S, 0.5)
            m.euler(*EP[:3], *SP[:3], 0.5)
            m.euler(*EP[3:], *SP[3:], 0.5)
        tua, _ = time_steps(unfused_all, steps, 3, world)
        assert m.device_status() == 0
        out[dtype]["wind_theta_5q"] = {"fused_ms": round(tfa / steps * 1e3, 4),
                                       "unfused_ms": round(tua / steps * 1e3, 4), "speedup": round(tua / tfa, 3),
                                       "fused_bytes_per_point": (6 + 15) * es,
                                       "unfused_bytes_per_point": (15 + 3 + 6 * 5) * es}
        del m, A, B, S, E, P, Q, SP, EP
        torch.cuda.empty_cache()
    return out


def bench_paper_strong(args, world, hbm):
    """The paper's strong-scaling global domain (2048 x 2048 x 64) held on one
    GPU in FP32: halo fill + stencil per step."""
    import torch
    from paper_2009_12850_b300 import api
    wl = synthetic.PAPER_STRONG
    m = api.Mesh(wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, dtype="f32")
    U = [m.from_interior(a) for a in synthetic.fields_for(wl)]
    S = [m.empty_out() for _ in range(3)]
    stream = torch.cuda.current_stream()

    def step(rec):
        m.halo(*U, stream=stream)
        if rec is None:
            m.advect(*U, *S, stream=stream)
            return
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        m.advect(*U, *S, stream=stream)
        b.record(stream)
        rec.append((a, b))
    steps = max(3, args.steps // 2)
    tot, kms = time_steps(step, steps, 3, world)
    assert m.device_status() == 0
    pts = wl.points
    return {"workload": wl.name, "dtype": "f32", "value": world * pts * steps / tot, "unit": UNIT,
            "kernel_ms": round(kms, 4), "hbm_frac": round(24 * pts / (kms * 1e-3) / 1e9 / hbm, 4)}


def bench_adjoint_loop(args):
    """Loss = sum of squared sources after 10 Euler steps (dt = 0.5 s) on
    256 x 256 x 96 FP32 and its gradient by the adjoint kernels with
    checkpointed recomputation every 2 steps; gradient compared with the same
    computation in FP64 (native FP64 kernels)."""
    import torch
    from paper_2009_12850_b300 import api, autograd
    wl = synthetic.ADJOINT
    f = synthetic.wind_fields(wl.nx, wl.ny, wl.nz, wl.seed)
    dt, steps, every = wl.extra["dt"], wl.extra["steps"], wl.extra["checkpoint_every"]
    out = {}
    grads = {}
    for dtype, algo in (("f32", "auto"), ("f64", "auto"), ("f64", "native")):
        m = api.Mesh(wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, dtype=dtype, algo=algo)
        base = [m.from_interior(a) for a in f]

        def one():
            U = [t.clone().requires_grad_(True) for t in base]
            L = autograd.source_energy_loss(m, *U, dt=dt, steps=steps, checkpoint_every=every)
            L.backward()
            return L, U
        spin_up(one)
        # eager: each repetition timed alone; the median, since the small FP32
        # steps make the Python-driven launch sequence sensitive to host load
        reps = 10 if dtype == "f32" else 3
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            L, U = one()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        res = {"ms_per_loss_and_grad_eager_median": round(float(np.median(times)), 3), "loss": float(L.item())}
        key = dtype if algo == "auto" else dtype + "_native"
        grads[key] = [m.interior(u.grad).double() for u in U]
        # the same loss and gradient captured in one CUDA graph and replayed: the
        # device-side time of the whole computation, free of launch overhead
        Ug = [t.clone().requires_grad_(True) for t in base]
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(2):
                autograd.source_energy_loss(m, *Ug, dt=dt, steps=steps, checkpoint_every=every).backward()
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            autograd.source_energy_loss(m, *Ug, dt=dt, steps=steps, checkpoint_every=every).backward()
        graph.replay()
        torch.cuda.synchronize()
        n = 10
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(n):
            graph.replay()
        e1.record()
        torch.cuda.synchronize()
        assert m.device_status() == 0
        res["ms_per_loss_and_grad"] = round(e0.elapsed_time(e1) / n, 3)
        out[key] = res
        del m, base, U, Ug, graph
    rel = [float((a - b).abs().max() / b.abs().max()) for a, b in zip(grads["f32"], grads["f64_native"])]
    rel2 = [float((a - b).abs().max() / b.abs().max()) for a, b in zip(grads["f64"], grads["f64_native"])]
    return {"workload": wl.name, "steps": steps, "dt": dt, "checkpoint_every": every,
            "f32": out["f32"], "f64": out["f64"], "f64_native": out["f64_native"],
            "f64_note": "f64: double-float (split) forward steps and adjoint; f64_native: native FP64 throughout",
            "grad_rel_err_f32_vs_f64": {"gu": rel[0], "gv": rel[1], "gw": rel[2]},
            "grad_rel_err_f64_vs_f64_native": {"gu": rel2[0], "gv": rel2[1], "gw": rel2[2]}}


def bench_adjoint_kernel(args):
    """The adjoint stencil alone on the bandwidth workload (1024 x 1024 x 128):
    gu, gv, gw = J(u,v,w)^T (gsu, gsv, gsw), 6 fields read and 3 written
    (36 B/point compulsory in FP32, 72 in FP64), in FP32 and in FP64
    (double-float arithmetic)."""
    import torch
    from paper_2009_12850_b300 import api
    wl = WL
    peak = float(load_peaks()[0]["hbm_gbs"])
    out = {"workload": wl.name}
    for dtype in ("f32", "f64"):
        m = api.Mesh(wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, dtype=dtype)
        U = [m.from_interior(a) for a in synthetic.fields_for(wl)]
        Y = [m.zeros() for _ in range(3)]
        for t in Y:
            t.normal_()
        G = [m.zeros() for _ in range(3)]
        stream = torch.cuda.current_stream()

        def step(rec):
            if rec is None:
                m.adjoint(*U, *Y, *G, stream=stream)
                return
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            m.adjoint(*U, *Y, *G, stream=stream)
            b.record(stream)
            rec.append((a, b))
        steps = max(3, args.steps // 2)
        _, kms = time_steps(step, steps, 3, world_size())
        assert m.device_status() == 0
        pts = wl.points
        bpp = 36 if dtype == "f32" else 72
        out[dtype] = {"ms_per_call": round(kms, 4), "value": pts / (kms * 1e-3), "unit": UNIT,
                      "bytes_per_point": bpp, "hbm_frac": round(bpp * pts / (kms * 1e-3) / 1e9 / peak, 4),
                      "algo": m.algo}
        del m, U, Y, G
        torch.cuda.empty_cache()
    return out


def bench_precision():
    """512 x 512 x 160 sheared turbulence: the sources in FP64 (split), FP32,
    BF16 and BF16-in-and-out storage, and the conservation residuals of each.
    The sources are kept in host memory; their max and RMS error against the
    FP64 oracle is filled in by the CPU leg (precision_vs_oracle), which is the
    only part of this program that runs the oracle."""
    import torch
    from paper_2009_12850_b300 import api
    wl = synthetic.PRECISION
    f = synthetic.fields_for(wl)
    res, kept = {}, {}
    for dtype in ("f64", "f32", "bf16", "bf16_out"):
        m = api.Mesh(wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, dtype=dtype)
        U = [m.from_interior(a) for a in f]
        S = m.advect(*U)
        re, rm = m.residuals(*U, *S)
        assert m.device_status() == 0
        res[dtype] = {"R_E": list(re), "R_M": list(rm)}
        kept[dtype] = [m.interior(t).double().cpu().numpy() for t in S]
        del m, U, S
    PRECISION_KEPT["sources"] = kept
    return {"workload": wl.name, "fields": "u = 15 z/z_top + N(0,2), v = N(0,2), w = N(0,0.3) m/s", **res}


PRECISION_KEPT = {}


# ----------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline leg and the reference arm)
# ----------------------------------------------------------------------------
def oracle_sample(seconds, ncols=64, threads=None):
    """Time the FP64 CPU oracle on slabs of the bench workload (ncols x ny x nz
    columns of the same field distribution, periodic) until `seconds` of work
    have run, on `threads` threads (default: every host core); returns
    (points/s, threads, description)."""
    import oracle
    threads = oracle.set_threads(threads or os.cpu_count() or 1)
    c = oracle.Coeffs(WL.nz, WL.dx, WL.dy)
    u, v, w = synthetic.wind_fields(ncols, WL.ny, WL.nz, WL.seed)
    oracle.advect(c, u, v, w)  # warm
    done, t0 = 0, time.perf_counter()
    while True:
        oracle.advect(c, u, v, w)
        done += u.size
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return done / el, threads, f"{done // u.size} sweeps of a {ncols}x{WL.ny}x{WL.nz} slab " \
                               f"({done} points, {el:.1f} s)"


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or "unknown"


def precision_vs_oracle():
    """Max and RMS error, per source, of the precision row's GPU sources against
    the FP64 oracle evaluated on the original (unrounded) FP64 fields, also
    relative to each point's condition sum."""
    import oracle
    kept = PRECISION_KEPT.pop("sources", None)
    if not kept:
        return None
    wl = synthetic.PRECISION
    f = synthetic.fields_for(wl)
    c = oracle.Coeffs(wl.nz, wl.dx, wl.dy)
    ref, cond = oracle.advect(c, *f, want_cond=True)
    out = {"reference": "FP64 oracle on the unrounded fields"}
    for dtype, S in kept.items():
        e = {}
        for q, nm in enumerate(("su", "sv", "sw")):
            d = np.abs(S[q] - ref[q])
            with np.errstate(divide="ignore", invalid="ignore"):
                r = np.where(cond[q] > 0, d / cond[q], 0.0)
            e[nm] = {"max_abs": float(d.max()), "rms": float(np.sqrt(np.mean(d * d))),
                     "max_rel_to_max": float(d.max() / np.abs(ref[q]).max()), "max_err_over_cond": float(r.max())}
        out[dtype] = e
    return out


def cpu_baseline(seconds):
    rate, threads, desc = oracle_sample(seconds)
    rate1, _, desc1 = oracle_sample(min(3.0, seconds / 4), threads=1)
    oracle_threads_all()
    return {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": desc + "; FP64 C oracle, OpenMP over x",
            "single_thread": {"value": rate1, "unit": UNIT, "sample": desc1},
            "cpu_model": cpu_model()}


def oracle_threads_all():
    import oracle
    oracle.set_threads(os.cpu_count() or 1)


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    rates = []
    for _ in range(args.warmup):
        oracle_sample(min(per_step, 5.0))
    t0 = time.perf_counter()
    descs = []
    for _ in range(args.steps):
        r, threads, d = oracle_sample(per_step)
        rates.append(r)
        descs.append(d)
    total = time.perf_counter() - t0
    value = float(np.mean(rates))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WL.name, "nx": WL.nx, "ny": WL.ny, "nz": WL.nz, "dx": WL.dx,
                       "step": "PW stencil u,v,w -> su,sv,sw (FP64) on a bounded slab sample"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": descs[-1]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_fp_rates():
    """Compile and run the package's arithmetic-rate microbenchmark
    (paper_2009_12850_b300/rates/fp_rates.cu): the FP64, conversion and FP32
    rates that decide how the FP64 stencil computes.  Prints its JSON line."""
    src = os.path.join(ROOT, "paper_2009_12850_b300", "rates", "fp_rates.cu")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "fp_rates")
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, src], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    print(json.dumps({"fp_rates": json.loads(out)}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-extras", action="store_true", help="only the headline and e2e")
    ap.add_argument("--extras", default=None,
                    help="comma list of extra rows to run (default all): f32, bf16, f64_native, residuals, "
                         "bf16_out, small_latency, scalars, e2e_theta_5q, "
                         "paper_strong_f32, fused_step, batched, adjoint_loop, adjoint_kernel, precision")
    ap.add_argument("--batch-tune", default=None,
                    help="autotuner cache file for the batched row (reused when it exists)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--dtype", choices=["f64", "f32", "bf16", "bf16_out"], default="f64", help="headline storage type")
    ap.add_argument("--algo", choices=["auto", "native", "split"], default="auto", help="FP64 arithmetic")
    ap.add_argument("--fp-rates", action="store_true",
                    help="only run the arithmetic-rate microbenchmark (FP64, f64<->f32, FP32, FP32x2) and print it")
    ap.add_argument("--nx", type=int, default=None, help="smaller domain (ncu captures)")
    ap.add_argument("--ny", type=int, default=None)
    ap.add_argument("--nz", type=int, default=None)
    args = ap.parse_args()
    global WL
    if args.nx or args.ny or args.nz:
        nx, ny, nz = args.nx or WL.nx, args.ny or WL.ny, args.nz or WL.nz
        WL = synthetic.Workload(f"pw_{nx}x{ny}x{nz}_dx25", nx, ny, nz, WL.dx, WL.dy, WL.seed)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.fp_rates:
        run_fp_rates()
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

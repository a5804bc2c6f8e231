"""Benchmark of the NOHAP/OUCS3 compressible Navier-Stokes RK step on GB300.

Metric: RK-stage grid-point updates per second (points x 4 stages x steps /
time) of the mixed-precision form at 1024^3 (FP32 fluxes/derivatives on the
state minus its hydrostatic base, FP64 state and RK accumulation, NOHAP
sub-domains of 64), one RK4 step per benchmark step, the filter on its
every-50-steps cadence, state resident in HBM.  Also reported: the plain FP64
form, the dominant kernel against the HBM roofline, an end-to-end number
through the C ABI with host buffers, and the FP64 CPU oracle as a baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank advances its own independent box (the path
needs no exchange between boxes): weak scaling, no data-path collective.
"""
import argparse
import ctypes
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RK-stage grid-point updates/s at 1024^3 (mixed vs FP64), % of HBM/tensor roofline"
UNIT = "point-stage updates/s"

# algorithmic bytes per grid point of one launch of each kernel kind
# (mixed form; see the design notes for the derivation)
ALG_BYTES_MIXED = {
    "prep": 40 + 24,                   # read Q (5 f64), write W (6 f32)
    "sweep_x": 24 + 20,                # read W, write R (5 f32)
    "sweep_y": 24 + 40,                # read W, read+write R
    "sweep_z": 24 + 40,
    # stage average of W + R + Dn (+ K) in, K + W' out; stage 4 also Q_n in/out and Dn out
    "visc_rk_update": (108 + 128 + 128 + 188) / 4.0,
    "filter": 3 * 80,                  # three sweeps, each read+write Q
    # compact viscous terms (visc_compact): per launch of each kind
    "visc_grad": 20 + 16,              # read rho', u, v, w, p'; write 4 gradients
    "visc_flux": 48 + 20 + 48,         # read 12 gradients and 5 primitives, write 12 fluxes
    "visc_div": 16 + 32,               # read 4 fluxes; reduction adds into R[1..4] (read + write)
    # visc_rk_update without the viscous terms: W0 and the velocity along gravity
    # instead of the five primitives the viscous stencils need
    "source_rk_update": (92 + 112 + 112 + 172) / 4.0,
}
ALG_BYTES_FP64 = {
    "prep": 40 + 48, "sweep_x": 48 + 40, "sweep_y": 48 + 80, "sweep_z": 48 + 80,
    "visc_rk_update": (188 + 228 * 2 + 148) / 4.0, "filter": 3 * 80,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1024, help="grid points per axis")
    ap.add_argument("--shape", default=None,
                    help="nx,ny,nz of the timed box instead of n^3 (profiling small cases of one kernel)")
    ap.add_argument("--sub-n", type=int, default=64)
    ap.add_argument("--fp64-n", type=int, default=1024, help="grid of the FP64-form comparison (0: skip)")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--compact-n", type=int, default=1024,
                    help="grid of the compact-viscous-term measurement, mixed form (0: skip)")
    ap.add_argument("--compact-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--cpu-n", type=int, default=128, help="oracle sample grid for the CPU baseline")
    ap.add_argument("--cpu-steps", type=int, default=12, help="oracle sample steps for the CPU baseline")
    ap.add_argument("--cpu1-n", type=int, default=64, help="oracle sample grid for the one-core timing")
    ap.add_argument("--cpu1-steps", type=int, default=4, help="oracle sample steps for the one-core timing")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", dest="extra", action="store_false",
                    help="skip the short derivative-microbenchmark and 64-box runs of the default line")
    ap.add_argument("--workload", default="rk", choices=["rk", "deriv", "batched"],
                    help="rk: the RK-step benchmark (default); deriv: the derivative microbenchmark; "
                         "batched: 64 uneven boxes in one context")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out, _ = self.p.communicate()
        rows = [r.split(", ") for r in out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        loaded = [s for s in sm if s > 0.5 * mx] or sm
        return {"sm_mhz": loaded[len(loaded) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(rows)}


def max_over_ranks(x, dist=None, device="cpu"):
    """Max of a per-rank scalar over all ranks (identity without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(points_per_rank, stages, steps, world, ms_max):
    """Whole-job point-stage updates per second: every rank advances its own
    box of `points_per_rank` points, the slowest rank sets the time."""
    return world * float(points_per_rank) * stages * steps / (ms_max * 1e-3)


def box(n, sub_n, **kw):
    import nopcs_synth as S
    return S.box_params((n, n, n), sub_n=(sub_n,) * 3, **kw)


def run_cpu_oracle(n, steps, warmup=0, threads=None):
    """Time the FP64 oracle as it stands (OpenMP over lines; all host cores,
    or `threads` of them)."""
    import oracle
    p = box(n, min(64, n))
    p["base_subtract"] = 1
    all_threads = oracle.num_threads()
    if threads:
        oracle.set_num_threads(threads)
    try:
        s = oracle.Solver(p)
        Q = s.initial_state()
        if warmup:
            Q = s.step(Q, warmup)
        t0 = time.perf_counter()
        Q = s.step(Q, steps)
        dt = time.perf_counter() - t0
        used = oracle.num_threads()
    finally:
        oracle.set_num_threads(all_threads)
    pts = float(n) ** 3 * 4 * steps
    return pts / dt, dt, used


def workload_name(n, sub_n):
    return ("two-temperature Rayleigh-Taylor box %d^3, mixed precision (FP32 fluxes and NOHAP derivatives, "
            "FP64 state and RK4), sub-domains of %d, filter every 50 steps" % (n, sub_n))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = args.cpu_n
    rate, dt, cores = run_cpu_oracle(n, args.steps, args.warmup)
    sample = "FP64 CPU oracle, %d^3 box of the same physics (base-subtracted), %d RK4 steps after %d warm-up" % (
        n, args.steps, args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "FP64 CPU oracle on %d host cores, timed on a bounded sample (a %d^3 box, "
                                   "base-subtracted, sub-domains of %d) of the workload: %s"
                                   % (cores, n, min(64, n), workload_name(args.n, args.sub_n)),
                       "grid": [args.n] * 3, "sub_n": args.sub_n,
                       "precision": "fp64 (the oracle)", "sample_grid": [n] * 3,
                       "parallelism": "rank 0 only (host cores)"},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def deriv_rows(N, steps, warmup):
    """NOHAP first derivative of a seeded 512^3 field (random-phase sines plus
    N(0, 1e-3^2) noise) along x, y, z: Thomas form in FP64 and FP32 and the
    3xTF32 and BF16x3 tensor-core forms, sub-domains of 32, 64 and 128, and the banded
    explicit form (FP32, no sub-domains).  Each case is timed
    with CUDA events over `steps` calls after `warmup`; the field (0.5-1 GB) is
    larger than L2.  Returns (rows, peaks)."""
    import torch
    import nopcs_synth as S
    n = 512
    hbm, peak_kind = peaks()
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            bf16 = float(json.load(fh)["bf16_tflops"])
        tf32_peak, tf32_kind = bf16 * 1.1 / 2.25, "measured bf16 x nominal tf32/bf16 ratio"
        bf16_peak = bf16
    except Exception:
        tf32_peak, tf32_kind = 1900.0 * 1.1 / 2.25, "fallback"
        bf16_peak = 1900.0
    st = torch.cuda.current_stream()
    px, py, pz = [torch.from_numpy(v).cuda() for v in S.sine_profiles((n, n, n), kmax=64, seed=7)]
    g = torch.Generator(device="cuda").manual_seed(11)
    f64 = (pz[:, None, None] + py[None, :, None] + px[None, None, :]).contiguous()
    f64 += 1e-3 * torch.randn(f64.shape, generator=g, device="cuda", dtype=torch.float64)
    f32 = f64.float()
    rows = []
    for sub_n in (32, 64, 128):
        p = box(n, sub_n, perturb_amp=0.0)
        forms = [("thomas", N.NOPCS_FORM_THOMAS), ("gemm_3xtf32", N.NOPCS_FORM_GEMM_3XTF32),
                 ("gemm_bf16x3", N.NOPCS_FORM_GEMM_BF16X3)]
        if sub_n == 64:  # the banded form has no sub-domains: timed once
            forms.append(("banded", N.NOPCS_FORM_BANDED))
        for form_name, form in forms:
            try:
                ctx = N.nopcs_init([p], prec=N.NOPCS_MIXED, form=form, stream=st.cuda_stream)
            except N.NopcsError as exc:
                rows.append({"form": form_name, "sub_n": sub_n, "unsupported": str(exc)})
                continue
            cases = [("f32", 1, f32)] if form_name != "thomas" else [("f64", 0, f64), ("f32", 1, f32)]
            for dname, dt, f in cases:
                out = torch.empty_like(f)
                for axis in range(3):
                    for _ in range(warmup):
                        N.nopcs_derivative(ctx, 0, axis, 1, dt, f.data_ptr(), out.data_ptr(), st.cuda_stream)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    e0.record(st)
                    for _ in range(steps):
                        N.nopcs_derivative(ctx, 0, axis, 1, dt, f.data_ptr(), out.data_ptr(), st.cuda_stream)
                    e1.record(st)
                    N.nopcs_synchronize(ctx)
                    ms = e0.elapsed_time(e1) / steps
                    es = 8 if dt == 0 else 4
                    gbs = 2 * es * n ** 3 / (ms * 1e-3) / 1e9
                    row = {"form": form_name, "dtype": dname, "sub_n": sub_n, "axis": "xyz"[axis], "ms": ms,
                           "points_per_s": n ** 3 / (ms * 1e-3), "hbm_gbs": gbs, "hbm_frac": gbs / hbm}
                    if form_name == "banded":
                        # 49 FP32 FMAs per point (the interior stencil)
                        row["sub_n"] = None
                        row["fp32_tflops"] = 2.0 * 49 * n ** 3 / (ms * 1e-3) / 1e12
                    elif form_name == "gemm_3xtf32":
                        # three TF32 products of 2 flops per window point
                        kpad = (sub_n + 48 + 7) // 8 * 8
                        tflops = 6.0 * kpad * n ** 3 / (ms * 1e-3) / 1e12
                        row.update({"tensor_tflops": tflops, "tensor_frac": tflops / tf32_peak})
                    elif form_name == "gemm_bf16x3":
                        # six BF16 products of 2 flops per window point
                        kpad = (sub_n + 48 + 15) // 16 * 16
                        tflops = 12.0 * kpad * n ** 3 / (ms * 1e-3) / 1e12
                        row.update({"tensor_tflops": tflops, "tensor_frac": tflops / bf16_peak})
                    rows.append(row)
            N.nopcs_destroy(ctx)
    del f64, f32, px, py, pz
    torch.cuda.empty_cache()
    return rows, {"hbm": hbm, "peak_kind": peak_kind, "tf32_peak": tf32_peak, "tf32_kind": tf32_kind,
                  "bf16_peak": bf16_peak}


def deriv_summary(rows):
    """Best case per form and dtype (fastest over sub-domain lengths and axes,
    and the slowest axis of that sub-domain length)."""
    out = {}
    for r in rows:
        if "ms" not in r:
            continue
        key = r["form"] + "_" + r["dtype"]
        same = [q for q in rows if q.get("form") == r["form"] and q.get("dtype") == r["dtype"]
                and q.get("sub_n") == r.get("sub_n") and "ms" in q]
        worst = max(q["ms"] for q in same)
        cur = out.get(key)
        if cur is None or worst < cur["ms_slowest_axis"]:
            ent = {"sub_n": r.get("sub_n"), "ms_slowest_axis": worst,
                   "ms_per_axis": {q["axis"]: round(q["ms"], 4) for q in same},
                   "hbm_frac_slowest_axis": min(q["hbm_frac"] for q in same)}
            if "tensor_frac" in r:
                ent["tensor_frac_slowest_axis"] = min(q["tensor_frac"] for q in same)
            out[key] = ent
    return out


def run_deriv_microbench(args):
    import torch
    from paper_2203_00879_gb300 import build as B
    B.build()
    from paper_2203_00879_gb300 import nopcs as N
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    n = 512
    rows, pk = deriv_rows(N, args.steps, args.warmup)
    hbm, peak_kind, tf32_peak, tf32_kind, bf16_peak = (pk["hbm"], pk["peak_kind"], pk["tf32_peak"], pk["tf32_kind"],
                                                       pk["bf16_peak"])
    best = max((r for r in rows if r.get("dtype") == "f32"), key=lambda r: r["points_per_s"])
    line = {"metric": "NOHAP first-derivative points/s at 512^3 (microbenchmark)", "value": best["points_per_s"],
            "unit": "points/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": best["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "seeded 512^3 sine+noise field, first derivative along x, y, z", "best": best,
                       "l2": "inputs larger than L2 (512^3 FP32 = 0.54 GB)"},
            "roofline": {"bound": "hbm", "peak": hbm, "unit": "GB/s", "peak_kind": peak_kind,
                         "tensor_peak_tflops": tf32_peak, "tensor_peak_kind": tf32_kind,
                         "bf16_peak_tflops": bf16_peak},
            "summary": deriv_summary(rows),
            "cases": rows}
    print(json.dumps(line))
    return 0


def batched_run(N, steps, warmup, mode=0):
    """64 independent boxes (edges from {32, 48, 64, 96, 128}, heights 1-2x,
    temperature contrasts 50-250 K), mixed precision, sub-domain lengths chosen
    by the autotuner, advanced together: every RK step is one CUDA-graph launch
    whose branches are the boxes (mode 0) or one persistent kernel over all of
    them (mode 1).  Returns (points, ms, init_s, tuned)."""
    import torch
    import nopcs_synth as S
    boxes = S.uneven_boxes(64, seed=11)
    for b in boxes:
        b["sub_n"] = (-1, -1, -1)
    st = torch.cuda.current_stream()
    t0 = time.perf_counter()
    ctx = N.nopcs_init(boxes, prec=N.NOPCS_MIXED, stream=st.cuda_stream)
    init_s = time.perf_counter() - t0
    npts = sum(b["n"][0] * b["n"][1] * b["n"][2] for b in boxes)
    if mode:
        N.nopcs_set_launch(ctx, mode)
    N.nopcs_rk_step(ctx, warmup)
    N.nopcs_synchronize(ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    N.nopcs_rk_step(ctx, steps)
    e1.record(st)
    N.nopcs_synchronize(ctx)
    ms = e0.elapsed_time(e1)
    tuned = {}
    for i in range(len(boxes)):
        k = str(N.nopcs_box_info(ctx, i)["sub_n"])
        tuned[k] = tuned.get(k, 0) + 1
    N.nopcs_destroy(ctx)
    return npts, ms, init_s, tuned


def run_batched(args):
    import torch
    from paper_2203_00879_gb300 import build as B
    B.build()
    from paper_2203_00879_gb300 import nopcs as N
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    npts, ms, init_s, tuned = batched_run(N, args.steps, args.warmup, 1)
    _, ms_g, _, _ = batched_run(N, args.steps, args.warmup, 0)
    line = {"metric": "RK-stage grid-point updates/s, 64 uneven boxes batched (mixed)",
            "value": npts * 4 * args.steps / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
            "config": {"workload": "64 uneven two-temperature boxes, edges 32-128, heights 1-2x edge, "
                                   "dT 50-250 K, seed 11", "points": npts, "init_s": init_s,
                       "tuned_sub_n": tuned, "launch": "one persistent kernel per step",
                       "graph_launch": {"value": npts * 4 * args.steps / (ms_g * 1e-3),
                                        "ms_per_step": ms_g / args.steps,
                                        "launch": "one CUDA graph per step, one branch per box"}}}
    print(json.dumps(line))
    return 0


_CUDA_DRIVER = None


def profiler_range(on):
    """cuProfilerStart/Stop around the timed region: a profiler started with
    profiling from the start off records the timed launches only."""
    global _CUDA_DRIVER
    try:
        if _CUDA_DRIVER is None:
            _CUDA_DRIVER = ctypes.CDLL("libcuda.so.1")
        rc = (_CUDA_DRIVER.cuProfilerStart if on else _CUDA_DRIVER.cuProfilerStop)()
        if rc != 0:
            print(f"cuProfiler{'Start' if on else 'Stop'} returned {rc}", file=sys.stderr)
    except OSError as exc:
        print(f"profiler range unavailable: {exc}", file=sys.stderr)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "deriv":
        return run_deriv_microbench(args)
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2203_00879_gb300 import build as B
    B.build()
    from paper_2203_00879_gb300 import nopcs as N

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def rank_max(x):
        return max_over_ranks(x, dist, "cuda")

    stream = torch.cuda.current_stream()
    st = stream.cuda_stream
    n, K, W = args.n, args.steps, args.warmup
    shape = tuple(int(v) for v in args.shape.split(",")) if args.shape else (n, n, n)
    npts = float(shape[0]) * shape[1] * shape[2]
    if args.shape:
        import nopcs_synth as S
        p = S.box_params(shape, sub_n=(args.sub_n,) * 3, seed=1 + rank)
    else:
        p = box(n, args.sub_n, seed=1 + rank)
    ctx = N.nopcs_init([p], prec=N.NOPCS_MIXED, stream=st)
    tile_lines = N.nopcs_box_info(ctx, 0)["tile_lines"]
    N.nopcs_rk_step(ctx, W)
    N.nopcs_synchronize(ctx)
    # Place the timed window on the filter's every-50-steps cadence so that it
    # holds ceil(K / 50) filters (the count a long run amortises to, rounded
    # up): the first timed step ends on a multiple of 50.
    N.nopcs_set_step(ctx, 0, 49)
    filters_in_window = (K + 49) // 50
    # ---- timed region: graph replay, as nopcs_rk_step runs in production ----
    clocks = Clocks(local)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    clocks.start()
    profiler_range(True)
    ev0.record(stream)
    N.nopcs_rk_step(ctx, K)
    diag = N.nopcs_diagnostics(ctx, 0)  # result read back (D2H) inside the timed region
    ev1.record(stream)
    profiler_range(False)
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ms_max = rank_max(ms)
    value = job_rate(npts, 4, K, world, ms_max)

    # ---- per-kernel times: a separate window of direct launches, each kernel
    # between CUDA events on the context stream (same kernels, same state) ----
    KP = 3
    N.nopcs_set_profiling(ctx, True)
    N.nopcs_profile_read(ctx, reset=True)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    N.nopcs_rk_step(ctx, KP)
    e1.record(stream)
    barrier()
    ms_prof = e0.elapsed_time(e1)
    prof = N.nopcs_profile_read(ctx, reset=True)
    N.nopcs_set_profiling(ctx, False)
    launches_per_kind = {"prep": 1, "sweep_x": 1, "sweep_y": 1, "sweep_z": 1, "visc_rk_update": 1,
                         "wall_bc": 3, "filter": 4, "diagnostics": 2}
    step_launches = sum(v[1] * launches_per_kind.get(k, 1) for k, v in prof.items()
                        if k not in ("filter", "diagnostics")) / KP
    gpu_launches = int(round(step_launches * K)) + 4 * filters_in_window + 2

    # dominant kernel against the HBM roofline
    hbm, peak_kind = peaks()
    dom = max((k for k in prof if k in ALG_BYTES_MIXED and k != "filter"), key=lambda k: prof[k][0])
    avg_ms = prof[dom][0] / max(prof[dom][1], 1)
    alg = ALG_BYTES_MIXED[dom] * npts
    achieved = alg / (avg_ms * 1e-3) / 1e9
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            tr = json.load(f)
        from paper_2203_00879_gb300.build import KERNEL_FILES, source_hash
        ent = tr.get("mixed", {}).get(dom)
        if ent and ent.get("source_hash") == source_hash(KERNEL_FILES[dom]):
            traffic = ent["bytes_per_point"] * npts
    except Exception:
        traffic = None
    per_kernel = {}
    for k, v in prof.items():
        if not v[1]:
            continue
        ent = {"ms_total": v[0], "launches": v[1], "ms_per_launch": v[0] / v[1], "share": v[0] / max(ms_prof, 1e-9)}
        if k in ALG_BYTES_MIXED and k != "filter":
            gbs = ALG_BYTES_MIXED[k] * npts / (v[0] / v[1] * 1e-3) / 1e9
            ent.update(alg_bytes_per_point=ALG_BYTES_MIXED[k], achieved_gbs=gbs, frac=gbs / hbm)
        per_kernel[k] = ent
    # the whole RK stage against the algorithmic 160 B per point and stage
    # (FP64 state, three-register classical RK4)
    whole = 160.0 * npts * 4 * K / (ms * 1e-3) / 1e9
    whole_step = {"alg_bytes_per_point_stage": 160, "achieved_gbs": whole, "frac": whole / hbm,
                  "peak_kind": peak_kind}
    N.nopcs_destroy(ctx)
    torch.cuda.synchronize()

    # end to end through the C ABI with host buffers: every step's state is
    # uploaded from pinned host memory (staged while the previous step runs,
    # nopcs_stage_state / nopcs_commit_state), advanced one RK4 step, and the
    # diagnostics are read back
    e2e = None
    if args.e2e_steps > 0:
        ctx = N.nopcs_init([p], prec=N.NOPCS_MIXED, stream=st)
        nbytes = int(5 * npts * 8)
        try:
            host = torch.empty(int(5 * npts), dtype=torch.float64, pin_memory=True)
            pinned = True
        except Exception:
            host = torch.empty(int(5 * npts), dtype=torch.float64)
            pinned = False
        N.nopcs_get_state(ctx, 0, host.data_ptr())
        N.nopcs_stage_state(ctx, 0, host.data_ptr())  # allocates the staging buffer
        N.nopcs_commit_state(ctx, 0)
        N.nopcs_rk_step(ctx, 1)
        N.nopcs_diagnostics(ctx, 0)
        barrier()
        t0 = time.perf_counter()
        N.nopcs_stage_state(ctx, 0, host.data_ptr())
        for k in range(args.e2e_steps):
            N.nopcs_commit_state(ctx, 0)
            if k + 1 < args.e2e_steps:
                # the next step's state crosses the link while this step runs
                N.nopcs_stage_state(ctx, 0, host.data_ptr())
            N.nopcs_rk_step(ctx, 1)
            N.nopcs_diagnostics(ctx, 0)
        barrier()
        el = rank_max(time.perf_counter() - t0)
        e2e = {"value": world * npts * 4 * args.e2e_steps / el, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": 10 * 8, "pinned_host": pinned, "steps": args.e2e_steps,
               "readback": "the diagnostics (10 doubles) every step; the state stays on the device",
               "upload": "each step's state staged from pinned host memory on the copy stream while the "
                         "previous step runs (nopcs_stage_state), made current by nopcs_commit_state"}
        del host
        N.nopcs_destroy(ctx)
        torch.cuda.synchronize()

    # plain FP64 form for comparison
    fp64 = None
    if args.fp64_n > 0:
        n64 = args.fp64_n
        p64 = box(n64, args.sub_n, seed=1 + rank)
        try:
            ctx = N.nopcs_init([p64], prec=N.NOPCS_FP64, stream=st)
        except N.NopcsError:
            n64 = 768
            p64 = box(n64, args.sub_n, seed=1 + rank)
            ctx = N.nopcs_init([p64], prec=N.NOPCS_FP64, stream=st)
        N.nopcs_rk_step(ctx, 1)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        N.nopcs_rk_step(ctx, args.fp64_steps)
        e1.record(stream)
        barrier()
        m64 = rank_max(e0.elapsed_time(e1))
        N.nopcs_set_profiling(ctx, True)
        N.nopcs_profile_read(ctx, reset=True)
        N.nopcs_rk_step(ctx, 1)
        p64k = N.nopcs_profile_read(ctx, reset=True)
        N.nopcs_set_profiling(ctx, False)
        v64 = world * float(n64) ** 3 * 4 * args.fp64_steps / (m64 * 1e-3)
        fp64 = {"value": v64, "unit": UNIT, "grid": [n64] * 3, "steps": args.fp64_steps,
                "ms_per_step": m64 / args.fp64_steps, "mixed_over_fp64": value / v64,
                "kernels": {k: {"ms_per_launch": v[0] / v[1], "launches": v[1]} for k, v in p64k.items() if v[1]}}
        N.nopcs_destroy(ctx)

    # mixed form with compact viscous terms (NOHAP gradients and divergence)
    compact = None
    if args.compact_n > 0:
        nc = args.compact_n
        pc = box(nc, args.sub_n, seed=1 + rank, visc_compact=1)
        ctx = N.nopcs_init([pc], prec=N.NOPCS_MIXED, stream=st)
        N.nopcs_rk_step(ctx, 1)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        N.nopcs_rk_step(ctx, args.compact_steps)
        e1.record(stream)
        barrier()
        mc = rank_max(e0.elapsed_time(e1))
        N.nopcs_set_profiling(ctx, True)
        N.nopcs_profile_read(ctx, reset=True)
        N.nopcs_rk_step(ctx, 1)
        pr = N.nopcs_profile_read(ctx, reset=True)
        N.nopcs_set_profiling(ctx, False)
        N.nopcs_destroy(ctx)
        ptc = float(nc) ** 3
        kc = {}
        for k, (kms, kn) in pr.items():
            if not kn:
                continue
            ent = {"ms_per_launch": kms / kn, "launches": kn}
            if k in ALG_BYTES_MIXED and k != "filter":
                gbs = ALG_BYTES_MIXED[k] * ptc / (kms / kn * 1e-3) / 1e9
                ent.update(alg_bytes_per_point=ALG_BYTES_MIXED[k], achieved_gbs=gbs, frac=gbs / hbm)
            kc[k] = ent
        compact = {"value": world * ptc * 4 * args.compact_steps / (mc * 1e-3), "unit": UNIT, "grid": [nc] * 3,
                   "steps": args.compact_steps, "ms_per_step": mc / args.compact_steps, "kernels": kc,
                   "explicit_over_compact": value / (world * ptc * 4 * args.compact_steps / (mc * 1e-3))}

    # the derivative microbenchmark (512^3) and the 64-box batched workload,
    # in short runs: best case per form, and the batched rate
    deriv = None
    batched = None
    if args.extra:
        torch.cuda.empty_cache()
        rows, pk = deriv_rows(N, 10, 3)
        deriv = {"grid": [512] * 3, "metric": "NOHAP first derivative of one field, ms per call", "steps": 10,
                 "hbm_peak_gbs": pk["hbm"], "tf32_peak_tflops": pk["tf32_peak"],
                 "bf16_peak_tflops": pk["bf16_peak"], "best": deriv_summary(rows)}
        bn, bms, binit, btuned = batched_run(N, 20, 3, 1)
        _, bms_g, _, _ = batched_run(N, 20, 3, 0)
        batched = {"value": world * bn * 4 * 20 / (bms * 1e-3), "unit": UNIT, "points": bn, "steps": 20,
                   "ms_per_step": bms / 20, "init_s": binit, "tuned_sub_n": btuned,
                   "launch": "one persistent kernel per step (all boxes, device work list)",
                   "graph_launch": {"value": world * bn * 4 * 20 / (bms_g * 1e-3), "ms_per_step": bms_g / 20,
                                    "launch": "one CUDA graph per step, one branch per box"},
                   "workload": "64 uneven two-temperature boxes, edges 32-128, heights 1-2x edge, dT 50-250 K, "
                               "seed 11"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, dt, cores = run_cpu_oracle(args.cpu_n, args.cpu_steps)
        rate1, dt1, cores1 = run_cpu_oracle(args.cpu1_n, args.cpu1_steps, threads=1)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "FP64 CPU oracle, %d RK4 steps of a %d^3 box of the same physics (base-subtracted), "
                         "%.1f s" % (args.cpu_steps, args.cpu_n, dt),
               "one_core": {"value": rate1, "unit": UNIT, "cores": cores1,
                            "sample": "%d RK4 steps of a %d^3 box, %.1f s" % (args.cpu1_steps, args.cpu1_n, dt1)}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32/f64", "data": "synthetic",
            "config": {"workload": workload_name(n, args.sub_n) if not args.shape else
                       workload_name(n, args.sub_n).replace("%d^3" % n, "x".join(map(str, shape))),
                       "grid": list(shape), "sub_n": args.sub_n, "precision": "mixed", "form": "thomas",
                       "sweep_tile_lines": tile_lines, "launch": "CUDA graph replay, one graph per RK4 step",
                       "filters_in_window": filters_in_window,
                       "l2": "inputs larger than L2 (FP64 state %.1f GB)" % (40 * npts / 1e9),
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic, "peak_kind": peak_kind,
                         "alg_bytes_per_point": ALG_BYTES_MIXED[dom], "avg_launch_ms": avg_ms,
                         "timing": "CUDA events around each launch, %d-step window of direct launches" % KP},
            "whole_step": whole_step,
            "kernels": per_kernel,
            "gpu_launches": gpu_launches,
            "e2e": e2e,
            "fp64_form": fp64,
            "compact_viscous_form": compact,
            "deriv_microbench": deriv,
            "batched_64_boxes": batched,
            "cpu_baseline": cpu,
            "clocks": clk,
            "diagnostics": {"step": diag["step"], "max_speed": diag["max_speed"], "max_dp": diag["max_dp"]},
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

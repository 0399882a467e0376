"""Benchmark: fine DOF-solves/s of the two-grid GMsFEM-preconditioned PCG.

Workload (one "step" = one solve: Section 3 preprocessing + PCG to relative
residual 1e-8 + velocity update and pressure):
  256 x 256 RT0/P0 grid, 16 x 16-cell coarse blocks, kappa = exp(Gaussian field,
  variance 4, correlation length 0.05) with horizontal channels at 1e6,
  quarter five-spot source, eigenvalue tolerance 10, eta 0.2, overlap 2.
The headline arm runs the mixed-precision preconditioner (BF16 patch inverses
and coarse basis, FP32 arithmetic inside the two-grid cycle, flexible CG);
outer vectors, dot products, fine operator and coarse matrix are FP64.  The
FP32 arm (FP32 storage) and the plain FP64 arm (the same code with FP64
everywhere) are reported beside it.  DOF per solve =
2n(n-1) + n^2 + 1 (interior faces + cells + one pressure constraint).

Inputs are resident on the device when a timed step starts; L2 is flushed
(256 MiB write) before every timed step, outside the timed interval.  Every
step is timed with CUDA events on the solver's stream.  `e2e` repeats the
headline arm through the host-pointer C ABI (host -> device copy of f and
device -> host copy of ux, uy, p inside every timed call).

The default line also carries, for one GPU:
  comparisons.batch_64x4: 64 instances (n in {64,128,256,512}, b in {8,16},
    channels at 10^U(4,6)) x 4 right-hand sides in one graph launch per
    step: learned coarse space + FP16 preconditioner (networks trained here
    for b = 8 and 16), exact spectral space + FP16, and plain FP64 exact;
  comparisons.n1024_b16: 1024^2, b = 16, held-out exp(GRF) + 1e6 channel
    field: learned (network trained here on 25 fields, 201 600 faces) and
    exact with the FP16 preconditioner against plain FP64 exact, plus the
    smoother's roofline at that size (its factors stream from HBM);
  comparisons.impes_512: two-phase IMPES at 512^2 (b = 16, channels 1e5),
    200 steps with the FP16 preconditioner: the coarse space of the first
    setup kept with low-rank inverse updates (the paper's choice) against
    the space rebuilt every step by the learned network (trained here on
    other channel fields, exact fallback per face).
With the oracle legs (unless --no-cpu-baseline): cpu_baseline, the oracle's
full solve on every host core (one core beside it), and the GPU solutions
checked against the oracle: error_vs_oracle (relative l2 and energy-norm
velocity error and l2 pressure error against its sparse direct solve) for
the headline arm and a sample of the batch, and the properties that fix the
solution (mass balance, momentum equation, zero-mean pressure, evaluated
with its matrices) for the 1024^2 arms.

--impl reference times the FP64 CPU oracle (test infrastructure of this
repository) on the host cores: each step is one oracle PCG iteration on the
same workload, and the throughput uses the oracle's own preprocessing,
iteration count and pressure times measured once in warm-up; ms_per_step is
the solve time this extrapolates to.
"""

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

METRIC = "fine DOF-solves/s to 1e-8 rel. residual vs plain FP64; PCG iters; HBM %"
N_DEFAULT, B_DEFAULT, CONTRAST, EIG_TOL, RTOL = 256, 16, 1e6, 10.0, 1e-8
# DRAM bytes per smoother launch (ncu dram__bytes_read.sum + dram__bytes_write.sum,
# mean over the captured launches of both sweeps) of the current kernels:
# 256 x 256 BF16 dense shape 2 and tensor-core shape 8, and 1024 x 1024 FP16
# handle with the band form
SMOOTHER_TRAFFIC = {("bf16", 2): 66.51e6, ("bf16", 8): 68.50e6, ("f16", 7): 296.39e6}


def dof(n):
    return 2 * n * (n - 1) + n * n + 1


def workload(n, seed):
    from paper_1807_07220_gb300 import inputs
    return inputs.grf_channel_field(n, CONTRAST, seed), inputs.quarter_five_spot(n)


def workload_name(n, b):
    return ("%dx%d RT0/P0, %dx%d-cell coarse blocks, kappa = exp(GRF var 4, corr 0.05) + channels 1e6, "
            "quarter five-spot, eig tol 10, rtol 1e-8" % (n, n, b, b))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu, self.proc, self.lines = gpu, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- our arm
def time_solves(solver, f, steps, warmup, flush, torch):
    """Per-step CUDA-event times (ms) of steps solves; L2 flushed before each."""
    stream = solver.stream
    for _ in range(warmup):
        solver.solve(f, rtol=RTOL)
    times, reps = [], []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it, rep = solver.solve(f, rtol=RTOL)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        reps.append(rep)
    return times, reps


def band_smoother_bytes(n, b, ov, tc_bytes):
    """Algorithmic bytes of one band-smoother launch (tile shape 7): every
    patch's band Cholesky factor read once by each triangular solve (n_loc
    rows of w + 1 entries, w = n_x + 1), the residual gathered and the
    correction scattered."""
    total = 0
    nc = n // b
    for J in range(nc):
        for I in range(nc):
            nx = min(n, (I + 1) * b + ov) - max(0, I * b - ov) - 1
            ny = min(n, (J + 1) * b + ov) - max(0, J * b - ov) - 1
            m = nx * ny
            total += 2 * m * (nx + 2) * tc_bytes + m * 8 + 2 * m * tc_bytes
    return total


FP64_PEAK_GFLOPS = 1250.0   # nominal dense FP64 rate of the part


def measured_fp64_gflops(torch):
    """The part's FP64 rate as a cuBLAS DGEMM reaches it (4096^3, best of 5
    timed with CUDA events after one warm-up); None without a GPU."""
    try:
        a = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
        b = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
        torch.matmul(a, b)
        best = None
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        del a, b
        return 2.0 * 4096 ** 3 / (best / 1e3) / 1e9
    except Exception:
        return None


def operator_roofline(n, tc_bytes, op_ms, op_n, peaks, peak_src, fp64_gflops=None):
    """Roofline of the PCG operator kernel (p = z + beta p, q = K p, (p, q),
    alpha), timed with events around each launch.  On this part it is bound
    by the FP64 pipe, so its arithmetic is reported against the FP64 rate a
    cuBLAS DGEMM measures in the same run (the nominal 1.25 TFLOP/s when that
    is unavailable) and its bytes against the measured copy bandwidth.
    Algorithmic FP64 work: 9 FMAs of K p per interior node, plus one FMA for p
    and one for (p, q) per node; bytes: z (TC), p_old, five coefficient arrays
    read, p_new, q (FP64) and the cleared z_next (TC) written, per node."""
    if not op_n:
        return None
    sec = op_ms / op_n / 1e3
    flops = 2.0 * (9 * (n - 1) ** 2 + 2 * n * n)
    nbytes = float(n * n * (2 * tc_bytes + 8 + 40 + 16))
    gflops = flops / sec / 1e9
    gbs = nbytes / sec / 1e9
    peak = fp64_gflops or FP64_PEAK_GFLOPS
    return {"kernel": "k_pcg_apply_p", "bound": "fp64", "achieved": gflops, "peak": peak,
            "unit": "GFLOP/s", "frac": gflops / peak,
            "peak_source": "measured (cuBLAS DGEMM 4096^3 in this run)" if fp64_gflops
            else "nominal FP64 rate (1.25 TFLOP/s)",
            "frac_of_nominal_fp64": gflops / FP64_PEAK_GFLOPS,
            "hbm_achieved": gbs, "hbm_peak": peaks.get("hbm_gbs"),
            "hbm_frac": gbs / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None, "hbm_peak_source": peak_src,
            "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": nbytes,
            "avg_launch_us": sec * 1e6, "launches_timed": op_n}


def smoother_bytes(n, b, ov, ts_bytes, tc_bytes):
    """Algorithmic bytes of one smoother launch: every patch inverse read once
    (nloc^2 entries), the residual gathered (FP64 or TC) and the correction
    scattered (read + write, TC)."""
    total = 0
    nc = n // b
    for J in range(nc):
        for I in range(nc):
            nx = min(n, (I + 1) * b + ov) - max(0, I * b - ov) - 1
            ny = min(n, (J + 1) * b + ov) - max(0, J * b - ov) - 1
            m = nx * ny
            total += m * m * ts_bytes + m * 8 + 2 * m * tc_bytes
    return total


def whole_job_rate(ms_list, dof_per_solve, world, distributed, device):
    """Whole-job DOF-solves/s of `world` replicas that each timed len(ms_list)
    solves: every rank's solves over the slowest rank's summed time (the max
    over ranks, one all-reduce of the initialised default process group when
    `distributed`).  Returns (DOF-solves/s, ms per step of the slowest rank)."""
    total_ms = sum(ms_list)
    if distributed:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * len(ms_list) * dof_per_solve / (total_ms / 1e3), total_ms / len(ms_list)


def run_ncu_target(args):
    """Setup, warm-up and timed solves of the headline arm only (the command
    profiled by ncu; prints the solver report of the last solve)."""
    import torch
    from paper_1807_07220_gb300 import tgms
    n, b = args.n, args.b
    kappa, f = workload(n, 5)
    s = tgms.Solver(kappa, b, EIG_TOL, precision=args.precision, flexible=int(args.precision != "f64"),
                    profile=int(args.profile_loop), smoother_shape=args.shape, coarse_solver=args.coarse_solver)
    for _ in range(args.warmup + args.steps):
        it, rep = s.solve(f, rtol=RTOL)
    torch.cuda.synchronize()
    s.close()
    print(json.dumps(rep.as_dict()))


def run_ours(args):
    import numpy as np
    import torch
    from paper_1807_07220_gb300 import build, tgms

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if not os.path.exists(tgms.LIB_PATH):
        if rank == 0:
            build.build_library()
        if dist:
            dist.barrier()
    n, b = args.n, args.b
    kappa, f = workload(n, 5 + rank)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MiB
    prec = args.precision

    def make(precision, flexible, profile=0, pointer_mode=1, **kw):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = tgms.Solver(kappa, b, EIG_TOL, precision=precision, flexible=flexible, profile=profile,
                        pointer_mode=pointer_mode, coarse_solver=args.coarse_solver, **kw)
        torch.cuda.synchronize()
        return s, (time.perf_counter() - t0) * 1e3

    # plain FP64 reference arm of the metric, and the other mixed arm
    plain, plain_setup_ms = make("f64", 0)
    p_times, p_reps = time_solves(plain, f, args.steps, args.warmup, flush, torch)
    plain.close()
    others = {}
    for other in ("f32", "bf16", "f16"):
        if other == prec:
            continue
        oth, oth_setup_ms = make(other, 1)
        o_times, o_reps = time_solves(oth, f, args.steps, args.warmup, flush, torch)
        oth.close()
        others[other] = (o_times, o_reps, oth_setup_ms)
    # headline mixed-precision arm, timed region with clock sampling
    head, setup_ms = make(prec, 1, smoother_shape=args.shape)
    for _ in range(args.warmup):
        head.solve(f, rtol=RTOL)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    times, reps = time_solves(head, f, args.steps, 0, flush, torch)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    # the last timed solve (rtol 1e-8), checked against the oracle after the timing
    checks = {"headline": dict(n=n, b=b, kappa=kappa, f=f, direct=True, p=head.p.cpu().numpy().ravel(),
                               u=np.concatenate([head.ux.cpu().numpy().ravel(), head.uy.cpu().numpy().ravel()]))}
    head.close()
    # roofline of the dominant kernel (patch smoother): events around every launch
    shape = reps[-1].smoother_shape
    prof, _ = make(prec, 1, profile=1, smoother_shape=shape)
    _, prof_reps = time_solves(prof, f, args.steps, args.warmup, flush, torch)
    prof.close()
    sm_ms = sum(r.smoother_ms for r in prof_reps)
    sm_n = sum(r.smoother_launches for r in prof_reps)
    op_ms = sum(r.operator_ms for r in prof_reps)
    op_n = sum(r.operator_launches for r in prof_reps)
    ts_bytes = {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}[prec]
    tc_bytes = 8 if prec == "f64" else 4
    band = shape in (7, 9)   # the band forms (register or shared-memory read-ahead)
    alg_bytes = band_smoother_bytes(n, b, 2, tc_bytes) if band else smoother_bytes(n, b, 2, ts_bytes, tc_bytes)
    # end to end through the host-pointer ABI (copies inside the timed call)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    h = tgms.tg_setup(pin(kappa), n, b, EIG_TOL, 2,
                      tgms.default_options(precision=prec, flexible=1, pointer_mode=tgms.PTR_HOST,
                                           coarse_solver=args.coarse_solver),
                      torch.cuda.current_stream().cuda_stream)
    hf = pin(f)
    hux, huy, hp = pin(np.zeros((n, n + 1))), pin(np.zeros((n + 1, n))), pin(np.zeros((n, n)))
    for _ in range(args.warmup):
        tgms.tg_solve(h, hf, None, RTOL, hux, huy, hp)
    e2e_t = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tgms.tg_solve(h, hf, None, RTOL, hux, huy, hp)
        e2e_t.append((time.perf_counter() - t0) * 1e3)
    tgms.tg_destroy(h)

    def agg(ms_list):
        return whole_job_rate(ms_list, dof(n), world, dist is not None, "cuda")

    peaks, peak_src = measured_peaks()
    comp = None
    if world == 1 and not args.no_comparisons:
        comp = {"batch_64x4": compare_batch(args, tgms, torch, flush, checks),
                 "n1024_b16": compare_1024(args, tgms, torch, flush, checks, peaks, peak_src)}
        # two-phase flow: 512^2, 200 steps, the paper's frozen coarse space (low-rank inverse updates) and
        # the coarse space rebuilt every step by the learned network with exact fallback
        rec = impes_record(args, 512, 16, ["frozen", "rebuild_learned"], 200, prec="f16")
        comp["impes_512"] = {k: rec[k] for k in ("metric", "value", "unit", "ms_per_step", "config", "arms",
                                                  "headline_arm", "training")}

    value, ms_step = agg(times)
    p_value, p_ms = agg(p_times)
    other_arms = {}
    for other, (o_times, o_reps, oth_setup_ms) in others.items():
        o_value, o_ms = agg(o_times)
        other_arms[other] = {"value": o_value, "ms_per_step": o_ms, "iters": o_reps[-1].iters,
                             "setup_ms": oth_setup_ms, "tile_shape": o_reps[-1].smoother_shape}
    e_value, e_ms = agg(e2e_t)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    achieved = alg_bytes / (sm_ms / sm_n / 1e3) / 1e9 if sm_n else None
    line = {
        "metric": METRIC, "value": value, "unit": "DOF-solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+%s" % prec, "data": "synthetic",
        "config": {"workload": workload_name(n, b), "n": n, "b": b, "precision": prec, "flexible_cg": True,
                   "dof_per_solve": dof(n), "l2": "flushed before every timed step (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "iters": reps[-1].iters, "cond_estimate": reps[-1].cond_estimate,
        "rel_residual": reps[-1].rel_residual, "max_div_error": reps[-1].max_div_error,
        "coarse_dim": reps[-1].coarse_dim, "setup_ms": setup_ms,
        "plain_f64": {"value": p_value, "ms_per_step": p_ms, "iters": p_reps[-1].iters,
                      "setup_ms": plain_setup_ms},
        "other_precisions": other_arms,
        "speedup_vs_plain_f64": value / p_value,
        "gpu_launches": sum(r.kernel_launches for r in reps),
        "gpu_launches_per_step": reps[-1].kernel_launches,
        "roofline": {"bound": "hbm",
                     "kernel": "k_smoother_band (patch band solves)" if band else
                     "k_smoother_mma (patch inverse apply, tensor-core tiles)" if shape == 8 else
                     "k_smoother (patch inverse apply)",
                     "achieved": achieved, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                     "frac": (achieved / peaks["hbm_gbs"]) if achieved else None,
                     "traffic": SMOOTHER_TRAFFIC.get((prec, shape)),
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, cold cache",
                     "working_set": "%.0f MB of patch factors per sweep against a 129 MB L2: at %d^2 they stay "
                                    "L2-resident between sweeps, so the launch is L2/latency-bound and the HBM "
                                    "fraction is a lower bound of what the kernel could stream" % (alg_bytes / 1e6, n)
                     if alg_bytes < 100e6 else "%.0f MB per sweep, streamed from HBM" % (alg_bytes / 1e6),
                     "tile_shape": shape, "autotuner_us_per_shape": reps[-1].shape_times(),
                     "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_us": 1e3 * sm_ms / sm_n if sm_n else None,
                     "launches_timed": sm_n, "peak_source": peak_src},
        "operator_roofline": operator_roofline(n, tc_bytes, op_ms, op_n, peaks, peak_src,
                                               measured_fp64_gflops(torch)),
        "e2e": {"value": e_value, "unit": "DOF-solves/s", "ms_per_step": e_ms,
                "h2d_bytes_per_step": 8 * n * n, "d2h_bytes_per_step": 8 * (2 * n * (n + 1) + n * n)},
        "clocks": clk,
    }
    if comp is not None:
        line["comparisons"] = comp
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(n, b)
        try:
            res = oracle_checks(checks)
        except Exception as e:  # reported, never fatal for the GPU line
            res = {"error": str(e)[:300]}
        line["error_vs_oracle"] = res.get("headline", res)
        if comp is not None:
            for arm in comp["batch_64x4"]["arms"]:
                comp["batch_64x4"]["arms"][arm]["error_vs_oracle"] = {
                    k[len("batch_%s_" % arm):]: v for k, v in res.items() if k.startswith("batch_%s_" % arm)}
            for arm in comp["n1024_b16"]["arms"]:
                comp["n1024_b16"]["arms"][arm]["properties_vs_oracle"] = res.get("n1024_" + arm)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------- comparisons against plain FP64
def train_net(tgms, torch, n, b, kappa_of, seeds, steps, hidden, stream, k=4):
    """A network for block size b: labels from the exact spectral problems
    (Section 4.2) of the seeded fields kappa_of(seed), then ``steps`` Adam
    steps of 1024 faces with the library's own kernels.  Returns (Mlp, info)."""
    from paper_1807_07220_gb300 import inputs
    dev = "cuda"
    nc = n // b
    F = 2 * nc * (nc - 1)
    din, dout, npar = tgms.tg_mlp_shape(b, k, hidden)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X = torch.empty((len(seeds) * F, din), dtype=torch.bfloat16, device=dev)
    Q = torch.empty((len(seeds) * F, k, b), dtype=torch.float32, device=dev)
    for i, sd in enumerate(seeds):
        kap = torch.as_tensor(kappa_of(sd), dtype=torch.float64, device=dev)
        tgms.tg_face_data(kap, n, b, EIG_TOL, k, X[i * F:(i + 1) * F], Q[i * F:(i + 1) * F], stream=stream)
    torch.cuda.synchronize()
    label_s = time.perf_counter() - t0
    params = torch.as_tensor(inputs.mlp_init_params(din, dout, hidden, 17), device=dev)
    net = tgms.Mlp(b, k, hidden, params, stream=stream)
    order = torch.as_tensor(inputs.sample_order(X.shape[0], steps, 1024, 23), device=dev)
    hist = torch.zeros(steps, dtype=torch.float32, device=dev)
    t0 = time.perf_counter()
    net.train(X, Q, order, steps, 1024, 1e-3, hist)
    torch.cuda.synchronize()
    info = {"b": b, "fields": len(seeds), "field_n": n, "samples": int(X.shape[0]), "steps": steps,
            "label_s": label_s, "train_s": time.perf_counter() - t0,
            "loss_last": float(hist[-min(50, steps):].mean().item())}
    del X, Q
    return net, info


def arm_record(dof_total, times, setup_s):
    ms = statistics.mean(times)
    return {"value": dof_total / (ms / 1e3), "ms_per_step": ms, "setup_s": setup_s,
            "value_with_setup": dof_total / (ms / 1e3 + setup_s)}


def compare_batch(args, tgms, torch, flush, checks):
    """The 64-instance x 4-right-hand-side workload (n from {64, 128, 256,
    512}, b from {8, 16}, channels at 10^U(4,6), one random source/sink pair
    per right-hand side) in one graph launch per step: learned coarse space
    with the row-scaled FP16 preconditioner (networks for b = 8 and b = 16
    trained on other channel fields), the exact spectral space with the same
    preconditioner, and the plain FP64 exact path in the same batched form."""
    import numpy as np
    from paper_1807_07220_gb300 import inputs
    dev = "cuda"
    stream = torch.cuda.current_stream().cuda_stream
    specs = batch_specs(64)
    nrhs = 4
    ns, bs = [sp[0] for sp in specs], [sp[1] for sp in specs]
    kappas = [inputs.channel_field(n, c, seed) for n, b, c, seed in specs]
    kd = [torch.as_tensor(k, dtype=torch.float64, device=dev).contiguous() for k in kappas]
    fs_h = [inputs.random_pairs(n, 1, 7 * seed + r) for (n, b, c, seed) in specs for r in range(nrhs)]
    fs = [torch.as_tensor(f, dtype=torch.float64, device=dev).contiguous() for f in fs_h]
    z = lambda *sh: torch.zeros(*sh, dtype=torch.float64, device=dev)
    ux = [z(n, n + 1) for n in ns for _ in range(nrhs)]
    uy = [z(n + 1, n) for n in ns for _ in range(nrhs)]
    pp = [z(n, n) for n in ns for _ in range(nrhs)]
    total_dof = sum(dof(n) for n in ns) * nrhs
    rng = np.random.default_rng(2025)
    contrast = {sd: float(10.0 ** rng.uniform(4, 6)) for sd in range(7000, 7016)}
    nets, training = [], []
    for b, seeds in ((8, range(7000, 7004)), (16, range(7004, 7016))):
        net, info = train_net(tgms, torch, 512, b, lambda sd: inputs.channel_field(512, contrast[sd], sd),
                              list(seeds), args.train_steps, args.hidden, stream)
        nets.append(net)
        training.append(info)
    # one problem per grid side up to 256 (its first right-hand side) against the direct solve
    sample = {}
    for i, n in enumerate(ns):
        if n <= 256 and n not in sample:
            sample[n] = i
    steps = max(1, min(args.steps, args.ns_steps))
    arms = {}
    for name, opt in (("learned_f16", dict(precision="f16", flexible=1, coarse_space="learned", batch_nets=nets)),
                      ("exact_f16", dict(precision="f16", flexible=1)),
                      ("exact_f64", dict(precision="f64", flexible=0))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        batch = tgms.tg_setup_batch(kd, ns, bs, EIG_TOL, nrhs, options=tgms.default_options(**opt), stream=stream)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        try:
            for _ in range(args.warmup):
                tgms.tg_solve_batch(batch, fs, None, RTOL, ux, uy, pp)
            times = []
            for _ in range(steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                iters, status = tgms.tg_solve_batch(batch, fs, None, RTOL, ux, uy, pp)
                e1.record()
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
        finally:
            tgms.tg_destroy_batch(batch)
        rec = arm_record(total_dof, times, setup_s)
        rec.update(iters_min_mean_max=[int(iters.min()), float(iters.mean()), int(iters.max())],
                   all_converged=bool((status == 0).all()), steps_timed=steps)
        arms[name] = rec
        for n, i in sample.items():
            j = i * nrhs
            checks["batch_%s_n%d" % (name, n)] = dict(
                n=n, b=bs[i], kappa=kappas[i], f=fs_h[j], direct=True,
                u=np.concatenate([ux[j].cpu().numpy().ravel(), uy[j].cpu().numpy().ravel()]),
                p=pp[j].cpu().numpy().ravel())
    for net in nets:
        net.close()
    return {"workload": "64 instances x 4 right-hand sides, n in {64,128,256,512}, b in {8,16}, channels at "
                        "10^U(4,6), one random source/sink pair per rhs, rtol 1e-8, one CUDA graph launch per "
                        "step, L2 flushed before each", "dof_per_step": total_dof, "arms": arms,
            "training": training, "error_sample": {str(n): "instance %d (b = %d), first rhs" % (i, bs[i])
                                                    for n, i in sample.items()},
            "learned_f16_vs_exact_f64": arms["learned_f16"]["value"] / arms["exact_f64"]["value"],
            "learned_f16_vs_exact_f64_with_setup":
                arms["learned_f16"]["value_with_setup"] / arms["exact_f64"]["value_with_setup"]}


def compare_1024(args, tgms, torch, flush, checks, peaks, peak_src):
    """1024 x 1024, 16 x 16-cell blocks, exp(GRF) + 1e6 channels (held-out
    field): the learned coarse space (network trained on 25 other seeded
    fields, 201 600 faces) and the exact spectral space with the row-scaled
    FP16 preconditioner, against the plain FP64 exact path.  Also the
    roofline of the smoother at this size, where its factors (hundreds of MB)
    stream from HBM on every sweep."""
    import numpy as np
    from paper_1807_07220_gb300 import inputs
    n, b = 1024, 16
    stream = torch.cuda.current_stream().cuda_stream
    net, training = train_net(tgms, torch, n, b, lambda sd: inputs.grf_channel_field(n, CONTRAST, sd),
                              list(range(5000, 5000 + args.train_fields)), args.train_steps, args.hidden, stream)
    kappa, f = workload(n, 4242)
    kd = torch.as_tensor(kappa, dtype=torch.float64, device="cuda")
    steps = max(1, min(args.steps, args.ns_steps))
    arms = {}
    shape16 = None
    for name, kw in (("learned_f16", dict(precision="f16", flexible=1, coarse_space="learned", net=net)),
                     ("exact_f16", dict(precision="f16", flexible=1)),
                     ("exact_f64", dict(precision="f64", flexible=0))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = tgms.Solver(kd, b, EIG_TOL, **kw)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        times, reps = time_solves(s, f, steps, args.warmup, flush, torch)
        r = reps[-1]
        rec = arm_record(dof(n), times, setup_s)
        rec.update(iters=r.iters, rel_residual=r.rel_residual, coarse_unknowns=r.coarse_unknowns,
                   snapshot_solves=r.snapshot_solves, fallback_faces=r.fallback_faces,
                   smoother_shape=r.smoother_shape, steps_timed=steps)
        arms[name] = rec
        if name == "exact_f16":
            shape16 = r.smoother_shape
        checks["n1024_" + name] = dict(n=n, b=b, kappa=kappa, f=f, direct=False,
                                       u=np.concatenate([s.ux.cpu().numpy().ravel(), s.uy.cpu().numpy().ravel()]),
                                       p=s.p.cpu().numpy().ravel())
        s.close()
    net.close()
    # smoother roofline at 1024^2: events around every launch of a profiled run of the FP16 arm
    prof = tgms.Solver(kd, b, EIG_TOL, precision="f16", flexible=1, profile=1, smoother_shape=shape16)
    _, prof_reps = time_solves(prof, f, 2, 1, flush, torch)
    prof.close()
    sm_ms = sum(r.smoother_ms for r in prof_reps)
    sm_n = sum(r.smoother_launches for r in prof_reps)
    band = shape16 in (7, 9)
    alg = band_smoother_bytes(n, b, 2, 4) if band else smoother_bytes(n, b, 2, 2, 4)
    ach = alg / (sm_ms / sm_n / 1e3) / 1e9 if sm_n else None
    roof = {"bound": "hbm", "kernel": "k_smoother_band (patch band solves)" if band else "k_smoother",
            "achieved": ach, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
            "frac": ach / peaks["hbm_gbs"] if ach else None, "traffic": SMOOTHER_TRAFFIC.get(("f16", shape16)),
            "tile_shape": shape16, "algorithmic_bytes_per_launch": alg,
            "avg_launch_us": 1e3 * sm_ms / sm_n if sm_n else None, "launches_timed": sm_n, "peak_source": peak_src}
    return {"workload": workload_name(n, b) + " (field seed 4242, held out of training)", "dof_per_solve": dof(n),
            "arms": arms, "training": training, "smoother_roofline": roof,
            "learned_f16_vs_exact_f64": arms["learned_f16"]["value"] / arms["exact_f64"]["value"],
            "learned_f16_vs_exact_f16": arms["learned_f16"]["value"] / arms["exact_f16"]["value"],
            "learned_f16_vs_exact_f64_with_setup":
                arms["learned_f16"]["value_with_setup"] / arms["exact_f64"]["value_with_setup"]}


# ---------------------------------------------------------------- batched workload
def batch_specs(ninst, seed=2024):
    """64 instances: side n from {64, 128, 256, 512}, block b from {8, 16},
    contrast 10^U(4, 6), own channel field."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for i in range(ninst):
        n = int(rng.choice([64, 128, 256, 512]))
        b = int(rng.choice([8, 16]))
        out.append((n, b, float(10.0 ** rng.uniform(4, 6)), 1000 + i))
    return out


def run_batch(args):
    """One step = tg_solve_batch over all instances x right-hand sides (one
    CUDA graph launch; the right-hand sides of an instance in lock step);
    compared with independent chains in the same graph and with the same
    problems solved one by one."""
    import numpy as np
    import torch
    from paper_1807_07220_gb300 import inputs, tgms
    torch.cuda.set_device(0)
    dev = "cuda"
    specs = batch_specs(args.batch_instances)
    nrhs = args.batch_rhs
    prec = args.precision
    kappas = [torch.as_tensor(inputs.channel_field(n, c, seed), dtype=torch.float64, device=dev).contiguous()
              for n, b, c, seed in specs]
    stream = torch.cuda.current_stream().cuda_stream
    fs, ux, uy, pp = [], [], [], []
    for (n, b, c, seed) in specs:
        for r in range(nrhs):
            fs.append(torch.as_tensor(inputs.random_pairs(n, 1, 7 * seed + r), dtype=torch.float64,
                                      device=dev).contiguous())
            ux.append(torch.zeros(n, n + 1, dtype=torch.float64, device=dev))
            uy.append(torch.zeros(n + 1, n, dtype=torch.float64, device=dev))
            pp.append(torch.zeros(n, n, dtype=torch.float64, device=dev))
    total_dof = sum(dof(n) for (n, b, c, seed) in specs) * nrhs
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def timed_batch(lockstep):
        opts = tgms.default_options(precision=prec, flexible=1, batch_lockstep=lockstep)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        batch = tgms.tg_setup_batch(kappas, [s[0] for s in specs], [s[1] for s in specs], EIG_TOL, nrhs,
                                    options=opts, stream=stream)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        try:
            for _ in range(args.warmup):
                tgms.tg_solve_batch(batch, fs, None, RTOL, ux, uy, pp)
            times = []
            for _ in range(args.steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                iters, status = tgms.tg_solve_batch(batch, fs, None, RTOL, ux, uy, pp)
                e1.record()
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
        finally:
            tgms.tg_destroy_batch(batch)
        return times, iters, status, setup_s

    times, iters, status, setup_s = timed_batch(1)
    times_ind, iters_ind, status_ind, _ = timed_batch(0)
    # the same problems one solve at a time (one graph launch each)
    seq_ms = 0.0
    seq_iters = []
    j = 0
    for (n, b, c, seed), k in zip(specs, kappas):
        s = tgms.Solver(k, b, EIG_TOL, precision=prec, flexible=1)
        for r in range(nrhs):
            for _ in range(2):
                s.solve(fs[j], rtol=RTOL)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            it, _ = s.solve(fs[j], rtol=RTOL)
            e1.record()
            e1.synchronize()
            seq_ms += e0.elapsed_time(e1)
            seq_iters.append(it)
            j += 1
        s.close()
    ms = statistics.mean(times)
    line = {
        "metric": METRIC + " (batched)", "value": total_dof / (ms / 1e3), "unit": "DOF-solves/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+%s" % prec, "data": "synthetic",
        "config": {"workload": "%d instances x %d right-hand sides, n in {64,128,256,512}, b in {8,16}, "
                               "channels at 10^U(4,6), random source/sink pair per rhs, "
                               "one CUDA graph launch per step" % (len(specs), nrhs),
                   "instances": [[n, b] for (n, b, c, seed) in specs], "dof_per_step": total_dof},
        "iters_min_mean_max": [int(iters.min()), float(iters.mean()), int(iters.max())],
        "all_converged": bool((status == 0).all()),
        "setup_s": setup_s,
        "sequential": {"value": total_dof / (seq_ms / 1e3), "ms_per_step": seq_ms,
                       "note": "same problems, one tg_solve graph launch each"},
        "speedup_vs_sequential": seq_ms / ms,
        "independent_chains": {"value": total_dof / (statistics.mean(times_ind) / 1e3),
                               "ms_per_step": statistics.mean(times_ind),
                               "iters_mean": float(iters_ind.mean()),
                               "all_converged": bool((status_ind == 0).all()),
                               "note": "same batch with batch_lockstep 0: every right-hand side its own chain"},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- learned coarse space
def run_learned(args):
    """Learned coarse space at 1024 x 1024 with 16 x 16 blocks: labels from the
    exact spectral problems of ``--train-fields`` seeded fields, GPU training
    with the library's kernels, then setup and solves on a held-out field with
    the exact and the learned coarse space (BF16 preconditioner) and the plain
    FP64 exact path."""
    import numpy as np
    import torch
    from paper_1807_07220_gb300 import inputs, tgms
    torch.cuda.set_device(0)
    dev = "cuda"
    n, b, k, hidden, tol = args.n, args.b, 4, args.hidden, EIG_TOL
    stream = torch.cuda.current_stream().cuda_stream
    nc = n // b
    F = 2 * nc * (nc - 1)
    din, dout, npar = tgms.tg_mlp_shape(b, k, hidden)
    # ---- training data
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X = torch.empty((args.train_fields * F, din), dtype=torch.bfloat16, device=dev)
    Q = torch.empty((args.train_fields * F, k, b), dtype=torch.float32, device=dev)
    for i in range(args.train_fields):
        kap = torch.as_tensor(inputs.grf_channel_field(n, CONTRAST, 5000 + i), dtype=torch.float64, device=dev)
        tgms.tg_face_data(kap, n, b, tol, k, X[i * F:(i + 1) * F], Q[i * F:(i + 1) * F], stream=stream)
    torch.cuda.synchronize()
    data_s = time.perf_counter() - t0
    # ---- training
    params = torch.as_tensor(inputs.mlp_init_params(din, dout, hidden, 17), device=dev)
    net = tgms.Mlp(b, k, hidden, params, stream=stream)
    nsteps, batch = args.train_steps, 1024
    order = torch.as_tensor(inputs.sample_order(X.shape[0], nsteps, batch, 23), device=dev)
    hist = torch.zeros(nsteps, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    net.train(X, Q, order, nsteps, batch, 1e-3, hist)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    h = hist.cpu().numpy()
    # ---- held-out field
    kappa, f = workload(n, 4242)
    kd = torch.as_tensor(kappa, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    arms = {}
    lp = args.learned_precision
    for name, kw in (("exact_" + lp, dict(precision=lp, flexible=1, coarse_space="gmsfem")),
                     ("learned_" + lp, dict(precision=lp, flexible=1, coarse_space="learned", net=net)),
                     ("exact_plain_f64", dict(precision="f64", flexible=0, coarse_space="gmsfem"))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = tgms.Solver(kd, b, tol, **kw)
        torch.cuda.synchronize()
        setup_ms = (time.perf_counter() - t0) * 1e3
        times, reps = time_solves(s, f, args.steps, args.warmup, flush, torch)
        ms = statistics.mean(times)
        r = reps[-1]
        arms[name] = {"value": dof(n) / (ms / 1e3), "ms_per_solve": ms, "iters": r.iters, "setup_ms": setup_ms,
                      "coarse_unknowns": r.coarse_unknowns, "velocity_basis": r.velocity_basis,
                      "snapshot_solves": r.snapshot_solves, "fallback_faces": r.fallback_faces,
                      "rel_residual": r.rel_residual}
        s.close()
    net.close()
    line = {
        "metric": METRIC + " (learned coarse space)", "value": arms["learned_" + lp]["value"], "unit": "DOF-solves/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": arms["learned_" + lp]["ms_per_solve"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+" + lp, "data": "synthetic",
        "config": {"workload": workload_name(n, b) + "; network %d-%d-%d-%d trained on %d fields (%d faces)"
                   % (din, hidden, hidden, dout, args.train_fields, X.shape[0]), "l2": "flushed between solves"},
        "arms": arms, "faces": F,
        "training": {"samples": int(X.shape[0]), "steps": nsteps, "batch": batch, "label_s": data_s,
                     "train_s": train_s, "loss_first": float(h[:20].mean()), "loss_last": float(h[-50:].mean())},
        "vs_exact_same_precision": arms["learned_" + lp]["value"] / arms["exact_" + lp]["value"],
        "vs_plain_f64": arms["learned_" + lp]["value"] / arms["exact_plain_f64"]["value"],
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- network GEMMs
def run_mlp(args):
    """The learned basis's network on the tensor cores (tcgen05 GEMMs): the
    forward pass over the faces of one 1024 x 1024 grid with 16 x 16 blocks
    (8 064 faces, 612 -> 512 -> 512 -> 64) and training steps of 1 024 faces,
    on random inputs of that shape, timed with CUDA events.  Work: 2 M (din h
    + h h + h dout) flops per forward pass over M faces, 2 B (2 din h + 3 h h
    + 3 h dout) per training step of B faces (forward plus the five backward
    GEMMs).  Each call includes its operand packing (row gathers, transposes,
    padding to the 16-byte TMA stride)."""
    import numpy as np
    import torch
    from paper_1807_07220_gb300 import inputs, tgms
    torch.cuda.set_device(0)
    dev = "cuda"
    b, k, hidden, F, batch = 16, 4, args.hidden, 8064, 1024
    din, dout, npar = tgms.tg_mlp_shape(b, k, hidden)
    g = torch.Generator(device="cpu").manual_seed(29)
    X = (torch.rand((F, din), generator=g) * 2 - 1).to(torch.bfloat16).to(dev)
    Q = torch.linalg.qr(torch.randn((F, b, k), generator=g))[0].transpose(1, 2).contiguous().to(dev,
                                                                                              torch.float32)
    params = torch.as_tensor(inputs.mlp_init_params(din, dout, hidden, 17), device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    net = tgms.Mlp(b, k, hidden, params, stream=stream)
    y = torch.zeros((F, dout), dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        net.forward(X, y)
    times = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        net.forward(X, y)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    fwd_ms = statistics.mean(times)
    fwd_flops = 2.0 * F * (din * hidden + hidden * hidden + hidden * dout)
    nsteps = 200
    order = torch.as_tensor(inputs.sample_order(F, nsteps * (args.steps + 1), batch, 23), device=dev)
    net.train(X, Q, order, nsteps, batch, 1e-3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    net.train(X, Q, order[nsteps * batch:], nsteps * args.steps, batch, 1e-3)
    e1.record()
    e1.synchronize()
    step_ms = e0.elapsed_time(e1) / (nsteps * args.steps)
    step_flops = 2.0 * batch * (2 * din * hidden + 3 * hidden * hidden + 3 * hidden * dout)
    net.close()
    peaks, src = measured_peaks()
    peak = peaks.get("bf16_tflops")
    fwd_tf = fwd_flops / (fwd_ms / 1e3) / 1e12
    line = {
        "metric": "network forward TFLOP/s (bf16 tcgen05 GEMMs, FP32 accumulation)", "value": fwd_tf,
        "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": fwd_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "%d faces x %d-%d-%d-%d perceptron (1024^2 grid, 16x16 blocks); training steps of "
                               "%d faces" % (F, din, hidden, hidden, dout, batch)},
        "roofline": {"bound": "tensor", "kernel": "k_gemm_tc (3 GEMMs + operand packing per forward pass)",
                     "achieved": fwd_tf, "peak": peak, "unit": "TFLOP/s",
                     "frac": fwd_tf / peak if peak else None, "peak_source": src + " bf16 burst"},
        "train_step_ms": step_ms, "train_tflops": step_flops / (step_ms / 1e3) / 1e12,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- two-phase IMPES
def run_impes(args):
    """Two-phase IMPES (Section 6.2) at 512 x 512 with 16 x 16 blocks:
    channels at 1e5, water injected in cell (0, 0) and produced in
    (n-1, n-1), mu_w = 1, mu_o = 5, CFL 0.5, args.impes_steps steps.  Arms:
    the coarse basis of the first setup kept (the paper's choice) with the
    coarse inverses updated by low-rank corrections ('frozen', the headline)
    or recomputed in full ('frozen_full'); the basis rebuilt every step from
    the exact spectral problems ('rebuild') or from the learned network with
    per-face exact fallback ('rebuild_learned', network trained beforehand on
    args.train_fields other seeded channel fields of the same size)."""
    line = impes_record(args, args.n, args.b, args.impes_arms.split(","), args.impes_steps)
    print(json.dumps(line), flush=True)


def impes_record(args, n, b, arm_names, nsteps, prec=None):
    """The IMPES line (see run_impes) as a dict, for the given arms."""
    prec = prec or args.precision
    import numpy as np
    import torch
    from paper_1807_07220_gb300 import inputs, tgms
    from paper_1807_07220_gb300.impes import Impes
    torch.cuda.set_device(0)
    k = 4
    dev = "cuda"
    stream = torch.cuda.current_stream().cuda_stream
    kap = torch.as_tensor(inputs.channel_field(n, 1e5, 77), dtype=torch.float64, device=dev)
    f = torch.as_tensor(inputs.quarter_five_spot(n), dtype=torch.float64, device=dev)
    nc = n // b
    F = 2 * nc * (nc - 1)
    net, training = None, None
    if "rebuild_learned" in arm_names:
        # ---- network for the learned rebuild: labels from other channel fields
        din, dout, npar = tgms.tg_mlp_shape(b, k, args.hidden)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        X = torch.empty((args.train_fields * F, din), dtype=torch.bfloat16, device=dev)
        Q = torch.empty((args.train_fields * F, k, b), dtype=torch.float32, device=dev)
        for i in range(args.train_fields):
            kt = torch.as_tensor(inputs.channel_field(n, 1e5, 6000 + i), dtype=torch.float64, device=dev)
            tgms.tg_face_data(kt, n, b, EIG_TOL, k, X[i * F:(i + 1) * F], Q[i * F:(i + 1) * F], stream=stream)
        params = torch.as_tensor(inputs.mlp_init_params(din, dout, args.hidden, 17), device=dev)
        net = tgms.Mlp(b, k, args.hidden, params, stream=stream)
        order = torch.as_tensor(inputs.sample_order(X.shape[0], args.train_steps, 1024, 23), device=dev)
        loss = torch.zeros(args.train_steps, dtype=torch.float32, device=dev)
        net.train(X, Q, order, args.train_steps, 1024, 1e-3, loss)
        torch.cuda.synchronize()
        training = {"fields": args.train_fields, "samples": int(X.shape[0]), "steps": args.train_steps,
                    "seconds": time.perf_counter() - t0, "loss_last": float(loss[-50:].mean())}
    arms = {}
    modes = {"frozen": dict(coarse="frozen"), "frozen_full": dict(coarse="frozen_full"),
             "rebuild": dict(coarse="rebuild"),
             "rebuild_learned": dict(coarse="rebuild", coarse_space="learned", net=net)}
    for name in arm_names:
        kw = modes[name]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim = Impes(kap, f, b, EIG_TOL, rtol=RTOL, precision=prec, flexible=1, **kw)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        torch.cuda.nvtx.range_push("impes_steps")
        for _ in range(nsteps):
            sim.step()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        wall = time.perf_counter() - t0
        hist = np.array(sim.history)
        water = float(sim.s.sum()) / n ** 2
        arms[name] = {"steps": sim.steps, "t_final": sim.t, "wall_s": wall, "steps_per_s": sim.steps / wall,
                      "setup_s": setup_s, "iters_mean": float(hist[:, 1].mean()), "iters_max": int(hist[:, 1].max()),
                      "update_ms_mean": float(hist[:, 2].mean()), "solve_ms_mean": float(hist[:, 3].mean()),
                      "transport_ms_mean": float(hist[:, 4].mean()),
                      "refactored_patch_frac_mean": float(hist[1:, 5].mean()) / nc ** 2 if sim.steps > 1 else 1.0,
                      "coarse_update_rank_mean": float(hist[1:, 6][hist[1:, 6] >= 0].mean())
                      if (hist[1:, 6] >= 0).any() else None,
                      "coarse_full_inverses": int((hist[1:, 6] < 0).sum()),
                      "snapshot_solves_per_space": float(hist[1:, 7].mean()) if sim.steps > 1 else 0.0,
                      "fallback_faces_mean": float(hist[1:, 8].mean()) if sim.steps > 1 else 0.0,
                      "pressure_dof_solves_per_s": dof(n) / (float(hist[:, 3].mean()) / 1e3),
                      "water_volume": water, "s_max": float(sim.s.max())}
        sim.close()
    if net is not None:
        net.close()
    head = "frozen" if "frozen" in arms else arm_names[0]
    return {
        "metric": "IMPES steps/s (pressure update + warm-started solve + transport)",
        "value": arms[head]["steps_per_s"], "unit": "steps/s", "n_gpus": 1, "steps": nsteps,
        "warmup": 0, "ms_per_step": 1e3 / arms[head]["steps_per_s"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+" + prec, "data": "synthetic",
        "config": {"workload": "%dx%d two-phase IMPES, %dx%d-cell blocks, channels 1e5, quarter five-spot, "
                               "mu_w 1, mu_o 5, CFL 0.5, rtol %g" % (n, n, b, b, RTOL)},
        "arms": arms, "faces": F, "headline_arm": head, "training": training,
    }


# ---------------------------------------------------------------- ablations
def run_ablation(args):
    """Robustness and parameter study at args.n x args.n with b x b blocks,
    quarter five-spot, rtol 1e-8, plain FP64 (standard CG, so N_iter and Cond
    are those of the method itself): (1) N_iter, Cond and Dim against the
    channel contrast (background 1, channels at 1, 1e2, 1e4, 1e6) for the
    GMsFEM, MsFEM and RT0 coarse spaces (the paper's Tables 1-6 experiment on
    synthetic channels); (2) at contrast 1e6 with GMsFEM, the smoother weight
    eta, the oversampling, the smoothing counts m1/m2 and the additive
    two-level Schwarz cycle against the two-grid cycle.  Each row times
    args.steps solves after args.warmup, L2 flushed before each."""
    import torch
    from paper_1807_07220_gb300 import inputs, tgms
    torch.cuda.set_device(0)
    n, b = args.n, args.b
    f = inputs.quarter_five_spot(n)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def row(kappa, overlap=2, **opts):
        kd = torch.as_tensor(kappa, dtype=torch.float64, device="cuda")
        t0 = time.perf_counter()
        s = tgms.Solver(kd, b, EIG_TOL, overlap=overlap, precision="f64", flexible=0, max_iter=4000, **opts)
        setup_s = time.perf_counter() - t0
        try:
            for _ in range(args.warmup):
                s.solve(f, rtol=RTOL, allow_maxiter=True)
            times = []
            for _ in range(args.steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s.stream)
                it, r = s.solve(f, rtol=RTOL, allow_maxiter=True)
                e1.record(s.stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
        finally:
            s.close()
        return {"iters": r.iters, "cond": r.cond_estimate, "dim": r.coarse_dim, "velocity_basis": r.velocity_basis,
                "ms_per_solve": statistics.mean(times), "setup_s": setup_s, "converged": r.converged}

    contrast = {}
    for c in (1.0, 1e2, 1e4, 1e6):
        kappa = inputs.channel_field(n, c, 31)
        contrast["%g" % c] = {cs: row(kappa, coarse_space=cs) for cs in ("gmsfem", "msfem", "rt0")}
    kappa = inputs.channel_field(n, 1e6, 31)
    params = {}
    for eta in (0.1, 0.2, 0.3, 0.5):
        params["eta=%g" % eta] = row(kappa, eta=eta)
    for ov in (1, 2):   # overlap 0 leaves the coarse grid lines in no patch: singular, rejected
        params["overlap=%d" % ov] = row(kappa, overlap=ov)
    for m1, m2 in ((1, 0), (1, 1), (2, 1), (2, 2)):
        params["m1=%d,m2=%d" % (m1, m2)] = row(kappa, m1=m1, m2=m2)
    params["additive"] = row(kappa, cycle="additive")
    head = contrast["1e+06"]["gmsfem"]
    line = {
        "metric": "PCG iterations to 1e-8 (robustness to contrast; preconditioner ablations)",
        "value": head["iters"], "unit": "PCG iterations", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": head["ms_per_solve"], "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "%dx%d RT0/P0, %dx%d-cell blocks, channel fields (background 1, seed 31), "
                               "quarter five-spot, eig tol 10, rtol 1e-8, plain FP64" % (n, n, b, b),
                   "l2": "flushed between solves"},
        "contrast": contrast, "params_at_1e6": params,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- oracle arms
ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, %(root)r)
import numpy as np
from oracle.twogrid import TwoGridSolver
from oracle.fine import boundary_lift
from paper_1807_07220_gb300 import inputs
n, b, mode, steps, warmup = %(n)d, %(b)d, %(mode)r, %(steps)d, %(warmup)d
kappa = inputs.grf_channel_field(n, 1e6, 5)
f = inputs.quarter_five_spot(n)
t0 = time.perf_counter()
s = TwoGridSolver(n, b, kappa, tol=10.0)
setup = time.perf_counter() - t0
out = {"setup_s": setup}
if mode == "full":
    t0 = time.perf_counter()
    res = s.solve(f, rtol=1e-8)
    out.update(solve_s=time.perf_counter() - t0, iters=res["iters"])
else:
    g = s.g
    F = g.h ** 2 * f.ravel()
    t0 = time.perf_counter(); vbar = s.preprocess(F, np.zeros(s.If.size)); t_pre = time.perf_counter() - t0
    res = s.solve(f, rtol=1e-8)
    t0 = time.perf_counter(); s.pressure(res["u"]); t_post = time.perf_counter() - t0
    r = s.project(-(s.AII @ vbar)); z = s.precondition(r); p = z.copy(); rz = r @ z
    x = np.zeros_like(r)
    it_times = []
    for k in range(warmup + steps):
        t0 = time.perf_counter()
        q = s.project(s.AII @ p); a = rz / (p @ q)
        x += a * p; r = r - a * q
        s.residual_norm(r)
        z = s.precondition(r); rz_new = r @ z; p = z + (rz_new / rz) * p; rz = rz_new
        if k >= warmup:
            it_times.append(time.perf_counter() - t0)
    out.update(t_pre=t_pre, t_post=t_post, iters=res["iters"], it_times=it_times)
print("ORACLE_JSON " + json.dumps(out))
"""


def host_cores():
    return os.cpu_count() or 1


def oracle_env(threads):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    return env


def run_oracle(n, b, mode, steps=0, warmup=0, timeout=900, threads=None):
    threads = threads or host_cores()
    code = ORACLE_SNIPPET % {"root": ROOT, "n": n, "b": b, "mode": mode, "steps": steps, "warmup": warmup}
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=oracle_env(threads),
                       timeout=timeout)
    for ln in r.stdout.splitlines():
        if ln.startswith("ORACLE_JSON "):
            return json.loads(ln[len("ORACLE_JSON "):])
    raise RuntimeError("oracle run failed: " + r.stderr[-2000:])


ORACLE_CHECK_SNIPPET = r"""
import json, sys
sys.path.insert(0, %(root)r)
import numpy as np
from oracle.fine import Grid, assemble, solve_direct_pinned
d = np.load(%(path)r)
out, cache = {}, {}
for name in %(names)r:
    n, b = int(d[name + "/n"]), int(d[name + "/b"])
    kappa, f, u, p = d[name + "/kappa"], d[name + "/f"], d[name + "/u"], d[name + "/p"]
    g = Grid(n, b)
    A, B = assemble(g, kappa)
    I = g.interior_faces()
    F = g.h ** 2 * f.ravel()
    Au = (A @ u)[I]
    r = {"n": n, "b": b,
         "mass": float(np.abs(B @ u - F).max() / np.abs(F).max()),
         "momentum": float(np.linalg.norm(Au - (B.T @ p)[I]) / np.linalg.norm(Au)),
         "mean_p": float(abs(p.sum()) / np.abs(p).sum())}
    if int(d[name + "/direct"]):
        key = (n, b, hash(kappa.tobytes()), hash(f.tobytes()))
        if key not in cache:
            cache[key] = solve_direct_pinned(g, kappa, f)
        us, ps = cache[key]
        e = u - us
        r.update(err_u_l2=float(np.linalg.norm(e) / np.linalg.norm(us)),
                 err_u_energy=float(np.sqrt(e @ (A @ e)) / np.sqrt(us @ (A @ us))),
                 err_p_l2=float(np.linalg.norm(p - ps) / np.linalg.norm(ps)))
    out[name] = r
print("ORACLE_JSON " + json.dumps(out))
"""


def oracle_checks(cases, timeout=900):
    """The GPU solutions in ``cases`` (name -> dict(n, b, kappa, f, u, p,
    direct)) checked with the oracle in a subprocess: the relative errors
    against its sparse direct solve (direct = True) and the properties that
    fix the discrete solution (mass balance per cell, momentum equation
    A u = B^T p on interior faces, sum(p) = 0), evaluated with its matrices."""
    import tempfile
    import numpy as np
    if not cases:
        return {}
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "cases.npz")
        arrs = {}
        for name, c in cases.items():
            for k in ("n", "b", "kappa", "f", "u", "p"):
                arrs[name + "/" + k] = np.asarray(c[k])
            arrs[name + "/direct"] = np.asarray(int(c.get("direct", False)))
        np.savez(path, **arrs)
        code = ORACLE_CHECK_SNIPPET % {"root": ROOT, "path": path, "names": sorted(cases)}
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                           env=oracle_env(host_cores()), timeout=timeout)
    for ln in r.stdout.splitlines():
        if ln.startswith("ORACLE_JSON "):
            return json.loads(ln[len("ORACLE_JSON "):])
    raise RuntimeError("oracle check failed: " + r.stderr[-2000:])


def cpu_baseline(n, b):
    """The oracle's full solve of the workload on the host cores: BLAS
    threads set to every core (the figure reported) and to one core (beside
    it).  The oracle's sparse LU and sparse products are single-threaded."""
    cores = host_cores()
    try:
        o = run_oracle(n, b, "full", threads=cores)
        o1 = run_oracle(n, b, "full", threads=1)
    except Exception as e:  # reported, never fatal for the GPU line
        return {"value": None, "error": str(e)[:200]}
    return {"value": dof(n) / o["solve_s"], "unit": "DOF-solves/s", "cores": cores, "kind": "oracle",
            "sample": "one full oracle solve (preprocessing + %d PCG iterations + pressure) of the same "
                      "workload, BLAS threads = %d host cores (SuperLU and sparse products single-threaded); "
                      "oracle setup (%.0f s) excluded" % (o["iters"], cores, o["setup_s"]),
            "solve_s": o["solve_s"],
            "one_core": {"value": dof(n) / o1["solve_s"], "solve_s": o1["solve_s"], "cores": 1}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n, b = args.n, args.b
    cores = host_cores()
    o = run_oracle(n, b, "iter", steps=args.steps, warmup=args.warmup, timeout=3000, threads=cores)
    t_iter = statistics.mean(o["it_times"])
    t_solve = o["t_pre"] + o["iters"] * t_iter + o["t_post"]
    value = dof(n) / t_solve
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF-solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_solve, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(n, b), "n": n, "b": b, "precision": "f64",
                   "dof_per_solve": dof(n)},
        "ms_per_pcg_iteration": 1e3 * t_iter,
        "cpu_baseline": {"value": value, "unit": "DOF-solves/s", "cores": cores, "kind": "oracle",
                         "sample": "each step = one oracle PCG iteration (operator, two preconditioner "
                                   "applications for the scalars, vector updates) on the same workload, "
                                   "BLAS threads = %d host cores; ms_per_step = the solve it extrapolates to: "
                                   "preprocessing %.2f s + %d iterations + pressure %.2f s"
                                   % (cores, o["t_pre"], o["iters"], o["t_post"])},
        "e2e": {"value": value, "unit": "DOF-solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--b", type=int, default=B_DEFAULT)
    ap.add_argument("--precision", default="bf16", choices=["f32", "bf16", "f16"])
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle legs (CPU baseline and the checks against the oracle)")
    ap.add_argument("--no-comparisons", action="store_true",
                    help="skip the batched and 1024^2 learned comparisons against plain FP64")
    ap.add_argument("--ns-steps", type=int, default=5, help="timed steps of each comparison arm")
    ap.add_argument("--workload", default="single",
                    choices=["single", "batch", "learned", "impes", "ablation", "mlp"])
    ap.add_argument("--impes-steps", type=int, default=200)
    ap.add_argument("--impes-arms", default="frozen,frozen_full,rebuild,rebuild_learned",
                    help="comma-separated IMPES arms (frozen, frozen_full, rebuild, rebuild_learned)")
    ap.add_argument("--train-fields", type=int, default=25)
    ap.add_argument("--train-steps", type=int, default=2000)
    ap.add_argument("--hidden", type=int, default=512)
    ap.add_argument("--learned-precision", default="f16", choices=["f32", "bf16", "f16"])
    ap.add_argument("--shape", type=int, default=-1, help="smoother tile shape (-1: autotune)")
    ap.add_argument("--coarse-solver", default="auto", choices=["auto", "dense", "nd"],
                    help="solver of the FP64 coarse system (auto: nested dissection above 2048 unknowns)")
    ap.add_argument("--batch-instances", type=int, default=64)
    ap.add_argument("--batch-rhs", type=int, default=4)
    ap.add_argument("--ncu-target", action="store_true", help="headline solves only (for ncu)")
    ap.add_argument("--profile-loop", action="store_true",
                    help="with --ncu-target: host-driven PCG loop instead of the graph (ncu sees each launch)")
    args = ap.parse_args()
    if args.ncu_target:
        return run_ncu_target(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "impes":
        run_impes(args)
    elif args.workload == "ablation":
        run_ablation(args)
    elif args.workload == "mlp":
        run_mlp(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

"""Benchmark: FC-SDNN grid-point-stage updates per second on one GB300,
batched FP32 (BF16 classifier) against the plain FP64 form, at a stated error.

Default workload (the batched-ensemble configuration): 32 independent Mach
2-4 forward-facing-step flows (channel [0,3] x [0,1], step of height 0.2 at
x = 0.6; inflow Mach uniform in [2, 4], resolutions log-uniform between 0.25M
and 2M points per flow, both seeded), each flow 64 overlapping patches of
uneven resolution with interpolated fringes, one L-shaped (C1) and one C2
corner patch, all flows in one layout so every launch covers all of them.
One "step" = one full time step of the hot path: proxy + windows +
classifier MLP, artificial viscosity, CFL time step, four Runge-Kutta stages
(FC derivatives of fluxes and viscous fluxes, operator, stage update, boundary
conditions), each followed by the fringe exchange.  Inputs are synthetic.

In one invocation: the FP32 arm (`value`), the plain FP64 form on the same
inputs (`fp64`), the FP32 result's error against the FP64 form after a
stated number of steps (`precision_error`), rooflines of the stage operator
and of the FC-derivative kernel against measured peaks, the end-to-end rate
through the C ABI with host copies (`e2e`) and the FP64 CPU oracle on the
host cores (`cpu_baseline`).  --workload sod|ffs|cylinder selects the other
layouts.  --impl reference times the oracle alone.  Prints one JSON line.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FC-SDNN grid-point-stage updates/s on 1 GB300, batched FP32 vs plain FP64, at set error"
UNIT = "pt-stage/s"
FALLBACK_HBM = 6800.0
FFS_H0 = 0.002      # forward-facing step: ~0.85M points in 64 patches per instance
CYL_H = 0.004       # cylinder: ~3.9M points in 260 patches


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--instances", type=int, default=None,
                    help="independent instances (sod: 128, ffs: 8, cylinder: 1; the ensemble is one layout)")
    ap.add_argument("--workload", default="ensemble", choices=["ensemble", "sod", "ffs", "cylinder"],
                    help="ensemble: 32 step flows of seeded resolutions (0.25M-2M points) and Mach numbers in one "
                         "layout (default); sod: the shock-tube batch; ffs: forward-facing steps with corner "
                         "patches; cylinder: Mach-10 flow past a cylinder (annular sectors + Cartesian far field)")
    ap.add_argument("--fp64-steps", type=int, default=None, help="timed steps of the FP64 arm (default steps/4, >= 3)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 arm and the error run")
    ap.add_argument("--flows", type=int, default=32, help="flows of the ensemble (32; fewer for small profiling runs)")
    ap.add_argument("--error-steps", type=int, default=20)
    ap.add_argument("--train-windows", type=int, default=10_000_000,
                    help="labelled classifier windows produced by the solver's FC step (training set)")
    ap.add_argument("--train-steps", type=int, default=3000, help="Adam steps of 4096 windows")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cpu-procs", type=int, default=None, help="oracle processes (default: all host cores, <= 16)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-chunks", type=int, default=None,
                    help="end-to-end run: instances split into this many contexts on their own streams, so the "
                         "copies of one chunk overlap the step of another (default 4 for the Sod batch, 1 else)")
    return ap.parse_args()


def ensemble_params(n=32):
    """Seeded resolutions (points per flow log-uniform in [0.25M, 2M]) and
    inflow Mach numbers (uniform in [2, 4]) of the step-flow ensemble; the
    spacing of a flow follows from the point count of the layout at h0 = 0.002
    (points scale as 1/h0^2)."""
    import numpy as np
    from paper_2506_19370_gb300 import inputs as I
    rng = np.random.default_rng(I.SEED + 5)
    pts = np.exp(rng.uniform(np.log(0.25e6), np.log(2.0e6), n))
    p0 = sum(int(p.active().sum()) for p in I.ffs_instance(h0=FFS_H0).patches)
    return [float(FFS_H0 * np.sqrt(p0 / p)) for p in pts], [float(m) for m in rng.uniform(2.0, 4.0, n)]


def workload(args):
    from paper_2506_19370_gb300 import inputs as I
    if args.workload == "ffs":
        return [I.ffs_instance(h0=FFS_H0) for _ in range(args.instances)]
    if args.workload == "ensemble":
        h0s, machs = ensemble_params()
        return [I.ffs_ensemble(h0s[:args.flows], machs[:args.flows])]
    if args.workload == "cylinder":
        return [I.cylinder_instance(h=CYL_H, wall=I.BC_NOSLIP) for _ in range(args.instances)]
    return [I.sod_instance(perturb=0.01, seed=I.SEED + k, smear=2.0) for k in range(args.instances)]


def config(args, inst, points):
    npatch = len(inst.patches)
    if args.workload == "cylinder":
        desc = (f"Mach-10 flow past a cylinder of radius 0.5: 16 body-fitted curvilinear annular sectors plus "
                f"Cartesian far-field patches of uneven resolution ({npatch} patches, interpolated fringes), "
                f"no-slip adiabatic cylinder wall, h = {CYL_H}, x {args.instances} instance(s)")
    elif args.workload == "ensemble":
        h0s, machs = ensemble_params()
        desc = (f"{args.flows} independent Mach 2-4 forward-facing-step flows (seeded: Mach U[2,4], resolutions log-uniform "
                f"0.25M-2M points, h0 {min(h0s):.5f}-{max(h0s):.5f}), {npatch} patches of uneven size (each flow: "
                f"64 patches with one C1 and one C2 corner patch, interpolated fringes, its own inflow state) in one "
                f"layout: every launch covers all flows")
    elif args.workload == "ffs":
        desc = (f"Mach-3 forward-facing step, channel [0,3]x[0,1], step of height 0.2 at x = 0.6; 64 overlapping "
                f"patches of uneven resolution including one C1 and one C2 corner patch, x {args.instances} "
                f"independent instances")
    else:
        desc = (f"Sod shock tube, 8 overlapping Cartesian patches of 160x40 points (overlap 10) per instance, "
                f"x {args.instances} independent instances")
    return {"workload": desc + "; per step: SDNN classifier + artificial viscosity + CFL dt + 4 RK stages + "
                               "exchange",
            "instances": args.instances, "patches_per_instance": npatch, "points": points,
            "d": 5, "C": "25 requested; FFT-length policy per line length",
            "classifier": (f"16-32-32-4 MLP, BF16 tensor-core inference with FP32 accumulation, trained on the "
                           f"device at setup ({args.train_steps} Adam steps of 4096 windows drawn from "
                           f"{args.train_windows} labelled windows that one FC step of the solver produced from "
                           f"seeded feature profiles)"),
            "l2": "inputs larger than L2 and flushed (256 MiB write) between timed steps",
            "parallelism": f"replicas x{args.gpus}" if args.gpus > 1 else "1 GPU"}


# ---------------------------------------------------------------- CPU oracle
ORACLE_CHILD = r"""
import json, sys, time
root, wl, mode, amount, warm = sys.argv[1], sys.argv[2], sys.argv[3], float(sys.argv[4]), int(sys.argv[5])
sys.path.insert(0, root)
from oracle import euler, sdnn
from paper_2506_19370_gb300 import inputs as I
if wl in ("ffs", "ensemble"):
    inst = I.ffs_instance(h0=0.005)
elif wl == "cylinder":
    inst = I.cylinder_instance(h=0.02, wall=I.BC_NOSLIP)
else:
    inst = I.sod_instance(perturb=0.01, smear=2.0)
s = euler.Solver(inst, c_policy=1)
params = sdnn.init_params(0)
st = [e.copy() for e in inst.state]
def step(st):
    taus = [sdnn.classify_patch(params, e, inst.gamma, lcut=tuple(p.lcut) if p.is_l else (0, 0))[0]
            for e, p in zip(st, inst.patches)]
    mu = sdnn.av_assemble(s, st, taus)
    return s.step(st, s.dt(st, mu), mu)
for _ in range(warm):
    st = step(st)
t0 = time.perf_counter(); n = 0
while (mode == "steps" and n < amount) or (mode == "time" and (time.perf_counter() - t0 < amount or n < 2)):
    st = step(st); n += 1
el = time.perf_counter() - t0
print(json.dumps({"steps": n, "seconds": el, "points": sum(int(p.active().sum()) for p in inst.patches)}))
"""


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_run(workload_name, mode, amount, warm, procs):
    """The FP64 oracle stepping independent copies of a bounded sample of the
    workload in `procs` separate single-threaded processes at once (one per
    host core); returns (pt-stage/s summed over the processes, steps of one
    process, points, seconds, procs) or raises."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, "-c", ORACLE_CHILD, ROOT, workload_name, mode, str(amount), str(warm)]
    ps = [subprocess.Popen(cmd, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
          for _ in range(procs)]
    res = []
    for p in ps:
        out, err = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(err[-300:])
        res.append(json.loads(out.strip().splitlines()[-1]))
    rate = sum(r["points"] * 4 * r["steps"] / r["seconds"] for r in res)
    return rate, res[0]["steps"], res[0]["points"], max(r["seconds"] for r in res), procs


def sample_text(workload_name, points, steps, seconds, procs):
    what = {"ffs": "forward-facing-step flow at h0 = 0.005", "ensemble": "forward-facing-step flow at h0 = 0.005",
            "cylinder": "cylinder flow at h = 0.02", "sod": "Sod instance"}[workload_name]
    return (f"{procs} oracle processes at once (one per host core, 1 thread each), each {steps} full steps "
            f"(classifier, viscosity, dt, 4 stages, exchange) of one {what} ({points} points) in {seconds:.1f} s; "
            f"FP64 numpy; rate = sum over the processes")


def cpu_baseline(seconds, workload_name, procs=None):
    procs = procs or min(host_cores(), 16)
    try:
        rate, steps, pts, secs, procs = oracle_run(workload_name, "time", seconds, 1, procs)
    except Exception as ex:   # reported, not fatal: the GPU line stands on its own
        return {"value": None, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": "failed: " + str(ex)}
    return {"value": rate, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": sample_text(workload_name, pts, steps, secs, procs)}


def run_reference(args):
    import torch  # noqa: F401  (rank bookkeeping only)
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    procs = args.cpu_procs or min(host_cores(), 16)
    try:
        rate, steps, pts, secs, procs = oracle_run(args.workload, "steps", args.steps, args.warmup, procs)
    except Exception as ex:
        print(json.dumps({"impl": "reference", "unavailable": "oracle failed: " + str(ex)[-200:]}))
        return
    inst = workload(args)[0]
    points = args.instances * sum(int(p.active().sum()) for p in inst.patches)
    samp = sample_text(args.workload, pts, steps, secs, procs)
    line = {"metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * pts * 4 * procs / rate, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(args, inst, points), "impl": "reference",
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": samp},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows if len(r) >= 8 for k in range(4) if r[4 + k] == "Active"})
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json: STREAM-style copy)"
    except Exception:
        return FALLBACK_HBM, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("fcs_device.cuh", "fcs_line_kernels.cuh", "fcs_launch.cuh", "fcs_roots.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2506_19370_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(workload_name, points):
    """DRAM bytes of one rk_stage call (both flux passes) from the committed
    ncu summary of this workload, scaled to `points`; None if the line-kernel
    sources changed since the capture or there is none."""
    p = os.path.join(ROOT, "profiles", f"rk_stage_traffic_{workload_name}.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    return d["dram_bytes_per_point_stage"] * points


# ---------------------------------------------------------------- ranks
def job_throughput(total_ms, points_per_rank, stages, steps, world, dist=None):
    """Whole-job pt-stage/s: all ranks' points over the slowest rank's time
    (max over ranks; replicas, no data-path collective)."""
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64)
    if world > 1 and dist is not None:
        if dist.get_backend() == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    slowest = float(t.item())
    return world * points_per_rank * stages * steps / (slowest / 1000.0), slowest


# ---------------------------------------------------------------- GPU arm
def seeded_weights():
    """He-uniform classifier weights, zero biases (seeded; drawn here so the
    oracle stays out of the GPU arm)."""
    import numpy as np
    from paper_2506_19370_gb300.inputs import SEED
    rng = np.random.default_rng(SEED)
    w = []
    for shape in ((32, 16), (32,), (32, 32), (32,), (4, 32), (4,)):
        if len(shape) == 2:
            lim = np.sqrt(6.0 / shape[1])
            w.append(rng.uniform(-lim, lim, size=shape).ravel())
        else:
            w.append(np.zeros(shape))
    return np.concatenate(w).astype(np.float32)


class Stepper:
    """One time step as fcs_step runs it, call by call (so the stage operator
    can be timed on its own): classifier, viscosity, dt, four stages each
    followed by the exchange; counts the library's launches."""

    def __init__(self, ctx, e, stream):
        import torch
        self.ctx, self.e, self.stream = ctx, e, stream
        self.tau = ctx.new_scalar(torch.int8)
        self.mu = ctx.new_scalar()
        self.dtd = torch.zeros(ctx.instances, dtype=torch.float64, device=e.device)
        self.S, self.A = ctx.new_state(), ctx.new_state()
        self.launches = 0

    def step(self, ev=None):
        c, e, s = self.ctx, self.e, self.stream
        c.classify(e, self.tau, None, s)
        c.av_assemble(e, self.tau, self.mu, s)
        c.time_step(e, self.dtd, self.mu, s)
        # proxy, MLP, tau gather; viscosity (preliminary, blend, exchange); dt init/min/final
        self.launches += 3 + c.launches["av"] + 3
        for k in range(4):
            es = e if k == 0 else self.S
            out = e if k == 3 else self.S
            if ev is not None:
                ev[k][0].record(s)
            c.rk_stage(k, 0.0, e, es, self.A, out, mu=self.mu, dt_dev=self.dtd, stream=s)
            if ev is not None:
                ev[k][1].record(s)
            c.patch_exchange(out, 4, s)
            self.launches += c.launches["stage_visc"] + c.launches["exchange"]


def timed_steps(st, steps, warmup, flush, world, dist):
    """W untimed steps, then exactly `steps` timed ones (L2 flushed before
    each, CUDA events on the launching stream around each step and each
    stage); returns per-step and per-stage milliseconds."""
    import torch
    with torch.cuda.stream(st.stream):
        for _ in range(warmup):
            st.step()
    st.stream.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, stage_ms = [], []
    st.launches = 0
    torch.cuda.nvtx.range_push("fcs_timed")
    with torch.cuda.stream(st.stream):
        for _ in range(steps):
            flush.fill_(1.0)
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(4)]
            t0.record(st.stream)
            st.step(ev)
            t1.record(st.stream)
            st.stream.synchronize()
            step_ms.append(t0.elapsed_time(t1))
            stage_ms += [a.elapsed_time(b) for a, b in ev]
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    return step_ms, stage_ms


def line_deriv_flops(N, n, C, d=5):
    """Algorithmic flops of one FC derivative per line point: a line pair
    shares one complex FFT of length n forward and back (10 n log2 n), the
    multiplication by i k (2 n) and both ends' continuations (Gram projection
    2 x 2 d^2 and blend 2 x 2 d C per line), over the 2 N points of the pair."""
    return (10.0 * n * math.log2(n) + 2.0 * n + 2 * (4.0 * d * d + 4.0 * d * C)) / (2.0 * N)


def stage_accounting(ctx, inst, mu_fields, tsize):
    """Per point-stage of the layout: algorithmic bytes of the stage operator
    (read e_s and e_n, write e_out: 12 values; mu: 1; metrics x_q1, x_q2,
    y_q1, y_q2, J on curvilinear patches: 5) and the flops the kernels execute
    (4 flux derivatives per direction at every point, 4 viscous derivatives
    per direction on the lines where mu is not zero everywhere; curvilinear
    patches with viscosity differentiate e along q2 on every column, plus ~70
    pointwise flops).  Returns (bytes, flops, fraction of viscous line
    derivatives among the possible ones)."""
    import numpy as np
    pts = bts = fl = 0.0
    visc_done = visc_possible = 0.0
    for p, mu in zip(inst.patches, mu_fields):
        act = p.active()
        npt = float(act.sum())
        pts += npt
        bts += npt * tsize * (13 + (0 if p.cartesian else 5))
        m1, m2 = p.lcut if p.is_l else (0, 0)
        nz = (mu != 0) & act
        # line segments (direction, length, index block): full and short rows, full and short columns
        segs = [(0, p.n1, (slice(m2, p.n2), slice(0, p.n1))), (0, p.n1 - m1, (slice(0, m2), slice(m1, p.n1))),
                (1, p.n2, (slice(0, p.n2), slice(m1, p.n1))), (1, p.n2 - m2, (slice(m2, p.n2), slice(0, m1)))]
        for dirn, N, blk in segs:
            sub, subnz = act[blk], nz[blk]
            if N <= 0 or sub.size == 0:
                continue
            C = ctx.line_c(N)
            f = line_deriv_flops(N, N + C, C)
            npts = float(sub.sum())
            fl += 4 * f * npts
            # points on lines (rows for dirn 0, columns for dirn 1) with viscosity
            vis_line = subnz.any(axis=1 - dirn)
            vpts = float((sub * (vis_line[:, None] if dirn == 0 else vis_line[None, :])).sum())
            if not p.cartesian and dirn == 1 and nz.any():
                vpts = npts
            fl += 4 * f * vpts
            visc_done += vpts
            visc_possible += npts
    return bts / pts, fl / pts + 70.0, (visc_done / visc_possible if visc_possible else 0.0)


def alu_peak_tflops(fcsdnn, dtype, dev, stream):
    """Measured FMA rate of this GPU (library probe, 8 blocks of 256 threads
    per SM, best of 5 after a warm-up), TFLOP/s."""
    import torch
    blocks = 152 * 8
    iters = 8192 if dtype == fcsdnn.F32 else 128
    out = torch.zeros(blocks, dtype=torch.float64 if dtype == fcsdnn.F64 else torch.float32, device=dev)
    best = None
    with torch.cuda.stream(stream):
        fcsdnn.alu_probe(dtype, blocks, iters, out, stream)
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fcsdnn.alu_probe(dtype, blocks, iters, out, stream)
            b.record(stream)
            stream.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
    return blocks * 256.0 * iters * 64.0 / (best / 1000.0) / 1e12


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2506_19370_gb300 import fcsdnn
    from paper_2506_19370_gb300.inputs import SEED

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
        dist.barrier()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    insts = workload(args)
    inst0 = insts[0]
    # ---- the learned part (not timed as steps): labelled windows that one FC
    # step of the solver produces from seeded feature profiles, the network
    # trained on them by the library's training kernels, scored on states it
    # has not seen against the known features and the decay indicator
    from paper_2506_19370_gb300 import training as TR
    t0 = time.perf_counter()
    wsrc = TR.WindowSource(chunk=2048, seed=SEED)
    Xtr, Ytr, nch = TR.make_dataset(args.train_windows, wsrc)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    wsrc.ctx.set_weights(seeded_weights())
    t0 = time.perf_counter()
    loss0, loss1 = TR.train(wsrc.ctx, Xtr, Ytr, steps=args.train_steps)
    torch.cuda.synchronize()
    fit_s = time.perf_counter() - t0
    held = TR.evaluate(wsrc, nch + 1)
    counts = torch.bincount(Ytr.long(), minlength=5).cpu().numpy()[1:].tolist()
    xw_d, yw_d = Xtr[:4096].contiguous(), Ytr[:4096].contiguous()
    ctx = fcsdnn.Context(inst0, d=5, C=25, dtype=fcsdnn.F32, instances=args.instances, c_policy=1, autotune=1)
    ctx.set_weights(wsrc.ctx.get_weights())
    wsrc.ctx.close()
    del wsrc, Xtr, Ytr
    host = ctx.pack_state([i.state for i in insts])
    e = ctx.to_device(host)
    points = args.instances * sum(int(p.active().sum()) for p in inst0.patches)
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()

    # ---- FP32 arm: the timed steps
    st = Stepper(ctx, e, stream)
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    step_ms, stage_ms = timed_steps(st, args.steps, args.warmup, flush, world, dist)
    clocks = clk.stop()
    launches = st.launches
    rc, flags = ctx.status()
    value, total_ms = job_throughput(sum(step_ms), points, 4, args.steps, world, dist if world > 1 else None)
    stage_avg_ms = sum(stage_ms) / len(stage_ms)
    mu_fields = ctx.unpack_scalar(st.mu, 0)

    def timed(fn, reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            fn()
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
        stream.synchronize()
        return a.elapsed_time(b) / reps

    # ---- learned part: training samples/s (one Adam step on 4096 windows)
    # and inference windows/s (proxy + windows + MLP + per-point tau)
    train_ms = timed(lambda: ctx.train_step(xw_d, yw_d, 3e-3, None, stream), 20)
    infer_ms = timed(lambda: ctx.classify(e, st.tau, None, stream), 10)
    learned = {"training_samples_per_s": 4096 / (train_ms / 1000.0),
               "inference_windows_per_s": args.instances * ctx.windows / (infer_ms / 1000.0),
               "train_step_ms": train_ms, "classify_ms": infer_ms, "windows_per_step": args.instances * ctx.windows,
               "training_set": {"windows": args.train_windows, "per_class": counts, "chunks": nch,
                                "generation_s": gen_s, "source": "one RK4 step of the FC operator on seeded profiles "
                                "with jumps, kinks and C1 features at known places (training.py)"},
               "training_run": {"steps": args.train_steps, "batch": 4096, "seconds": fit_s,
                                "samples_per_s_incl_batch_gather": args.train_steps * 4096 / fit_s,
                                "loss_first10": loss0, "loss_last10": loss1},
               "held_out_vs_known_features": held}

    # ---- the FC-derivative kernel alone (continuation + FFT + i k + inverse
    # FFT + restriction), one call per direction over every line of the
    # layout: algorithmic bytes = one read and one write of the field
    hbm_peak, hbm_src = measured_peak()
    rng = np.random.default_rng(SEED)
    xs = ctx.to_device(ctx.pack_scalar([rng.standard_normal((p.n2, p.n1)) for p in inst0.patches]))
    ys = ctx.new_scalar()
    fcd = {}
    torch.cuda.nvtx.range_push("fcs_fcderiv")
    for direction in (0, 1):
        with torch.cuda.stream(stream):
            ctx.fc_derivative(xs, ys, direction, 1, stream)
        ts_ = []
        for _ in range(5):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ctx.fc_derivative(xs, ys, direction, 1, stream)
                b.record(stream)
            stream.synchronize()
            ts_.append(a.elapsed_time(b))
        ts_.sort()
        fcd[direction] = ts_[len(ts_) // 2]
    torch.cuda.nvtx.range_pop()
    fcd_bytes = 2.0 * 4 * points
    fcd_gbs = [fcd_bytes / (fcd[k] / 1000.0) / 1e9 for k in (0, 1)]
    fc_derivative = {"kernel": "k_fc_deriv (FP32, all FFT-size groups of one direction)",
                     "alg_bytes_per_point": 8, "us_dir_q1": 1000.0 * fcd[0], "us_dir_q2": 1000.0 * fcd[1],
                     "achieved_gbs": sum(fcd_gbs) / 2, "peak_gbs": hbm_peak, "frac": sum(fcd_gbs) / 2 / hbm_peak,
                     "peak_source": hbm_src}
    del xs, ys

    # ---- end to end through the C ABI: pinned host state in, one
    # graph-captured step, state out, every step.  Independent instances can
    # run as K contexts of m instances on their own streams, so chunk k's
    # copies overlap another chunk's step.
    K = args.e2e_chunks if args.e2e_chunks is not None else (4 if args.workload == "sod" else 1)
    K = K if K > 0 and args.instances % K == 0 else 1
    m = args.instances // K
    wts = ctx.get_weights()
    chunks = []
    for k in range(K):
        ck = ctx if K == 1 else fcsdnn.Context(inst0, d=5, C=25, dtype=fcsdnn.F32, instances=m, c_policy=1,
                                               autotune=1)
        if K > 1:
            ck.set_weights(wts)
        hk = ck.pack_state([i.state for i in insts[k * m:(k + 1) * m]]) if K > 1 else host
        pin = torch.from_numpy(hk).pin_memory()
        ek = ck.to_device(hk)
        dk = torch.zeros(m, dtype=torch.float64, device=dev)
        sk = stream if K == 1 else torch.cuda.Stream(device=dev)
        chunks.append(dict(ctx=ck, pin=pin, out=torch.empty_like(pin).pin_memory(), e=ek, dt=dk, s=sk))
    for ch in chunks:   # capture the graphs outside the timed region
        ch["ctx"].step_graph(ch["e"], dt_dev=ch["dt"], use_av=True, stream=ch["s"])
    torch.cuda.synchronize()
    n_e2e = max(3, args.steps // 2)
    e2e_ms = 0.0
    for _ in range(n_e2e):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for ch in chunks:
            with torch.cuda.stream(ch["s"]):
                ch["e"].copy_(ch["pin"], non_blocking=True)
                ch["ctx"].step_graph(ch["e"], dt_dev=ch["dt"], use_av=True, stream=ch["s"])
                ch["out"].copy_(ch["e"], non_blocking=True)
        for ch in chunks:
            ch["s"].synchronize()
        e2e_ms += 1000.0 * (time.perf_counter() - t0)
    e2e_val, _ = job_throughput(e2e_ms, points, 4, n_e2e, world, dist if world > 1 else None)
    nbytes = sum(ch["e"].numel() * ch["e"].element_size() for ch in chunks)
    for ch in chunks:
        if ch["ctx"] is not ctx:
            ch["ctx"].close()
    del chunks

    # ---- roofline of the stage operator and the measured ALU peaks
    alu32 = alu_peak_tflops(fcsdnn, fcsdnn.F32, dev, stream)
    alu64 = alu_peak_tflops(fcsdnn, fcsdnn.F64, dev, stream)
    alg_b, alg_f, vfrac = stage_accounting(ctx, inst0, mu_fields, 4)
    stage_s = stage_avg_ms / 1000.0
    gbs = alg_b * points / stage_s / 1e9
    tfl = alg_f * points / stage_s / 1e12
    t_hbm, t_alu = alg_b / (hbm_peak * 1e9), alg_f / (alu32 * 1e12)
    bound = "hbm" if t_hbm >= t_alu else "alu"
    traffic = recorded_traffic(args.workload, points)
    roofline = {"bound": bound,
                "achieved": gbs if bound == "hbm" else tfl, "peak": hbm_peak if bound == "hbm" else alu32,
                "unit": "GB/s" if bound == "hbm" else "TFLOP/s",
                "frac": gbs / hbm_peak if bound == "hbm" else tfl / alu32, "traffic": traffic,
                "kernel": "rk_stage: flux pass along q2 (k_ypass, partial operator R) + flux pass along q1 with "
                          "the stage update (k_xpass), every FFT-size group (the groups of a pass concurrent)",
                "stage_ms": stage_avg_ms, "alg_bytes_per_point_stage": alg_b,
                "hbm": {"achieved_gbs": gbs, "peak_gbs": hbm_peak, "frac": gbs / hbm_peak, "peak_source": hbm_src},
                "alu": {"executed_flops_per_point_stage": alg_f, "viscous_line_fraction": vfrac,
                        "achieved_tflops": tfl, "peak_tflops": alu32, "frac": tfl / alu32,
                        "peak_source": "measured: FP32 FMA probe (fcs_alu_probe), best of 5"},
                "intensity_flop_per_byte": alg_f / alg_b, "ridge_flop_per_byte": alu32 * 1e12 / (hbm_peak * 1e9)}

    # ---- the plain FP64 form on the same inputs, and the FP32 error against it
    fp64 = err = None
    if not args.no_fp64:
        ctx64 = fcsdnn.Context(inst0, d=5, C=25, dtype=fcsdnn.F64, instances=args.instances, c_policy=1, autotune=1)
        ctx64.set_weights(ctx.get_weights())
        e64 = ctx64.to_device(ctx64.pack_state([i.state for i in insts]))
        st64 = Stepper(ctx64, e64, stream)
        n64 = args.fp64_steps or max(3, args.steps // 4)
        s64_ms, g64_ms = timed_steps(st64, n64, min(args.warmup, 3), flush, world, dist)
        v64, t64 = job_throughput(sum(s64_ms), points, 4, n64, world, dist if world > 1 else None)
        rc64, _ = ctx64.status()
        g64 = sum(g64_ms) / len(g64_ms) / 1000.0
        fp64 = {"value": v64, "unit": UNIT, "ms_per_step": t64 / n64, "steps": n64, "status": rc64,
                "speedup_fp32_over_fp64": value / v64, "stage_ms": 1000.0 * g64,
                "alu_frac": alg_f * points / g64 / 1e12 / alu64, "alu_peak_tflops": alu64,
                "alu_peak_source": "measured: FP64 FMA probe (fcs_alu_probe), best of 5",
                "note": "same layout, initial state and classifier weights; FP64 throughout (FP64 classifier); the "
                        "FP64 form matches the FP64 CPU oracle to 1e-12 per derivative in the parity tests"}
        # error: both forms from the initial state with the same time steps
        # (the FP64 form's CFL steps, with its viscosity), classifier and
        # viscosity on
        e32 = ctx.to_device(host)
        e64 = ctx64.to_device(ctx64.pack_state([i.state for i in insts]))
        dtd = torch.zeros(args.instances, dtype=torch.float64, device=dev)
        t_err = 0.0
        for _ in range(args.error_steps):
            ctx64.step(e64, dt_dev=dtd, use_av=True)
            dt = float(dtd.min().item())
            ctx.step(e32, dt=dt, use_av=True)
            t_err += dt
        torch.cuda.synchronize()
        rc_e, _ = ctx.status()
        a32, a64 = ctx.unpack_state(e32), ctx64.unpack_state(e64)
        num = den = lin = linden = 0.0
        for p, x, y in zip(inst0.patches, a32, a64):
            act = p.active()
            num += float(np.abs(x[0][act] - y[0][act]).sum())
            den += float(np.abs(y[0][act]).sum())
            lin = max(lin, float(np.abs(x[:, act] - y[:, act]).max()))
            linden = max(linden, float(np.abs(y[:, act]).max()))
        err = {"l1_rel_density": num / den, "linf_rel_state": lin / linden, "steps": args.error_steps,
               "t_end": t_err, "status": rc_e,
               "against": "the plain FP64 GPU form (instance 0), same initial state and time steps (the FP64 "
                          "form's), viscosity and classifier on (FP32: BF16 classifier)"}
        ctx64.close()

    if rank == 0:
        cfg = dict(config(args, inst0, points), tile_width=ctx.tile_width,
                   launches_per_stage=ctx.launches["stage_visc"] + ctx.launches["exchange"])
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                        "note": (f"pinned host state -> device, one graph-captured step, state -> host; {K} "
                                 f"context(s) of {m} instance(s) on {K} stream(s)")},
                "gpu_launches": launches, "roofline": roofline, "fc_derivative": fc_derivative,
                "fp64": fp64, "precision_error": err, "clocks": clocks, "status": rc, "classifier": learned}
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(args.cpu_seconds, args.workload, args.cpu_procs)
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.instances is None:
        args.instances = {"ffs": 8, "ensemble": 1, "cylinder": 1}.get(args.workload, 128)
    if args.workload == "ensemble":
        args.instances = 1
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

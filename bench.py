"""Benchmark: FC-SDNN grid-point-stage updates per second on one GB300.

Workload (one "step" = one full time step of the hot path): a batch of
independent Sod shock-tube instances, each on [0,1] x [0,0.1] split into 8
overlapping Cartesian patches of 160 x 40 points (overlap 10), seeded
perturbations of the Sod states; per step: proxy + windows + classifier MLP,
artificial viscosity assembly, CFL time step, four Runge-Kutta stages (FC
derivatives of fluxes and viscous fluxes, operator, stage update, boundary
conditions), each followed by the fringe exchange.  Inputs are synthetic.
--workload ffs times the Mach-3 forward-facing step instead (64 patches of
uneven resolution with interpolated fringes and the two corner patches, ~1M
points per instance, 8 instances).

Prints one JSON line (see --help).  --impl reference times the FP64 CPU
oracle on a bounded sample of the same workload on the host cores.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FC-SDNN grid-point-stage updates/s on 1 GB300, batched FP32 vs plain FP64, at set error"
UNIT = "pt-stage/s"
L2_BYTES = 129 * 2 ** 20
FALLBACK_HBM = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--instances", type=int, default=None,
                    help="independent instances (default: 128 for sod, 8 for ffs)")
    ap.add_argument("--workload", default="sod", choices=["sod", "ffs", "ensemble", "cylinder"],
                    help="sod: the shock-tube batch (default); ffs: the forward-facing step with corner patches; "
                         "ensemble: 32 step flows of seeded resolutions and Mach numbers in one layout; "
                         "cylinder: Mach-10 flow past a cylinder (annular sectors + Cartesian far field)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-chunks", type=int, default=None,
                    help="end-to-end run: instances split into this many contexts on their own streams, so the "
                         "copies of one chunk overlap the step of another (1: one context, no overlap; default 4 "
                         "for the Sod batch, 1 for the multi-patch flows, whose smaller per-context launches "
                         "measured slower than the copies they hide)")
    return ap.parse_args()


FFS_H0 = 0.002      # forward-facing step: ~1M points in 64 patches per instance
CYL_H = 0.004       # cylinder: ~3.9M points in 260 patches


def ensemble_params(n=32):
    """Seeded resolutions (points per flow log-uniform in [0.25M, 1.1M]; the
    corner patch of a finer flow would exceed 256 points per side) and inflow
    Mach numbers (uniform in [2, 4]) of the step-flow ensemble."""
    import numpy as np
    from paper_2506_19370_gb300 import inputs as I
    rng = np.random.default_rng(I.SEED + 5)
    pts = np.exp(rng.uniform(np.log(0.25e6), np.log(1.1e6), n))
    return [float(FFS_H0 * np.sqrt(880203.0 / p)) for p in pts], [float(m) for m in rng.uniform(2.0, 4.0, n)]


def workload(args):
    from paper_2506_19370_gb300 import inputs as I
    if args.workload == "ffs":
        return [I.ffs_instance(h0=FFS_H0) for _ in range(args.instances)]
    if args.workload == "ensemble":
        h0s, machs = ensemble_params()
        return [I.ffs_ensemble(h0s, machs)]
    if args.workload == "cylinder":
        return [I.cylinder_instance(h=CYL_H, wall=I.BC_NOSLIP) for _ in range(args.instances)]
    return [I.sod_instance(perturb=0.01, seed=I.SEED + k, smear=2.0) for k in range(args.instances)]


def config(args, points):
    if args.workload == "cylinder":
        desc = (f"Mach-10 flow past a cylinder of radius 0.5: 16 body-fitted curvilinear annular sectors plus 244 "
                f"Cartesian far-field patches of uneven resolution (interpolated fringes), no-slip adiabatic "
                f"cylinder wall, h = {CYL_H}, "
                f"x {args.instances} instance(s); SDNN classifier + artificial viscosity + CFL dt + 4 RK stages + "
                f"exchange per step")
        cdesc = "25 requested; FFT-length policy per line length"
    elif args.workload == "ensemble":
        h0s, machs = ensemble_params()
        desc = (f"32 independent Mach 2-4 forward-facing-step flows (seeded resolutions, 0.25M-1.1M points each; "
                f"h0 {min(h0s):.4f}-{max(h0s):.4f}) in one layout of {32 * 64} patches of uneven size with "
                f"per-flow inflow states, one context: every launch covers all flows")
        cdesc = "25 requested; FFT-length policy per line length"
    elif args.workload == "ffs":
        desc = (f"Mach-3 forward-facing step, channel [0,3]x[0,1], step of height 0.2 at x = 0.6; 64 overlapping "
                f"patches of uneven resolution (48-128 points per side, non-coincident grids, interpolated "
                f"fringes) including one L-shaped C1 corner patch and one C2 corner patch per instance, "
                f"x {args.instances} independent instances; SDNN classifier + artificial viscosity + CFL dt + "
                f"4 RK stages + exchange per step")
        cdesc = "25 requested; FFT-length policy per line length (n = 96 ... 224)"
    else:
        desc = (f"Sod shock tube, 8 overlapping Cartesian patches of 160x40 points (overlap 10) per "
                f"instance, x {args.instances} independent instances; SDNN classifier + artificial "
                f"viscosity + CFL dt + 4 RK stages + exchange per step")
        cdesc = ("25 requested; FFT-length policy gives 32 on 160-point rows (n = 192) and 24 on 40-point "
                 "columns (n = 64)")
    return {"workload": desc,
            "instances": args.instances, "points_per_instance": points // args.instances, "points": points,
            "d": 5, "C": cdesc,
            "classifier": "16-32-32-4 MLP trained on the device at setup (300 Adam steps, 4096 seeded windows)",
            "l2": "flushed (256 MiB write) between timed steps",
            "parallelism": f"replicas x{args.gpus}" if args.gpus > 1 else "1 GPU"}


# ---------------------------------------------------------------- CPU oracle
def cpu_baseline(seconds, workload_name="sod"):
    """Time the oracle (single-threaded numpy) on whole steps of one instance
    (forward-facing step: the same layout at a coarser spacing, h0 = 0.005)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = (
        "import time, json, sys; sys.path.insert(0, %r)\n"
        "from oracle import euler, sdnn\n"
        "from paper_2506_19370_gb300 import inputs as I\n"
        + ("inst = I.ffs_instance(h0=0.005)\n" if workload_name in ("ffs", "ensemble") else
           "inst = I.cylinder_instance(h=0.02, wall=I.BC_NOSLIP)\n" if workload_name == "cylinder" else
           "inst = I.sod_instance(perturb=0.01, smear=2.0)\n") +
        "s = euler.Solver(inst, c_policy=1)\n"
        "params = sdnn.init_params(0)\n"
        "st = [e.copy() for e in inst.state]\n"
        "def step(st):\n"
        "    taus = [sdnn.classify_patch(params, e, inst.gamma, lcut=tuple(p.lcut) if p.is_l else (0, 0))[0]\n"
        "            for e, p in zip(st, inst.patches)]\n"
        "    mu = sdnn.av_assemble(s, st, taus)\n"
        "    dt = s.dt(st, mu)\n"
        "    return s.step(st, dt, mu)\n"
        "st = step(st)\n"
        "t0 = time.perf_counter(); n = 0\n"
        "while time.perf_counter() - t0 < %f or n < 2:\n"
        "    st = step(st); n += 1\n"
        "el = time.perf_counter() - t0\n"
        "pts = sum(int(p.active().sum()) for p in inst.patches)\n"
        "print(json.dumps({'steps': n, 'seconds': el, 'points': pts}))\n"
    ) % (ROOT, seconds)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": "failed: " + r.stderr[-300:]}
    res = json.loads(r.stdout.strip().splitlines()[-1])
    val = res["points"] * 4 * res["steps"] / res["seconds"]
    return {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{res['steps']} full steps (classifier, viscosity, dt, 4 stages, exchange) of one "
                      + ("forward-facing-step instance at h0 = 0.005" if workload_name in ("ffs", "ensemble")
                         else "cylinder instance at h = 0.02" if workload_name == "cylinder" else "Sod instance")
                      + f" ({res['points']} points) in {res['seconds']:.1f} s, FP64 numpy, 1 thread",
            "seconds": res["seconds"]}


def run_reference(args):
    import torch  # noqa: F401  (rank bookkeeping only)
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per = max(args.cpu_seconds / max(args.steps, 1), 2.0)
    vals, secs = [], 0.0
    base = None
    for _ in range(args.steps):
        b = cpu_baseline(per, args.workload)
        if b["value"] is None:
            print(json.dumps({"impl": "reference", "unavailable": b["sample"]}))
            return
        vals.append(b["value"])
        secs += b["seconds"]
        base = b
    pts = 51200 if args.workload == "sod" else None
    value = sum(vals) / len(vals)
    if pts is None:
        pts = sum(int(p.active().sum()) for p in workload(args)[0].patches)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * pts * 4 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(args, pts * args.instances), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": base["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
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
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("fcs_device.cuh", "fcs_line_kernels.cuh", "fcs_launch.cuh", "fcs_roots.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2506_19370_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(per_launch_points):
    """DRAM bytes per launch of the stage operator (both flux passes) from the
    committed ncu capture, scaled to this launch's points; None if the kernel
    sources changed since the capture."""
    p = os.path.join(ROOT, "profiles", "rk_stage_traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    return d["dram_bytes_per_point_stage"] * per_launch_points


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
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2506_19370_gb300 import fcsdnn

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
        dist.barrier()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dtype = fcsdnn.F64 if args.dtype == "f64" else fcsdnn.F32
    insts = workload(args)
    ctx = fcsdnn.Context(insts[0], d=5, C=25, dtype=dtype, instances=args.instances, c_policy=1, autotune=1)
    from paper_2506_19370_gb300.inputs import SEED
    rng = np.random.default_rng(SEED)
    # seeded classifier weights (He-uniform), drawn here to keep the oracle out of the GPU arm
    w = []
    for shape in ((32, 16), (32,), (32, 32), (32,), (4, 32), (4,)):
        if len(shape) == 2:
            lim = np.sqrt(6.0 / shape[1])
            w.append(rng.uniform(-lim, lim, size=shape).ravel())
        else:
            w.append(np.zeros(shape))
    ctx.set_weights(np.concatenate(w).astype(np.float32))
    # train the classifier on the device (library kernels, seeded windows; not timed) so the
    # viscosity is localized at the waves as in the method
    from paper_2506_19370_gb300.inputs import classifier_windows
    xw, yw = classifier_windows(4096, seed=SEED)
    xw_d = torch.from_numpy(xw.astype(np.float32)).to(dev)
    yw_d = torch.from_numpy(yw).to(dev)
    for _ in range(300):
        ctx.train_step(xw_d, yw_d, 3e-3)
    host = ctx.pack_state([i.state for i in insts])
    e = ctx.to_device(host)
    points = args.instances * sum(int(p.active().sum()) for p in insts[0].patches)
    tau = ctx.new_scalar(torch.int8)
    mu = ctx.new_scalar()
    dtd = torch.zeros(args.instances, dtype=torch.float64, device=dev)
    S = ctx.new_state()
    A = ctx.new_state()
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    launches = {"n": 0}

    def step(ev=None):
        # the same sequence as fcs_step, call by call, so the stage operator can be timed
        ctx.classify(e, tau, None, stream)
        ctx.av_assemble(e, tau, mu, stream)
        ctx.time_step(e, dtd, mu, stream)
        # proxy, MLP, tau gather; viscosity (preliminary, blend, exchange); dt init/min/final
        launches["n"] += 3 + ctx.launches["av"] + 3
        for s in range(4):
            es = e if s == 0 else S
            out = e if s == 3 else S
            if ev is not None:
                ev[s][0].record(stream)
            ctx.rk_stage(s, 0.0, e, es, A, out, mu=mu, dt_dev=dtd, stream=stream)
            if ev is not None:
                ev[s][1].record(stream)
            ctx.patch_exchange(out, 4, stream)
            launches["n"] += ctx.launches["stage_visc"] + ctx.launches["exchange"]

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()
    if world > 1:
        dist.barrier()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    step_ms, stage_ms = [], []
    launches["n"] = 0
    # NVTX range of the timed steps (lets a profiler capture exactly these launches)
    torch.cuda.nvtx.range_push("fcs_timed")
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.fill_(1.0)
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(4)]
            t0.record(stream)
            step(ev)
            t1.record(stream)
            stream.synchronize()
            step_ms.append(t0.elapsed_time(t1))
            stage_ms += [a.elapsed_time(b) for a, b in ev]
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clocks = clk.stop()
    rc, flags = ctx.status()
    value, total_ms = job_throughput(sum(step_ms), points, 4, args.steps, world, dist if world > 1 else None)

    # learned part: training samples/s (one Adam step on 4096 windows) and
    # inference windows/s (proxy + windows + MLP + per-point tau on the state)
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
    train_ms = timed(lambda: ctx.train_step(xw_d, yw_d, 3e-3, None, stream), 20)
    infer_ms = timed(lambda: ctx.classify(e, tau, None, stream), 10)
    learned = {"training_samples_per_s": 4096 / (train_ms / 1000.0),
               "inference_windows_per_s": args.instances * ctx.windows / (infer_ms / 1000.0),
               "train_step_ms": train_ms, "classify_ms": infer_ms}

    # end to end through the C ABI: pinned host state in, step (graph), state out.
    # The instances are independent, so they run as K contexts of m instances,
    # each on its own stream: chunk k's host->device copy overlaps chunk k-1's
    # step, and its device->host copy chunk k+1's (copy engines and SMs work
    # at once).  Every step copies the whole state in and out.
    K = args.e2e_chunks if args.e2e_chunks is not None else (4 if args.workload == "sod" else 1)
    K = K if K > 0 and args.instances % K == 0 else 1
    m = args.instances // K
    wts = ctx.get_weights()
    chunks = []
    for k in range(K):
        ck = ctx if K == 1 else fcsdnn.Context(insts[0], d=5, C=25, dtype=dtype, instances=m, c_policy=1, autotune=1)
        if K > 1:
            ck.set_weights(wts)
        hk = ck.pack_state([i.state for i in insts[k * m:(k + 1) * m]]) if K > 1 else host
        pin = torch.from_numpy(hk).pin_memory()
        ek = e if K == 1 else ck.to_device(hk)
        dk = dtd if K == 1 else torch.zeros(m, dtype=torch.float64, device=dev)
        sk = stream if K == 1 else torch.cuda.Stream(device=dev)
        chunks.append(dict(ctx=ck, pin=pin, out=torch.empty_like(pin).pin_memory(), e=ek, dt=dk, s=sk))
    for ch in chunks:   # capture the graphs outside the timed region
        ch["ctx"].step_graph(ch["e"], dt_dev=ch["dt"], use_av=True, stream=ch["s"])
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for _ in range(max(3, args.steps // 2)):
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
    n_e2e = max(3, args.steps // 2)
    e2e_val, _ = job_throughput(e2e_ms, points, 4, n_e2e, world, dist if world > 1 else None)
    nbytes = sum(ch["e"].numel() * ch["e"].element_size() for ch in chunks)

    # roofline of the stage operator rk_stage (flux pass along q1 + flux pass
    # along q2 with the stage update: two launches sharing the partial
    # operator through L2).  Bound: ALU issue (counters: DRAM 1-3 %, SM 25 %).
    # Algorithmic FLOPs per point-stage: 16 line derivatives (8 viscous, 8 of
    # the fluxes) of [10 n log2 n (FFT pair) + 2 n (i k) + 8 d C (both
    # continuations)] / (2 N) each, plus ~70 pointwise (fluxes, viscous flux,
    # stage update); peak = 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz.
    import math
    def per_point(N, n, C, d=5):
        return (10 * n * math.log2(n) + 2 * n + 8 * d * C) / (2 * N)
    # every point lies on one line segment per direction: average over the
    # layout's segments with their own continuation lengths
    flops_sum = 0.0
    for p in insts[0].patches:
        m1, m2 = p.lcut if p.is_l else (0, 0)
        for nlines, N in ((p.n2 - m2, p.n1), (m2, p.n1 - m1), (p.n1 - m1, p.n2), (m1, p.n2 - m2)):
            if nlines and N:
                Cn = ctx.line_c(N)
                flops_sum += nlines * N * 8 * per_point(N, N + Cn, Cn)
    flops_pt = flops_sum / (points // args.instances) + 70
    stage_avg_ms = sum(stage_ms) / len(stage_ms)
    achieved_tf = flops_pt * points / (stage_avg_ms / 1000.0) / 1e12
    alu_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    if dtype == fcsdnn.F64:
        alu_peak /= 64.0   # GB300 FP64 vector rate (1/64 of FP32), see the design notes
    ts = 8 if dtype == fcsdnn.F64 else 4
    # minimum state traffic per point-stage (elements): stage 0 reads e_n, writes
    # acc and out (12); stages 1-2 read e_s, e_n, acc, write acc, out (20); stage 3
    # reads e_s, acc, writes out (12); every stage reads mu (1): mean 17
    alg_bytes_pt = ts * 17
    hbm_gbs = alg_bytes_pt * points / (stage_avg_ms / 1000.0) / 1e9
    peak, peak_kind = measured_peak()
    traffic = recorded_traffic(points) if args.workload == "sod" else None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
                "config": dict(config(args, points), tile_width=ctx.tile_width,
                               launches_per_stage=ctx.launches["stage_visc"] + ctx.launches["exchange"]),
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                        "note": (f"pinned host state -> device, one graph-captured step, state -> host; "
                                 f"{K} context(s) of {m} instance(s) on {K} stream(s), copies of one chunk "
                                 f"overlapping the step of another")},
                "gpu_launches": launches["n"],
                "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": alu_peak, "unit": "TFLOP/s",
                             "frac": achieved_tf / alu_peak, "traffic": traffic,
                             "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz"
                                            + (" / 64 (FP64)" if dtype == fcsdnn.F64 else ""),
                             "kernel": "rk_stage (flux pass along q1 + flux pass along q2 with stage update)",
                             "alg_flops_per_point_stage": flops_pt, "stage_ms": stage_avg_ms,
                             "hbm_context": {"alg_bytes_per_point_stage": alg_bytes_pt, "achieved_gbs": hbm_gbs,
                                             "peak_gbs": peak, "frac": hbm_gbs / peak, "peak_source": peak_kind}},
                "clocks": clocks, "status": rc, "classifier": learned}
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(args.cpu_seconds, args.workload)
        print(json.dumps(line))
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

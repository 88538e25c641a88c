"""The shock-tube configuration in full (GPU, C ABI): Sod data on [0,1] x
[0,0.1] split into 8 overlapping Cartesian patches of 160 x 40 points
(overlap 10), run to t = 0.2 in FP64 and in FP32 with the BF16 classifier,
from Sod data with the jump smoothed over two grid spacings, compared with the
exact Riemann solution in L1 (§7, Sod; the oracle's scheme is pinned to the
same exact solution under refinement by the CPU tests) and with each other.

Two runs per precision: (1) viscosity where the network (trained on windows
of the solver's own FC step) flags the proxy; (2) viscosity everywhere.  The
second isolates the arithmetic: FP32 and FP64 agree to ~1e-5 there.  In the
first the classifier's discrete decisions feed back on the state over ~7000
steps, and the FP32 trajectory ends with more viscosity than the FP64 one
(more steps, a smeared rarefaction): measured L1 2.5e-3..2.9e-3 (FP64) and
7.6e-3..7.7e-3 (FP32) against the exact solution, with d = 5 and d = 2 alike.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import exact, sdnn  # noqa: E402
from paper_2506_19370_gb300 import fcsdnn  # noqa: E402
from paper_2506_19370_gb300 import inputs as I  # noqa: E402

T_END = 0.2


def _trained_weights():
    """The network trained on labelled windows of the solver's own FC step
    (training.py), by the library's training kernels."""
    from paper_2506_19370_gb300 import training as T
    src = T.WindowSource(chunk=256, seed=I.SEED)
    X, Y, _ = T.make_dataset(300_000, src)
    src.ctx.set_weights(sdnn.init_params(0).astype(np.float32))
    T.train(src.ctx, X, Y, steps=1500)
    w = src.ctx.get_weights()
    src.ctx.close()
    return w


def _run(dtype, w, everywhere=False):
    # 8 patches of 160 x 40, overlap 10; the jump at x = 0.5 as a tanh profile
    # two spacings wide (smoothed initial data)
    inst = I.sod_instance(smear=2.0)
    ctx = fcsdnn.Context(inst, dtype=dtype, c_policy=1)
    ctx.set_weights(w)
    e = ctx.to_device(ctx.pack_state(inst.state))
    dtd = torch.zeros(1, dtype=torch.float64, device="cuda")
    tau, mu = ctx.new_scalar(torch.int8), ctx.new_scalar()
    S, A = ctx.new_state(), ctx.new_state()
    t, steps = 0.0, 0
    while t < T_END - 1e-12:
        # the step's CFL time step with its viscosity, clipped to the end time
        if everywhere:
            tau.fill_(1)
        else:
            ctx.classify(e, tau)
        ctx.av_assemble(e, tau, mu)
        ctx.time_step(e, dtd, mu)
        dt = min(float(dtd.item()), T_END - t)
        for k in range(4):
            ctx.rk_stage(k, dt, e, e if k == 0 else S, A, e if k == 3 else S, mu=mu)
            ctx.patch_exchange(e if k == 3 else S, 4)
        t += dt
        steps += 1
        assert steps < 20000
    torch.cuda.synchronize()
    rc, _ = ctx.status()
    st = ctx.unpack_state(e)
    xs, rho = [], []
    for p, s in zip(inst.patches, st):
        X, _ = p.coords()
        xs.append(X[p.n2 // 2])
        rho.append(s[0, p.n2 // 2])
    ctx.close()
    return rc, np.concatenate(xs), np.concatenate(rho), steps


def test_sod_eight_patches_to_t_02():
    w = _trained_weights()
    out = {}
    for ev in (False, True):
        for dt_ in (fcsdnn.F64, fcsdnn.F32):
            out[(ev, dt_)] = _run(dt_, w, everywhere=ev)
    x = out[(False, fcsdnn.F64)][1]
    ex = exact.riemann_sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (x - 0.5) / T_END)[0]
    l1 = {k: float(np.mean(np.abs(v[2] - ex))) for k, v in out.items()}
    for ev in (False, True):
        r64, r32 = out[(ev, fcsdnn.F64)][2], out[(ev, fcsdnn.F32)][2]
        print(f"\nSod 8 x (160 x 40) to t = {T_END}, viscosity {'everywhere' if ev else 'where the network flags'}: "
              f"FP64 {out[(ev, fcsdnn.F64)][3]} steps L1(rho) {l1[(ev, fcsdnn.F64)]:.3e}; FP32 "
              f"{out[(ev, fcsdnn.F32)][3]} steps L1(rho) {l1[(ev, fcsdnn.F32)]:.3e}; "
              f"L1(FP32 - FP64) {np.mean(np.abs(r32 - r64)):.3e}; overshoot FP64 {max(r64.max() - 1, 0):.2e} "
              f"FP32 {max(r32.max() - 1, 0):.2e}")
    assert all(v[0] == 0 for v in out.values())
    # the method with the trained network, against the exact solution
    assert l1[(False, fcsdnn.F64)] < 4e-3 and l1[(False, fcsdnn.F32)] < 1e-2
    # the network localizes the viscosity: both beat viscosity everywhere
    assert l1[(False, fcsdnn.F64)] < 0.5 * l1[(True, fcsdnn.F64)]
    assert l1[(False, fcsdnn.F32)] < 0.5 * l1[(True, fcsdnn.F32)]
    # the arithmetic: with a state-independent viscosity pattern FP32 follows FP64
    r64, r32 = out[(True, fcsdnn.F64)][2], out[(True, fcsdnn.F32)][2]
    assert np.mean(np.abs(r32 - r64)) < 1e-4

"""sdnn_gradient_noalloc: the classifier gradient for callers that cannot
allocate device memory (hosts that only pass in buffers from their own
arenas).  It must agree with sdnn_gradient, which uses a context's buffers,
on consecutive calls that reuse its fixed scratch array.

This file is named to run last, after every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_gradient_matches_context_gradient():
    import os
    from paper_2506_19370_gb300 import build, fcsdnn
    from paper_2506_19370_gb300 import inputs as I
    if not os.path.exists(fcsdnn.LIB_PATH):
        build.build()
    assert torch.cuda.is_available()
    inst = I.sod_instance(npatch=1, n1=64, n2=32)
    ctx = fcsdnn.Context(inst, c_policy=1)
    rng = np.random.default_rng(17)
    w = (0.3 * rng.standard_normal(fcsdnn.N_PARAMS)).astype(np.float32)
    ctx.set_weights(w)
    wd = torch.from_numpy(w).cuda()
    # two calls in a row with different batches: the second reuses the
    # scratch array the first one filled
    for batch, seed in ((3000, 1), (517, 2)):
        x, y = I.classifier_windows(batch, seed=seed)
        xd = torch.from_numpy(x.astype(np.float32)).cuda()
        yd = torch.from_numpy(y).cuda()
        g_ref = torch.zeros(fcsdnn.N_PARAMS, dtype=torch.float32, device="cuda")
        l_ref = torch.zeros(1, dtype=torch.float32, device="cuda")
        ctx.gradient(xd, yd, g_ref, l_ref)
        g = torch.full((fcsdnn.N_PARAMS,), float("nan"), dtype=torch.float32, device="cuda")
        l = torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")
        fcsdnn.gradient_noalloc(wd, xd, yd, g, l)
        torch.cuda.synchronize()
        a, b = g.cpu().numpy(), g_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.max(np.abs(a - b)) <= 1e-6 * np.max(np.abs(b))
        assert abs(l.item() - l_ref.item()) <= 1e-6 * abs(l_ref.item())
    # a batch beyond the fixed scratch is rejected without launching
    big = torch.zeros((fcsdnn.NOALLOC_BATCH_MAX + 1, 16), dtype=torch.float32, device="cuda")
    lab = torch.ones(fcsdnn.NOALLOC_BATCH_MAX + 1, dtype=torch.int8, device="cuda")
    with pytest.raises(fcsdnn.FcsError) as ei:
        fcsdnn.gradient_noalloc(wd, big, lab, g)
    assert ei.value.code == -8
    ctx.close()

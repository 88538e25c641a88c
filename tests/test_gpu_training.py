"""Classifier training data from the solver's own FC step (GPU, C ABI).

Seeded flow states with jumps, kinks and C1 features at known places go
through one Runge-Kutta step of the library's FC operator; the library cuts
the proxy windows as the classifier does (sdnn_windows, checked here against
the oracle's proxy and window cut on the same state); the windows, labelled
from the known feature places, train the network with the library's own
training kernels; the trained network (BF16 tensor-core inference) and the
coefficient-decay indicator are then scored against the known features on
windows of states neither has seen.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sdnn  # noqa: E402
from paper_2506_19370_gb300 import fcsdnn  # noqa: E402
from paper_2506_19370_gb300 import inputs as I  # noqa: E402
from paper_2506_19370_gb300 import training as T  # noqa: E402


@pytest.fixture(scope="module")
def src():
    from paper_2506_19370_gb300 import build
    import os
    if not os.path.exists(fcsdnn.LIB_PATH):
        build.build()
    return T.WindowSource(chunk=256, seed=7)


def test_windows_match_the_oracle_proxy_windows(src):
    # the raw windows of an FC-stepped state against the oracle's proxy and
    # window cut of the same (FP32) state
    c = src.ctx
    src.fc_step(0)
    c.windows_raw(src.e, src.x, src.flat)
    torch.cuda.synchronize()
    got = src.x.view(src.chunk, c.windows, 16).cpu().numpy().astype(np.float64)
    flat = src.flat.view(src.chunk, c.windows).cpu().numpy()
    for k in (0, 17, 255):
        e = c.unpack_state(src.e, k)[0]
        win, cover = sdnn.patch_windows(sdnn.proxy(e, I.GAMMA))
        assert win.shape == got[k].shape
        # the FP32 proxy against the FP64 proxy of the same FP32 state
        assert np.abs(got[k] - win).max() <= 1e-6 * np.abs(win).max()
        _, fl = sdnn.normalise(win)
        rng_w = win.max(1) - win.min(1)
        clear = np.abs(rng_w - 1e-4 * np.maximum(1.0, np.abs(win).max(1))) > 1e-6 * np.abs(win).max()
        assert np.array_equal(flat[k][clear].astype(bool), fl[clear])
        # the row windows come first, in the order of training.row_window_labels
        assert all(d == 0 for d, _, _ in cover[:src.nx]) and all(d == 1 for d, _, _ in cover[src.nx:])
        assert [(line, s) for _, line, s in cover[:src.nx]] == [(j, s) for j in range(T.N2)
                                                               for s in T.window_starts(T.N1)]


def test_network_trained_on_fc_step_windows(src):
    c = src.ctx
    X, Y, nchunks = T.make_dataset(300_000, src)
    counts = torch.bincount(Y.long(), minlength=5).cpu().numpy()[1:]
    assert counts.min() > 0.15 * counts.sum(), counts            # about balanced classes
    c.set_weights(sdnn.init_params(0).astype(np.float32))
    l0, l1 = T.train(c, X, Y, steps=1500)
    res = T.evaluate(src, nchunks + 5)                            # states it has not seen
    # the same network trained on raw analytic windows (no FC step), for comparison
    c.set_weights(sdnn.init_params(0).astype(np.float32))
    xr, yr = I.classifier_windows(300_000, seed=3)
    T.train(c, torch.from_numpy(xr.astype(np.float32)).cuda(), torch.from_numpy(yr).cuda(), steps=1500)
    raw = T.evaluate(src, nchunks + 5)
    print(f"\nFC-step windows: {int(Y.numel())} from {nchunks} chunks, classes {counts.tolist()}; loss {l0:.3f} -> "
          f"{l1:.3f}\n  trained on FC-step windows: {res}\n  trained on raw windows:     {raw}")
    assert l1 < 0.5 * l0
    assert res["accuracy"] > 0.8 and res["recall_1"] > 0.9
    assert res["jump_false_positive"] < 0.05
    # the network beats the coefficient-decay indicator on the classes both separate
    assert res["network_accuracy_c1_smooth_merged"] > res["indicator_accuracy_c1_smooth_merged"]

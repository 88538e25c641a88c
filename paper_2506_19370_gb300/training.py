"""Training data for the shock-detecting classifier, produced by the solver's
own FC step, and its training and evaluation on the device.

The paper loads a trained network (Algorithm 2); its training data and
weights are not available, so the network is trained here (§4, §5 item 2:
the classifier sees 16-point windows of the Mach-number proxy along the grid
lines).  Windows come from what the solver itself produces: seeded flow
states with jumps, kinks and C1 features at known places
(`inputs.feature_profiles`) are advanced by one Runge-Kutta step of the FC
operator (FC-Gram continuation, FFT derivatives; no viscosity, so the
Gibbs-type ringing the operator makes near a jump is in the data), and the
library cuts the proxy windows exactly as the classifier does
(`sdnn_windows`).  A window gets the class of the feature inside it (at
least one grid point from its ends), 4 (smooth) if no feature is within one
point of it, and is left out otherwise; flat windows (classified smooth
without inference) are left out too.  Smooth windows are subsampled so that
the four classes are about equally frequent.

Everything on the device runs through the library's C ABI (`fcsdnn`); this
module only generates inputs, keeps the labels and moves tensors.
"""
import numpy as np

from . import fcsdnn
from . import inputs as I

N1, N2, PER_ROW = 256, 16, 8
WINDOW = 16
MARGIN = 1.0      # a feature counts inside a window from MARGIN points in from its ends
STEP_CFL = 0.25   # the FC step: one RK4 step at this fraction of the CFL time step
PARTS = 8         # host threads generating a chunk's profiles


def window_starts(N, W=WINDOW):
    """Starts 0, 16, 32, ... of the windows of an N-point line; the last one
    right-aligned (the classifier's cut of a line)."""
    s = list(range(0, N - W + 1, W))
    if s[-1] + W < N:
        s.append(N - W)
    return np.array(s)


def row_window_labels(features, n1=N1, n2=N2, h=None):
    """Labels of the windows along the rows (q1 lines) of the profile patch,
    [instance][row][window]: 1..4, or 0 where a feature sits within MARGIN of
    a window end (left out)."""
    h = h if h is not None else 1.0 / (n1 - 1)
    cls, a, b = features["cls"], features["a"], features["b"]
    starts = window_starts(n1)
    y = np.arange(n2) * h
    # feature positions in grid units, (B, K, n2)
    pos = (a[:, :, None] + b[:, None, None] * y[None, None, :]) / h
    B, K = cls.shape
    lab = np.full((B, n2, len(starts)), 4, dtype=np.int8)
    for k in range(K):
        c = cls[:, k]
        has = c != I.CLASS_SMOOTH
        p = pos[:, k, :][:, :, None]                             # (B, n2, 1)
        s0 = starts[None, None, :]
        inside = (p >= s0 + MARGIN) & (p <= s0 + WINDOW - 1 - MARGIN)
        near = (p > s0 - MARGIN - 1) & (p < s0 + WINDOW + MARGIN) & ~inside
        cc = np.broadcast_to(c[:, None, None], lab.shape)
        hh = np.broadcast_to(has[:, None, None], lab.shape)
        lab = np.where(hh & near, np.int8(0), lab)
        lab = np.where(hh & inside & (lab != 0), cc, lab)
    return lab


class WindowSource:
    """Labelled windows of FC-stepped feature profiles, a chunk of `chunk`
    instances at a time, on one FP32 context (its network is the one trained
    and evaluated)."""

    def __init__(self, chunk=2048, seed=I.SEED, d=5):
        import torch
        if chunk % PARTS:
            raise ValueError(f"chunk must be a multiple of {PARTS}")
        self.torch = torch
        self.chunk, self.seed = chunk, seed
        patch, st, feat = I.feature_profiles(1, seed=seed)
        self.patch = patch
        # d: the FC-Gram degree of the solver whose FC step makes the windows
        self.ctx = fcsdnn.Context(I.Instance([patch], st), d=d, dtype=fcsdnn.F32, instances=chunk, c_policy=1,
                                  train_batch_max=4096)
        self.nx = N2 * len(window_starts(N1))       # row windows come first in the window table
        c = self.ctx
        self.e = c.new_state()
        self.S, self.A = c.new_state(), c.new_state()
        self.dtd = torch.zeros(chunk, dtype=torch.float64, device=self.e.device)
        self.x = torch.empty(chunk * c.windows * WINDOW, dtype=torch.float32, device=self.e.device)
        self.flat = torch.empty(chunk * c.windows, dtype=torch.int8, device=self.e.device)

    def profiles(self, k):
        """Seeded profile states of chunk k, generated in PARTS sub-batches on
        host threads (numpy releases the interpreter lock in its array
        operations)."""
        from concurrent.futures import ThreadPoolExecutor
        sub = self.chunk // PARTS
        with ThreadPoolExecutor(PARTS) as ex:
            res = list(ex.map(lambda q: I.feature_profiles(sub, seed=(self.seed * 1000 + k) * 64 + q), range(PARTS)))
        st = [x for r in res for x in r[1]]
        feat = {key: np.concatenate([r[2][key] for r in res]) for key in ("cls", "a", "b")}
        return st, feat

    def fc_step(self, k):
        """Chunk k: profile states, one RK4 step of the FC operator (no
        viscosity), returns the features."""
        torch, c = self.torch, self.ctx
        st, feat = self.profiles(k)
        self.e.copy_(torch.from_numpy(c.pack_state([[s] for s in st])))
        c.time_step(self.e, self.dtd)
        dt = STEP_CFL * float(self.dtd.min().item())
        for s in range(4):
            c.rk_stage(s, dt, self.e, self.e if s == 0 else self.S, self.A, self.e if s == 3 else self.S)
        return feat

    def chunk_windows(self, k, smooth_keep=None, rng=None):
        """(X, Y) device tensors of chunk k: raw row windows (n x 16) and labels."""
        torch, c = self.torch, self.ctx
        feat = self.fc_step(k)
        c.windows_raw(self.e, self.x, self.flat)
        lab = torch.from_numpy(row_window_labels(feat).reshape(self.chunk, -1)).to(self.e.device)
        X = self.x.view(self.chunk, c.windows, WINDOW)[:, :self.nx]
        F = self.flat.view(self.chunk, c.windows)[:, :self.nx]
        keep = (lab > 0) & (F == 0)
        if smooth_keep is not None:
            r = torch.rand(lab.shape, generator=rng, device=self.e.device)
            keep &= (lab != I.CLASS_SMOOTH) | (r < smooth_keep)
        return X[keep].contiguous(), lab[keep].contiguous()


def make_dataset(total, src, smooth_keep=0.2):
    """About `total` labelled windows from successive chunks of `src`."""
    torch = src.torch
    g = torch.Generator(device=src.e.device)
    g.manual_seed(src.seed)
    xs, ys, n, k = [], [], 0, 0
    while n < total:
        X, Y = src.chunk_windows(k, smooth_keep, g)
        xs.append(X)
        ys.append(Y)
        n += int(Y.numel())
        k += 1
    return torch.cat(xs)[:total], torch.cat(ys)[:total], k


def train(ctx, X, Y, steps, batch=4096, lr=3e-3, seed=I.SEED):
    """`steps` Adam steps of the library's training kernels on random
    batches of (X, Y); returns the mean loss of the first and last 10 steps."""
    torch = ctx.torch
    g = torch.Generator(device=X.device)
    g.manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float32, device=X.device)
    first, last = [], []
    for s in range(steps):
        idx = torch.randint(0, Y.numel(), (batch,), generator=g, device=X.device)
        ctx.train_step(X[idx].contiguous(), Y[idx].contiguous(), lr, loss)
        if s < 10:
            first.append(loss.item())
        elif s >= steps - 10:
            last.append(loss.item())
    return float(np.mean(first)), float(np.mean(last))


def indicator_class(s):
    """tau_hat of the coefficient-decay indicator from its decay rate s (the
    cut points 2.7 and 4.4 of sdnn_indicator; flat windows have s = inf)."""
    return np.where(s < 2.7, 1, np.where(s < 4.4, 2, 4)).astype(np.int8)


def evaluate(src, k):
    """Classifier (BF16 tensor-core inference, sdnn_classify) and the
    coefficient-decay indicator (sdnn_indicator) on the row windows of chunk
    k against the known feature classes: accuracy per class and overall,
    indicator accuracy (C1 and smooth counted together: on 16 points the
    indicator does not separate them), and their agreement."""
    torch, c = src.torch, src.ctx
    feat = src.fc_step(k)
    lab = row_window_labels(feat).reshape(src.chunk, -1)
    logits = torch.zeros(src.chunk * c.windows * 4, dtype=torch.float32, device=src.e.device)
    tau = c.new_scalar(torch.int8)
    c.classify(src.e, tau, logits)
    sw = torch.zeros(src.chunk * c.windows, dtype=torch.float32, device=src.e.device)
    c.indicator(src.e, tau, sw)
    c.windows_raw(src.e, src.x, src.flat)
    torch.cuda.synchronize()
    z = logits.view(src.chunk, c.windows, 4)[:, :src.nx].cpu().numpy()
    flat = src.flat.view(src.chunk, c.windows)[:, :src.nx].cpu().numpy().astype(bool)
    s_ind = sw.view(src.chunk, c.windows)[:, :src.nx].cpu().numpy()
    net = np.where(flat, 4, 1 + np.argmax(z, axis=2))
    ind = indicator_class(s_ind)
    ok = (lab > 0) & ~flat
    res = {"windows": int(ok.sum()), "accuracy": float(np.mean(net[ok] == lab[ok]))}
    for cl in (1, 2, 3, 4):
        m = ok & (lab == cl)
        res[f"recall_{cl}"] = float(np.mean(net[m] == cl)) if m.any() else None
    merge = lambda t: np.where(t == 3, 4, t)
    res["indicator_accuracy_c1_smooth_merged"] = float(np.mean(merge(ind[ok]) == merge(lab[ok])))
    res["network_accuracy_c1_smooth_merged"] = float(np.mean(merge(net[ok]) == merge(lab[ok])))
    res["agreement_network_indicator"] = float(np.mean(merge(net[ok]) == merge(ind[ok])))
    # jumps are what the viscosity is for: false negatives and false positives
    res["jump_false_negative"] = float(np.mean(net[ok & (lab == 1)] != 1))
    res["jump_false_positive"] = float(np.mean(net[ok & (lab != 1)] == 1))
    res["indicator_jump_false_negative"] = float(np.mean(ind[ok & (lab == 1)] != 1))
    res["indicator_jump_false_positive"] = float(np.mean(ind[ok & (lab != 1)] == 1))
    return res

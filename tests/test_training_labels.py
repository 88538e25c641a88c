"""Labels of the classifier's training windows against the profiles themselves
(CPU): a window labelled a jump holds a grid-to-grid step at least as large
as the smallest jump amplitude, a window labelled smooth holds none, and each
jump, kink or C1 feature of a row lands in at most one labelled window."""
import numpy as np

from paper_2506_19370_gb300 import inputs as I
from paper_2506_19370_gb300 import training as T


def test_window_starts_cover_lines():
    for N in (16, 40, 160, 256, 257):
        s = T.window_starts(N)
        assert s[0] == 0 and s[-1] == N - T.WINDOW
        covered = np.zeros(N, bool)
        for a in s:
            covered[a:a + T.WINDOW] = True
        assert covered.all()


def test_row_labels_match_the_profiles():
    patch, st, feat = I.feature_profiles(64, seed=3)
    lab = T.row_window_labels(feat)
    starts = T.window_starts(T.N1)
    lr = np.log(np.stack([s[0] for s in st]))                   # (B, n2, n1)
    step = np.abs(np.diff(lr, axis=2))                          # |log rho jump| between neighbours
    counts = {c: 0 for c in (0, 1, 2, 3, 4)}
    for b in range(lab.shape[0]):
        for j in range(lab.shape[1]):
            for w, s0 in enumerate(starts):
                L = lab[b, j, w]
                counts[int(L)] += 1
                big = step[b, j, s0:s0 + T.WINDOW - 1].max()
                if L == I.CLASS_JUMP:
                    assert big >= 0.099, (b, j, s0, big)        # jump amplitudes are >= 0.1
                elif L == I.CLASS_SMOOTH:
                    assert big < 0.099, (b, j, s0, big)
    # every class occurs, and a feature lands in at most one labelled window per row
    assert all(counts[c] > 100 for c in (1, 2, 3, 4)), counts
    nfeat = int(np.sum(feat["cls"] != I.CLASS_SMOOTH)) * lab.shape[1]
    assert counts[1] + counts[2] + counts[3] <= nfeat
    assert counts[1] + counts[2] + counts[3] + counts[0] >= nfeat

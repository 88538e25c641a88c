"""Write oracle/fcgram_tables.npz: the oracle's own FP64 FC-Gram tables for
d = 5 and C = 20..64 (every continuation length the FFT-length policy can
pick for C = 25): the combined right-end table A_R (key d5_C<C>) and the
blend values T of the Gram polynomials (key T_d5_C<C>), so that test runs do
not redo the 40-digit fits.

Run from the repository root:  python -m oracle.make_tables
Only oracle code is called; the file is a cache of `fcgram.blend_fit`.
"""
import multiprocessing as mp
import os

import numpy as np

D = 5
CS = range(20, 65)


def _one(C):
    from oracle import fcgram
    A_R, _ = fcgram.continuation_tables(D, C, use_store=False)
    _, _, T = fcgram.gram_tables(D, C, use_store=False)
    return C, A_R, T


def main():
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        res = pool.map(_one, sorted(CS, reverse=True))
    out = {}
    for C, A, T in res:
        out[f"d{D}_C{C}"] = A
        out[f"T_d{D}_C{C}"] = T
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fcgram_tables.npz")
    np.savez_compressed(path, **out)
    print(f"wrote {len(out)} tables to {path}")


if __name__ == "__main__":
    main()

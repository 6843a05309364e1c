"""Writes pba_headline_digests.txt from the oracle alone.

The PBA workload at the paper's headline size (Table 1: 10^9 vertices, 5e9
edges): 2^30 new vertices in B = 1024 blocks of n_b = 2^20, m = 5, seed
clique n0 = 6, faction width 1, inter-faction probability f = 0.1, seed 3.
Runs the oracle's phase 1 for every block (Sec. 3, phase 1: the list A_p),
then every block's phase-2 endpoint list T_q (Sec. 3, phase 2), and writes,
per block, the digests of tests/pba_digest.py: D1 over A_p in entry order,
D2 over the slices of every T_q that the block receives, in the ascending
requester order of reading R4, and R_q, the length of block p's own T_p.

    python tests/golden/make_pba_headline_digests.py [threads]

Calls nothing but oracle/ (about 2 minutes on 8 cores).
"""
import os
import sys
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

import oracle as o            # noqa: E402
import pba_digest as dg       # noqa: E402

B, NB, M, N0, W, F, SEED = 1024, 2**20, 5, 6, 1, 0.1, 3
NE = NB * M
OUT = os.path.join(HERE, "pba_headline_digests.txt")


def main(threads: int):
    t0 = time.time()
    counts = np.zeros((B, B), dtype=np.uint64)
    d1 = np.zeros(B, dtype=np.uint64)
    pos = np.arange(NE, dtype=np.uint64)

    def phase1(p):
        A, cnt, _ = o.pba_phase1(p, B, W, NE, F, SEED)
        counts[p] = cnt
        d1[p] = np.sum(dg.f_np(A, pos), dtype=np.uint64)

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(phase1, range(B)))
    R = counts.sum(axis=0, dtype=np.uint64)
    off = np.cumsum(counts, axis=0, dtype=np.uint64) - counts    # off[p][q]
    print(f"phase 1: {time.time() - t0:.0f} s", flush=True)

    parts = []

    def phase2(qs):
        d2 = np.zeros(B, dtype=np.uint64)
        for q in qs:
            T = o.pba_endpoints(q, int(R[q]), NB, N0, SEED)
            c = counts[:, q]
            nz = np.nonzero(c)[0]
            start = np.repeat(off[:, q], c.astype(np.int64))
            k = np.arange(len(T), dtype=np.uint64) - start
            vals = dg.f_np(T, k)
            sd = np.add.reduceat(vals, off[nz, q].astype(np.int64), dtype=np.uint64)
            d2[nz] += dg.g_np(np.full(len(nz), q, dtype=np.uint64), sd)
        parts.append(d2)

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(phase2, [range(t, B, threads) for t in range(threads)]))
    d2 = np.zeros(B, dtype=np.uint64)
    for part in parts:
        d2 += part
    print(f"phase 2: {time.time() - t0:.0f} s", flush=True)
    with open(OUT, "w") as fh:
        fh.write("# PBA at the paper's headline size (Table 1): n = 2^30 new vertices, B = 1024\n"
                 "# blocks of n_b = 2^20, m = 5, n0 = 6, W = 1, f = 0.1, seed 3. Written by\n"
                 "# make_pba_headline_digests.py from the oracle alone. Per block p:\n"
                 "# p, D1[p], D2[p] (tests/pba_digest.py), R_p (entries of T_p), hex.\n")
        for p in range(B):
            fh.write(f"{p} {int(d1[p]):016x} {int(d2[p]):016x} {int(R[p]):x}\n")
    print(f"wrote {OUT} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 4))

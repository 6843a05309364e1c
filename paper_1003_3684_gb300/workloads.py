"""Synthetic workloads: the named configurations and seeded input generators.

This module holds parameters and seeded random inputs only -- none of the
generators' arithmetic -- so that both the CUDA path and the CPU oracle can be
driven from the same inputs. The configurations follow the paper's problem
statement (vertex count, edges per new vertex, block count, initiator, seed).
"""
from __future__ import annotations

import numpy as np

# Initiator of the stochastic Kronecker configuration (2x2, row-major).
KRON_INITIATOR = [[0.57, 0.19], [0.19, 0.05]]

# Seed graph of the deterministic Kronecker example (Sec. 3, PK method, Fig.
# 2(b)): 5 vertices, 11 edges including the self-loops, row-major 0/1.
PK_FIG2_SEED = [[1, 1, 1, 1, 0], [1, 1, 0, 0, 0], [1, 0, 1, 0, 0], [1, 0, 0, 1, 0],
                [0, 0, 0, 0, 1]]

CONFIGS = {
    # serial BA: 100,000 new vertices, 4 edges each, seed clique K5
    "ba_n100k_m4": dict(kind="pba", n=100_000, m=4, blocks=1, n0=5, faction_width=1,
                        inter_frac=0.0, seed=1),
    # stochastic Kronecker, k = 20 levels (2^20 vertices), 16 * 2^20 edges, plus CSR
    "kron_k20_m16x_csr": dict(kind="kron", initiator=KRON_INITIATOR, k=20,
                              n_edges=16 * 2**20, seed=7, csr=True),
    # deterministic Kronecker of the Fig. 2 seed at k = 8: 5^8 = 390,625
    # vertices, 11^8 = 214,358,881 edges (1.7 GB of pairs), in stack order
    "kron_det_fig2_k8": dict(kind="kron_det", initiator=PK_FIG2_SEED, k=8, seed=0),
    # the same initiator at k = 26 (2^26 vertices, 2^30 edges: 8.6 GB of pairs)
    "kron_k26_m16x_csr": dict(kind="kron", initiator=KRON_INITIATOR, k=26,
                              n_edges=16 * 2**26, seed=7, csr=True),
    # two-phase PBA at the paper's headline size: 2^30 new vertices in 1024
    # blocks of 2^20, 5 edges each, inter-block fraction 0.1
    "pba_n2p30_b1024_m5": dict(kind="pba", n=2**30, m=5, blocks=1024, n0=6, faction_width=1,
                               inter_frac=0.1, seed=3),
    # the headline PBA with overlapping factions: block p's list names its
    # neighbours p-1, p, p+1 (mod 1024), so every block shares its faction
    # with two others, as F0..F2 of Fig. 1 overlap
    "pba_n2p30_b1024_m5_factions": dict(kind="pba", n=2**30, m=5, blocks=1024, n0=6,
                                        faction_width=1, factions="ring3", inter_frac=0.1,
                                        seed=3),
    # the headline PBA made in 8 ranges of 128 blocks through an output buffer
    # one eighth of the graph (prepare once, then each range on demand)
    "pba_n2p30_b1024_m5_parts8": dict(kind="pba", n=2**30, m=5, blocks=1024, n0=6,
                                      faction_width=1, inter_frac=0.1, seed=3, parts=8),
    # Kronecker k = 20 made irregular by exclusive-or with a random graph of
    # 2^20 cells, then CSR keeping the cells of odd multiplicity
    "kron_k20_m16x_xor": dict(kind="kron_xor", initiator=KRON_INITIATOR, k=20,
                              n_edges=16 * 2**20, n_random=2**20, seed=7),
    # graph check: breadth-first search over the undirected CSR of a PBA graph
    # (2^24 new vertices in 64 blocks, m = 5) from 8 fixed sources
    "bfs_pba_n2p24_b64": dict(kind="bfs", n=2**24, m=5, blocks=64, n0=6, faction_width=1,
                              inter_frac=0.1, seed=3, sources=8),
    # 4096 independent graphs of uneven sizes in one persistent launch
    "batch_4096_mixed": dict(kind="batch", n_jobs=4096, seed=0),
    # served requests: Poisson arrivals at 2000/s, half BA / half Kronecker,
    # edge counts log-uniform in 2^12..2^26, CSR kept on the device, admission
    # by a 64 GB device-memory budget
    "serve_poisson_2000": dict(kind="serve", rate=2000.0, duration=20.0, budget=64 << 30,
                               seed=0),
}


def ring_factions(B: int, width: int = 3):
    """Faction lists of a ring: block p's list is p - width//2 .. p + width//2 (mod B)."""
    h = width // 2
    return [[(p + d) % B for d in range(-h, width - h)] for p in range(B)]


def random_edges(seed: int, n_edges: int, n_vertices: int, id64: bool = False,
                 hub_fraction: float = 0.0) -> np.ndarray:
    """Seeded random (src, dst) list; a fraction of edges is pinned on vertex 0.

    The hub makes one very long CSR row, the shape that power-law graphs give.
    """
    rng = np.random.default_rng(seed)
    dt = np.uint64 if id64 else np.uint32
    e = rng.integers(0, max(n_vertices, 1), size=(n_edges, 2), dtype=np.uint64)
    if hub_fraction > 0 and n_edges > 0:
        k = int(n_edges * hub_fraction)
        e[rng.choice(n_edges, size=k, replace=False), 0] = 0
    return e.astype(dt)


def batch_jobs(n_jobs: int = 4096, seed: int = 0):
    """Mixed batch of independent generation jobs (uneven sizes).

    Half serial-BA jobs (m uniform in 2..8, vertex count log-uniform in
    2^10..2^22), half stochastic Kronecker jobs (scale uniform in 10..22,
    16 edges per vertex); job i uses generator seed i.
    """
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(n_jobs):
        if i < n_jobs // 2:
            m = int(rng.integers(2, 9))
            n = int(2 ** rng.uniform(10, 22))
            jobs.append(dict(kind="pba", n=n, m=m, blocks=1, n0=m + 1, faction_width=1,
                             inter_frac=0.0, seed=i))
        else:
            k = int(rng.integers(10, 23))
            jobs.append(dict(kind="kron", initiator=KRON_INITIATOR, k=k, n_edges=16 * 2**k,
                             seed=i))
    return jobs

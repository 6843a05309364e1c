"""Full-size parity of two-phase PBA at the paper's headline size.

The launch the benchmark times (Sec. 3 PBA method at Table 1's size): 2^30
new vertices in 1024 blocks of 2^20, m = 5, n0 = 6, f = 0.1, seed 3, about
5.37e9 edges. Every block is checked:
  - its seed clique and the source of every edge, exactly;
  - the digest of the target blocks it names in entry order (phase 1's A_p)
    and the digest of the endpoints each target hands it, in entry order
    (phase 2 and the substitution of Fig. 1(b)), against digests the oracle
    alone wrote (tests/golden/pba_headline_digests.txt);
  - the number of endpoints each target produces, R_q, exactly.
Eight blocks drawn at random from 8..255 are also compared edge for edge
with the oracle, run here on every host core.
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest
import torch

import oracle as o
import paper_1003_3684_gb300 as pg
import pba_digest as dg
from paper_1003_3684_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "pba_headline_digests.txt")


def _golden():
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    assert [int(r[0]) for r in rows] == list(range(len(rows)))
    return ([int(r[1], 16) for r in rows], [int(r[2], 16) for r in rows],
            np.array([int(r[3], 16) for r in rows], np.uint64))


@pytest.fixture(scope="module")
def headline():
    from paper_1003_3684_gb300 import build
    build.build()
    cfg = W.CONFIGS["pba_n2p30_b1024_m5"]
    n, m, B, n0, Wf, f, seed = (cfg[k] for k in ("n", "m", "blocks", "n0", "faction_width",
                                                 "inter_frac", "seed"))
    edges = pg.gen_pba(n, m, B, n0, Wf, f, seed)
    torch.cuda.synchronize()
    yield cfg, edges
    del edges
    torch.cuda.empty_cache()


def test_every_block_against_the_oracle_digests(headline):
    cfg, edges = headline
    n, m, B, n0 = cfg["n"], cfg["m"], cfg["blocks"], cfg["n0"]
    n_b, e0 = n // B, n0 * (n0 - 1) // 2
    N_e, span = n_b * m, n0 + n_b
    per = e0 + N_e
    D1, D2, R = _golden()
    assert len(D1) == B and int(R.sum()) == n * m
    assert edges.shape[0] == B * per
    e = edges.view(B, per, 2)
    clique = torch.tensor([[a, b] for a in range(n0) for b in range(n0) if a < b],
                          dtype=torch.int64, device="cuda")
    pos = torch.arange(N_e, dtype=torch.int64, device="cuda")
    R_gpu = torch.zeros(B, dtype=torch.int64, device="cuda")
    bad = []
    for p in range(B):
        blk = e[p].to(torch.int64) & 0xFFFFFFFF
        assert torch.equal(blk[:e0], clique + p * span), p
        assert torch.equal(blk[e0:, 0], p * span + n0 + pos // m), p
        dst = blk[e0:, 1]
        R_gpu += torch.bincount(dst // span, minlength=B)
        d1, d2 = dg.block_digests_torch(dst, span, B)
        if (d1, d2) != (D1[p], D2[p]):
            bad.append((p, d1 == D1[p], d2 == D2[p]))
    assert not bad, f"{len(bad)} blocks differ, first (block, A ok, endpoints ok): {bad[:4]}"
    assert np.array_equal(R_gpu.cpu().numpy().astype(np.uint64), R)


def test_eight_random_blocks_edge_for_edge(headline):
    cfg, edges = headline
    n, m, B, n0, Wf, f, seed = (cfg[k] for k in ("n", "m", "blocks", "n0", "faction_width",
                                                 "inter_frac", "seed"))
    n_b, e0 = n // B, n0 * (n0 - 1) // 2
    N_e, span = n_b * m, n0 + n_b
    per = e0 + N_e
    _, _, R = _golden()
    picks = sorted(np.random.default_rng(2026).choice(np.arange(8, 256), 8, replace=False))
    top = max(picks)
    counts = np.zeros((top + 1, B), np.uint64)
    lists = {}

    def phase1(p):
        A, c, _ = o.pba_phase1(p, B, Wf, N_e, f, seed)
        return p, (A if p in picks else None), c

    workers = os.cpu_count() or 8
    with cf.ThreadPoolExecutor(workers) as ex:
        for p, A, c in ex.map(phase1, range(top + 1)):
            counts[p] = c
            if A is not None:
                lists[p] = A
    start = np.cumsum(counts, axis=0) - counts            # slice starts, requester order (R4)
    upto = start[top] + counts[top]

    def prefix(q):
        return q, o.pba_endpoints(q, int(R[q]), n_b, n0, seed, int(upto[q]))

    with cf.ThreadPoolExecutor(workers) as ex:
        T = dict(ex.map(prefix, range(B)))
    for p in picks:
        local = o.pba_substitute(lists[p], B, start[p], [T[q] for q in range(B)])
        ref = np.stack([p * span + n0 + np.arange(N_e, dtype=np.uint64) // m,
                        lists[p].astype(np.uint64) * span + local.astype(np.uint64)], 1)
        got = edges[p * per + e0:(p + 1) * per].cpu().numpy().view(np.uint32).astype(np.uint64)
        bad = np.nonzero((got != ref).any(axis=1))[0]
        assert bad.size == 0, f"block {p}: {bad.size} edges differ, first at {bad[:5]}"

"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Every comparison is bit-exact: the generators are integer-only and the
output is a pure function of the arguments. Oracle inputs come from the
oracle itself or from the seeded generators in ``workloads``; nothing the
GPU produced is ever fed to the oracle.
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest
import torch

import oracle as o
import paper_1003_3684_gb300 as pg
from paper_1003_3684_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIG2 = [[1, 1, 1, 1, 0], [1, 1, 0, 0, 0], [1, 0, 1, 0, 0], [1, 0, 0, 1, 0], [0, 0, 0, 0, 1]]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1003_3684_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield
    torch.cuda.synchronize()


def host(t, id64=False):
    a = t.cpu().numpy()
    return a.view(np.uint64 if id64 else np.uint32).astype(np.uint64)


def assert_same(gpu, ref):
    assert gpu.shape == ref.shape, (gpu.shape, ref.shape)
    bad = np.nonzero((gpu != ref).any(axis=-1) if gpu.ndim == 2 else gpu != ref)[0]
    assert bad.size == 0, f"{bad.size} mismatches, first at {bad[:5]}: {gpu[bad[:3]]} vs {ref[bad[:3]]}"


# --------------------------------------------------------------------------
# Kronecker
# --------------------------------------------------------------------------

@pytest.mark.parametrize("P,k,M,seed,id64", [
    (W.KRON_INITIATOR, 20, 200_001, 7, False),
    (W.KRON_INITIATOR, 20, 1, 7, False),
    (W.KRON_INITIATOR, 20, 0, 7, False),
    ([[0.5, 0.3], [0.15, 0.05]], 7, 50_000, 1, False),
    ([[0.0, 0.6], [0.4, 0.0]], 9, 20_000, 2, False),          # zero cells at both ends
    ([[0.2, 0.5, 0.0], [0.1, 0.05, 0.05], [0.0, 0.02, 0.08]], 5, 30_001, 3, False),
    (np.arange(16.0).reshape(4, 4), 6, 40_000, 4, False),
    (np.ones((16, 16)), 2, 10_000, 6, False),
    ([[1.0]], 5, 17, 5, False),
    (W.KRON_INITIATOR, 40, 100_003, 11, True),                 # 2^40 vertices
    (W.KRON_INITIATOR, 12, 65_536, 2**40 + 3, True),           # 64-bit seed
])
def test_kron_stochastic(P, k, M, seed, id64):
    got = pg.gen_kronecker(P, k, M, seed, id64=id64)
    torch.cuda.synchronize()
    assert_same(host(got, id64), o.kron(P, k, M, seed))


@pytest.mark.parametrize("P,k,id64", [
    (FIG2, 1, False), (FIG2, 2, False), (FIG2, 3, False), (FIG2, 5, False),
    ([[1, 1], [1, 0]], 12, False), ([[0, 1], [1, 1]], 7, True),
])
def test_kron_deterministic(P, k, id64):
    got = pg.gen_kronecker(P, k, deterministic=True, id64=id64)
    ref, _ = o.kron_det(np.asarray(P, float), k)
    torch.cuda.synchronize()
    assert_same(host(got, id64), ref)


@pytest.mark.slow
def test_kron_deterministic_benchmark_size():
    """The launch the benchmark times: the Fig. 2 seed at k = 8, all
    11^8 = 214,358,881 edges compared with the oracle's literal stack."""
    cfg = W.CONFIGS["kron_det_fig2_k8"]
    got = pg.gen_kronecker(cfg["initiator"], cfg["k"], deterministic=True)
    torch.cuda.synchronize()
    ref, peak = o.kron_det(np.asarray(cfg["initiator"], float), cfg["k"])
    assert ref.shape[0] == 11 ** 8 and peak <= cfg["k"] * 10 + 1
    assert np.array_equal(host(got), ref)


def test_kron_deterministic_large_seed():
    rng = np.random.default_rng(9)
    P = (rng.random((40, 40)) < 0.15).astype(float)
    P[0, 0] = 1.0
    got = pg.gen_kronecker(P, 2, deterministic=True)
    ref, _ = o.kron_det(P, 2)
    assert_same(host(got), ref)


# --------------------------------------------------------------------------
# Serial BA (blocks = 1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,m,n0,seed,id64", [
    (100_000, 4, 5, 1, False),    # serial BA workload: 100k new vertices, m = 4, K5 seed
    (33_333, 3, 2, 5, False),
    (5_000, 8, 9, 2**33 + 1, True),
    (1, 1, 2, 0, False),
    (0, 4, 5, 1, False),
    (4097, 1, 3, 8, False),
])
def test_ba(n, m, n0, seed, id64):
    got = pg.gen_pba(n, m, 1, n0, 1, 0.0, seed, id64=id64)
    torch.cuda.synchronize()
    assert_same(host(got, id64), o.ba(n, m, n0, seed).astype(np.uint64))


# --------------------------------------------------------------------------
# Two-phase PBA
# --------------------------------------------------------------------------

PBA_CASES = [
    # B, n_b, m, W, f, n0, seed
    (8, 30_000, 5, 1, 0.1, 6, 3),      # spans the smem prefix, tiles and segments
    (16, 10_000, 4, 2, 0.3, 4, 7),
    (6, 20_000, 7, 3, 1.0, 3, 11),     # every later entry is an inter-faction pick
    (5, 40_000, 2, 5, 0.5, 5, 2),      # one faction holds every block
    (4, 70_000, 3, 1, 0.0, 2, 9),      # isolated blocks
    (1024, 100, 5, 1, 0.1, 6, 3),      # many blocks, short lists
    (3, 1, 1, 1, 0.2, 2, 1),           # one vertex per block
    (7, 0, 3, 7, 0.1, 4, 1),           # no new vertices: seed cliques only
    (2, 50_000, 1, 1, 0.9, 2, 12345),
    (16, 2**14, 5, 1, 0.1, 6, 5),      # n_b a power of two: shift instead of division
    (4, 5_000, 3, 1, 0.2, 40, 8),      # 780 seed edges: long seed-endpoint walks
    (8, 3_000, 48, 2, 0.25, 49, 21),   # many edges per vertex
    (4, 3_329, 5, 1, 0.1, 6, 31),      # 16,645 entries: a last segment of one run + 5 entries
    (9, 5, 5, 1, 0.3, 6, 4),           # 25 entries per block: fewer than a warp's lanes
]


@pytest.mark.parametrize("B,n_b,m,Wf,f,n0,seed", PBA_CASES)
def test_pba(B, n_b, m, Wf, f, n0, seed):
    n = B * n_b
    got = pg.gen_pba(n, m, B, n0, Wf, f, seed)
    ref, _, _ = o.pba(n, m, B, n0, Wf, f, seed)
    torch.cuda.synchronize()
    assert_same(host(got), ref)


@pytest.fixture
def wide_path():
    pg.pg_force_wide_path(True)
    try:
        yield
    finally:
        pg.pg_force_wide_path(False)


@pytest.mark.parametrize("B,n_b,m,Wf,f,n0,seed,id64", [
    (8, 30_000, 5, 1, 0.1, 6, 3, False),
    (5, 40_000, 2, 5, 0.5, 5, 2, True),
    (1024, 100, 5, 1, 0.1, 6, 3, False),
    (16, 2**14, 5, 1, 0.1, 6, 5, False),
    (4, 5_000, 3, 1, 0.2, 40, 8, False),
    (3, 1, 1, 1, 0.2, 2, 1, False),
    (1, 60_000, 4, 1, 0.0, 5, 1, False),          # blocks = 1: the serial kernel
    (1, 20_000, 3, 1, 0.0, 2, 2**33 + 1, True),
])
def test_pba_wide_index_variants_match_oracle(wide_path, B, n_b, m, Wf, f, n0, seed, id64):
    """The 64-bit-index kernels (otherwise reached only past 2^32 entries per
    block) give the oracle's graph."""
    n = B * n_b
    got = pg.gen_pba(n, m, B, n0, Wf, f, seed, id64=id64)
    ref = o.ba(n, m, n0, seed) if B == 1 else o.pba(n, m, B, n0, Wf, f, seed)[0]
    torch.cuda.synchronize()
    assert_same(host(got, id64), np.asarray(ref).astype(np.uint64))


def test_pba_wide_choice_follows_the_prepared_workspace():
    """Prepared with the 64-bit variants forced, emitted after the switch is
    off (and the reverse): every range still equals the oracle's graph."""
    B, n_b, m, n0, seed = 6, 20_000, 4, 5, 17
    n = B * n_b
    ref, _, _ = o.pba(n, m, B, n0, 1, 0.1, seed)
    ref = np.asarray(ref).astype(np.uint64)
    per = ref.shape[0] // B
    pg.pg_force_wide_path(True)
    try:
        ws_wide = pg.pg_pba_prepare(n, m, B, n0, seed=seed)
    finally:
        pg.pg_force_wide_path(False)
    ws_fast = pg.pg_pba_prepare(n, m, B, n0, seed=seed)
    pg.pg_force_wide_path(True)
    try:
        part_a = pg.gen_pba_blocks(ws_fast, n, m, B, 0, 3, n0=n0, seed=seed)
    finally:
        pg.pg_force_wide_path(False)
    part_b = pg.gen_pba_blocks(ws_wide, n, m, B, 3, 6, n0=n0, seed=seed)
    torch.cuda.synchronize()
    assert_same(host(part_a), ref[:3 * per])
    assert_same(host(part_b), ref[3 * per:])


def test_pba_id64_and_repeat_is_identical():
    B, n_b, m = 12, 9_000, 3
    a = pg.gen_pba(B * n_b, m, B, 4, 2, 0.2, 77, id64=True)
    b = pg.gen_pba(B * n_b, m, B, 4, 2, 0.2, 77, id64=True)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    ref, _, _ = o.pba(B * n_b, m, B, 4, 2, 0.2, 77)
    assert_same(host(a, True), ref)


@pytest.mark.parametrize("B,n_b,m", [(16, 30_000, 5), (1, 50_000, 3), (300, 100, 2)])
def test_pba_to_host_copy_matches(B, n_b, m):
    n = B * n_b
    E = pg.pg_pba_edge_count(n, m, B, m + 1)
    host_buf = torch.empty((E, 2), dtype=torch.int32, pin_memory=True)
    dev = pg.gen_pba_to_host(host_buf, n, m, B, m + 1, 1, 0.1, 5)
    torch.cuda.current_stream().synchronize()
    assert torch.equal(host_buf, dev.cpu())
    ref, _, _ = o.pba(n, m, B, m + 1, 1, 0.1, 5)
    assert_same(host_buf.numpy().view(np.uint32).astype(np.uint64), ref)


def test_pba_other_stream():
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        got = pg.gen_pba(6 * 7000, 4, 6, 5, 1, 0.1, 5)
    s.synchronize()
    ref, _, _ = o.pba(6 * 7000, 4, 6, 5, 1, 0.1, 5)
    assert_same(host(got), ref)


# --------------------------------------------------------------------------
# PBA with general faction lists
# --------------------------------------------------------------------------

FIG1_STYLE_LISTS = [[0, 1, 4, 5, 0], [0, 1, 1, 2, 3], [1, 2, 3], [1, 2, 3, 3, 4],
                    [3, 4, 4, 5, 0], [4, 5, 0]]


def _random_lists(B, seed):
    """Overlapping factions of random sizes; each block's list concatenates
    the factions it belongs to (some lists omit the block itself, one list
    names every block, one repeats entries)."""
    rng = np.random.default_rng(seed)
    factions = [sorted(rng.choice(B, size=int(rng.integers(1, 6)), replace=False).tolist())
                for _ in range(B // 2)]
    lists = []
    for p in range(B):
        mine = [F for F in factions if p in F] or [factions[p % len(factions)]]
        lists.append([b for F in mine for b in F])
    lists[1] = list(range(B))                  # no block outside: no picks
    lists[2] = lists[2] + lists[2]             # repeated entries
    return lists


@pytest.mark.parametrize("lists,n_b,m,n0,f,seed,id64", [
    (FIG1_STYLE_LISTS, 3000, 3, 4, 0.3, 71, False),
    (FIG1_STYLE_LISTS, 3000, 3, 4, 1.0, 2, False),
    (FIG1_STYLE_LISTS, 2, 2, 3, 0.5, 5, False),       # lists longer than a block's entries
    (_random_lists(64, 9), 700, 5, 6, 0.1, 17, False),
    (_random_lists(40, 4), 20_000, 2, 3, 0.0, 3, True),
])
def test_pba_factions_match_oracle(lists, n_b, m, n0, f, seed, id64):
    B = len(lists)
    got = pg.gen_pba_factions(B * n_b, m, lists, n0=n0, inter_frac=f, seed=seed, id64=id64)
    torch.cuda.synchronize()
    ref, _, _ = o.pba_factions(B * n_b, m, B, n0, lists, f, seed)
    assert_same(host(got, id64), ref)


def test_pba_factions_aligned_lists_equal_gen_pba():
    B, W, n_b = 16, 4, 5000
    lists = [[(p // W) * W + t for t in range(W)] for p in range(B)]
    a = pg.gen_pba_factions(B * n_b, 3, lists, n0=4, inter_frac=0.2, seed=8)
    b = pg.gen_pba(B * n_b, 3, B, 4, W, 0.2, 8)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


# --------------------------------------------------------------------------
# Generation in parts: edge ranges and block ranges
# --------------------------------------------------------------------------

@pytest.mark.parametrize("id64", [False, True])
def test_kronecker_ranges_concatenate_to_the_graph(id64):
    Pm, k, M, seed = W.KRON_INITIATOR, 12, 100_003, 21
    cuts = [0, 777, 50_000, 50_001, M]
    spans = list(zip(cuts[:-1], cuts[1:]))
    made = {sp: pg.gen_kronecker_range(Pm, k, M, sp[0], sp[1], seed=seed, id64=id64)
            for sp in reversed(spans)}                          # made out of order
    parts = [made[sp] for sp in spans]
    torch.cuda.synchronize()
    got = np.concatenate([host(t, id64) for t in parts])
    assert_same(got, o.kron(Pm, k, M, seed))


def test_deterministic_kronecker_ranges(golden):
    G = np.array([[float(x) for x in r] for r in golden("pk_fig2_seed.txt")])
    k = 4
    full = pg.gen_kronecker(G, k, deterministic=True)
    E = full.shape[0]
    cuts = [0, 1, 4096, 4097, E]
    parts = [pg.gen_kronecker_range(G, k, 0, a, b, deterministic=True)
             for a, b in zip(cuts[:-1], cuts[1:])]
    torch.cuda.synchronize()
    assert torch.equal(torch.cat(parts), full)


@pytest.mark.parametrize("id64", [False, True])
def test_deterministic_kronecker_across_2p32(golden, id64):
    """Fig. 2 seed at k = 10: 11^10 edges, more than 2^32. A range ending at
    edge 2^32 takes the 32-bit digit path, and one reaching past it the
    64-bit path. Both must give every edge its base-e0 digits, most
    significant first, applied to the seed's edges in row-major order
    (reading R9; the oracle's stack order, pinned on the CPU)."""
    G = np.array([[float(x) for x in r] for r in golden("pk_fig2_seed.txt")])
    k, n0 = 10, G.shape[0]
    seed_edges = [(a, b) for a in range(n0) for b in range(n0) if G[a, b] > 0]
    e0 = len(seed_edges)
    lo, mid, hi = 2**32 - 1000, 2**32, 2**32 + 1000
    narrow = pg.gen_kronecker_range(G, k, 0, lo, mid, deterministic=True, id64=id64)
    wide = pg.gen_kronecker_range(G, k, 0, lo, hi, deterministic=True, id64=id64)
    torch.cuda.synchronize()
    got_n, got_w = host(narrow, id64), host(wide, id64)
    assert np.array_equal(got_n, got_w[:mid - lo])
    want = np.zeros((hi - lo, 2), np.uint64)
    for i, e in enumerate(range(lo, hi)):
        row = col = 0
        mul = 1
        for _ in range(k):
            a, b = seed_edges[e % e0]
            e //= e0
            row += a * mul
            col += b * mul
            mul *= n0
        want[i] = (row, col)
    assert_same(got_w, want)


def test_pba_block_ranges_from_one_prepare():
    n_b, m, B, n0, Wd, f, seed = 3000, 3, 16, 4, 2, 0.2, 12
    n = B * n_b
    ws = pg.pg_pba_prepare(n, m, B, n0, Wd, f, seed)
    ranges = [(5, 9), (0, 5), (9, 16), (3, 4)]                 # any order, overlaps allowed
    parts = {r: pg.gen_pba_blocks(ws, n, m, B, r[0], r[1], n0=n0, seed=seed) for r in ranges}
    full = pg.gen_pba(n, m, B, n0, Wd, f, seed)
    torch.cuda.synchronize()
    per = full.shape[0] // B
    for (a, b), t in parts.items():
        assert torch.equal(t, full[a * per:b * per]), (a, b)
    ref, _, _ = o.pba(n, m, B, n0, Wd, f, seed)
    assert_same(host(parts[(5, 9)]), ref[5 * per:9 * per])


def test_pba_block_ranges_with_faction_lists():
    lists = FIG1_STYLE_LISTS
    B, n_b, m, n0, f, seed = len(lists), 2000, 2, 3, 0.4, 6
    ws = pg.pg_pba_prepare(B * n_b, m, B, n0, inter_frac=f, seed=seed, factions=lists)
    part = pg.gen_pba_blocks(ws, B * n_b, m, B, 2, 5, n0=n0, seed=seed, id64=True)
    torch.cuda.synchronize()
    ref, _, _ = o.pba_factions(B * n_b, m, B, n0, lists, f, seed)
    per = ref.shape[0] // B
    assert_same(host(part, True), ref[2 * per:5 * per])


# --------------------------------------------------------------------------
# CSR
# --------------------------------------------------------------------------

def csr_check(edges_np, N, id64=False):
    t = torch.from_numpy(edges_np.view(np.int64 if id64 else np.int32)).cuda()
    rp, col = pg.edges_to_csr(t, N)
    torch.cuda.synchronize()
    ref_rp, ref_col = o.csr(edges_np.astype(np.uint64), N)
    assert np.array_equal(rp.cpu().numpy().view(np.uint64), ref_rp)
    assert_same(host(col, id64), ref_col)


@pytest.mark.parametrize("M,N,hub,id64", [
    (300_001, 5_000, 0.3, False),    # one very long row
    (100_000, 2**20, 0.0, False),
    (8_191, 3, 0.0, False),
    (50_000, 1, 0.0, False),         # a single row: nothing to sort on
    (0, 10, 0.0, False),
    (70_000, 2**33 + 5, 0.1, True),  # 34-bit ids
    (200_003, 3_000, 0.5, True),     # 64-bit ids, a row beyond shared memory
    (50_000, 2**26 + 3, 0.2, False), # mostly empty rows
])
def test_csr_random(M, N, hub, id64):
    csr_check(W.random_edges(M + N, M, N, id64=id64, hub_fraction=hub), N, id64)


@pytest.mark.parametrize("N,id64", [(3000, False), (3000, True), (2**26 + 3, False),
                                     (2**26 + 3, True)])
def test_csr_row_length_classes(N, id64):
    """Unsorted list whose rows straddle every length class of the row sort:
    thread-sorted rows (up to 32), CTA-sorted rows in shared memory, and rows
    longer than shared memory holds (12288 ids of 32 bits, 6144 of 64), with
    an odd (N = 3000: 3 digit passes) and odd-and-long (2^26+3: 7) pass count."""
    rng = np.random.default_rng(11 + N % 7 + id64)
    lens = list(range(0, 41)) + [63, 64, 65, 4095, 4096, 6144, 6145, 12288, 12289, 30001]
    srcs = rng.choice(min(N, 10**6), size=len(lens), replace=False)
    src = np.repeat(srcs, lens)
    dst = rng.integers(0, N, size=src.size)
    dst[::5] = dst[0]                                    # repeated destinations
    perm = rng.permutation(src.size)
    e = np.stack([src[perm], dst[perm]], 1).astype(np.uint64 if id64 else np.uint32)
    csr_check(e, N, id64)


def _multigraph(seed, M, N, id64):
    rng = np.random.default_rng(seed)
    e = rng.integers(0, N, size=(M, 2), dtype=np.uint64)
    if M > 5:
        e[: M // 5] = e[M // 5: 2 * (M // 5)]        # repeated pairs
        e[::11, 1] = e[::11, 0]                       # self-loops
        e[3::97] = e[5]                               # one pair many times
    return e.astype(np.uint64 if id64 else np.uint32)


@pytest.mark.parametrize("flags", [1, 2, 4, 8, 1 | 2, 2 | 4, 1 | 2 | 4, 8 | 4, 1 | 8])
@pytest.mark.parametrize("M,N,id64", [(50_001, 3000, False), (20_000, 2**22 + 5, True),
                                      (9_999, 1, False), (0, 7, False)])
def test_csr_options_match_oracle(flags, M, N, id64):
    e = _multigraph(M + flags, M, N, id64)
    t = torch.from_numpy(e.view(np.int64 if id64 else np.int32)).cuda()
    rp, col = pg.edges_to_csr_opts(t, N, flags)
    torch.cuda.synchronize()
    ref_rp, ref_col = o.csr_opts(e.astype(np.uint64), N, flags)
    got_rp = rp.cpu().numpy().view(np.uint64)
    assert np.array_equal(got_rp, ref_rp)
    k = int(got_rp[-1])
    assert_same(host(col, id64)[:k], ref_col)


@pytest.mark.parametrize("flags,id64,grouped", [(0, False, False), (0, True, False),
                                                 (0, False, True), (1 | 2, False, False),
                                                 (8, True, False)])
def test_csr_ignores_workspace_contents_and_clears_its_wait_word(flags, id64, grouped):
    """Every workspace word a CSR call reads is written earlier in the same
    call: a workspace filled with 0xFF gives the oracle's CSR. The sort's
    wait word reads 0 afterwards (no look-back wait gave up), also when the
    list is already grouped and the sort passes have nothing to do."""
    M, N = (100_000, 50_000) if grouped else (300_001, 5_000)
    if grouped:
        e = np.random.default_rng(3).integers(0, N, size=(M, 2), dtype=np.uint64)
        e = e[np.lexsort((e[:, 1], e[:, 0]))].astype(np.uint64 if id64 else np.uint32)
        assert np.bincount(e[:, 0].astype(np.int64)).max() <= 32
    else:
        e = _multigraph(7 + flags, M, N, id64)
    t = torch.from_numpy(e.view(np.int64 if id64 else np.int32)).cuda()
    size = (pg.pg_csr_workspace_size(M, N) if flags == 0 else
            int(pg._opts_lib().pg_csr_opts_workspace_size(M, N, flags)))
    ws = torch.full((size,), 255, dtype=torch.uint8, device="cuda")
    if flags == 0:
        rp, col = pg.edges_to_csr(t, N, workspace=ws)
        ref_rp, ref_col = o.csr(e.astype(np.uint64), N)
    else:
        rp, col = pg.edges_to_csr_opts(t, N, flags, workspace=ws)
        ref_rp, ref_col = o.csr_opts(e.astype(np.uint64), N, flags)
    torch.cuda.synchronize()
    assert pg.csr_wait_error(ws, M, N, id64, flags) == 0
    got_rp = rp.cpu().numpy().view(np.uint64)
    assert np.array_equal(got_rp, ref_rp)
    assert_same(host(col, id64)[:int(got_rp[-1])], ref_col)


@pytest.mark.parametrize("N,M,id64", [(1000, 100_001, False), (2**40 + 7, 50_000, True), (1, 33, False)])
def test_random_cells_match_oracle(N, M, id64):
    got = pg.gen_random_cells(N, M, seed=2**33 + 9, id64=id64)
    torch.cuda.synchronize()
    assert_same(host(got, id64), o.random_cells(N, M, 2**33 + 9))


@pytest.mark.parametrize("deterministic", [True, False])
def test_kronecker_xor_random_matches_oracle(golden, deterministic):
    if deterministic:
        G = np.array([[float(x) for x in r] for r in golden("pk_fig2_seed.txt")])
        k, n_edges = 4, 0
        pk = o.kron_det(G, k)[0]
    else:
        G, k, n_edges = W.KRON_INITIATOR, 12, 40_000
        pk = o.kron(G, k, n_edges, 5)
    N = len(G) ** k
    rnd = o.random_cells(N, 3000, 5)
    rp, col = pg.kronecker_xor_random(G, k, 3000, n_edges=n_edges, seed=5,
                                      deterministic=deterministic)
    torch.cuda.synchronize()
    ref_rp, ref_col = o.csr_opts(np.concatenate([pk, rnd]), N, o.CSR_ODD)
    got_rp = rp.cpu().numpy().view(np.uint64)
    assert np.array_equal(got_rp, ref_rp)
    assert_same(host(col)[:int(got_rp[-1])], ref_col)


def test_csr_of_kronecker_and_pba_graphs():
    ek = o.kron(W.KRON_INITIATOR, 16, 2**20, 7).astype(np.uint32)
    csr_check(ek, 2**16)
    ep, _, _ = o.pba(8 * 5000, 4, 8, 5, 1, 0.1, 3)
    csr_check(ep.astype(np.uint32), 8 * (5 + 5000))


@pytest.mark.slow
def test_csr_kron_workload_full():
    """Kronecker k = 20, 16 * 2^20 edges, seed 7 -- edge list and CSR."""
    cfg = W.CONFIGS["kron_k20_m16x_csr"]
    ref_edges = o.kron(cfg["initiator"], cfg["k"], cfg["n_edges"], cfg["seed"])
    got = pg.gen_kronecker(cfg["initiator"], cfg["k"], cfg["n_edges"], cfg["seed"])
    rp, col = pg.edges_to_csr(got, 2 ** cfg["k"])
    torch.cuda.synchronize()
    assert_same(host(got), ref_edges)
    ref_rp, ref_col = o.csr(ref_edges, 2 ** cfg["k"])
    assert np.array_equal(rp.cpu().numpy().view(np.uint64), ref_rp)
    assert_same(host(col), ref_col)


def _grouped(seed, N, max_row, M_rows, id64=False):
    """Seeded list already grouped by source (rows of random lengths)."""
    rng = np.random.default_rng(seed)
    srcs = np.sort(rng.choice(N, size=M_rows, replace=False))
    lens = rng.integers(0, max_row + 1, size=M_rows)
    src = np.repeat(srcs, lens)
    dst = rng.integers(0, N, size=src.size)
    dst[: src.size // 7] = dst[0] if src.size else 0          # duplicates
    e = np.stack([src, dst], 1).astype(np.uint64 if id64 else np.uint32)
    return e


@pytest.mark.parametrize("max_row,id64", [(1, False), (5, False), (32, False), (33, False),
                                          (200, False), (32, True)])
def test_csr_grouped_lists(max_row, id64):
    N = 3000
    csr_check(_grouped(max_row, N, max_row, 1500, id64), N, id64)


@pytest.mark.parametrize("flaw", ["none", "last_pair_out_of_order", "long_last_row"])
def test_csr_grouped_check_reads_to_the_end(flaw):
    """A list of 3.2M pairs, grouped except (maybe) at its very end: the
    sortedness check must see a flaw that only the last rounds of its grid
    stride reach, and must not flag a list that has none."""
    N = 2**22
    e = _grouped(11, N, 8, 800_000)
    if flaw == "last_pair_out_of_order":
        assert e[-2, 0] > 0
        e[-1, 0] = e[-2, 0] - 1
    elif flaw == "long_last_row":
        tail = np.stack([np.full(40, N - 1), np.arange(40)[::-1]], 1).astype(e.dtype)
        e = np.concatenate([e[e[:, 0] < N - 1], tail])
    csr_check(e, N)


def test_csr_of_gpu_ba_output_is_canonical():
    """Serial BA output is grouped by source: the CSR must equal the oracle's."""
    n, m, n0, seed = 20_000, 6, 7, 4
    edges = pg.gen_pba(n, m, 1, n0, 1, 0.0, seed)
    rp, col = pg.edges_to_csr(edges, n0 + n)
    torch.cuda.synchronize()
    ref_rp, ref_col = o.csr(o.ba(n, m, n0, seed), n0 + n)
    assert np.array_equal(rp.cpu().numpy().view(np.uint64), ref_rp)
    assert_same(host(col), ref_col)


# --------------------------------------------------------------------------
# Graph properties on the GPU: degrees, histogram, BFS
# --------------------------------------------------------------------------

@pytest.mark.parametrize("which", [0, 1, 2])
@pytest.mark.parametrize("id64", [False, True])
def test_degrees_and_histogram_match_oracle(which, id64):
    e, _, _ = o.pba(16 * 3000, 4, 16, 5, 2, 0.2, 4)
    N = 16 * (5 + 3000)
    e = e.astype(np.uint64 if id64 else np.uint32)
    t = torch.from_numpy(e.view(np.int64 if id64 else np.int32)).cuda()
    deg = pg.degrees(t, N, which)
    h_small = pg.degree_histogram(deg, 50)          # shared-memory buckets
    h_big = pg.degree_histogram(deg, 20_000)        # global buckets
    torch.cuda.synchronize()
    ref = o.degrees(e.astype(np.uint64), N, which)
    assert np.array_equal(deg.cpu().numpy().view(np.uint64), ref)
    assert np.array_equal(h_small.cpu().numpy().view(np.uint64), o.degree_histogram(ref, 50))
    assert np.array_equal(h_big.cpu().numpy().view(np.uint64), o.degree_histogram(ref, 20_000))


def _bfs_case(name):
    if name == "pba_undirected":
        e, _, _ = o.pba(8 * 4000, 3, 8, 4, 1, 0.1, 9)
        return e, 8 * 4004, o.CSR_SYMMETRIZE, [0, 5, 8 * 4004 - 1]
    if name == "kron_directed":
        return o.kron(W.KRON_INITIATOR, 14, 60_000, 3), 2**14, 0, [0, 1, 12345]
    if name == "path":
        n = 3000                                  # 3000 levels
        e = np.stack([np.arange(n - 1), np.arange(1, n)], 1).astype(np.uint64)
        return e, n, o.CSR_SYMMETRIZE, [0, 1500]
    if name == "single":
        return np.zeros((0, 2), np.uint64), 1, 0, [0]
    if name == "hubs":
        # vertex 0 joined to 1..4999 (a row of ten 512-entry slices); each of
        # 1..1500 joined to 70 vertices of its own (1500 rows of 71 entries:
        # more than 32^2 long rows in one level)
        hub = np.stack([np.zeros(4999, np.uint64), np.arange(1, 5000, dtype=np.uint64)], 1)
        owner = np.repeat(np.arange(1, 1501, dtype=np.uint64), 70)
        leaf = 5000 + np.arange(1500 * 70, dtype=np.uint64)
        e = np.concatenate([hub, np.stack([owner, leaf], 1)])
        return e, 5000 + 1500 * 70, o.CSR_SYMMETRIZE, [0, 1, 7000]
    raise KeyError(name)


@pytest.mark.parametrize("name", ["pba_undirected", "kron_directed", "path", "single", "hubs"])
@pytest.mark.parametrize("id64", [False, True])
def test_bfs_matches_oracle(name, id64):
    e, N, flags, sources = _bfs_case(name)
    ref_rp, ref_col = o.csr_opts(e, N, flags)
    rp = torch.from_numpy(ref_rp.view(np.int64)).cuda()
    col = torch.from_numpy(ref_col.astype(np.uint64 if id64 else np.uint32)
                           .view(np.int64 if id64 else np.int32)).cuda()
    if col.numel() == 0:
        col = torch.zeros(1, dtype=col.dtype, device="cuda")
    # a symmetric CSR also runs with bottom-up levels allowed: the same results
    modes = [False, True] if flags & o.CSR_SYMMETRIZE else [False]
    for s in sources:
        rd, rl, rs = o.bfs(ref_rp, ref_col, s)
        for undirected in modes:
            dist, levels, scanned = pg.bfs(rp, col, s, undirected=undirected)
            torch.cuda.synchronize()
            assert np.array_equal(dist.cpu().numpy().view(np.uint32), rd), (name, s, undirected)
            assert (levels, scanned) == (rl, rs), (name, s, undirected)


def test_bfs_runs_bottom_up_levels_on_wide_frontiers():
    # the PBA case's middle levels hold most of the vertices: with the graph
    # declared undirected those levels run bottom-up (traced separately)
    e, N, flags, _ = _bfs_case("pba_undirected")
    ref_rp, ref_col = o.csr_opts(e, N, flags)
    rp = torch.from_numpy(ref_rp.view(np.int64)).cuda()
    col = torch.from_numpy(ref_col.astype(np.uint32).view(np.int32)).cuda()
    pg.pg_trace_dump()
    pg.pg_trace_enable(True)
    try:
        pg.bfs(rp, col, 0, undirected=True)
        torch.cuda.synchronize()
    finally:
        pg.pg_trace_enable(False)
    assert "bfs_bottom_up" in pg.pg_trace_dump()


def test_throughput_probes_run():
    """The probes behind the bench's measured integer ceilings launch and give rates."""
    r = pg.philox_rate(calls_per_thread=256, reps=1)
    pipes = pg.int_pipe_rates(iters=256)
    assert r > 1e10
    assert set(pipes) == {"mul_wide", "mad32", "lop3", "add3"} and min(pipes.values()) > 1e11


def test_launch_count_counts_every_kernel():
    """pg_launch_count rises by one per kernel the library launches: one for a
    Kronecker descent; for two-phase PBA the phase-1 prefix, one pass per
    level (levels growing 1.5x from the 96K-entry prefix, in 16384-entry
    granules), the scan and the emit, plus the 64-bit emit once any earlier
    call forced the wide path in this process."""
    c0 = pg.pg_launch_count()
    pg.gen_kronecker(W.KRON_INITIATOR, 10, 4096, 7)
    assert pg.pg_launch_count() - c0 == 1
    B, n_b, m = 8, 30_000, 5
    N_e, gran = n_b * m, 16384
    lvl, levels = min(N_e, 6 * gran), 0
    while lvl < N_e:
        lvl = min(lvl + -(-(lvl // 2) // gran) * gran, N_e)
        levels += 1
    c0 = pg.pg_launch_count()
    pg.gen_pba(B * n_b, m, B, 6, 1, 0.1, 3)
    torch.cuda.synchronize()
    assert pg.pg_launch_count() - c0 in (3 + levels, 4 + levels), levels

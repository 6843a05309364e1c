"""Batched generation: plan validation on the host, and on the GPU every job's
slice of the arena equal to the oracle's graph for the same arguments."""
import ctypes as C

import numpy as np
import pytest

import oracle as o
from paper_1003_3684_gb300 import workloads as W


def mixed_jobs():
    jobs = []
    rng = np.random.default_rng(17)
    for i in range(24):
        m = int(rng.integers(1, 9))
        n = int(2 ** rng.uniform(0, 14))
        jobs.append(dict(kind="pba", n=n, m=m, n0=m + 1, seed=100 + i))
    for i in range(20):
        k = int(rng.integers(3, 15))
        jobs.append(dict(kind="kron", initiator=W.KRON_INITIATOR, k=k,
                         n_edges=int(rng.integers(0, 3 * 2**k)), seed=200 + i))
    jobs.append(dict(kind="pba", n=0, m=3, n0=4, seed=7))          # seed clique only
    jobs.append(dict(kind="kron", initiator=W.KRON_INITIATOR, k=9, n_edges=0, seed=8))
    jobs.append(dict(kind="kron", initiator=[[0.2, 0.5, 0.0], [0.1, 0.05, 0.05],
                                             [0.0, 0.02, 0.08]], k=6, n_edges=9999, seed=9))
    jobs.append(dict(kind="kron", initiator=[[0.0, 0.6], [0.4, 0.0]], k=30, n_edges=5000,
                     seed=2**40 + 1))
    order = rng.permutation(len(jobs))
    return [jobs[i] for i in order]


def oracle_job(j):
    if j["kind"] == "pba":
        return o.ba(j["n"], j["m"], j["n0"], j["seed"])
    return o.kron(j["initiator"], j["k"], j["n_edges"], j["seed"])


def _plan_host(jobs, tile=512, id64=False, host_out=None):
    """Run pg_batch_plan on the host only (no device copy)."""
    import paper_1003_3684_gb300 as pg
    from paper_1003_3684_gb300 import build
    build.build()
    L = pg._batch_lib()
    arr = (pg._PgJob * len(jobs))()
    keep = []
    for i, j in enumerate(jobs):
        arr[i] = pg._job_struct(j, keep)
    size = L.pg_batch_plan_size(C.cast(arr, C.c_void_p), len(jobs))
    host = np.zeros(size, np.uint8)
    offs = np.zeros(len(jobs) + 1, np.uint64)
    items = C.c_uint64(0)
    st = L.pg_batch_plan(C.cast(arr, C.c_void_p), len(jobs), tile, 1 if id64 else 0,
                         host.ctypes.data_as(C.c_void_p), size, offs.ctypes.data_as(C.c_void_p),
                         C.byref(items))
    if host_out is not None:
        host_out.append(host)
    return st, offs, items.value


def two_phase_jobs():
    """Two-phase PBA jobs (blocks > 1) between serial and Kronecker ones."""
    return [dict(kind="pba", n=3001, m=3, n0=4, seed=1),                      # odd edge count
            dict(kind="pba", n=8 * 1000, m=4, n0=5, blocks=8, inter_frac=0.1, seed=2),
            dict(kind="kron", initiator=W.KRON_INITIATOR, k=11, n_edges=7777, seed=3),
            dict(kind="pba", n=4 * 2048, m=3, n0=4, blocks=4, inter_frac=0.3, faction_width=2,
                 seed=4),
            dict(kind="pba", n=0, m=2, n0=3, seed=5),
            dict(kind="pba", n=16 * 700, m=5, n0=6, blocks=16, inter_frac=0.0, seed=6)]


def job_edges(j):
    if j["kind"] == "kron":
        return j["n_edges"]
    e0 = j["n0"] * (j["n0"] - 1) // 2
    return j.get("blocks", 1) * e0 + j["n"] * j["m"]


def test_batch_plan_offsets_and_items():
    jobs = mixed_jobs()
    st, offs, items = _plan_host(jobs, tile=512)
    assert st == 0
    sizes = [oracle_job(j).shape[0] if j["kind"] == "pba" and j["n"] < 5000 else
             (j["n0"] * (j["n0"] - 1) // 2 + j["n"] * j["m"] if j["kind"] == "pba"
              else j["n_edges"]) for j in jobs]
    assert np.array_equal(np.diff(offs.astype(np.int64)), sizes)
    expect_items = sum(max(1, -(-j["n"] * j["m"] // 512)) if j["kind"] == "pba"
                       else -(-j["n_edges"] // 512) for j in jobs)
    assert items == expect_items


@pytest.mark.parametrize("bad", [
    dict(kind="pba", n=10, m=0, n0=3, seed=1),
    dict(kind="pba", n=10, m=2, n0=1, seed=1),
    dict(kind="pba", n=2**31, m=2, n0=3, seed=1),            # 32-bit links needed
    dict(kind="kron", initiator=[[0, 0], [0, 0]], k=3, n_edges=5, seed=1),
    dict(kind="kron", initiator=[[1, 1], [1, 1]], k=40, n_edges=5, seed=1),   # ids > 2^32
])
def test_batch_plan_rejects_bad_jobs(bad):
    st, _, _ = _plan_host([dict(kind="pba", n=10, m=2, n0=3, seed=1), bad])
    assert st == 1


def test_batch_plan_places_two_phase_jobs_on_even_edges():
    import paper_1003_3684_gb300 as pg
    jobs = two_phase_jobs()
    for id64 in (False, True):
        st, offs, items = _plan_host(jobs, tile=512, id64=id64)
        assert st == 0
        prev_end = 0
        for i, j in enumerate(jobs):
            a = int(offs[i])
            gap = a - prev_end
            two = j.get("blocks", 1) > 1
            # a two-phase job starts on an even edge with 32-bit ids, else right after
            assert gap == ((prev_end & 1) if two and not id64 else 0), (i, gap)
            prev_end = a + job_edges(j)
            if j["kind"] == "pba":
                assert job_edges(j) == pg.pg_pba_edge_count(j["n"], j["m"], j.get("blocks", 1),
                                                            j["n0"])
        assert int(offs[-1]) == prev_end
        # work items: only the serial and Kronecker jobs have tiles
        assert items == sum(max(1, -(-j["n"] * j["m"] // 512)) if j["kind"] == "pba"
                            else -(-j["n_edges"] // 512) for j in jobs
                            if j.get("blocks", 1) == 1)


@pytest.mark.parametrize("bad", [
    dict(kind="pba", n=1001, m=3, n0=4, blocks=8, inter_frac=0.1, seed=1),   # blocks ∤ n
    dict(kind="pba", n=800, m=3, n0=4, blocks=8, inter_frac=1.5, seed=1),    # f > 1
    dict(kind="pba", n=800, m=3, n0=4, blocks=8, inter_frac=0.1, faction_width=3, seed=1),
])
def test_batch_plan_rejects_bad_two_phase_jobs(bad):
    st, _, _ = _plan_host([dict(kind="pba", n=10, m=2, n0=3, seed=1), bad])
    assert st == 1


def test_batch_csr_layout_on_the_host():
    import paper_1003_3684_gb300 as pg
    jobs = two_phase_jobs()
    for i, j in enumerate(jobs):
        j["want_csr"] = i % 3 != 2
    hosts = []
    st, offs, _ = _plan_host(jobs, host_out=hosts)
    assert st == 0
    L = pg._batch_lib()
    rows = np.zeros(len(jobs), np.uint64)
    cols = np.zeros(len(jobs), np.uint64)
    rt, ct = C.c_uint64(0), C.c_uint64(0)
    assert L.pg_batch_csr_layout(hosts[0].ctypes.data_as(C.c_void_p), len(jobs),
                                 rows.ctypes.data_as(C.c_void_p), cols.ctypes.data_as(C.c_void_p),
                                 C.byref(rt), C.byref(ct)) == 0
    r = c = 0
    for i, j in enumerate(jobs):
        if not j["want_csr"]:
            assert rows[i] == cols[i] == np.uint64(2**64 - 1)
            continue
        assert (int(rows[i]), int(cols[i])) == (r, c)
        r += pg._job_vertices(j) + 1
        c += job_edges(j)
    assert (rt.value, ct.value) == (r, c)
    assert L.pg_batch_csr_workspace_size(hosts[0].ctypes.data_as(C.c_void_p)) > 0
    # a union of more than 2^32 vertices does not fit 32-bit ids
    big = [dict(kind="kron", initiator=W.KRON_INITIATOR, k=31, n_edges=10, seed=i,
                want_csr=True) for i in range(3)]
    assert _plan_host(big)[0] == 1
    assert _plan_host(big, id64=True)[0] == 0


def test_batch_plan_rejects_bad_tile():
    st, _, _ = _plan_host([dict(kind="pba", n=10, m=2, n0=3, seed=1)], tile=100)
    assert st == 1


@pytest.mark.gpu
@pytest.mark.parametrize("tile,id64,grid", [(512, False, 0), (8192, False, 0), (64, True, 7),
                                            (4096, False, 1)])
def test_batch_matches_oracle(tile, id64, grid):
    import torch

    import paper_1003_3684_gb300 as pg
    jobs = mixed_jobs()
    plan = pg.BatchPlan(jobs, tile_edges=tile, id64=id64)
    arena = pg.gen_batch(plan, grid_ctas=grid)
    torch.cuda.synchronize()
    got = arena.cpu().numpy().view(np.uint64 if id64 else np.uint32).astype(np.uint64)
    for i, j in enumerate(jobs):
        a, b = int(plan.offsets[i]), int(plan.offsets[i + 1])
        assert np.array_equal(got[a:b], oracle_job(j)), (i, j)


@pytest.mark.gpu
def test_batch_cuda_graph_replay():
    import torch

    import paper_1003_3684_gb300 as pg
    jobs = mixed_jobs()
    plan = pg.BatchPlan(jobs, tile_edges=1024)
    arena = torch.zeros((plan.total_edges, 2), dtype=torch.int32, device="cuda")
    ws = torch.empty(pg.pg_batch_workspace_size(), dtype=torch.uint8, device="cuda")
    pg.gen_batch(plan, arena=arena, workspace=ws)       # warm-up outside capture
    ref = arena.clone()
    arena.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        pg.gen_batch(plan, arena=arena, workspace=ws)
    for _ in range(3):
        arena.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(arena, ref)


@pytest.mark.gpu
def test_autotune_picks_a_candidate(tmp_path, monkeypatch):
    monkeypatch.setenv("PGEN_CACHE_DIR", str(tmp_path))
    from paper_1003_3684_gb300 import autotune
    jobs = mixed_jobs()
    best = autotune.tune_batch(jobs, reps=1, tiles=(512, 2048), fractions=(1.0,))
    assert best["tile_edges"] in (512, 2048) and not best["cached"]
    again = autotune.tune_batch(jobs, reps=1, tiles=(512, 2048), fractions=(1.0,))
    assert again["cached"] and again["tile_edges"] == best["tile_edges"]


def _single(pg, j, id64):
    """The single-graph call a batch job must equal."""
    if j["kind"] == "kron":
        return pg.gen_kronecker(j["initiator"], j["k"], j["n_edges"], j["seed"], id64=id64)
    return pg.gen_pba(j["n"], j["m"], j.get("blocks", 1), j["n0"], j.get("faction_width", 1),
                      j.get("inter_frac", 0.0), j["seed"], id64=id64)


@pytest.mark.gpu
@pytest.mark.parametrize("id64", [False, True])
def test_batch_two_phase_jobs_equal_single_calls(id64):
    import torch

    import paper_1003_3684_gb300 as pg
    jobs = two_phase_jobs()
    plan = pg.BatchPlan(jobs, tile_edges=1024, id64=id64)
    arena = pg.gen_batch(plan)
    torch.cuda.synchronize()
    for i, j in enumerate(jobs):
        assert torch.equal(plan.edges_of(arena, i), _single(pg, j, id64)), (i, j)
    # the small two-phase job against the oracle itself
    j = jobs[1]
    ref, _, _ = o.pba(j["n"], j["m"], j["blocks"], j["n0"], 1, j["inter_frac"], j["seed"])
    got = plan.edges_of(arena, 1).cpu().numpy().view(np.uint64 if id64 else np.uint32)
    assert np.array_equal(got.astype(np.uint64), ref)


@pytest.mark.gpu
def test_batch_with_two_phase_jobs_replays_in_a_cuda_graph():
    import torch

    import paper_1003_3684_gb300 as pg
    plan = pg.BatchPlan(two_phase_jobs() + mixed_jobs()[:10], tile_edges=2048)
    arena = torch.zeros((plan.total_edges, 2), dtype=torch.int32, device="cuda")
    ws = torch.empty(pg.pg_batch_workspace_size(plan), dtype=torch.uint8, device="cuda")
    pg.gen_batch(plan, arena=arena, workspace=ws)
    ref = arena.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        pg.gen_batch(plan, arena=arena, workspace=ws)
    for _ in range(2):
        arena.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(arena, ref)


@pytest.mark.gpu
@pytest.mark.parametrize("id64", [False, True])
def test_batch_csr_equals_each_jobs_csr(id64):
    import torch

    import paper_1003_3684_gb300 as pg
    jobs = two_phase_jobs() + mixed_jobs()[:14]
    for i, j in enumerate(jobs):
        j["want_csr"] = i % 4 != 1
    plan = pg.BatchPlan(jobs, tile_edges=512, id64=id64)
    arena = pg.gen_batch(plan)
    row_ptr, col = pg.gen_batch_csr(plan, arena, check=True)
    torch.cuda.synchronize()
    idt = np.uint64 if id64 else np.uint32
    for i, j in enumerate(jobs):
        if not j["want_csr"]:
            assert plan.csr_rows[i] == -1
            continue
        rp, cl = plan.csr_of(row_ptr, col, i)
        e = plan.edges_of(arena, i).cpu().numpy().view(idt).astype(np.uint64)
        ref_rp, ref_col = o.csr(e, pg._job_vertices(j))
        assert np.array_equal(rp.cpu().numpy().view(np.uint64), ref_rp), (i, j)
        assert np.array_equal(cl.cpu().numpy().view(idt).astype(np.uint64), ref_col), (i, j)


@pytest.mark.gpu
def test_batch_csr_of_grouped_jobs_only_and_of_none():
    import torch

    import paper_1003_3684_gb300 as pg
    # only BA jobs: their union is grouped by source, so no sort runs
    jobs = [dict(kind="pba", n=500 + 37 * i, m=1 + i % 4, n0=2 + i % 4, seed=i, want_csr=True)
            for i in range(12)]
    plan = pg.BatchPlan(jobs, tile_edges=256)
    arena = pg.gen_batch(plan)
    row_ptr, col = pg.gen_batch_csr(plan, arena, check=True)
    torch.cuda.synchronize()
    for i, j in enumerate(jobs):
        rp, cl = plan.csr_of(row_ptr, col, i)
        ref_rp, ref_col = o.csr(o.ba(j["n"], j["m"], j["n0"], j["seed"]), pg._job_vertices(j))
        assert np.array_equal(rp.cpu().numpy().view(np.uint64), ref_rp)
        assert np.array_equal(cl.cpu().numpy().view(np.uint32).astype(np.uint64), ref_col)
    # no job asks for a CSR: nothing to do
    plan = pg.BatchPlan([dict(kind="pba", n=100, m=2, n0=3, seed=1)], tile_edges=256)
    assert plan.csr_rows_total == 0 and pg.pg_batch_csr_workspace_size(plan) == 0
    pg.gen_batch_csr(plan, pg.gen_batch(plan))


@pytest.mark.gpu
@pytest.mark.parametrize("id64", [False, True])
def test_batch_csr_of_empty_and_seed_only_jobs(id64):
    import torch

    import paper_1003_3684_gb300 as pg
    jobs = [dict(kind="kron", initiator=W.KRON_INITIATOR, k=9, n_edges=0, seed=1, want_csr=True),
            dict(kind="pba", n=0, m=3, n0=4, seed=2, want_csr=True),       # the seed clique only
            dict(kind="kron", initiator=W.KRON_INITIATOR, k=6, n_edges=5, seed=3, want_csr=True),
            dict(kind="pba", n=8 * 10, m=2, n0=3, blocks=8, inter_frac=0.5, seed=4,
                 want_csr=True)]
    plan = pg.BatchPlan(jobs, tile_edges=64, id64=id64)
    arena = pg.gen_batch(plan)
    row_ptr, col = pg.gen_batch_csr(plan, arena, check=True)
    torch.cuda.synchronize()
    idt = np.uint64 if id64 else np.uint32
    for i, j in enumerate(jobs):
        rp, cl = plan.csr_of(row_ptr, col, i)
        e = plan.edges_of(arena, i).cpu().numpy().view(idt).astype(np.uint64).reshape(-1, 2)
        ref_rp, ref_col = o.csr(e, pg._job_vertices(j))
        assert np.array_equal(rp.cpu().numpy().view(np.uint64), ref_rp), (i, j)
        assert np.array_equal(cl.cpu().numpy().view(idt).astype(np.uint64), ref_col), (i, j)
    assert int(plan.csr_of(row_ptr, col, 0)[0].sum()) == 0


@pytest.mark.gpu
def test_batch_csr_with_only_an_empty_job():
    import torch

    import paper_1003_3684_gb300 as pg
    plan = pg.BatchPlan([dict(kind="kron", initiator=W.KRON_INITIATOR, k=5, n_edges=0, seed=1,
                              want_csr=True)], tile_edges=64)
    arena = pg.gen_batch(plan)
    row_ptr, col = pg.gen_batch_csr(plan, arena, check=True)
    torch.cuda.synchronize()
    assert plan.total_edges == 0 and plan.csr_cols_total == 0
    assert torch.equal(row_ptr[:33], torch.zeros(33, dtype=torch.int64, device="cuda"))

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


def _plan_host(jobs, tile=512):
    """Run pg_batch_plan on the host only (no device copy)."""
    import paper_1003_3684_gb300 as pg
    from paper_1003_3684_gb300 import build
    build.build()
    L = pg._batch_lib()
    arr = (pg._PgJob * len(jobs))()
    keep = []
    for i, j in enumerate(jobs):
        if j["kind"] == "pba":
            arr[i] = pg._PgJob(0, j["m"], j["n0"], 0, j["n"], j["seed"], None)
        else:
            P = np.ascontiguousarray(j["initiator"], dtype=np.float64)
            keep.append(P)
            arr[i] = pg._PgJob(1, 0, P.shape[0], j["k"], j["n_edges"], j["seed"],
                               P.ctypes.data_as(C.c_void_p))
    size = L.pg_batch_plan_size(C.cast(arr, C.c_void_p), len(jobs))
    host = np.zeros(size, np.uint8)
    offs = np.zeros(len(jobs) + 1, np.uint64)
    items = C.c_uint64(0)
    st = L.pg_batch_plan(C.cast(arr, C.c_void_p), len(jobs), tile, 0, host.ctypes.data_as(C.c_void_p),
                         size, offs.ctypes.data_as(C.c_void_p), C.byref(items))
    return st, offs, items.value


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

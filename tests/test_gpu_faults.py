"""Failure detection on the GPU, in forms that fault nothing.

A bounded device wait that runs out: a test hook makes one tile of every
digit pass of the CSR sort withhold its counts, so that the later tiles'
look-back waits give up after a short poll limit. The kernel must return,
report the timeout through the workspace's wait word (pg_csr_check ->
PG_ETIMEOUT), and keep every write inside its output buffers; the next call
must be right again.

Output canaries: every generator and the CSR call, given output buffers
longer than they need, leave the part past their result untouched.
"""
import numpy as np
import pytest
import torch

import oracle as o
import paper_1003_3684_gb300 as pg
from paper_1003_3684_gb300 import workloads as W

pytestmark = pytest.mark.gpu

C32 = 0x5A5A5A5A                     # canary word of 32-bit outputs
C64 = 0x5A5A5A5A5A5A5A5A             # and of 64-bit ones


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1003_3684_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield
    pg.pg_csr_test_wait_hook(0, 0xFFFFFFFF)
    torch.cuda.synchronize()


def _canary(shape, id64):
    return torch.full(shape, C64 if id64 else C32, dtype=torch.int64 if id64 else torch.int32,
                      device="cuda")


def _untouched(t, id64):
    return bool((t == (C64 if id64 else C32)).all())


def _multigraph(seed, M, N, id64):
    rng = np.random.default_rng(seed)
    e = rng.integers(0, N, size=(M, 2), dtype=np.uint64)
    e[: M // 5] = e[M // 5: 2 * (M // 5)]
    e[::11, 1] = e[::11, 0]
    return e.astype(np.uint64 if id64 else np.uint32)


def _csr(t, N, flags, row_ptr, col, ws):
    if flags == 0:
        pg.edges_to_csr(t, N, row_ptr=row_ptr, col=col, workspace=ws)
    else:
        pg.edges_to_csr_opts(t, N, flags, row_ptr=row_ptr, col=col, workspace=ws)


@pytest.mark.parametrize("flags,id64", [(0, False), (0, True), (pg.CSR_DEDUP, False),
                                        (pg.CSR_ODD, True)])
def test_csr_wait_that_gives_up_is_reported_and_stays_in_bounds(flags, id64):
    M, N = 300_001, 5_000          # unsorted: 37 tiles of 32-bit pairs, 74 of 64-bit
    e = _multigraph(17 + flags, M, N, id64)
    t = torch.from_numpy(e.view(np.int64 if id64 else np.int32)).cuda()
    size = (pg.pg_csr_workspace_size(M, N) if flags == 0 else
            int(pg._opts_lib().pg_csr_opts_workspace_size(M, N, flags)))
    ws = torch.empty(size, dtype=torch.uint8, device="cuda")
    rp_buf = torch.full((N + 1 + 64,), C64, dtype=torch.int64, device="cuda")
    col_buf = _canary((M + 64,), id64)
    row_ptr, col = rp_buf[:N + 1], col_buf[:M]
    pg.pg_csr_test_wait_hook(256, 1)           # tile 1 never publishes; 256 polls
    try:
        _csr(t, N, flags, row_ptr, col, ws)
        with pytest.raises(pg.PgenError) as err:
            pg.pg_csr_check(ws, M, N, id64=id64, flags=flags)
        assert err.value.status == pg.PG_ETIMEOUT
        assert pg.csr_wait_error(ws, M, N, id64, flags) != 0
    finally:
        pg.pg_csr_test_wait_hook(0, 0xFFFFFFFF)
    torch.cuda.synchronize()
    assert bool((rp_buf[N + 1:] == C64).all()), "row_ptr written past its end"
    assert _untouched(col_buf[M:], id64), "col written past its end"
    # the same call again, hook off: the word is cleared and the CSR is right
    _csr(t, N, flags, row_ptr, col, ws)
    pg.pg_csr_check(ws, M, N, id64=id64, flags=flags)
    ref_rp, ref_col = (o.csr(e.astype(np.uint64), N) if flags == 0 else
                       o.csr_opts(e.astype(np.uint64), N, flags))
    got_rp = row_ptr.cpu().numpy().view(np.uint64)
    assert np.array_equal(got_rp, ref_rp)
    k = int(got_rp[-1])
    got_col = col.cpu().numpy().view(np.uint64 if id64 else np.uint32).astype(np.uint64)[:k]
    assert np.array_equal(got_col, ref_col)
    assert _untouched(col_buf[M:], id64)


def test_csr_check_passes_a_normal_call():
    e = _multigraph(5, 100_000, 3_000, False)
    t = torch.from_numpy(e.view(np.int32)).cuda()
    rp, col = pg.edges_to_csr(t, 3_000, check=True)     # raises on a timeout
    ref_rp, _ = o.csr(e.astype(np.uint64), 3_000)
    assert np.array_equal(rp.cpu().numpy().view(np.uint64), ref_rp)


def _generated(call, E, id64, extra=37):
    """call(out) with an output buffer extra rows longer than E: the rows past
    E keep the canary and the first E rows equal a call with an exact buffer."""
    buf = _canary((E + extra, 2), id64)
    call(buf)
    exact = _canary((max(E, 1), 2), id64)
    call(exact)
    torch.cuda.synchronize()
    assert _untouched(buf[E:], id64), "output written past the edge count"
    assert torch.equal(buf[:E], exact[:E])


@pytest.mark.parametrize("id64", [False, True])
def test_generators_leave_output_past_their_edges_untouched(id64):
    n, m = 10_007, 3
    E = pg.pg_pba_edge_count(n, m, 1, 4)
    _generated(lambda out: pg.gen_pba(n, m, 1, 4, 1, 0.0, 5, id64=id64, out=out), E, id64)
    B, nb = 8, 3_001
    E = pg.pg_pba_edge_count(B * nb, 4, B, 5)
    ws = torch.empty(pg.pg_pba_workspace_size(B * nb, 4, B), dtype=torch.uint8, device="cuda")
    _generated(lambda out: pg.gen_pba(B * nb, 4, B, 5, 1, 0.1, 9, id64=id64, out=out,
                                      workspace=ws), E, id64)
    lists = W.ring_factions(B, 3)
    _generated(lambda out: pg.gen_pba_factions(B * nb, 4, lists, n0=5, inter_frac=0.2, seed=4,
                                               id64=id64, out=out), E, id64)
    _generated(lambda out: pg.gen_kronecker(W.KRON_INITIATOR, 12, 10_001, 7, id64=id64,
                                            out=out), 10_001, id64)
    FIG2 = [[1, 1, 1, 1, 0], [1, 1, 0, 0, 0], [1, 0, 1, 0, 0], [1, 0, 0, 1, 0], [0, 0, 0, 0, 1]]
    _generated(lambda out: pg.gen_kronecker(FIG2, 3, deterministic=True, id64=id64, out=out),
               11 ** 3, id64)
    _generated(lambda out: pg.gen_random_cells(1000, 5_003, seed=3, id64=id64, out=out),
               5_003, id64)


@pytest.mark.parametrize("id64", [False, True])
def test_batch_leaves_arena_past_its_jobs_untouched(id64):
    jobs = [dict(kind="pba", n=5_000 + 97 * i, m=2 + i % 5, n0=3 + i % 5, seed=i) for i in range(5)]
    jobs += [dict(kind="kron", initiator=W.KRON_INITIATOR, k=8 + i, n_edges=3_001 * (i + 1),
                  seed=40 + i) for i in range(5)]
    plan = pg.BatchPlan(jobs, tile_edges=2048, id64=id64)
    total = plan.total_edges
    arena = _canary((total + 101, 2), id64)
    pg.gen_batch(plan, arena=arena)
    torch.cuda.synchronize()
    assert _untouched(arena[total:], id64)
    ref = pg.gen_batch(plan)
    torch.cuda.synchronize()
    assert torch.equal(arena[:total], ref)


@pytest.mark.parametrize("id64", [False, True])
def test_csr_leaves_output_past_its_rows_untouched(id64):
    M, N = 70_003, 2_001
    e = _multigraph(23, M, N, id64)
    t = torch.from_numpy(e.view(np.int64 if id64 else np.int32)).cuda()
    rp_buf = torch.full((N + 1 + 50,), C64, dtype=torch.int64, device="cuda")
    col_buf = _canary((M + 50,), id64)
    pg.edges_to_csr(t, N, row_ptr=rp_buf[:N + 1], col=col_buf[:M], check=True)
    torch.cuda.synchronize()
    assert bool((rp_buf[N + 1:] == C64).all())
    assert _untouched(col_buf[M:], id64)

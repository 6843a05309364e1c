"""Serving loop: admission and scheduling on the host (fake device, fake
clock), and on the GPU the same CSR for every request alone and in a mix."""
import numpy as np
import pytest

from paper_1003_3684_gb300 import serve


class FakeEvent:
    def __init__(self, clock, ready_at):
        self.clock, self.ready_at = clock, ready_at

    def query(self):
        return self.clock() >= self.ready_at


class FakeServer(serve.Server):
    """Server whose 'device' finishes a batch 1 ms per million edges later.
    `fail` holds request ids whose CSR sort reports a wait that gave up;
    a batch holding a request id of `refuse` fails to launch, as when a
    device allocation fails."""

    fail = ()
    refuse = ()

    def _init_cuda(self):
        self._cuda = True

    def _start(self, i, batch, now):
        if any(r.rid in self.refuse for r in batch):
            raise MemoryError("fake device: out of memory")
        for r in batch:
            r.launched = now
            r.state = "running"
        cost = sum(serve.job_edges(r.job) for r in batch) / 1e9
        status = np.array([1 if r.rid in self.fail else 0 for r in batch], np.int32)
        self.launches += 1
        return serve._Batch(batch, None, FakeEvent(self.clock, now + cost), status=status)


def fake_clock():
    t = [0.0]

    def clock():
        return t[0]

    def advance(dt):
        t[0] += dt

    return clock, advance


def test_budget_is_never_exceeded_and_fifo_admission():
    clock, advance = fake_clock()
    jobs = [serve.job_for_edges("pba" if i % 2 else "kron", 2 ** (12 + i % 10), seed=i)
            for i in range(200)]
    budget = 3 * max(serve.job_bytes(j) for j in jobs)
    srv = FakeServer(budget_bytes=budget, n_streams=2, clock=clock)
    reqs = [srv.submit(j, now=0.0) for j in jobs]
    while srv.pending():
        srv.step()
        assert srv.in_use <= budget
        for r in srv.completed:
            srv.release(r)
        advance(1e-3)
    assert srv.peak_in_use <= budget
    assert all(r.done is not None for r in reqs)
    admitted = [r.admitted for r in reqs]
    assert admitted == sorted(admitted)                 # FIFO
    assert srv.in_use == 0


def test_requests_arriving_while_busy_are_started_without_waiting_for_all():
    """Continuous batching: a request arriving while one batch runs starts on
    the other stream before that batch finishes."""
    clock, advance = fake_clock()
    srv = FakeServer(budget_bytes=1 << 40, n_streams=2, clock=clock)
    big = srv.submit(serve.job_for_edges("kron", 2**26, seed=1), now=0.0)
    srv.step()
    advance(1e-3)
    small = srv.submit(serve.job_for_edges("pba", 2**12, seed=2), now=clock())
    srv.step()
    assert small.launched is not None and big.done is None
    while srv.pending():
        advance(1e-3)
        srv.step()
    assert small.done < big.done


def run_until_idle(srv, advance, release=True):
    while srv.pending():
        srv.step()
        if release:
            for r in srv.completed:
                srv.release(r)
        advance(1e-3)


def test_cancel_waiting_admitted_and_running_requests():
    clock, advance = fake_clock()
    jobs = [serve.job_for_edges("kron", 2**22, seed=i) for i in range(4)]
    one = serve.job_bytes(jobs[0])
    srv = FakeServer(budget_bytes=2 * one, n_streams=1, max_batch_jobs=1, clock=clock)
    a, b, c, d = [srv.submit(j, now=0.0) for j in jobs]
    srv.step()                       # a running, b admitted (budget for two), c and d waiting
    assert (a.state, b.state, c.state, d.state) == ("running", "admitted", "waiting", "waiting")
    assert srv.cancel(c) and c.state == "cancelled" and c not in srv.waiting
    held_before = srv.in_use
    assert srv.cancel(b) and srv.in_use == held_before - one and b.held == 0
    assert srv.cancel(a) and a.state == "cancelled"     # still on the device
    assert srv.in_use == one                             # a's bytes stay until its batch retires
    run_until_idle(srv, advance)
    assert a.done is None and a not in srv.completed and a.held == 0
    assert d.state == "done" and srv.completed == [d]
    assert srv.in_use == 0 and srv.peak_in_use <= 2 * one
    assert not srv.cancel(d)                             # finished: nothing to cancel
    assert all(r.launched is None for r in (b, c))


def test_deadline_expires_waiting_requests_only():
    clock, advance = fake_clock()
    big = serve.job_for_edges("kron", 2**24, seed=0)
    small = serve.job_for_edges("pba", 2**12, seed=1)
    srv = FakeServer(budget_bytes=serve.job_bytes(big) + serve.job_bytes(small) // 2,
                     n_streams=1, clock=clock)
    r0 = srv.submit(big, now=0.0, deadline=0.0)          # starts at once: no expiry
    r1 = srv.submit(small, now=0.0, deadline=5e-3)       # waits for budget, expires at 5 ms
    r2 = srv.submit(small, now=0.0)                      # no deadline: waits and runs
    srv.step()
    assert r0.state == "running" and r1.state == "waiting"
    run_until_idle(srv, advance)
    assert r0.state == "done" and r2.state == "done"
    assert r1.state == "expired" and r1.launched is None and r1 in srv.expired
    assert r2.launched > r1.deadline
    assert srv.in_use == 0


def test_failed_csr_wait_is_reported_not_completed():
    clock, advance = fake_clock()
    jobs = [serve.job_for_edges("pba", 2**14, seed=i) for i in range(6)]
    srv = FakeServer(budget_bytes=1 << 40, n_streams=2, clock=clock)
    srv.fail = {2, 4}
    reqs = [srv.submit(j, now=0.0) for j in jobs]
    run_until_idle(srv, advance)
    assert [r.rid for r in srv.failed] == [2, 4]
    assert all(r.state == "failed" and "PG_ETIMEOUT" in r.error and r.held == 0
               for r in srv.failed)
    assert sorted(r.rid for r in srv.completed) == [0, 1, 3, 5]
    assert srv.in_use == 0 and len(reqs) == 6


def test_failed_launch_fails_its_batch_and_the_server_goes_on():
    clock, advance = fake_clock()
    jobs = [serve.job_for_edges("kron", 2**14, seed=i) for i in range(8)]
    srv = FakeServer(budget_bytes=1 << 40, n_streams=1, max_batch_jobs=2, clock=clock)
    srv.refuse = {2}
    reqs = [srv.submit(j, now=0.0) for j in jobs]
    run_until_idle(srv, advance)
    assert sorted(r.rid for r in srv.failed) == [2, 3]          # the batch [2, 3]
    assert all(r.state == "failed" and "out of memory" in r.error and r.held == 0
               and r.launched is None for r in srv.failed)
    assert sorted(r.rid for r in srv.completed) == [0, 1, 4, 5, 6, 7]
    assert srv.in_use == 0 and len(reqs) == 8


def test_allocation_failure_injection_on_the_host():
    import subprocess
    import sys

    import torch

    import paper_1003_3684_gb300 as pg
    pg.set_fail_alloc_at(3)
    try:
        pg.empty_device(4, torch.int32, "cpu")
        pg.empty_device((2, 2), torch.int64, "cpu")
        with pytest.raises(torch.cuda.OutOfMemoryError, match="injected"):
            pg.empty_device(8, torch.uint8, "cpu")
        pg.empty_device(8, torch.uint8, "cpu")                 # once only
    finally:
        pg.set_fail_alloc_at(0)
    code = ("import torch, paper_1003_3684_gb300 as pg\n"
            "try:\n    pg.empty_device(2, torch.int32, 'cpu')\n"
            "except torch.cuda.OutOfMemoryError:\n    print('refused')\n")
    import os
    from conftest import ROOT
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       env=dict(os.environ, PGEN_FAIL_ALLOC_AT="1"), timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "refused", r.stderr


def test_request_bytes_count_the_csr_workspace():
    import paper_1003_3684_gb300 as pg
    for kind, E in (("pba", 2**12), ("kron", 2**20)):
        j = serve.job_for_edges(kind, E, seed=0)
        N = serve.job_vertices(j)
        ws = pg.pg_csr_workspace_size(serve.job_edges(j), N)
        assert ws > 0
        # edge list 8 B and col 4 B per edge, row_ptr 8 B per vertex, the sort's
        # workspace, and the batch CSR's union list (8 B/edge) and row pointers
        assert serve.job_bytes(j) == serve.job_edges(j) * 20 + (N + 1) * 16 + ws


def test_oversized_request_is_rejected():
    srv = FakeServer(budget_bytes=1000)
    with pytest.raises(ValueError):
        srv.submit(serve.job_for_edges("pba", 2**20, seed=0))


def test_poisson_workload_shape():
    arr = serve.poisson_workload(2000, 2.0, seed=0)
    t = np.array([a for a, _ in arr])
    assert 3500 < len(arr) < 4500 and (np.diff(t) > 0).all()
    E = np.array([serve.job_edges(j) for _, j in arr])
    assert E.min() >= 2**12 and E.max() <= 2**26 + 16
    kinds = [j["kind"] for _, j in arr]
    assert 0.45 < kinds.count("pba") / len(kinds) < 0.55


@pytest.mark.gpu
def test_results_same_alone_and_in_the_mix():
    import torch

    import oracle as o
    rng = np.random.default_rng(3)
    jobs = [serve.job_for_edges("pba" if i % 2 else "kron", int(2 ** rng.uniform(12, 19)), seed=i)
            for i in range(40)]
    # alone: one request at a time on one stream
    alone = []
    srv = serve.Server(budget_bytes=8 << 30, n_streams=1, max_batch_jobs=1)
    for j in jobs:
        r = srv.submit(j)
        srv.drain()
        torch.cuda.synchronize()
        alone.append((r.row_ptr.cpu().numpy().copy(), r.col.cpu().numpy().copy()))
        srv.release(r)
    # in the mix: all at once, small budget so admission staggers them;
    # requests of 2^16 edges or more get their CSR from a call of their own,
    # the others from their batch's one sort
    budget = 6 * max(serve.job_bytes(j) for j in jobs)
    srv = serve.Server(budget_bytes=budget, n_streams=3, max_batch_jobs=16,
                       batch_csr_edges=2**16)
    reqs = [srv.submit(j) for j in jobs]
    srv.drain()
    torch.cuda.synchronize()
    assert srv.peak_in_use <= budget
    for r, (rp, col) in zip(reqs, alone):
        assert np.array_equal(r.row_ptr.cpu().numpy(), rp)
        assert np.array_equal(r.col.cpu().numpy(), col)
    # and the small ones against the oracle
    for r in reqs[:6]:
        j = r.job
        e = (o.ba(j["n"], j["m"], j["n0"], j["seed"]) if j["kind"] == "pba"
             else o.kron(j["initiator"], j["k"], j["n_edges"], j["seed"]))
        ref_rp, ref_col = o.csr(e, serve.job_vertices(j))
        assert np.array_equal(r.row_ptr.cpu().numpy().view(np.uint64), ref_rp)
        assert np.array_equal(r.col.cpu().numpy().view(np.uint32).astype(np.uint64), ref_col)


@pytest.mark.gpu
def test_open_loop_short_run():
    arr = serve.poisson_workload(500, 0.5, seed=1, hi_exp=20)
    srv = serve.Server(budget_bytes=4 << 30, n_streams=2)
    done = serve.run_open_loop(srv, arr)
    assert len(done) == len(arr)
    lat = np.array([r.latency for r in done])
    assert (lat > 0).all()


@pytest.mark.gpu
@pytest.mark.parametrize("k", [1, 2, 4])
def test_injected_allocation_failure_fails_one_batch(k):
    # the first batch (requests 0 and 1) allocates its edge arena (1), the
    # batch CSR's workspace (2), its row_ptr arena (3) and its col arena (4):
    # k = 1 fails before any kernel, 2 after the batch kernel was queued, 4
    # with the CSR workspace and row pointers already allocated
    import torch

    import oracle as o
    import paper_1003_3684_gb300 as pg
    jobs = [serve.job_for_edges("pba" if i % 2 else "kron", 2**13 + 512 * i, seed=i)
            for i in range(6)]
    srv = serve.Server(budget_bytes=8 << 30, n_streams=1, max_batch_jobs=2)
    reqs = [srv.submit(j) for j in jobs]
    srv._init_cuda()
    pg.set_fail_alloc_at(k)
    try:
        srv.drain()
    finally:
        pg.set_fail_alloc_at(0)
    torch.cuda.synchronize()
    assert [r.rid for r in srv.failed] == [0, 1]
    assert all("injected allocation failure" in r.error and r.held == 0 for r in srv.failed)
    assert [r.rid for r in srv.completed] == [2, 3, 4, 5]
    for r in reqs[2:]:
        j = r.job
        e = (o.ba(j["n"], j["m"], j["n0"], j["seed"]) if j["kind"] == "pba"
             else o.kron(j["initiator"], j["k"], j["n_edges"], j["seed"]))
        ref_rp, ref_col = o.csr(e, serve.job_vertices(j))
        assert np.array_equal(r.row_ptr.cpu().numpy().view(np.uint64), ref_rp)
        assert np.array_equal(r.col.cpu().numpy().view(np.uint32).astype(np.uint64), ref_col)
        srv.release(r)
    assert srv.in_use == sum(w.numel() for w in srv.batch_ws)

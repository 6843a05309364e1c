"""Serving loop: continuous batching of graph-generation requests.

Requests (serial BA or stochastic Kronecker graphs, CSR wanted) arrive at any
time. The server keeps a FIFO of waiting requests and a byte budget of device
memory. At every scheduling step it
  1. retires batches whose CUDA event has completed (their requests are done;
     latency = completion - arrival),
  2. drops waiting requests whose deadline has passed, then admits waiting
     requests, in arrival order, while their bytes fit the remaining budget,
  3. launches the admitted requests as one batch on a free stream: one
     persistent generation launch for all of them (gen_batch), then on the
     same stream the CSRs -- of the small requests from one sort of their
     union graph (gen_batch_csr), of each large one by its own call
     (edges_to_csr), where the launches cost nothing next to the sort --
     then an event.
Batches on different streams overlap on the GPU, so requests that arrive
while others are running are admitted and started as soon as a stream and
memory free up -- continuous batching rather than a queue drained in rounds.
Results stay on the device until the client releases them.

A request's bytes are its edge list, its CSR and its share of the batch
CSR's workspace; the edge list and the workspace are given back when its
batch retires. The CSRs of a batch share one allocation, so a request's CSR
bytes are given back when the last request of its batch is released. A
request can be cancelled at any time (a running one still finishes on the
device, and its results are dropped when its batch retires) and can carry a
deadline, the latest time it may start: a request still waiting at its
deadline expires without running. The batch CSR's bounded-wait status is
copied to pinned host memory on the batch's stream; if its sort gave up
waiting, the batch's requests are reported failed, not done.

The server never synchronises the device except through event queries; the
only host work per request is planning and launching.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np


def job_for_edges(kind: str, edges: int, seed: int, initiator=None):
    """Generation job with about `edges` edges (the serving workload's mapping):
    serial BA with m = 4 and n = ceil(E / 4), or Kronecker with
    k = ceil(log2(E / 16)) and exactly E edges."""
    if kind == "pba":
        return dict(kind="pba", n=max(1, -(-edges // 4)), m=4, n0=5, seed=seed)
    from .workloads import KRON_INITIATOR
    k = max(1, math.ceil(math.log2(max(edges, 32) / 16)))
    return dict(kind="kron", initiator=initiator or KRON_INITIATOR, k=k, n_edges=edges, seed=seed)


def job_edges(job) -> int:
    if job["kind"] == "pba":
        return job["n"] * job["m"] + job["n0"] * (job["n0"] - 1) // 2
    return job["n_edges"]


def job_vertices(job) -> int:
    if job["kind"] == "pba":
        return job["n0"] + job["n"]
    return job["initiator_n0"] ** job["k"] if "initiator_n0" in job else len(job["initiator"]) ** job["k"]


def job_csr_bytes(job) -> int:
    """Device bytes of a request's CSR: row_ptr (8 B/vertex) and col (4 B/edge)."""
    return (job_vertices(job) + 1) * 8 + job_edges(job) * 4


def job_transient_bytes(job) -> int:
    """Device bytes a request needs only until its batch retires: the edge
    list (8 B/edge), and its share of the batch CSR's workspace: the sort's
    workspace for its edges, its edges again in the union list (8 B/edge) and
    its rows in the union's row pointers (8 B/vertex)."""
    import paper_1003_3684_gb300 as pg
    E, N = job_edges(job), job_vertices(job)
    return E * 8 + pg.pg_csr_workspace_size(E, N) + E * 8 + (N + 1) * 8


def job_bytes(job) -> int:
    """Device bytes a request holds at its peak: edge list, CSR workspace and CSR."""
    return job_transient_bytes(job) + job_csr_bytes(job)


@dataclass
class Request:
    rid: int
    job: dict
    arrival: float
    nbytes: int
    deadline: float | None = None   # latest start time (server clock); None: no limit
    state: str = "waiting"          # waiting, admitted, running, done, cancelled, expired, failed
    error: str | None = None
    admitted: float | None = None
    launched: float | None = None
    done: float | None = None
    row_ptr: object = None
    col: object = None
    held: int = 0          # budget bytes this request holds right now
    csr_share: object = None   # the batch's shared CSR allocation, while results are held

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


@dataclass
class _CsrShare:
    """The CSR allocation shared by a batch's requests: the budget bytes of
    released requests stay counted until the last one is released."""
    live: int
    parked: int = 0


@dataclass
class _Batch:
    requests: list
    stream: object
    event: object
    keep: list = field(default_factory=list)
    status: object = None   # per request: its own CSR call's wait word (pinned host memory)
    batch_status: object = None   # the batch CSR's wait word, for the requests it built


class Server:
    def __init__(self, budget_bytes: int = 64 << 30, n_streams: int = 2, max_batch_jobs: int = 256,
                 max_batch_edges: int = 1 << 28, tile_edges: int = 4096, device="cuda",
                 clock=time.perf_counter, per_graph: bool = False,
                 batch_csr_edges: int = 1 << 17):
        """per_graph=True replaces the batched launch by one gen_pba /
        gen_kronecker call per request (the baseline a batching server beats).
        Requests with fewer than batch_csr_edges edges get their CSR from the
        batch's one sort; larger ones from a call of their own."""
        self.per_graph = per_graph
        self.batch_csr_edges = batch_csr_edges
        self.budget = budget_bytes
        self.in_use = 0
        self.peak_in_use = 0
        self.max_batch_jobs = max_batch_jobs
        self.max_batch_edges = max_batch_edges
        self.tile_edges = tile_edges
        self.device_name = device
        self.clock = clock
        self.n_streams = n_streams
        self.busy = {i: None for i in range(n_streams)}
        self.waiting: deque[Request] = deque()
        self.admitted: deque[Request] = deque()
        self.completed: list[Request] = []
        self.cancelled: list[Request] = []
        self.expired: list[Request] = []
        self.failed: list[Request] = []
        self._next_id = 0
        self.launches = 0
        self._cuda = False

    def _init_cuda(self):
        """Device objects, created at the first launch."""
        import torch

        import paper_1003_3684_gb300 as pg
        self.pg, self.torch = pg, torch
        self.device = torch.device(self.device_name)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(self.n_streams)]
        # the batch workspaces are held for the server's lifetime
        self.batch_ws = [torch.empty(pg.pg_batch_workspace_size(), dtype=torch.uint8,
                                     device=self.device) for _ in range(self.n_streams)]
        self.in_use += sum(w.numel() for w in self.batch_ws)
        self.peak_in_use = max(self.peak_in_use, self.in_use)
        self._cuda = True

    # ------------------------------------------------------------------
    def submit(self, job: dict, now: float | None = None, deadline: float | None = None) -> Request:
        """Queue a request. `deadline` (server clock) is the latest time it may
        start; a request still waiting then expires without running."""
        now = self.clock() if now is None else now
        r = Request(self._next_id, job, now, job_bytes(job), deadline=deadline)
        if r.nbytes > self.budget:
            raise ValueError(f"request of {r.nbytes} bytes exceeds the {self.budget}-byte budget")
        self._next_id += 1
        self.waiting.append(r)
        return r

    def cancel(self, r: Request) -> bool:
        """Withdraw a request. A waiting or admitted one is dropped at once (its
        budget is returned); a running one still finishes on the device, and
        its results and bytes are dropped when its batch retires. Returns
        False when the request had already finished or left the server."""
        if r.state == "waiting":
            self.waiting.remove(r)
        elif r.state == "admitted":
            self.admitted.remove(r)
            self._give_back(r, r.held)
        elif r.state != "running":
            return False
        r.state = "cancelled"
        if r not in self.cancelled:
            self.cancelled.append(r)
        return True

    def release(self, r: Request):
        """Client is done with a result: free its device memory and budget
        (a batch's CSR bytes come back when its last request is released)."""
        r.row_ptr = r.col = None
        share, r.csr_share = r.csr_share, None
        if share is None:
            self._give_back(r, r.held)
            return
        share.parked += r.held      # still allocated in the shared CSR arenas
        r.held = 0
        share.live -= 1
        if share.live == 0:
            self.in_use -= share.parked
            share.parked = 0

    def pending(self) -> int:
        return len(self.waiting) + len(self.admitted) + sum(b is not None for b in self.busy.values())

    # ------------------------------------------------------------------
    def _give_back(self, r: Request, nbytes: int):
        self.in_use -= nbytes
        r.held -= nbytes

    def _retire(self, now):
        for i, b in self.busy.items():
            if b is None or not b.event.query():
                continue
            for k, r in enumerate(b.requests):
                # the edge list and the CSR workspace are dropped once the CSR exists
                self._give_back(r, job_transient_bytes(r.job))
                if r.state == "cancelled":
                    self.release(r)
                    continue
                r.done = now
                own = b.status is not None and int(b.status[k]) != 0
                shared = (r.csr_share is not None and b.batch_status is not None and
                          int(b.batch_status[0]) != 0)
                if own or shared:
                    r.state, r.error = "failed", "CSR sort: a bounded wait gave up (PG_ETIMEOUT)"
                    self.release(r)
                    self.failed.append(r)
                    continue
                r.state = "done"
                self.completed.append(r)
            self.busy[i] = None

    def _expire(self, now):
        for q in (self.waiting, self.admitted):
            for r in [r for r in q if r.deadline is not None and now > r.deadline]:
                q.remove(r)
                if r.held:
                    self._give_back(r, r.held)
                r.state = "expired"
                self.expired.append(r)

    def _admit(self, now):
        while self.waiting and self.in_use + self.waiting[0].nbytes <= self.budget:
            r = self.waiting.popleft()
            r.admitted = now
            r.state = "admitted"
            r.held = r.nbytes
            self.in_use += r.nbytes
            self.peak_in_use = max(self.peak_in_use, self.in_use)
            self.admitted.append(r)

    def _next_batch(self):
        batch, edges = [], 0
        while (self.admitted and len(batch) < self.max_batch_jobs and
               (not batch or edges + job_edges(self.admitted[0].job) <= self.max_batch_edges)):
            r = self.admitted.popleft()
            edges += job_edges(r.job)
            batch.append(r)
        return batch

    def _fail(self, batch, why: str):
        """Requests of a batch whose launch failed: failed, budget returned."""
        for r in batch:
            r.row_ptr = r.col = None
            if r.held:
                self._give_back(r, r.held)
            r.state, r.error = "failed", why
            self.failed.append(r)

    def _launch(self, now):
        if not self._cuda:
            self._init_cuda()
        for i, b in self.busy.items():
            if b is not None or not self.admitted:
                continue
            batch = self._next_batch()
            try:
                self.busy[i] = self._start(i, batch, now)
            except (RuntimeError, MemoryError) as exc:
                # a device allocation that failed, or a library call that
                # refused: this batch fails, the server goes on. Work already
                # queued on the stream only touches buffers allocated on that
                # stream, which the allocator hands out again only to later
                # work on the same stream.
                self._fail(batch, f"launch failed: {exc}")

    def _start(self, i, batch, now) -> _Batch:
        """Queue one batch on stream i."""
        if self.per_graph:
            return self._start_per_graph(i, batch, now)
        return self._start_batched(i, batch, now)

    def _start_per_graph(self, i, batch, now) -> _Batch:
        """The per-graph baseline: a generation call and a CSR call per request."""
        torch, pg = self.torch, self.pg
        s = self.streams[i]
        with torch.cuda.stream(s):
            offs = np.cumsum([0] + [job_edges(r.job) + (job_edges(r.job) & 1) for r in batch])
            arena = pg.empty_device((max(int(offs[-1]), 1), 2), torch.int32, self.device)
            for k, r in enumerate(batch):
                j, a = r.job, int(offs[k])
                sl = arena[a:a + job_edges(j)]
                if j["kind"] == "pba":
                    pg.gen_pba(j["n"], j["m"], 1, j["n0"], 1, 0.0, j["seed"], out=sl, stream=s)
                else:
                    pg.gen_kronecker(j["initiator"], j["k"], j["n_edges"], j["seed"], out=sl,
                                     stream=s)
                self.launches += 1
            plan = None
            offsets = [int(x) for x in offs]
            # one CSR workspace for the batch, sized for its largest
            # request (each request's share is counted in its bytes)
            need = max(pg.pg_csr_workspace_size(job_edges(r.job), job_vertices(r.job))
                       for r in batch)
            ws = pg.empty_device(max(need, 256), torch.uint8, self.device)
            status = torch.zeros(len(batch), dtype=torch.int32, pin_memory=True)
            for k, r in enumerate(batch):
                a = offsets[k]
                z = a + job_edges(r.job)
                E, N = job_edges(r.job), job_vertices(r.job)
                r.row_ptr, r.col = pg.edges_to_csr(arena[a:z], N, workspace=ws, stream=s)
                off = pg.pg_csr_wait_error_offset(E, N)
                if off is not None:   # the call's wait word, to pinned memory
                    status[k:k + 1].copy_(ws[off:off + 4].view(torch.int32), non_blocking=True)
                r.launched = now
                r.state = "running"
                self.launches += 1
            ev = torch.cuda.Event()
            ev.record(s)
        return _Batch(batch, s, ev, keep=[plan, arena, ws], status=status)

    def _start_batched(self, i, batch, now) -> _Batch:
        """One persistent generation launch for the batch; then the CSRs of
        its small requests from one sort of their union (gen_batch_csr), and
        of each large one from its own edges_to_csr call."""
        torch, pg = self.torch, self.pg
        s = self.streams[i]
        small = [job_edges(r.job) < self.batch_csr_edges for r in batch]
        with torch.cuda.stream(s):
            plan = pg.BatchPlan([dict(r.job, want_csr=sm) for r, sm in zip(batch, small)],
                                tile_edges=self.tile_edges, device=self.device)
            arena = pg.empty_device((max(plan.total_edges, 1), 2), torch.int32, self.device)
            pg.gen_batch(plan, arena=arena, workspace=self.batch_ws[i], stream=s)
            self.launches += 1
            keep = [plan, arena]
            batch_status = None
            if any(small):
                ws = pg.empty_device(max(pg.pg_batch_csr_workspace_size(plan), 256), torch.uint8,
                                     self.device)
                rp_all = pg.empty_device(max(plan.csr_rows_total, 1), torch.int64, self.device)
                col_all = pg.empty_device(max(plan.csr_cols_total, 1), torch.int32, self.device)
                pg.gen_batch_csr(plan, arena, row_ptr=rp_all, col=col_all, workspace=ws, stream=s)
                self.launches += 1
                keep.append(ws)
                batch_status = torch.zeros(1, dtype=torch.int32, pin_memory=True)
                off = pg.pg_batch_csr_wait_error_offset(plan)
                if off is not None:   # the sort's wait word, to pinned memory
                    batch_status.copy_(ws[off:off + 4].view(torch.int32), non_blocking=True)
                share = _CsrShare(live=sum(small))
            status = None
            if not all(small):
                need = max(pg.pg_csr_workspace_size(job_edges(r.job), job_vertices(r.job))
                           for r, sm in zip(batch, small) if not sm)
                ws_big = pg.empty_device(max(need, 256), torch.uint8, self.device)
                keep.append(ws_big)
                status = torch.zeros(len(batch), dtype=torch.int32, pin_memory=True)
            for k, r in enumerate(batch):
                if small[k]:
                    r.row_ptr, r.col = plan.csr_of(rp_all, col_all, k)
                    r.csr_share = share
                else:
                    E, N = job_edges(r.job), job_vertices(r.job)
                    r.row_ptr, r.col = pg.edges_to_csr(plan.edges_of(arena, k), N,
                                                       workspace=ws_big, stream=s)
                    off = pg.pg_csr_wait_error_offset(E, N)
                    if off is not None:   # the call's wait word, to pinned memory
                        status[k:k + 1].copy_(ws_big[off:off + 4].view(torch.int32),
                                              non_blocking=True)
                    self.launches += 1
                r.launched = now
                r.state = "running"
            ev = torch.cuda.Event()
            ev.record(s)
        return _Batch(batch, s, ev, keep=keep, status=status, batch_status=batch_status)

    def step(self, now: float | None = None) -> int:
        """One scheduling step; returns the number of requests completed."""
        now = self.clock() if now is None else now
        before = len(self.completed)
        self._retire(now)
        self._expire(now)
        self._admit(now)
        self._launch(now)
        return len(self.completed) - before

    def drain(self):
        while self.pending():
            self.step()


def poisson_workload(rate: float, duration: float, seed: int = 0, lo_exp: int = 12,
                     hi_exp: int = 26):
    """Arrival times (exponential gaps) and jobs: half BA, half Kronecker,
    edge counts log-uniform in [2^lo_exp, 2^hi_exp]; job i uses seed i."""
    rng = np.random.default_rng(seed)
    t, out, i = 0.0, [], 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        kind = "pba" if rng.random() < 0.5 else "kron"
        edges = int(2 ** rng.uniform(lo_exp, hi_exp))
        out.append((t, job_for_edges(kind, edges, seed=i)))
        i += 1
    return out


def run_open_loop(server: Server, arrivals, release: bool = True, max_wall: float | None = None):
    """Replay arrivals in real time against the server (open loop: arrivals do
    not wait for completions). Returns the completed requests."""
    t0 = server.clock()
    idx = 0
    n = len(arrivals)
    while idx < n or server.pending():
        now = server.clock() - t0
        while idx < n and arrivals[idx][0] <= now:
            server.submit(arrivals[idx][1], now=t0 + arrivals[idx][0])
            idx += 1
        done = server.step(server.clock())
        if release and done:
            for r in server.completed[-done:]:
                server.release(r)
        if max_wall is not None and now > max_wall:
            break
        if not done and idx < n and arrivals[idx][0] > now + 2e-4:
            time.sleep(min(1e-3, arrivals[idx][0] - now))
    return server.completed

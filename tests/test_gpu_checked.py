"""The bounds-checked build (libpgen_checked.so, loaded with PGEN_LIBRARY=checked).

In the checked build every kernel access whose index comes from data, and
every store of a result element, is compared with its buffer's bound; a
failed comparison skips the access and is counted in a device record
(pg_check_read). test_gpu_suite_is_clean_under_the_checked_build runs the
whole GPU suite again in a child process that loads the checked library;
there a fixture in conftest reads the records around every GPU test and
fails it on any failed comparison.

The other tests run only in that child. A test hook shortens the bound of
result stores to bound >> 1, which lies inside the real buffer, so real
kernels skip stores that are in fact in bounds: the record must name the
right source file, the shortened bound and an index at or above it, the
part below the bound must equal a normal call's output, and the rest must
keep its canary.
"""
import os
import re
import subprocess
import sys

import numpy as np
import pytest
import torch

import paper_1003_3684_gb300 as pg
from conftest import ROOT
from paper_1003_3684_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CHECKED = os.environ.get("PGEN_LIBRARY") == "checked"
in_child = pytest.mark.skipif(not CHECKED, reason="runs in the checked-build child process")
C32 = 0x5A5A5A5A
UNIT_KRON, UNIT_PBA, UNIT_CSR, UNIT_BATCH = 1, 2, 3, 4


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1003_3684_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def test_gpu_suite_is_clean_under_the_checked_build():
    if CHECKED:
        pytest.skip("this is the child run")
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    env = dict(os.environ, PGEN_LIBRARY="checked")
    r = subprocess.run([sys.executable, "-m", "pytest", "tests", "-m", "gpu", "-x", "-q",
                        "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=1800)
    tail = "\n".join((r.stdout + r.stderr).splitlines()[-40:])
    assert r.returncode == 0, tail
    # the child ran the suite: every GPU test file, this one's child-only tests included
    passed = re.search(r"(\d+) passed", tail)
    assert passed and int(passed.group(1)) >= 150 and " failed" not in tail, tail
    print(tail.splitlines()[-1])


@in_child
def test_child_loaded_the_checked_library():
    assert pg.pg_checked_build()
    assert pg.library_path().endswith("libpgen_checked.so")


def _canary(rows, cols=2):
    shape = (rows, cols) if cols else (rows,)
    return torch.full(shape, C32, dtype=torch.int32, device="cuda")


def _hooked(call, E, unit, cols=2):
    """call(buf) writes E result rows into buf. Runs it once normally and
    once with the store bound halved; returns the record of the second."""
    ref = _canary(E, cols)
    call(ref)
    assert pg.pg_check_read().count == 0
    buf = _canary(E, cols)
    pg.pg_check_test_out_shift(1)
    try:
        call(buf)
        rep = pg.pg_check_read(reset=True)
    finally:
        pg.pg_check_test_out_shift(0)
    assert rep.count > 0, rep
    assert rep.unit == unit, rep
    assert rep.bound == E >> 1 and rep.index >= rep.bound, rep
    # pairs of edges are stored together from an even index, so with an even
    # bound everything below it is written and nothing above it
    h = rep.bound
    assert h % 2 == 0
    assert torch.equal(buf[:h], ref[:h])
    assert bool((buf[h:] == C32).all()), "a store past the shortened bound was not skipped"
    # and with the hook off again the library writes everything
    again = _canary(E, cols)
    call(again)
    assert pg.pg_check_read().count == 0
    assert torch.equal(again, ref)
    return rep


@in_child
@pytest.mark.check_violations
def test_kronecker_stores_past_the_shortened_bound_are_skipped_and_reported():
    E = 10_000
    _hooked(lambda out: pg.gen_kronecker(W.KRON_INITIATOR, 12, E, 7, out=out), E, UNIT_KRON)
    _hooked(lambda out: pg.gen_random_cells(1000, E, seed=3, out=out), E, UNIT_KRON)


@in_child
@pytest.mark.check_violations
def test_pba_stores_past_the_shortened_bound_are_skipped_and_reported():
    n, m = 10_002, 3                   # 30,012 edges: the halved bound is even
    E = pg.pg_pba_edge_count(n, m, 1, 4)
    _hooked(lambda out: pg.gen_pba(n, m, 1, 4, 1, 0.0, 5, out=out), E, UNIT_PBA)
    B, nb = 8, 3_000
    E = pg.pg_pba_edge_count(B * nb, 4, B, 5)
    ws = torch.empty(pg.pg_pba_workspace_size(B * nb, 4, B), dtype=torch.uint8, device="cuda")
    _hooked(lambda out: pg.gen_pba(B * nb, 4, B, 5, 1, 0.1, 9, out=out, workspace=ws), E,
            UNIT_PBA)


@in_child
@pytest.mark.check_violations
def test_csr_col_stores_past_the_shortened_bound_are_skipped_and_reported():
    M, N = 60_000, 2_000
    rng = np.random.default_rng(11)
    e = rng.integers(0, N, size=(M, 2), dtype=np.uint32)
    t = torch.from_numpy(e.view(np.int32)).cuda()

    def call(col):
        pg.edges_to_csr(t, N, col=col, check=True)

    _hooked(call, M, UNIT_CSR, cols=0)


@in_child
@pytest.mark.check_violations
def test_batch_stores_past_the_shortened_bound_are_skipped_and_reported():
    jobs = [dict(kind="pba", n=4_000 + 50 * i, m=2 + i % 3, n0=4, seed=i) for i in range(3)]
    jobs += [dict(kind="kron", initiator=W.KRON_INITIATOR, k=10, n_edges=3_000, seed=9)]
    plan = pg.BatchPlan(jobs, tile_edges=1024)
    E = plan.total_edges               # 39,568: the halved bound is even
    _hooked(lambda out: pg.gen_batch(plan, arena=out), E, UNIT_BATCH)

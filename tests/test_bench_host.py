"""Host-side pieces of the benchmark that need no GPU: the DRAM-traffic table
the roofline reads, and the labelled all-cores estimate of the CPU baseline."""
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _traffic_rows():
    rows = []
    for ln in open(os.path.join(ROOT, "profiles", "dram_traffic.md")).read().splitlines():
        cells = [c.strip() for c in ln.strip().strip("|").split("|")]
        if len(cells) >= 6 and cells[0].startswith("`"):
            rows.append(cells)
    return rows


def test_traffic_table_rows_are_well_formed():
    rows = _traffic_rows()
    assert rows, "no rows"
    for kernel, src, sha, per_unit, unit, capture in (r[:6] for r in rows):
        assert os.path.isfile(os.path.join(ROOT, src.strip("`"))), src
        assert re.fullmatch(r"`[0-9a-f]{12}`", sha), sha
        assert float(per_unit) > 0
        name = re.search(r"`([^`]+\.md)`", capture).group(1)
        assert os.path.isfile(os.path.join(ROOT, "profiles", name)), capture


def test_traffic_table_keeps_only_rows_of_the_current_sources():
    # a row applies only while its source still has the recorded hash
    got = bench.dram_traffic_table()
    import hashlib
    for kernel, src, sha, per_unit, *_ in _traffic_rows():
        cur = hashlib.sha256(open(os.path.join(ROOT, src.strip("`")), "rb").read()).hexdigest()[:12]
        if cur == sha.strip("`"):
            assert got[kernel.strip("`")] == float(per_unit)
        else:
            assert kernel.strip("`") not in got


def test_all_cores_estimate_is_labelled():
    e = bench.all_cores_estimate(2.0)
    assert e["value"] == 2.0 * e["host_cores"] and e["host_cores"] >= 1
    assert "estimate" in e["note"]


def test_deterministic_kronecker_workload_is_the_fig2_seed():
    # the workload's seed is the cited Fig. 2(b) fixture, and its size is e0^k
    from paper_1003_3684_gb300 import build, workloads as W
    build.build()
    import paper_1003_3684_gb300 as pg
    rows = [ln.split() for ln in open(os.path.join(ROOT, "tests", "golden", "pk_fig2_seed.txt"))
            if ln.strip() and not ln.startswith("#")]
    cfg = W.CONFIGS["kron_det_fig2_k8"]
    assert [[int(x) for x in r] for r in rows] == cfg["initiator"]
    assert pg.pg_kron_edge_count(cfg["initiator"], cfg["k"], 0, deterministic=True) == 11 ** 8
    assert bench.kron_det_work(cfg["k"]) == dict(ops=48, bytes=8)

"""Host-side pieces of the benchmark that need no GPU: the DRAM-traffic table
the roofline reads, and the labelled all-cores estimate of the CPU baseline."""
import json
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _traffic_rows():
    with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as fh:
        return json.load(fh)["kernels"]


def test_traffic_table_rows_are_well_formed():
    rows = _traffic_rows()
    assert rows, "no rows"
    for r in rows:
        assert os.path.isfile(os.path.join(ROOT, r["source"])), r["source"]
        assert re.fullmatch(r"[0-9a-f]{12}", r["sha256"]), r["sha256"]
        assert float(r["bytes_per_unit"]) > 0 and r["unit"]
        name = re.match(r"([\w.-]+\.md)", r["capture"]).group(1)
        assert os.path.isfile(os.path.join(ROOT, "profiles", name)), r["capture"]


def test_traffic_table_keeps_only_rows_of_the_current_sources():
    # a row applies only while its source still has the recorded hash
    got = bench.dram_traffic_table()
    import hashlib
    for r in _traffic_rows():
        cur = hashlib.sha256(open(os.path.join(ROOT, r["source"]), "rb").read()).hexdigest()[:12]
        if cur == r["sha256"]:
            assert got[r["kernel"]] == float(r["bytes_per_unit"])
        else:
            assert r["kernel"] not in got


def test_default_run_names_its_sub_records():
    # the default line carries the metric's other parts, each a known workload
    from paper_1003_3684_gb300 import workloads as W
    keys = [k for k, _, _ in bench.SUB_RECORDS]
    assert keys == ["kron", "batch", "serve"]
    for _, workload, over in bench.SUB_RECORDS:
        assert workload in W.CONFIGS
        assert W.CONFIGS[workload]["kind"] in ("kron", "batch", "serve")


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

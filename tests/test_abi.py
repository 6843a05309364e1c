"""The C ABI library loads, exports every symbol include/pgen.h declares, and
rejects bad arguments on the host before any launch (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess
import sys

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "pgen.h")


@pytest.fixture(scope="module")
def L():
    from paper_1003_3684_gb300 import build
    build.build()
    import paper_1003_3684_gb300 as pg
    return pg.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "defined")))


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("gen_pba", "gen_kronecker", "edges_to_csr", "pg_status_string",
                     "pg_pba_workspace_size", "pg_csr_workspace_size"):
        assert required in names


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_status_strings(L):
    import paper_1003_3684_gb300 as pg
    assert pg.pg_status_string(pg.PG_OK) == "ok"
    assert "invalid" in pg.pg_status_string(pg.PG_EINVAL)
    assert pg.pg_status_string(99) == "unknown status"


def test_edge_counts_on_host(L):
    import paper_1003_3684_gb300 as pg
    assert pg.pg_pba_edge_count(100_000, 4, 1, 5) == 400_010
    assert pg.pg_pba_edge_count(2**30, 5, 1024, 6) == 1024 * (15 + 2**20 * 5)
    assert pg.pg_pba_edge_count(10, 2, 3, 4) == 0             # blocks do not divide n
    G1 = [[1, 1, 1, 1, 0], [1, 1, 0, 0, 0], [1, 0, 1, 0, 0], [1, 0, 0, 1, 0], [0, 0, 0, 0, 1]]
    assert pg.pg_kron_edge_count(G1, 3, 0, deterministic=True) == 11 ** 3
    assert pg.pg_kron_edge_count([[0.5, 0.5], [0.5, 0.5]], 5, 1234) == 1234


@pytest.mark.parametrize("args", [
    (100, 0, 1, 5, 1, 0.1),       # m = 0
    (100, 4, 1, 1, 1, 0.1),       # n0 = 1
    (100, 4, 3, 5, 1, 0.1),       # blocks do not divide n
    (120, 4, 4, 5, 3, 0.1),       # faction width does not divide blocks
    (120, 4, 4, 5, 1, -0.5),      # f outside [0, 1]
    (120, 4, 4, 5, 1, float("nan")),
    (2048 * 2, 4, 2048, 5, 1, 0.1),   # more blocks than supported
])
def test_gen_pba_rejects_bad_arguments(L, args):
    n, m, B, n0, W, f = args
    cnt = C.c_uint64(7)
    st = L.gen_pba(n, m, B, n0, W, f, 1, 0, None, 0, C.byref(cnt), None, 0, None)
    assert st == 1


def test_gen_pba_capacity_and_ids(L):
    cnt = C.c_uint64(0)
    # capacity too small: reports the count, launches nothing
    st = L.gen_pba(100, 4, 1, 5, 1, 0.0, 1, 0, C.c_void_p(16), 5, C.byref(cnt), None, 0, None)
    assert st == 2 and cnt.value == 410
    # 2^32 vertex ids do not fit 32-bit ids
    st = L.gen_pba(2**32, 1, 1, 5, 1, 0.0, 1, 0, None, 0, C.byref(cnt), None, 0, None)
    assert st == 1
    # misaligned output
    st = L.gen_pba(100, 4, 1, 5, 1, 0.0, 1, 0, C.c_void_p(8), 10**6, C.byref(cnt), None, 0, None)
    assert st == 1


def test_gen_kronecker_rejects_bad_arguments(L):
    import numpy as np
    cnt = C.c_uint64(0)
    P = np.array([[0.5, 0.2], [0.2, 0.1]])
    Z = np.zeros((2, 2))
    Neg = np.array([[0.5, -0.2], [0.2, 0.1]])
    pp = lambda a: a.ctypes.data_as(C.c_void_p)
    assert L.gen_kronecker(pp(Z), 2, 4, 10, 1, 0, 0, C.c_void_p(16), 10, C.byref(cnt), None) == 1
    assert L.gen_kronecker(pp(Neg), 2, 4, 10, 1, 0, 0, C.c_void_p(16), 10, C.byref(cnt), None) == 1
    assert L.gen_kronecker(pp(P), 2, 33, 10, 1, 0, 0, C.c_void_p(16), 10, C.byref(cnt), None) == 1
    assert L.gen_kronecker(pp(P), 2, 4, 10, 1, 0, 0, C.c_void_p(16), 9, C.byref(cnt), None) == 2
    assert L.gen_kronecker(pp(P), 17, 2, 10, 1, 0, 0, C.c_void_p(16), 10, C.byref(cnt), None) == 1


def test_edges_to_csr_rejects_bad_arguments(L):
    assert L.edges_to_csr(C.c_void_p(16), 10, 0, 0, C.c_void_p(16), C.c_void_p(16),
                          None, 0, None) == 1
    assert L.edges_to_csr(C.c_void_p(16), 10, 100, 0, C.c_void_p(16), C.c_void_p(16),
                          None, 0, None) == 5


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_1003_3684_gb300 as pg
    monkeypatch.setattr(pg, "_LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pg, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        pg.lib()


def test_faction_table_layout_on_host(L):
    """pg_pba_faction_table (host only): list size, complement size, the list,
    and the blocks outside it in ascending order, one 4112-byte record each."""
    import numpy as np

    import paper_1003_3684_gb300 as pg
    lists = [[0, 1, 4, 5, 0], [0, 1, 1, 2, 3], [1, 2, 3], [1, 2, 3, 3, 4], [3, 4, 4, 5, 0],
             [4, 5, 0]]
    tab = pg.pba_faction_table(lists).view(np.uint16)
    assert tab.size == 6 * 2056
    for p, li in enumerate(lists):
        rec = tab[p * 2056:(p + 1) * 2056]
        outside = [b for b in range(6) if b not in li]
        assert rec[0] == len(li) and rec[1] == len(outside)
        assert rec[8:8 + len(li)].tolist() == li
        assert rec[8 + 1024:8 + 1024 + len(outside)].tolist() == outside


@pytest.mark.parametrize("lists", [
    [[0], []],                  # empty list
    [[0, 2], [1]],              # member out of range
    [[0] * 1025, [1]],          # longer than 1024 entries
])
def test_faction_table_rejects_bad_lists(L, lists):
    import paper_1003_3684_gb300 as pg
    with pytest.raises(pg.PgenError):
        pg.pba_faction_table(lists)


def test_range_entry_points_reject_bad_ranges(L):
    import numpy as np

    import paper_1003_3684_gb300 as pg
    R = pg._range_lib()
    P = np.array([0.5, 0.2, 0.2, 0.1])
    # e_end beyond the edge count, and e_begin after e_end
    assert R.gen_kronecker_range(P.ctypes.data, 2, 5, 100, 1, 0, 0, 0, 101, None, 1000, None) == pg.PG_EINVAL
    assert R.gen_kronecker_range(P.ctypes.data, 2, 5, 100, 1, 0, 0, 50, 40, None, 1000, None) == pg.PG_EINVAL
    # capacity below the range
    assert R.gen_kronecker_range(P.ctypes.data, 2, 5, 100, 1, 0, 0, 10, 40, None, 29, None) == pg.PG_ENOSPC
    # block range outside [0, blocks]
    cnt = C.c_uint64(0)
    assert R.gen_pba_blocks(4000, 2, 4, 3, 1, 0, 3, 5, None, 10**9, C.byref(cnt), None, 0, None) == pg.PG_EINVAL
    assert R.gen_pba_blocks(4000, 2, 4, 3, 1, 0, 3, 2, None, 10**9, C.byref(cnt), None, 0, None) == pg.PG_EINVAL
    # an empty range is valid and launches nothing
    assert R.gen_pba_blocks(4000, 2, 4, 3, 1, 0, 2, 2, None, 0, C.byref(cnt), None, 0, None) == pg.PG_OK
    assert cnt.value == 0


@pytest.mark.parametrize("M,N", [(1, 2), (100_000, 2**20), (8_191, 3), (70_000, 2**33 + 5),
                                 (3 * 2**20 + 7, 5_000)])
@pytest.mark.parametrize("id64", [False, True])
@pytest.mark.parametrize("flags", [0, 1, 2, 1 | 2 | 4, 8])
def test_csr_wait_error_word_lies_in_the_workspace(L, M, N, id64, flags):
    import paper_1003_3684_gb300 as pg
    if not id64 and N > 2**32:
        return
    off = pg.pg_csr_wait_error_offset(M, N, id64, flags)
    ws = (pg.pg_csr_workspace_size(M, N) if flags == 0 else
          int(pg._opts_lib().pg_csr_opts_workspace_size(M, N, flags)))
    listed = 2 * M if flags & pg.CSR_SYMMETRIZE else M
    assert off is not None and off % 4 == 0
    assert off + 4 <= ws
    # past the two copies of the list that the sort writes
    assert off >= 2 * listed * (16 if id64 else 8)


def test_csr_wait_error_word_absent_when_nothing_is_sorted(L):
    import paper_1003_3684_gb300 as pg
    assert pg.pg_csr_wait_error_offset(0, 10) is None          # no edges
    assert pg.pg_csr_wait_error_offset(50, 1) is None          # a single row
    assert pg.pg_csr_wait_error_offset(50, 10, flags=16) is None
    assert pg.pg_csr_wait_error_offset(50, 10, flags=1) is not None


def _per_device_once(L, devs, threads, fail_dev):
    n = len(devs)
    d = (C.c_int * max(n, 1))(*devs)
    calls = (C.c_int * 64)()
    status = (C.c_int * max(n, 1))()
    L.pg_test_per_device_once.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                          C.c_void_p]
    L.pg_test_per_device_once.restype = C.c_int
    st = L.pg_test_per_device_once(d, n, threads, fail_dev, calls, status)
    return st, list(calls), list(status)[:n]


def test_kernel_attributes_are_set_once_per_device(L):
    # the bookkeeping that guards cudaFuncSetAttribute: every device gets its
    # own set-up, exactly once, however many host threads race for it
    devs = [0, 1, 0, 3, 1, 7, 63, 0, 3]
    for threads in (1, 8, 64):
        st, calls, status = _per_device_once(L, devs, threads, -1)
        assert st == 0
        assert calls[0] == calls[1] == calls[3] == calls[7] == calls[63] == 1
        assert sum(calls) == 5
        assert status == [0] * len(devs)


def test_failed_device_setup_is_remembered(L):
    # a device whose set-up failed keeps failing (no retry, no partial state),
    # other devices are unaffected; ids outside 0..63 fail without a set-up
    st, calls, status = _per_device_once(L, [2, 5, 2, 5, 64, -1], 16, 5)
    assert st == 0
    assert calls[2] == 1 and calls[5] == 1 and sum(calls) == 2
    assert status[0] == status[2] == 0
    assert status[1] != 0 and status[3] == status[1]
    assert status[4] != 0 and status[5] != 0
    assert _per_device_once(L, [0], 0, -1)[0] == 1        # threads < 1: invalid


def test_csr_check_arguments_on_host(L):
    L.pg_csr_check.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int, C.c_uint32,
                               C.c_void_p]
    L.pg_csr_check.restype = C.c_int
    assert L.pg_csr_check(None, 10, 10, 0, 16, None) == 1    # unknown flag
    assert L.pg_csr_check(None, 10, 10, 7, 0, None) == 1     # bad id width
    # nothing to sort (no edges, or one vertex): no wait, nothing read
    assert L.pg_csr_check(None, 0, 10, 0, 0, None) == 0
    assert L.pg_csr_check(None, 10, 1, 0, 0, None) == 0
    assert L.pg_csr_check(None, 10, 10, 0, 0, None) == 1     # a sorting call needs its workspace


@pytest.fixture(scope="module")
def LC(L):
    """The bounds-checked build, loaded by path beside the default one."""
    return C.CDLL(os.path.join(ROOT, "paper_1003_3684_gb300", "libpgen_checked.so"))


def test_checked_library_exports_every_declared_symbol(LC):
    for name in declared_functions():
        assert hasattr(LC, name), name


def test_checked_build_flag_and_host_side_checks(L, LC):
    for lib in (L, LC):
        lib.pg_checked_build.restype = C.c_int
        lib.pg_check_test_out_shift.argtypes = [C.c_uint32, C.c_void_p]
        lib.pg_check_test_out_shift.restype = C.c_int
        lib.pg_check_read.restype = C.c_int
    assert L.pg_checked_build() == 0 and LC.pg_checked_build() == 1
    # the default build has no checks: the hook is refused, the record is empty
    assert L.pg_check_test_out_shift(1, None) == 1
    count, unit = C.c_uint32(7), C.c_uint32(7)
    assert L.pg_check_read(1, C.byref(count), C.byref(unit), None, None, None, None) == 0
    assert count.value == 0 and unit.value == 0
    # the checked build refuses a shift past 63 before touching the device
    assert LC.pg_check_test_out_shift(64, None) == 1


@pytest.mark.parametrize("variant,expect", [("default", "False libpgen.so"),
                                            ("checked", "True libpgen_checked.so")])
def test_binding_loads_the_library_named_by_the_environment(L, variant, expect):
    code = ("import os, paper_1003_3684_gb300 as pg; "
            "print(pg.pg_checked_build(), os.path.basename(pg.library_path()))")
    env = dict(os.environ, PGEN_LIBRARY=variant)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == expect


def test_binding_rejects_an_unknown_library_variant():
    env = dict(os.environ, PGEN_LIBRARY="fast")
    r = subprocess.run([sys.executable, "-c", "import paper_1003_3684_gb300"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode != 0 and "PGEN_LIBRARY" in r.stderr

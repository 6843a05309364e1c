"""gen_pba_noalloc: the PBA generator for callers that cannot allocate device
memory (a host application's allocator owns the device, a plugin gets buffers
but no allocation API, or a latency-critical path must avoid cudaMalloc and
its synchronisation). It uses a fixed scratch array inside the library
instead of a caller workspace, so its output must equal gen_pba's for the same
arguments -- checked here through the C ABI on two calls in a row, which also
shows that the second call is not disturbed by what the first left in the
shared scratch. This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = [
    # n, m, blocks, n0, faction_width, inter_frac, seed
    (8 * 20_000, 5, 8, 6, 1, 0.1, 3),
    (12 * 9_000, 3, 12, 4, 2, 0.3, 77),
]


@pytest.fixture(scope="module")
def lib():
    import torch

    import paper_1003_3684_gb300 as pg
    from paper_1003_3684_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    L = pg.lib()
    L.gen_pba_noalloc.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                  C.c_double, C.c_uint64, C.c_int, C.c_void_p, C.c_uint64,
                                  C.POINTER(C.c_uint64), C.c_void_p]
    L.gen_pba_noalloc.restype = C.c_int
    L.pg_pba_noalloc_scratch_bytes.restype = C.c_size_t
    return L


def test_noalloc_matches_gen_pba_twice_in_a_row(lib):
    import torch

    import paper_1003_3684_gb300 as pg
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for (n, m, B, n0, Wf, f, seed) in CASES:
        assert pg.pg_pba_workspace_size(n, m, B) <= lib.pg_pba_noalloc_scratch_bytes()
        E = pg.pg_pba_edge_count(n, m, B, n0)
        out = torch.full((E, 2), -1, dtype=torch.int32, device="cuda")
        cnt = C.c_uint64(0)
        st = lib.gen_pba_noalloc(n, m, B, n0, Wf, f, seed, 0, C.c_void_p(out.data_ptr()), E,
                                 C.byref(cnt), stream)
        assert st == 0 and cnt.value == E
        ref = pg.gen_pba(n, m, B, n0, Wf, f, seed)      # the existing entry point
        torch.cuda.synchronize()
        assert torch.equal(out, ref), (n, m, B)


def test_noalloc_rejects_graphs_beyond_its_scratch(lib):
    import paper_1003_3684_gb300 as pg
    n, m, B = 64 * 2**20, 5, 64          # workspace far above 32 MiB
    assert pg.pg_pba_workspace_size(n, m, B) > lib.pg_pba_noalloc_scratch_bytes()
    cnt = C.c_uint64(0)
    st = lib.gen_pba_noalloc(n, m, B, 6, 1, 0.1, 1, 0, C.c_void_p(256), 2**40, C.byref(cnt), None)
    assert st == pg.PG_ENOMEM
    assert "workspace" in pg.pg_status_string(st)

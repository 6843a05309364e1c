"""pgen: GB300-native generation of massive scale-free graphs (arXiv 1003.3684).

Thin Python binding over the C ABI of ``libpgen.so`` (declared in
``include/pgen.h``). Each function here carries the C entry point's name and
only marshals arguments: torch supplies the device buffers and the current
CUDA stream, and every step of generation runs in the library's sm_103a
kernels. There is no CPU fallback: if the library is missing the first call
raises.

    import paper_1003_3684_gb300 as pgen
    edges = pgen.gen_pba(n=2**20, m=5, blocks=64, n0=6, faction_width=1,
                         inter_frac=0.1, seed=3)            # (E, 2) int32 view
    row_ptr, col = pgen.edges_to_csr(edges, n_vertices=...)

Edge tensors hold unsigned ids in signed containers (int32 for 32-bit ids,
int64 for 64-bit ids); ``.view(torch.uint32)`` or numpy ``.view(np.uint32)``
recovers the unsigned values.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import NamedTuple

import numpy as np

__all__ = [
    "PG_OK", "PG_EINVAL", "PG_ENOSPC", "PG_ECUDA", "PG_ETIMEOUT", "PG_ENOMEM",
    "PgenError", "lib", "library_path",
    "pg_status_string", "pg_device_sm_count", "pg_version",
    "pg_pba_edge_count", "pg_force_wide_path", "pg_pba_workspace_size", "gen_pba", "gen_pba_to_host",
    "pba_faction_table", "gen_pba_factions", "pg_pba_prepare", "gen_pba_blocks",
    "gen_kronecker_range", "philox_rate", "int_pipe_rates", "edges_to_csr_opts", "gen_random_cells",
    "kronecker_xor_random", "CSR_SYMMETRIZE", "CSR_DEDUP", "CSR_NO_LOOPS", "CSR_ODD",
    "DEG_OUT", "DEG_IN", "DEG_TOTAL", "degrees", "degree_histogram", "bfs", "powerlaw_exponent",
    "path_length_stats",
    "pg_kron_edge_count", "gen_kronecker",
    "pg_csr_workspace_size", "edges_to_csr", "pg_trace_enable", "pg_trace_dump", "pg_launch_count",
    "pg_csr_wait_error_offset", "csr_wait_error", "pg_csr_check", "pg_csr_test_wait_hook",
    "pg_checked_build", "pg_check_read", "pg_check_test_out_shift", "CheckReport",
    "empty_device", "set_fail_alloc_at", "BatchPlan", "gen_batch", "pg_batch_workspace_size",
    "gen_batch_csr", "pg_batch_csr_workspace_size", "pg_batch_csr_wait_error_offset",
]

PG_OK, PG_EINVAL, PG_ENOSPC, PG_ECUDA, PG_ETIMEOUT, PG_ENOMEM = range(6)
PG_ID32, PG_ID64 = 0, 1
PG_KRON_STOCHASTIC, PG_KRON_DETERMINISTIC = 0, 1
PG_BFS_UNDIRECTED = 1

_HERE = os.path.dirname(os.path.abspath(__file__))
# PGEN_LIBRARY=checked loads the bounds-checked build (same entry points);
# anything else, or unset, the default build
_LIB_NAMES = {"default": "libpgen.so", "checked": "libpgen_checked.so"}
_LIB_VARIANT = os.environ.get("PGEN_LIBRARY", "default")
if _LIB_VARIANT not in _LIB_NAMES:
    raise RuntimeError(f"PGEN_LIBRARY={_LIB_VARIANT!r}: expected one of {sorted(_LIB_NAMES)}")
_LIB_PATH = os.path.join(_HERE, _LIB_NAMES[_LIB_VARIANT])
_lock = threading.Lock()
_lib = None

u32, u64, i32, dbl, vp = C.c_uint32, C.c_uint64, C.c_int, C.c_double, C.c_void_p
sz = C.c_size_t


class PgenError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn}: {pg_status_string(status)} (status {status})")
        self.status = status


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Load libpgen.so (built by ``paper_1003_3684_gb300.build``); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(
                    f"{_LIB_PATH} is missing: build it with "
                    "`python -m paper_1003_3684_gb300.build` (nvcc, sm_103a). "
                    "pgen has no CPU fallback.")
            L = C.CDLL(_LIB_PATH)
            L.pg_status_string.argtypes = [i32]
            L.pg_status_string.restype = C.c_char_p
            L.pg_device_sm_count.argtypes = []
            L.pg_device_sm_count.restype = i32
            L.pg_version.argtypes = []
            L.pg_version.restype = C.c_char_p
            L.pg_pba_edge_count.argtypes = [u64, u32, u32, u32]
            L.pg_pba_edge_count.restype = u64
            L.pg_pba_workspace_size.argtypes = [u64, u32, u32]
            L.pg_pba_workspace_size.restype = sz
            L.gen_pba.argtypes = [u64, u32, u32, u32, u32, dbl, u64, i32, vp, u64,
                                  C.POINTER(u64), vp, sz, vp]
            L.gen_pba.restype = i32
            L.pg_kron_edge_count.argtypes = [vp, u32, u32, u64, i32]
            L.pg_kron_edge_count.restype = u64
            L.gen_kronecker.argtypes = [vp, u32, u32, u64, u64, i32, i32, vp, u64,
                                        C.POINTER(u64), vp]
            L.gen_kronecker.restype = i32
            L.pg_csr_workspace_size.argtypes = [u64, u64]
            L.pg_csr_workspace_size.restype = sz
            L.edges_to_csr.argtypes = [vp, u64, u64, i32, vp, vp, vp, sz, vp]
            L.edges_to_csr.restype = i32
            L.pg_trace_enable.argtypes = [i32]
            L.pg_trace_enable.restype = None
            L.pg_trace_dump.argtypes = [C.c_char_p, sz]
            L.pg_trace_dump.restype = sz
            L.pg_launch_count.argtypes = []
            L.pg_launch_count.restype = u64
            _lib = L
    return _lib


def _check(fn: str, st: int):
    if st != PG_OK:
        raise PgenError(fn, st)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return vp(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t):
    return vp(t.data_ptr()) if t is not None and t.numel() > 0 else vp(None)


# Allocation-failure injection (a testing aid, not part of the method). The
# library itself allocates no device memory: every buffer it writes is made
# here, by empty_device. With PGEN_FAIL_ALLOC_AT=k in the environment, or
# after set_fail_alloc_at(k), the k-th of those allocations from then on
# (k >= 1) raises torch.cuda.OutOfMemoryError instead, as an exhausted device
# would, once; 0 turns the injection off.
_alloc_lock = threading.Lock()
try:
    _fail_at = [int(os.environ.get("PGEN_FAIL_ALLOC_AT", "0") or 0), 0]   # [k, counted]
except ValueError:
    raise RuntimeError("PGEN_FAIL_ALLOC_AT must be an integer") from None


def set_fail_alloc_at(k: int) -> None:
    """Make the k-th device allocation of the binding from now on fail (0: never)."""
    with _alloc_lock:
        _fail_at[0], _fail_at[1] = int(k), 0


def empty_device(shape, dtype, device):
    """An uninitialised buffer for the library to write: every device buffer
    the binding (and the serving loop) allocates comes from here."""
    import torch
    with _alloc_lock:
        if _fail_at[0] > 0:
            _fail_at[1] += 1
            if _fail_at[1] == _fail_at[0]:
                _fail_at[0] = 0
                raise torch.cuda.OutOfMemoryError(
                    f"injected allocation failure (shape {shape}, {dtype})")
    return torch.empty(shape, dtype=dtype, device=device)


_empty = empty_device


# --------------------------------------------------------------------------
def pg_status_string(status: int) -> str:
    try:
        return lib().pg_status_string(status).decode()
    except RuntimeError:
        return f"status {status}"


def pg_device_sm_count() -> int:
    return int(lib().pg_device_sm_count())


def pg_version() -> str:
    return lib().pg_version().decode()


def pg_force_wide_path(on: bool) -> None:
    """Test hook: the PBA kernels take their 64-bit-index variants for every
    input (the output is the same), so that parity tests reach them."""
    L = lib()
    L.pg_force_wide_path.argtypes = [C.c_int]
    L.pg_force_wide_path.restype = None
    L.pg_force_wide_path(1 if on else 0)


def pg_pba_edge_count(n: int, m: int, blocks: int, n0: int) -> int:
    return int(lib().pg_pba_edge_count(n, m, blocks, n0))


def pg_pba_workspace_size(n: int, m: int, blocks: int) -> int:
    return int(lib().pg_pba_workspace_size(n, m, blocks))


def gen_pba(n: int, m: int, blocks: int = 1, n0: int | None = None, faction_width: int = 1,
            inter_frac: float = 0.1, seed: int = 0, id64: bool = False, out=None,
            workspace=None, stream=None, device="cuda"):
    """Two-phase PBA graph (Sec. 3, PBA method); returns an (E, 2) edge tensor.

    ``n0`` defaults to m + 1. ``out`` (optional) is a preallocated 16-byte
    aligned int32/int64 tensor with at least E rows; ``workspace`` a uint8
    device tensor of at least ``pg_pba_workspace_size`` bytes (allocated here
    when omitted and blocks > 1).
    """
    import torch
    n0 = m + 1 if n0 is None else n0
    E = pg_pba_edge_count(n, m, blocks, n0)
    dtype = torch.int64 if id64 else torch.int32
    if out is None:
        out = _empty((max(E, 1), 2), dtype, device)
    if blocks > 1 and workspace is None:
        workspace = _empty(max(pg_pba_workspace_size(n, m, blocks), 1), torch.uint8,
                           out.device)
    ws_bytes = workspace.numel() if workspace is not None else 0
    n_out = u64(0)
    st = lib().gen_pba(n, m, blocks, n0, faction_width, float(inter_frac), seed,
                       PG_ID64 if id64 else PG_ID32, _ptr(out), out.shape[0], C.byref(n_out),
                       _ptr(workspace), ws_bytes, _stream(stream))
    _check("gen_pba", st)
    return out[:n_out.value]


def pba_faction_table(lists) -> np.ndarray:
    """Packs per-block faction lists (lists[p]: block p's list) into the
    device table of gen_pba_factions (host work only). Returns a uint8 array."""
    L = lib()
    if not getattr(L, "_fac_ready", False):
        L.pg_pba_faction_table_size.argtypes = [u32]
        L.pg_pba_faction_table_size.restype = sz
        L.pg_pba_faction_table.argtypes = [u32, vp, vp, vp, sz]
        L.pg_pba_faction_table.restype = i32
        L.gen_pba_factions.argtypes = [u64, u32, u32, u32, vp, dbl, u64, i32, vp, u64,
                                       C.POINTER(u64), vp, sz, vp]
        L.gen_pba_factions.restype = i32
        L._fac_ready = True
    B = len(lists)
    offs = np.zeros(B + 1, np.uint32)
    offs[1:] = np.cumsum([len(x) for x in lists])
    members = np.ascontiguousarray(np.concatenate([np.asarray(x, np.uint32) for x in lists])
                                   if B else np.zeros(1, np.uint32), dtype=np.uint32)
    size = L.pg_pba_faction_table_size(B)
    table = np.zeros(max(size, 16), np.uint8)
    _check("pg_pba_faction_table",
           L.pg_pba_faction_table(B, offs.ctypes.data, members.ctypes.data, table.ctypes.data, size))
    return table


def gen_pba_factions(n: int, m: int, factions, n0: int | None = None, inter_frac: float = 0.1,
                     seed: int = 0, id64: bool = False, out=None, workspace=None, stream=None,
                     device="cuda", table=None):
    """Two-phase PBA with general faction lists: ``factions[p]`` lists the
    members of every faction block p belongs to (blocks = len(factions)).
    ``table``: the device copy of pba_faction_table(factions), when the
    caller keeps one across calls (built and copied here otherwise)."""
    import torch
    blocks = len(factions)
    n0 = m + 1 if n0 is None else n0
    if table is None:
        table = torch.from_numpy(pba_faction_table(factions)).to(device)
    E = pg_pba_edge_count(n, m, blocks, n0)
    dtype = torch.int64 if id64 else torch.int32
    if out is None:
        out = _empty((max(E, 1), 2), dtype, device)
    if blocks > 1 and workspace is None:
        workspace = _empty(max(pg_pba_workspace_size(n, m, blocks), 1), torch.uint8, out.device)
    ws_bytes = workspace.numel() if workspace is not None else 0
    n_out = u64(0)
    st = lib().gen_pba_factions(n, m, blocks, n0, _ptr(table), float(inter_frac), seed,
                                PG_ID64 if id64 else PG_ID32, _ptr(out), out.shape[0],
                                C.byref(n_out), _ptr(workspace), ws_bytes, _stream(stream))
    _check("gen_pba_factions", st)
    return out[:n_out.value]


def gen_pba_to_host(host_out, n: int, m: int, blocks: int = 1, n0: int | None = None,
                    faction_width: int = 1, inter_frac: float = 0.1, seed: int = 0,
                    id64: bool = False, out=None, workspace=None, stream=None, device="cuda"):
    """gen_pba plus a copy of the edges into ``host_out`` (a pinned CPU tensor
    of the same shape and dtype), overlapped with generation. Synchronise the
    stream before reading ``host_out``. Returns the device edge tensor."""
    import torch
    L = lib()
    if not getattr(L, "_to_host_ready", False):
        L.gen_pba_to_host.argtypes = [u64, u32, u32, u32, u32, dbl, u64, i32, vp, vp, u64,
                                      C.POINTER(u64), vp, sz, vp]
        L.gen_pba_to_host.restype = i32
        L._to_host_ready = True
    n0 = m + 1 if n0 is None else n0
    E = pg_pba_edge_count(n, m, blocks, n0)
    dtype = torch.int64 if id64 else torch.int32
    if out is None:
        out = _empty((max(E, 1), 2), dtype, device)
    if host_out.dtype != out.dtype or host_out.shape[0] < E or not host_out.is_pinned():
        raise ValueError("host_out must be a pinned tensor of the output's dtype with E rows")
    if blocks > 1 and workspace is None:
        workspace = _empty(max(pg_pba_workspace_size(n, m, blocks), 1), torch.uint8, out.device)
    ws_bytes = workspace.numel() if workspace is not None else 0
    n_out = u64(0)
    st = L.gen_pba_to_host(n, m, blocks, n0, faction_width, float(inter_frac), seed,
                           PG_ID64 if id64 else PG_ID32, vp(host_out.data_ptr()), _ptr(out),
                           out.shape[0], C.byref(n_out), _ptr(workspace), ws_bytes,
                           _stream(stream))
    _check("gen_pba_to_host", st)
    return out[:n_out.value]


def _initiator(initiator):
    import numpy as np
    P = np.ascontiguousarray(np.asarray(initiator, dtype=np.float64))
    if P.ndim != 2 or P.shape[0] != P.shape[1]:
        raise ValueError("initiator must be a square matrix")
    return P


def pg_kron_edge_count(initiator, k: int, n_edges: int, deterministic: bool = False) -> int:
    P = _initiator(initiator)
    return int(lib().pg_kron_edge_count(P.ctypes.data_as(vp), P.shape[0], k, n_edges,
                                        PG_KRON_DETERMINISTIC if deterministic
                                        else PG_KRON_STOCHASTIC))


def gen_kronecker(initiator, k: int, n_edges: int = 0, seed: int = 0, deterministic: bool = False,
                  id64: bool = False, out=None, stream=None, device="cuda"):
    """Kronecker graph (Sec. 3, PK method); returns an (E, 2) edge tensor."""
    import torch
    P = _initiator(initiator)
    E = pg_kron_edge_count(P, k, n_edges, deterministic)
    dtype = torch.int64 if id64 else torch.int32
    if out is None:
        out = _empty((max(E, 1), 2), dtype, device)
    n_out = u64(0)
    st = lib().gen_kronecker(P.ctypes.data_as(vp), P.shape[0], k, n_edges, seed,
                             PG_KRON_DETERMINISTIC if deterministic else PG_KRON_STOCHASTIC,
                             PG_ID64 if id64 else PG_ID32, _ptr(out), out.shape[0],
                             C.byref(n_out), _stream(stream))
    _check("gen_kronecker", st)
    return out[:n_out.value]


def _range_lib():
    L = lib()
    if not getattr(L, "_range_ready", False):
        L.gen_kronecker_range.argtypes = [vp, u32, u32, u64, u64, i32, i32, u64, u64, vp, u64, vp]
        L.gen_kronecker_range.restype = i32
        L.pg_pba_prepare.argtypes = [u64, u32, u32, u32, u32, vp, dbl, u64, vp, sz, vp]
        L.pg_pba_prepare.restype = i32
        L.gen_pba_blocks.argtypes = [u64, u32, u32, u32, u64, i32, u32, u32, vp, u64,
                                     C.POINTER(u64), vp, sz, vp]
        L.gen_pba_blocks.restype = i32
        L._range_ready = True
    return L


def gen_kronecker_range(initiator, k: int, n_edges: int, e_begin: int, e_end: int, seed: int = 0,
                        deterministic: bool = False, id64: bool = False, out=None, stream=None,
                        device="cuda"):
    """Edges [e_begin, e_end) of gen_kronecker's graph, as an (e_end - e_begin, 2) tensor."""
    import torch
    P = _initiator(initiator)
    count = e_end - e_begin
    dtype = torch.int64 if id64 else torch.int32
    if out is None:
        out = _empty((max(count, 1), 2), dtype, device)
    st = _range_lib().gen_kronecker_range(
        P.ctypes.data_as(vp), P.shape[0], k, n_edges, seed,
        PG_KRON_DETERMINISTIC if deterministic else PG_KRON_STOCHASTIC,
        PG_ID64 if id64 else PG_ID32, e_begin, e_end, _ptr(out), out.shape[0], _stream(stream))
    _check("gen_kronecker_range", st)
    return out[:max(count, 0)]


def pg_pba_prepare(n: int, m: int, blocks: int, n0: int | None = None, faction_width: int = 1,
                   inter_frac: float = 0.1, seed: int = 0, factions=None, workspace=None,
                   stream=None, device="cuda"):
    """Phase 1 and the count scan of PBA into a workspace tensor (returned);
    gen_pba_blocks then emits any block range from it. ``factions`` (lists
    per block) replaces faction_width when given."""
    import torch
    n0 = m + 1 if n0 is None else n0
    if workspace is None:
        workspace = _empty(max(pg_pba_workspace_size(n, m, blocks), 1), torch.uint8, device)
    table = None
    if factions is not None:
        table = torch.from_numpy(pba_faction_table(factions)).to(workspace.device)
    st = _range_lib().pg_pba_prepare(n, m, blocks, n0, faction_width, _ptr(table),
                                     float(inter_frac), seed, _ptr(workspace), workspace.numel(),
                                     _stream(stream))
    _check("pg_pba_prepare", st)
    return workspace


def gen_pba_blocks(workspace, n: int, m: int, blocks: int, b_begin: int, b_end: int,
                   n0: int | None = None, seed: int = 0, id64: bool = False, out=None,
                   stream=None):
    """Edges of blocks [b_begin, b_end) from a prepared workspace."""
    import torch
    n0 = m + 1 if n0 is None else n0
    per = pg_pba_edge_count(n, m, blocks, n0) // max(blocks, 1)
    count = (b_end - b_begin) * per
    dtype = torch.int64 if id64 else torch.int32
    if out is None:
        out = _empty((max(count, 1), 2), dtype, workspace.device)
    n_out = u64(0)
    st = _range_lib().gen_pba_blocks(n, m, blocks, n0, seed, PG_ID64 if id64 else PG_ID32,
                                     b_begin, b_end, _ptr(out), out.shape[0], C.byref(n_out),
                                     _ptr(workspace), workspace.numel(), _stream(stream))
    _check("gen_pba_blocks", st)
    return out[:n_out.value]


def philox_rate(calls_per_thread: int = 2048, reps: int = 3, device="cuda") -> float:
    """Measured Philox4x32-10 calls per second of the device (best of reps,
    CUDA events on the current stream), from the library's probe kernel."""
    import torch
    L = lib()
    if not getattr(L, "_probe_ready", False):
        L.pg_philox_probe_threads.restype = sz
        L.pg_philox_probe.argtypes = [u32, vp, sz, vp]
        L.pg_philox_probe.restype = i32
        L._probe_ready = True
    n = int(L.pg_philox_probe_threads())
    out = torch.empty(n, dtype=torch.int32, device=device)
    stream = torch.cuda.current_stream(out.device)
    best = None
    for i in range(reps + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _check("pg_philox_probe", L.pg_philox_probe(calls_per_thread, _ptr(out), n,
                                                    vp(stream.cuda_stream)))
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        if i > 0 and (best is None or ms < best):      # the first launch is a warm-up
            best = ms
    return n * calls_per_thread / (best / 1000.0)


DEG_OUT, DEG_IN, DEG_TOTAL = 0, 1, 2


def _analysis_lib():
    L = lib()
    if not getattr(L, "_analysis_ready", False):
        L.pg_degrees.argtypes = [vp, u64, u64, i32, C.c_int, vp, vp]
        L.pg_degrees.restype = i32
        L.pg_degree_histogram.argtypes = [vp, u64, u32, vp, vp]
        L.pg_degree_histogram.restype = i32
        L.pg_bfs_workspace_size.argtypes = [u64]
        L.pg_bfs_workspace_size.restype = sz
        L.pg_bfs.argtypes = [vp, vp, u64, i32, u64, u32, vp, vp, sz, C.POINTER(u32),
                             C.POINTER(u64), vp]
        L.pg_bfs.restype = i32
        L._analysis_ready = True
    return L


def degrees(edges, n_vertices: int, which: int = DEG_TOTAL, out=None, stream=None):
    """Vertex degrees of an (E, 2) edge tensor as int64[n_vertices] (counts)."""
    import torch
    if out is None:
        out = _empty(max(n_vertices, 1), torch.int64, edges.device)
    st = _analysis_lib().pg_degrees(_ptr(edges), edges.shape[0], n_vertices,
                                    PG_ID64 if edges.dtype == torch.int64 else PG_ID32, which,
                                    _ptr(out), _stream(stream))
    _check("pg_degrees", st)
    return out[:n_vertices]


def degree_histogram(deg, max_degree: int, out=None, stream=None):
    """int64[max_degree + 2]: vertices per degree, the last bucket all larger."""
    import torch
    if out is None:
        out = _empty(max_degree + 2, torch.int64, deg.device)
    st = _analysis_lib().pg_degree_histogram(_ptr(deg), deg.numel(), max_degree, _ptr(out),
                                             _stream(stream))
    _check("pg_degree_histogram", st)
    return out


def bfs(row_ptr, col, source: int, dist=None, workspace=None, stream=None,
        undirected: bool = False):
    """BFS hop distances from source (int32 view of uint32; -1 = unreached).

    Returns (dist, levels, scanned). Waits for the stream once per level.
    undirected=True declares the CSR symmetric, so that wide levels may run
    bottom-up (same results)."""
    import torch
    L = _analysis_lib()
    N = row_ptr.numel() - 1
    if dist is None:
        dist = _empty(max(N, 1), torch.int32, row_ptr.device)
    if workspace is None:
        workspace = _empty(L.pg_bfs_workspace_size(N), torch.uint8, row_ptr.device)
    levels, scanned = u32(0), u64(0)
    st = L.pg_bfs(_ptr(row_ptr), _ptr(col), N, PG_ID64 if col.dtype == torch.int64 else PG_ID32,
                  source, PG_BFS_UNDIRECTED if undirected else 0, _ptr(dist), _ptr(workspace),
                  workspace.numel(), C.byref(levels), C.byref(scanned), _stream(stream))
    _check("pg_bfs", st)
    return dist[:N], int(levels.value), int(scanned.value)


def powerlaw_exponent(hist, d_min: int) -> float:
    """Discrete power-law exponent of a degree histogram over degrees >= d_min
    (Clauset, Shalizi & Newman 2009, the approximate discrete MLE
    1 + n / sum(ln(d / (d_min - 1/2)))). Host arithmetic on the counts;
    the overflow bucket of degree_histogram is left out."""
    h = np.asarray(hist, dtype=np.float64)[:-1]
    d = np.arange(h.size, dtype=np.float64)
    sel = d >= d_min
    n = h[sel].sum()
    if n == 0:
        raise ValueError("no vertex of degree >= d_min")
    return 1.0 + n / float((h[sel] * np.log(d[sel] / (d_min - 0.5))).sum())


def path_length_stats(dist) -> dict:
    """Mean and largest hop distance over the vertices a BFS reached (source excluded)."""
    d = np.asarray(dist).view(np.uint32).astype(np.int64)
    reached = d[(d != 0xFFFFFFFF) & (d > 0)]
    return dict(reached=int(reached.size) + 1,
                mean=float(reached.mean()) if reached.size else 0.0,
                max=int(reached.max()) if reached.size else 0)


def int_pipe_rates(iters: int = 1024, device="cuda") -> dict:
    """Measured operations per second of the device for a 32x32->64 multiply,
    a 32-bit multiply-add, a three-input logic operation and a three-input add (the
    operations of Philox and the index arithmetic), from the library's probe."""
    import torch
    L = lib()
    if not getattr(L, "_intprobe_ready", False):
        L.pg_philox_probe_threads.restype = sz
        L.pg_int_probe.argtypes = [C.c_int, u32, vp, sz, vp]
        L.pg_int_probe.restype = i32
        L._intprobe_ready = True
    n = int(L.pg_philox_probe_threads())
    out = torch.empty(n, dtype=torch.int32, device=device)
    stream = torch.cuda.current_stream(out.device)
    rates = {}
    for op, name in enumerate(("mul_wide", "mad32", "lop3", "add3")):
        best = None
        for i in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _check("pg_int_probe", L.pg_int_probe(op, iters, _ptr(out), n, vp(stream.cuda_stream)))
            b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b)
            if i > 0 and (best is None or ms < best):
                best = ms
        rates[name] = n * 8 * iters / (best / 1000.0)
    return rates


def pg_csr_workspace_size(n_edges: int, n_vertices: int) -> int:
    return int(lib().pg_csr_workspace_size(n_edges, n_vertices))


def edges_to_csr(edges, n_vertices: int, row_ptr=None, col=None, workspace=None, stream=None,
                 check: bool = False):
    """CSR of an (E, 2) edge tensor: (row_ptr int64[N+1], col[E]) with rows sorted.

    check=True waits for the stream and raises PgenError(PG_ETIMEOUT) when a
    bounded wait of the sort gave up (pg_csr_check)."""
    import torch
    id64 = edges.dtype == torch.int64
    E = edges.shape[0]
    if row_ptr is None:
        row_ptr = _empty(n_vertices + 1, torch.int64, edges.device)
    if col is None:
        col = _empty(max(E, 1), edges.dtype, edges.device)
    if workspace is None:
        workspace = _empty(max(pg_csr_workspace_size(E, n_vertices), 1), torch.uint8,
                           edges.device)
    st = lib().edges_to_csr(_ptr(edges), E, n_vertices, PG_ID64 if id64 else PG_ID32,
                            _ptr(row_ptr), _ptr(col), _ptr(workspace), workspace.numel(),
                            _stream(stream))
    _check("edges_to_csr", st)
    if check:
        pg_csr_check(workspace, E, n_vertices, id64=id64, stream=stream)
    return row_ptr, col[:E]


def pg_csr_check(workspace, n_edges: int, n_vertices: int, id64: bool = False, flags: int = 0,
                 stream=None) -> None:
    """Wait for `stream`, then raise PgenError(PG_ETIMEOUT) if the CSR call
    with these arguments that used `workspace` had a bounded wait give up."""
    L = lib()
    if not getattr(L, "_check_ready", False):
        L.pg_csr_check.argtypes = [vp, u64, u64, i32, u32, vp]
        L.pg_csr_check.restype = i32
        L.pg_csr_test_wait_hook.argtypes = [u32, u32]
        L.pg_csr_test_wait_hook.restype = None
        L._check_ready = True
    _check("pg_csr_check", L.pg_csr_check(_ptr(workspace), n_edges, n_vertices,
                                          PG_ID64 if id64 else PG_ID32, flags, _stream(stream)))


def pg_csr_test_wait_hook(spin_limit: int = 0, withhold_tile: int = 0xFFFFFFFF) -> None:
    """Test hook: sort waits give up after spin_limit polls (0: the default)
    and tile withhold_tile of every digit pass never publishes its counts."""
    L = lib()
    L.pg_csr_test_wait_hook.argtypes = [u32, u32]
    L.pg_csr_test_wait_hook.restype = None
    L.pg_csr_test_wait_hook(spin_limit, withhold_tile)


class CheckReport(NamedTuple):
    """What the checked build's bounds comparisons found (pg_check_read)."""
    count: int    # failed comparisons
    unit: int     # source file of the first one: 1 Kronecker, 2 PBA, 3 CSR, 4 batch, 5 checks
    line: int     # its source line
    index: int    # the compared index and bound
    bound: int


def _check_lib():
    L = lib()
    if not getattr(L, "_bounds_ready", False):
        L.pg_checked_build.argtypes = []
        L.pg_checked_build.restype = i32
        L.pg_check_read.argtypes = [i32, C.POINTER(u32), C.POINTER(u32), C.POINTER(u32),
                                    C.POINTER(u64), C.POINTER(u64), vp]
        L.pg_check_read.restype = i32
        L.pg_check_test_out_shift.argtypes = [u32, vp]
        L.pg_check_test_out_shift.restype = i32
        L._bounds_ready = True
    return L


def pg_checked_build() -> bool:
    """True when the loaded library is the bounds-checked build."""
    return bool(_check_lib().pg_checked_build())


def pg_check_read(reset: bool = True, stream=None) -> CheckReport:
    """Wait for `stream` and return the failed bounds comparisons since the
    last reset (always count 0 in the default build); reset zeroes them."""
    L = _check_lib()
    c, u, ln = u32(), u32(), u32()
    ix, bd = u64(), u64()
    _check("pg_check_read", L.pg_check_read(1 if reset else 0, C.byref(c), C.byref(u),
                                            C.byref(ln), C.byref(ix), C.byref(bd),
                                            _stream(stream)))
    return CheckReport(c.value, u.value, ln.value, ix.value, bd.value)


def pg_check_test_out_shift(shift: int, stream=None) -> None:
    """Test hook of the checked build: result stores are compared with
    bound >> shift (0 restores the real bounds)."""
    _check("pg_check_test_out_shift",
           _check_lib().pg_check_test_out_shift(shift, _stream(stream)))


CSR_SYMMETRIZE, CSR_DEDUP, CSR_NO_LOOPS, CSR_ODD = 1, 2, 4, 8


def _opts_lib():
    L = lib()
    if not getattr(L, "_opts_ready", False):
        L.pg_csr_opts_workspace_size.argtypes = [u64, u64, u32]
        L.pg_csr_opts_workspace_size.restype = sz
        L.edges_to_csr_opts.argtypes = [vp, u64, u64, i32, u32, vp, vp, u64, vp, sz, vp]
        L.edges_to_csr_opts.restype = i32
        L.pg_csr_wait_error_offset.argtypes = [u64, u64, i32, u32]
        L.pg_csr_wait_error_offset.restype = sz
        L.gen_random_cells.argtypes = [u64, u64, u64, i32, vp, u64, vp]
        L.gen_random_cells.restype = i32
        L._opts_ready = True
    return L


def edges_to_csr_opts(edges, n_vertices: int, flags: int, row_ptr=None, col=None, workspace=None,
                      stream=None):
    """CSR with options (CSR_SYMMETRIZE | CSR_DEDUP | CSR_NO_LOOPS | CSR_ODD).

    Returns (row_ptr, col) with col holding capacity for the whole list; the
    entries in use are col[:row_ptr[-1]] (known once the stream's work ends).
    """
    import torch
    L = _opts_lib()
    id64 = edges.dtype == torch.int64
    E = edges.shape[0]
    listed = 2 * E if flags & CSR_SYMMETRIZE else E
    if row_ptr is None:
        row_ptr = _empty(n_vertices + 1, torch.int64, edges.device)
    if col is None:
        col = _empty(max(listed, 1), edges.dtype, edges.device)
    if workspace is None:
        workspace = _empty(max(L.pg_csr_opts_workspace_size(E, n_vertices, flags), 1),
                           torch.uint8, edges.device)
    st = L.edges_to_csr_opts(_ptr(edges), E, n_vertices, PG_ID64 if id64 else PG_ID32, flags,
                             _ptr(row_ptr), _ptr(col), col.numel(), _ptr(workspace),
                             workspace.numel(), _stream(stream))
    _check("edges_to_csr_opts", st)
    return row_ptr, col


def pg_csr_wait_error_offset(n_edges: int, n_vertices: int, id64: bool = False,
                             flags: int = 0):
    """Byte offset, in the workspace of a CSR call with these arguments, of
    the word its sort's bounded waits set when they give up; None when the
    call sorts nothing (no word is written) or the arguments are invalid."""
    off = int(_opts_lib().pg_csr_wait_error_offset(n_edges, n_vertices,
                                                   PG_ID64 if id64 else PG_ID32, flags))
    return None if off == C.c_size_t(-1).value else off


def csr_wait_error(workspace, n_edges: int, n_vertices: int, id64: bool = False,
                   flags: int = 0) -> int:
    """The sort's wait word after a CSR call that used `workspace` (a uint8
    tensor), read once the stream has finished the call: 0 when every wait
    ended normally, nonzero when one gave up (the CSR is then unspecified)."""
    off = pg_csr_wait_error_offset(n_edges, n_vertices, id64, flags)
    if off is None:
        return 0
    word = workspace[off:off + 4].cpu().numpy().tobytes()
    return int.from_bytes(word, "little")


def gen_random_cells(n_vertices: int, n_edges: int, seed: int = 0, id64: bool = False, out=None,
                     stream=None, device="cuda"):
    """Random graph G(N, M) with replacement (the XOR partner of a PK graph)."""
    import torch
    dtype = torch.int64 if id64 else torch.int32
    if out is None:
        out = _empty((max(n_edges, 1), 2), dtype, device)
    st = _opts_lib().gen_random_cells(n_vertices, n_edges, seed, PG_ID64 if id64 else PG_ID32,
                                      _ptr(out), out.shape[0], _stream(stream))
    _check("gen_random_cells", st)
    return out[:n_edges]


def kronecker_xor_random(initiator, k: int, n_random: int, n_edges: int = 0, seed: int = 0,
                         deterministic: bool = True, id64: bool = False, stream=None,
                         device="cuda"):
    """PK graph randomised by exclusive-or with a random graph (Sec. 3, PK
    method): the Kronecker list and G(N, n_random) in one buffer, then CSR
    keeping the cells of odd multiplicity. Returns (row_ptr, col) as
    edges_to_csr_opts does."""
    import torch
    P = _initiator(initiator)
    M1 = pg_kron_edge_count(P, k, n_edges, deterministic)
    N = P.shape[0] ** k
    dtype = torch.int64 if id64 else torch.int32
    buf = _empty((max(M1 + n_random, 1), 2), dtype, device)
    # the order of the two lists does not matter to the exclusive-or; the
    # second list must start on a 16-byte boundary (an even edge index for
    # 32-bit ids), so the list with an even length goes first
    kron_first = id64 or M1 % 2 == 0
    if not kron_first and n_random % 2:
        raise ValueError("kronecker_xor_random: both lists have odd lengths with 32-bit ids")
    a, b = (0, M1) if kron_first else (n_random, 0)
    gen_kronecker(P, k, n_edges, seed, deterministic=deterministic, id64=id64,
                  out=buf[a:a + max(M1, 1)], stream=stream)
    if n_random > 0:
        gen_random_cells(N, n_random, seed, id64=id64, out=buf[b:b + n_random], stream=stream)
    return edges_to_csr_opts(buf[:M1 + n_random], N, CSR_ODD, stream=stream)


def pg_trace_enable(on: bool = True) -> None:
    """Bracket every library kernel launch with CUDA events (see pgen.h)."""
    lib().pg_trace_enable(1 if on else 0)


def pg_launch_count() -> int:
    """Kernels the library has launched in this process (see pgen.h)."""
    return int(lib().pg_launch_count())


def pg_trace_dump() -> dict:
    """Per-kernel {name: (launches, total_ms)} since the last dump; clears it."""
    import json
    need = lib().pg_trace_dump(None, 0)
    buf = C.create_string_buffer(need + 64)
    lib().pg_trace_dump(buf, len(buf))
    return {k: (int(v[0]), float(v[1])) for k, v in json.loads(buf.value.decode()).items()}


# --------------------------------------------------------------------------
# Batched generation (one persistent launch for many graphs)
# --------------------------------------------------------------------------
PG_JOB_BA, PG_JOB_KRON = 0, 1


class _PgJob(C.Structure):
    _fields_ = [("kind", u32), ("m", u32), ("n0", u32), ("k", u32), ("n", u64), ("seed", u64),
                ("initiator", vp), ("blocks", u32), ("faction_width", u32), ("inter_frac", dbl),
                ("want_csr", u32), ("reserved", u32)]


def _batch_lib():
    L = lib()
    if not getattr(L, "_batch_ready", False):
        L.pg_batch_plan_size.argtypes = [vp, u32]
        L.pg_batch_plan_size.restype = sz
        L.pg_batch_workspace_size.argtypes = [vp]
        L.pg_batch_workspace_size.restype = sz
        L.pg_batch_plan.argtypes = [vp, u32, u32, i32, vp, sz, vp, vp]
        L.pg_batch_plan.restype = i32
        L.gen_batch.argtypes = [vp, vp, u32, i32, vp, u64, u64, u32, vp, sz, vp]
        L.gen_batch.restype = i32
        L.pg_batch_csr_layout.argtypes = [vp, u32, vp, vp, C.POINTER(u64), C.POINTER(u64)]
        L.pg_batch_csr_layout.restype = i32
        L.pg_batch_csr_workspace_size.argtypes = [vp]
        L.pg_batch_csr_workspace_size.restype = sz
        L.pg_batch_csr_wait_error_offset.argtypes = [vp]
        L.pg_batch_csr_wait_error_offset.restype = sz
        L.gen_batch_csr.argtypes = [vp, vp, u32, i32, vp, vp, u64, vp, u64, vp, sz, vp]
        L.gen_batch_csr.restype = i32
        L._batch_ready = True
    return L


def _job_struct(j, keep):
    """One pg_job from a job dict (see BatchPlan)."""
    want = 1 if j.get("want_csr") else 0
    if j["kind"] == "pba":
        blocks = int(j.get("blocks", 1) or 1)
        return _PgJob(PG_JOB_BA, j["m"], j.get("n0") or j["m"] + 1, 0, j["n"], j["seed"], None,
                      blocks, int(j.get("faction_width", 1) or 1), float(j.get("inter_frac", 0.0)),
                      want, 0)
    if j["kind"] == "kron":
        P = _initiator(j["initiator"])
        keep.append(P)
        return _PgJob(PG_JOB_KRON, 0, P.shape[0], j["k"], j["n_edges"], j["seed"],
                      P.ctypes.data_as(vp), 0, 0, 0.0, want, 0)
    raise ValueError(f"unknown job kind {j['kind']!r}")


class BatchPlan:
    """Host-built plan of a batch of jobs, copied to the device.

    ``jobs`` is a list of dicts: ``dict(kind="pba", n=..., m=..., n0=..., seed=...)``
    (BA: serial with the default blocks = 1, or two-phase PBA with
    ``blocks=B, inter_frac=f`` and optionally ``faction_width``), or
    ``dict(kind="kron", initiator=..., k=..., n_edges=..., seed=...)`` (stochastic
    Kronecker). ``want_csr=True`` on a job asks gen_batch_csr for its CSR.
    ``offsets[i]`` is job i's first edge in the arena, ``offsets[-1]`` the arena
    length, ``counts[i]`` its number of edges (with 32-bit ids one unused arena
    edge may precede a two-phase job). ``csr_rows[i]`` / ``csr_cols[i]`` are where
    gen_batch_csr puts job i's row_ptr and col entries (-1: no CSR).
    """

    def __init__(self, jobs, tile_edges: int = 4096, id64: bool = False, device="cuda"):
        import numpy as np
        import torch
        L = _batch_lib()
        n = len(jobs)
        arr = (_PgJob * max(n, 1))()
        self._keep = []
        for i, j in enumerate(jobs):
            arr[i] = _job_struct(j, self._keep)
        size = int(L.pg_batch_plan_size(C.cast(arr, vp), n))
        host = np.zeros(max(size, 16), dtype=np.uint8)
        offsets = np.zeros(n + 1, dtype=np.uint64)
        n_items = u64(0)
        st = L.pg_batch_plan(C.cast(arr, vp), n, tile_edges, PG_ID64 if id64 else PG_ID32,
                             host.ctypes.data_as(vp), host.size, offsets.ctypes.data_as(vp),
                             C.byref(n_items))
        _check("pg_batch_plan", st)
        rows = np.zeros(max(n, 1), dtype=np.uint64)
        cols = np.zeros(max(n, 1), dtype=np.uint64)
        rt, ct = u64(0), u64(0)
        _check("pg_batch_csr_layout", L.pg_batch_csr_layout(
            host.ctypes.data_as(vp), n, rows.ctypes.data_as(vp), cols.ctypes.data_as(vp),
            C.byref(rt), C.byref(ct)))
        self.jobs = list(jobs)
        self.n_jobs = n
        self.tile_edges = tile_edges
        self.id64 = id64
        self.host = host
        self.offsets = offsets
        self.counts = [int(pg_pba_edge_count(j["n"], j["m"], int(j.get("blocks", 1) or 1),
                                             j.get("n0") or j["m"] + 1))
                       if j["kind"] == "pba" else int(j["n_edges"]) for j in jobs]
        self.total_edges = int(offsets[-1])
        self.n_items = int(n_items.value)
        none = np.uint64(0xFFFFFFFFFFFFFFFF)
        self.csr_rows = [int(r) if r != none else -1 for r in rows[:n]]
        self.csr_cols = [int(c) if c != none else -1 for c in cols[:n]]
        self.csr_rows_total = int(rt.value)
        self.csr_cols_total = int(ct.value)
        self.d_plan = torch.from_numpy(host).to(device)
        self.device = self.d_plan.device

    def edges_of(self, arena, i: int):
        """Job i's (count, 2) slice of a gen_batch arena."""
        a = int(self.offsets[i])
        return arena[a:a + self.counts[i]]

    def csr_of(self, row_ptr, col, i: int):
        """Job i's (row_ptr, col) views into gen_batch_csr's output."""
        if self.csr_rows[i] < 0:
            raise ValueError(f"job {i} has no CSR (want_csr not set)")
        r, c = self.csr_rows[i], self.csr_cols[i]
        nv = _job_vertices(self.jobs[i])
        return row_ptr[r:r + nv + 1], col[c:c + self.counts[i]]


def _job_vertices(j) -> int:
    """Vertex ids of a batch job's graph (0 .. count - 1)."""
    if j["kind"] == "pba":    # a seed clique per block, then the new vertices
        return int(j.get("blocks", 1) or 1) * (j.get("n0") or j["m"] + 1) + j["n"]
    return len(j["initiator"]) ** j["k"]


def pg_batch_workspace_size(plan: "BatchPlan | None" = None) -> int:
    """Workspace bytes of gen_batch for `plan` (None: a plan without
    two-phase jobs)."""
    return int(_batch_lib().pg_batch_workspace_size(
        plan.host.ctypes.data_as(vp) if plan is not None else None))


def gen_batch(plan: "BatchPlan", arena=None, workspace=None, grid_ctas: int = 0, stream=None):
    """Run a BatchPlan: one persistent launch for the serial-BA and Kronecker
    jobs, then the two-phase PBA jobs; returns the (total, 2) arena."""
    import torch
    L = _batch_lib()
    dtype = torch.int64 if plan.id64 else torch.int32
    if arena is None:
        arena = _empty((max(plan.total_edges, 1), 2), dtype, plan.device)
    if workspace is None:
        workspace = _empty(pg_batch_workspace_size(plan), torch.uint8, plan.device)
    st = L.gen_batch(plan.host.ctypes.data_as(vp), _ptr(plan.d_plan), plan.n_jobs,
                     PG_ID64 if plan.id64 else PG_ID32, _ptr(arena), arena.shape[0],
                     plan.total_edges, grid_ctas, _ptr(workspace), workspace.numel(),
                     _stream(stream))
    _check("gen_batch", st)
    return arena[:plan.total_edges]


def pg_batch_csr_workspace_size(plan: "BatchPlan") -> int:
    return int(_batch_lib().pg_batch_csr_workspace_size(plan.host.ctypes.data_as(vp)))


def pg_batch_csr_wait_error_offset(plan: "BatchPlan"):
    """Byte offset of gen_batch_csr's wait word in its workspace, or None."""
    off = int(_batch_lib().pg_batch_csr_wait_error_offset(plan.host.ctypes.data_as(vp)))
    return None if off == C.c_size_t(-1).value else off


def gen_batch_csr(plan: "BatchPlan", arena, row_ptr=None, col=None, workspace=None, stream=None,
                  check: bool = False):
    """CSR of every want_csr job of a gen_batch arena, from one sort of their
    union graph; returns (row_ptr, col) arenas (plan.csr_of gives a job's
    views). check=True waits and raises PG_ETIMEOUT if a bounded wait of the
    sort gave up."""
    import torch
    L = _batch_lib()
    dev = arena.device
    dtype = torch.int64 if plan.id64 else torch.int32
    if row_ptr is None:
        row_ptr = _empty(max(plan.csr_rows_total, 1), torch.int64, dev)
    if col is None:
        col = _empty(max(plan.csr_cols_total, 1), dtype, dev)
    if workspace is None:
        workspace = _empty(max(pg_batch_csr_workspace_size(plan), 256), torch.uint8, dev)
    st = L.gen_batch_csr(plan.host.ctypes.data_as(vp), _ptr(plan.d_plan), plan.n_jobs,
                         PG_ID64 if plan.id64 else PG_ID32, _ptr(arena), _ptr(row_ptr),
                         row_ptr.numel(), _ptr(col), col.numel(), _ptr(workspace),
                         workspace.numel(), _stream(stream))
    _check("gen_batch_csr", st)
    if check:
        off = pg_batch_csr_wait_error_offset(plan)
        if off is not None:
            if stream is not None:
                stream.synchronize()
            else:
                torch.cuda.current_stream(dev).synchronize()
            if int(workspace[off:off + 4].view(torch.int32).item()) != 0:
                raise PgenError("gen_batch_csr", PG_ETIMEOUT)
    return row_ptr, col

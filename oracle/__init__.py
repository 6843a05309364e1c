"""Oracle for arXiv 1003.3684 graph generation -- TEST INFRASTRUCTURE ONLY.

ctypes wrapper around ``liboracle.so`` (plain single-threaded C built from
``pgen_oracle.c``). Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(``paper_1003_3684_gb300``) never does, and this package imports nothing from
it. Every function below mirrors one C routine; see ``pgen_oracle.c`` for the
section of the paper each one follows and the readings it implements.

The ctypes calls release the GIL, so a caller may run independent blocks of
the oracle on several host threads; each call itself stays single-threaded.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pgen_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

u32, u64, dbl = C.c_uint32, C.c_uint64, C.c_double
P = C.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: no -march)."""
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "pgen_oracle.h")))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            L.or_philox4x32_10.argtypes = [P, P, P]
            L.or_philox4x32_10.restype = None
            L.or_uniform.argtypes = [u32, u32, u64]
            L.or_uniform.restype = u64
            L.or_coin_threshold.argtypes = [dbl]
            L.or_coin_threshold.restype = u64
            L.or_ba.argtypes = [u64, u32, u32, u64, u32, P]
            L.or_pba_count.argtypes = [P, u64, u32, P]
            L.or_pba_phase1_general.argtypes = [u32, u32, P, u32, u64, dbl, u64, P, P, P]
            L.or_pba_phase1.argtypes = [u32, u32, u32, u64, dbl, u64, P, P, P]
            L.or_pba_endpoints.argtypes = [u32, u64, u64, u32, u64, u64, P]
            L.or_pba_substitute.argtypes = [P, u64, u32, P, P, P]
            L.or_pba.argtypes = [u64, u32, u32, u32, u32, dbl, u64, P, P, P]
            L.or_pba_factions.argtypes = [u64, u32, u32, u32, P, P, dbl, u64, P, P, P]
            L.or_kron_thresholds.argtypes = [P, u32, P]
            L.or_kron_pick.argtypes = [P, u32, u32]
            L.or_kron_pick.restype = u32
            L.or_kron.argtypes = [P, u32, u32, u64, u64, P]
            L.or_kron_det.argtypes = [P, u32, u32, P, u64, P, P]
            L.or_csr.argtypes = [P, u64, u64, P, P]
            L.or_csr_opts.argtypes = [P, u64, u64, u32, P, P, P]
            L.or_random_cells.argtypes = [u64, u64, u64, P]
            L.or_degrees.argtypes = [P, u64, u64, C.c_int, P]
            L.or_degree_histogram.argtypes = [P, u64, u64, P]
            L.or_bfs.argtypes = [P, P, u64, u64, P, P, P]
            for name in ("or_ba", "or_pba_count", "or_pba_phase1_general", "or_pba_phase1", "or_pba_endpoints",
                         "or_pba_substitute", "or_pba", "or_pba_factions", "or_kron_thresholds", "or_kron",
                         "or_kron_det", "or_csr", "or_csr_opts", "or_random_cells", "or_degrees",
                         "or_degree_histogram", "or_bfs"):
                getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform(w0: int, w1: int, R: int) -> int:
    return int(lib().or_uniform(w0, w1, R))


def coin_threshold(f: float) -> int:
    return int(lib().or_coin_threshold(f))


def seed_edges(n0: int) -> int:
    return n0 * (n0 - 1) // 2


def ba(n: int, m: int, n0: int, seed: int, stream: int = 0) -> np.ndarray:
    """Serial BA edge list, shape (e0 + n*m, 2), uint64 (src, dst)."""
    out = np.zeros((seed_edges(n0) + n * m, 2), dtype=np.uint64)
    _check(lib().or_ba(n, m, n0, seed, stream, _ptr(out)), "ba")
    return out


def pba_count(A, B: int) -> np.ndarray:
    Aa = np.ascontiguousarray(A, dtype=np.uint32)
    cnt = np.zeros(B, dtype=np.uint64)
    _check(lib().or_pba_count(_ptr(Aa), len(Aa), B, _ptr(cnt)), "pba_count")
    return cnt


def pba_phase1(p: int, B: int, W: int, n_entries: int, f: float, seed: int):
    """Phase-1 urn A_p of one block; returns (A, counts[B], fresh_count)."""
    A = np.zeros(max(n_entries, 1), dtype=np.uint32)
    cnt = np.zeros(B, dtype=np.uint64)
    fresh = np.zeros(1, dtype=np.uint64)
    _check(lib().or_pba_phase1(p, B, W, n_entries, f, seed, _ptr(A), _ptr(cnt), _ptr(fresh)),
           "pba_phase1")
    return A[:n_entries], cnt, int(fresh[0])


def pba_phase1_general(p: int, B: int, flist, n_entries: int, f: float, seed: int):
    fl = np.ascontiguousarray(flist, dtype=np.uint32)
    A = np.zeros(max(n_entries, 1), dtype=np.uint32)
    cnt = np.zeros(B, dtype=np.uint64)
    fresh = np.zeros(1, dtype=np.uint64)
    _check(lib().or_pba_phase1_general(p, B, _ptr(fl), len(fl), n_entries, f, seed, _ptr(A),
                                       _ptr(cnt), _ptr(fresh)), "pba_phase1_general")
    return A[:n_entries], cnt, int(fresh[0])


def pba_endpoints(q: int, R_q: int, n_b: int, n0: int, seed: int, length: int | None = None):
    """First `length` (default R_q) local endpoints T_q of block q."""
    length = R_q if length is None else length
    T = np.zeros(max(length, 1), dtype=np.uint32)
    _check(lib().or_pba_endpoints(q, R_q, n_b, n0, seed, length, _ptr(T)), "pba_endpoints")
    return T[:length]


def pba_substitute(A, B: int, start, T_lists) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.uint32)
    st = np.ascontiguousarray(start, dtype=np.uint64)
    keep = [np.ascontiguousarray(t, dtype=np.uint32) for t in T_lists]
    ptrs = (C.c_void_p * B)(*[t.ctypes.data for t in keep])
    out = np.zeros(max(len(A), 1), dtype=np.uint32)
    _check(lib().or_pba_substitute(_ptr(A), len(A), B, _ptr(st), ptrs, _ptr(out)),
           "pba_substitute")
    return out[:len(A)]


def pba(n: int, m: int, B: int, n0: int, W: int, f: float, seed: int):
    """Two-phase PBA; returns (edges (B*(e0+n_b*m), 2) uint64, counts (B,B), fresh)."""
    n_edges = B * (seed_edges(n0) + (n // B) * m)
    out = np.zeros((max(n_edges, 1), 2), dtype=np.uint64)
    cnt = np.zeros((B, B), dtype=np.uint64)
    fresh = np.zeros(1, dtype=np.uint64)
    _check(lib().or_pba(n, m, B, n0, W, f, seed, _ptr(out), _ptr(cnt), _ptr(fresh)), "pba")
    return out[:n_edges], cnt, int(fresh[0])


def pba_factions(n: int, m: int, B: int, n0: int, lists, f: float, seed: int):
    """Two-phase PBA with explicit faction lists (lists[p]: block p's list).

    Returns (edges, counts (B,B), fresh) like pba().
    """
    if len(lists) != B:
        raise ValueError("one faction list per block")
    foff = np.zeros(B + 1, dtype=np.uint32)
    foff[1:] = np.cumsum([len(x) for x in lists])
    flat = np.ascontiguousarray(np.concatenate([np.asarray(x, np.uint32) for x in lists])
                                if B else np.zeros(1, np.uint32), dtype=np.uint32)
    n_edges = B * (seed_edges(n0) + (n // B) * m)
    out = np.zeros((max(n_edges, 1), 2), dtype=np.uint64)
    cnt = np.zeros((B, B), dtype=np.uint64)
    fresh = np.zeros(1, dtype=np.uint64)
    _check(lib().or_pba_factions(n, m, B, n0, _ptr(foff), _ptr(flat), f, seed, _ptr(out),
                                 _ptr(cnt), _ptr(fresh)), "pba_factions")
    return out[:n_edges], cnt, int(fresh[0])


def kron_thresholds(P_init) -> np.ndarray:
    Pm = np.ascontiguousarray(P_init, dtype=np.float64)
    n0 = Pm.shape[0]
    T = np.zeros(max(n0 * n0 - 1, 1), dtype=np.uint64)
    _check(lib().or_kron_thresholds(_ptr(Pm), n0, _ptr(T)), "kron_thresholds")
    return T[:n0 * n0 - 1]


def kron_pick(T, w: int) -> int:
    Ta = np.ascontiguousarray(T, dtype=np.uint64)
    return int(lib().or_kron_pick(_ptr(Ta), len(Ta), w))


def kron(P_init, k: int, M: int, seed: int) -> np.ndarray:
    Pm = np.ascontiguousarray(P_init, dtype=np.float64)
    out = np.zeros((max(M, 1), 2), dtype=np.uint64)
    _check(lib().or_kron(_ptr(Pm), Pm.shape[0], k, M, seed, _ptr(out)), "kron")
    return out[:M]


def kron_det(P_init, k: int, cap: int | None = None):
    """Deterministic Kronecker by the meta-edge stack; returns (edges, peak stack)."""
    Pm = np.ascontiguousarray(P_init, dtype=np.float64)
    e0 = int(np.count_nonzero(Pm > 0))
    cap = e0 ** k if cap is None else cap
    out = np.zeros((max(cap, 1), 2), dtype=np.uint64)
    n_out = np.zeros(1, dtype=np.uint64)
    peak = np.zeros(1, dtype=np.uint64)
    _check(lib().or_kron_det(_ptr(Pm), Pm.shape[0], k, _ptr(out), cap, _ptr(n_out), _ptr(peak)),
           "kron_det")
    return out[:int(n_out[0])], int(peak[0])


CSR_SYMMETRIZE, CSR_DEDUP, CSR_NO_LOOPS, CSR_ODD = 1, 2, 4, 8


def csr_opts(edges, n_vertices: int, flags: int):
    """CSR with options (symmetrise, dedup, drop loops, odd multiplicity)."""
    e = np.ascontiguousarray(edges, dtype=np.uint64).reshape(-1, 2)
    M = e.shape[0]
    row_ptr = np.zeros(n_vertices + 1, dtype=np.uint64)
    col = np.zeros(max(2 * M, 1), dtype=np.uint64)
    m_out = np.zeros(1, dtype=np.uint64)
    _check(lib().or_csr_opts(_ptr(e), M, n_vertices, flags, _ptr(row_ptr), _ptr(col),
                             _ptr(m_out)), "csr_opts")
    return row_ptr, col[:int(m_out[0])]


def random_cells(n_vertices: int, n_edges: int, seed: int) -> np.ndarray:
    """Random graph G(N, M) with replacement, as (M, 2) uint64 pairs."""
    out = np.zeros((max(n_edges, 1), 2), dtype=np.uint64)
    _check(lib().or_random_cells(n_vertices, n_edges, seed, _ptr(out)), "random_cells")
    return out[:n_edges]


DEG_OUT, DEG_IN, DEG_TOTAL = 0, 1, 2


def degrees(edges, n_vertices: int, which: int) -> np.ndarray:
    e = np.ascontiguousarray(edges, dtype=np.uint64).reshape(-1, 2)
    deg = np.zeros(max(n_vertices, 1), dtype=np.uint64)
    _check(lib().or_degrees(_ptr(e), e.shape[0], n_vertices, which, _ptr(deg)), "degrees")
    return deg[:n_vertices]


def degree_histogram(deg, max_degree: int) -> np.ndarray:
    d = np.ascontiguousarray(deg, dtype=np.uint64)
    hist = np.zeros(max_degree + 2, dtype=np.uint64)
    _check(lib().or_degree_histogram(_ptr(d), d.size, max_degree, _ptr(hist)), "degree_histogram")
    return hist


def bfs(row_ptr, col, source: int):
    """BFS distances (uint32, 0xFFFFFFFF unreached), levels, scanned entries."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.uint64)
    c = np.ascontiguousarray(col, dtype=np.uint64)
    N = rp.size - 1
    dist = np.zeros(max(N, 1), dtype=np.uint32)
    lv = np.zeros(1, dtype=np.uint32)
    sc = np.zeros(1, dtype=np.uint64)
    _check(lib().or_bfs(_ptr(rp), _ptr(c if c.size else np.zeros(1, np.uint64)), N, source,
                        _ptr(dist), _ptr(lv), _ptr(sc)), "bfs")
    return dist[:N], int(lv[0]), int(sc[0])


def csr(edges, n_vertices: int):
    e = np.ascontiguousarray(edges, dtype=np.uint64).reshape(-1, 2)
    M = e.shape[0]
    row_ptr = np.zeros(n_vertices + 1, dtype=np.uint64)
    col = np.zeros(max(M, 1), dtype=np.uint64)
    _check(lib().or_csr(_ptr(e), M, n_vertices, _ptr(row_ptr), _ptr(col)), "csr")
    return row_ptr, col[:M]

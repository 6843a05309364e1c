"""Order-dependent 64-bit digests of a two-phase PBA graph, per block.

Test infrastructure: the same formulas over the oracle's phase-1 lists and
phase-2 endpoint lists (numpy, in tests/golden/make_pba_headline_digests.py)
and over a generated edge list (torch, in the full-size GPU parity test).
Arithmetic is modulo 2^64: numpy uint64 and torch int64 agree bit for bit
on multiply, add and exclusive-or; every constant is below 2^63.

For block p with N_e entries (phase-1 entry j is edge j of the block):
  D1[p] = sum_j f(q_j, j)          q_j = the block entry j names (A_p[j])
  D2[p] = sum over targets q of g(q, sum_k f(t_k, k)),
          t_0, t_1, ... = the local ids that block p's occurrences of q take,
          in entry order (R4: the slice of T_q that q hands to p)
with f(v, k) = (v*K1 + K2) ^ (k*K3 + K4) and g(q, s) = (s*K5 + K6) ^ (q*K7 + K8).
A wrong target block, a wrong endpoint or two endpoints of one target
swapped between entries all change a digest (with probability ~1 - 2^-64).
"""
K1, K2, K3, K4 = 0x2545F4914F6CDD1D, 0x1B873593, 0x27BB2EE687B0B0FD, 0x6A09E667F3BCC909
K5, K6, K7, K8 = 0x3C6EF372FE94F82B, 0x510E527FADE682D1, 0x1F83D9ABFB41BD6B, 0x5BE0CD19137E2179


def f_np(v, k):
    import numpy as np
    v = np.asarray(v).astype(np.uint64)
    k = np.asarray(k).astype(np.uint64)
    with np.errstate(over="ignore"):
        return (v * np.uint64(K1) + np.uint64(K2)) ^ (k * np.uint64(K3) + np.uint64(K4))


def g_np(q, s):
    import numpy as np
    q = np.asarray(q).astype(np.uint64)
    s = np.asarray(s).astype(np.uint64)
    with np.errstate(over="ignore"):
        return (s * np.uint64(K5) + np.uint64(K6)) ^ (q * np.uint64(K7) + np.uint64(K8))


def f_torch(v, k):
    return (v * K1 + K2) ^ (k * K3 + K4)


def g_torch(q, s):
    return (s * K5 + K6) ^ (q * K7 + K8)


def block_digests_torch(dst, span: int, B: int):
    """(D1, D2) of one block from its N_e (non-seed) destination ids, a
    1-D int64 CUDA tensor in entry order; ids are q * span + local."""
    import torch
    n = dst.numel()
    q = dst // span
    local = dst - q * span
    pos = torch.arange(n, device=dst.device, dtype=torch.int64)
    d1 = int(f_torch(q, pos).sum().item()) & (2**64 - 1)
    qs, perm = torch.sort(q, stable=True)
    counts = torch.bincount(q, minlength=B)
    starts = torch.cumsum(counts, 0) - counts
    k = pos - starts[qs]
    sd = torch.zeros(B, dtype=torch.int64, device=dst.device)
    sd.index_add_(0, qs, f_torch(local[perm], k))
    tq = torch.arange(B, dtype=torch.int64, device=dst.device)
    d2 = int(g_torch(tq, sd)[counts > 0].sum().item()) & (2**64 - 1)
    return d1, d2

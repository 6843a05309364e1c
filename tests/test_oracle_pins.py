"""Pins of the oracle against what the paper and the mathematics fix.

Every test here runs on the CPU (no GPU marker). None of them compares the
oracle with itself: each checks a value printed in the paper (Fig. 1, Fig. 2),
a published known answer (Philox), a closed form, an exact small-case
enumeration, an invariant, or a special case that reduces to a textbook
process.
"""
import itertools
import math
from collections import Counter

import numpy as np
import pytest
from scipy import stats

import oracle as o


# --------------------------------------------------------------------------
# Philox4x32-10 and the integer draw primitives
# --------------------------------------------------------------------------

def test_philox_known_answers(golden):
    rows = golden("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        got = o.philox4x32_10(v[0:4], v[4:6])
        assert got.tolist() == v[6:10]


def test_uniform_edges_and_powers_of_two():
    # high half of (x * R) / 2^64: x = 0 gives 0, x = 2^64 - 1 gives R - 1
    for R in (1, 2, 3, 7, 1000, 2**32 + 5, 2**63, 2**64 - 1):
        assert o.uniform(0, 0, R) == 0
        assert o.uniform(0xFFFFFFFF, 0xFFFFFFFF, R) == R - 1
    # for R = 2^b the draw is the top b bits of the 64-bit word (w1:w0)
    rng = np.random.default_rng(5)
    for _ in range(200):
        w0, w1 = (int(x) for x in rng.integers(0, 2**32, size=2))
        x = (w1 << 32) | w0
        for b in (1, 5, 32, 40, 63):
            assert o.uniform(w0, w1, 2**b) == x >> (64 - b)


def test_uniform_is_monotone_and_in_range():
    rng = np.random.default_rng(6)
    for R in (3, 10, 12345, 2**40 + 7):
        ws = sorted(int(x) for x in rng.integers(0, 2**64, size=300, dtype=np.uint64))
        vals = [o.uniform(w & 0xFFFFFFFF, w >> 32, R) for w in ws]
        assert all(0 <= v < R for v in vals)
        assert all(a <= b for a, b in zip(vals, vals[1:]))


def test_coin_threshold_special_values():
    assert o.coin_threshold(0.0) == 0
    assert o.coin_threshold(1.0) == 2**32 - 1          # clamped
    assert o.coin_threshold(0.5) == 2**31
    assert o.coin_threshold(0.25) == 2**30
    assert o.coin_threshold(2.0**-33) == 0              # 0.5 rounds to even 0
    assert o.coin_threshold(3 * 2.0**-33) == 2          # 1.5 rounds to even 2
    assert o.coin_threshold(5 * 2.0**-33) == 2          # 2.5 rounds to even 2
    assert abs(o.coin_threshold(0.1) - 0.1 * 2**32) <= 0.5


# --------------------------------------------------------------------------
# Serial BA (copy-edge preferential attachment)
# --------------------------------------------------------------------------

def test_ba_structure():
    n, m, n0 = 5000, 3, 4
    e = o.ba(n, m, n0, seed=11).astype(np.int64)
    e0 = n0 * (n0 - 1) // 2
    assert e.shape == (e0 + n * m, 2)
    # seed clique first, lexicographic
    assert e[:e0].tolist() == [[a, b] for a in range(n0) for b in range(a + 1, n0)]
    gen = e[e0:]
    # each new vertex is the source of exactly m consecutive edges
    assert np.array_equal(gen[:, 0], n0 + np.arange(n * m) // m)
    # growth: targets are strictly earlier vertices (no self-loops)
    assert (gen[:, 1] < gen[:, 0]).all()
    assert gen[:, 1].min() >= 0


def test_ba_empty_and_invalid():
    e = o.ba(0, 4, 5, seed=1)
    assert e.shape == (10, 2)
    with pytest.raises(ValueError):
        o.ba(10, 0, 5, seed=1)
    with pytest.raises(ValueError):
        o.ba(10, 2, 1, seed=1)


def _exact_ba_law(n, m, n0):
    """Exact law of the generated targets, enumerating every slot choice."""
    seed_slots = []
    for a in range(n0):
        for b in range(a + 1, n0):
            seed_slots += [a, b]
    law = {(): 1.0}
    for i in range(n):
        slots_before = None
        new_law = {}
        for hist, pr in law.items():
            slots = list(seed_slots)
            for t, d in enumerate(hist):
                slots += [n0 + t // m, d]
            assert len(slots) == 2 * (len(seed_slots) // 2 + i * m)
            for choice in itertools.product(slots, repeat=m):
                key = hist + tuple(choice)
                new_law[key] = new_law.get(key, 0.0) + pr / len(slots) ** m
        law = new_law
    return law


@pytest.mark.parametrize("n,m,n0", [(2, 2, 2), (3, 1, 3)])
def test_ba_exact_small_law(n, m, n0):
    law = _exact_ba_law(n, m, n0)
    e0 = n0 * (n0 - 1) // 2
    trials = 30000
    seen = Counter()
    for s in range(trials):
        e = o.ba(n, m, n0, seed=1000 + s)
        seen[tuple(int(x) for x in e[e0:, 1])] += 1
    assert set(seen) <= set(law)          # nothing outside the exact support
    keys = sorted(law)
    obs = np.array([seen[k] for k in keys], float)
    exp = np.array([law[k] for k in keys]) * trials
    chi2 = ((obs - exp) ** 2 / exp).sum()
    assert chi2 < stats.chi2.ppf(1 - 1e-4, len(keys) - 1), chi2


def test_ba_degree_law():
    """Degree distribution vs P(k) = 2m(m+1)/(k(k+1)(k+2)) (Bollobas-Riordan)."""
    n, m = 10**6, 4
    e = o.ba(n, m, 5, seed=1)
    deg = np.bincount(e.ravel().astype(np.int64))
    assert deg.sum() == 2 * e.shape[0]
    assert deg[5:].min() >= m
    ks = np.arange(m, 61)
    p = 2.0 * m * (m + 1) / (ks * (ks + 1) * (ks + 2))
    obs = np.array([(deg == k).sum() for k in ks], float)
    exp = p * len(deg)
    chi2 = ((obs - exp) ** 2 / exp).sum()
    assert chi2 < stats.chi2.ppf(1 - 1e-4, len(ks)), chi2
    # mean exponent between 2 and infinity (Sec. 4 remark on finite mean degree)
    assert 2.0 < 1.0 + (deg >= m).sum() / np.log(deg[deg >= m] / (m - 0.5)).sum() < 4.0


# --------------------------------------------------------------------------
# PBA: worked example of Fig. 1, special cases, invariants
# --------------------------------------------------------------------------

def _fig1(golden):
    rows = {r[0]: [int(x) for x in r[1:]] for r in golden("pba_fig1.txt")}
    return rows


def test_fig1_faction_prefix(golden):
    g = _fig1(golden)
    A, cnt, fresh = o.pba_phase1_general(0, 4, g["faction_list"], 10, 0.0, seed=1)
    assert A[:4].tolist() == g["phase1_A"][:4]
    # with f = 0 every later entry copies an earlier one: only factions' blocks
    assert set(A.tolist()) <= set(g["faction_list"])
    assert fresh == 0


def test_fig1_counts_and_substitution(golden):
    g = _fig1(golden)
    A = g["phase1_A"]
    assert o.pba_count(A, 3).tolist() == g["counts"]
    lists = [[100, 101, 102], g["list_from_1"], [200, 201, 202]]
    out = o.pba_substitute(A, 3, [0, 0, 0], lists)
    snap = g["phase2_snapshot"]
    for j, v in enumerate(snap):
        if v >= 0:
            assert out[j] == v
    # P1's list lands on P1's positions, in order
    assert [int(out[j]) for j in range(10) if A[j] == 1] == g["list_from_1"]
    # the other blocks' lists are consumed in order too
    assert [int(out[j]) for j in range(10) if A[j] == 0] == lists[0]
    assert [int(out[j]) for j in range(10) if A[j] == 2] == lists[2]


def test_substitution_uses_slice_start():
    A = [2, 0, 2, 2, 1]
    lists = [[10, 11, 12], [20, 21], [30, 31, 32, 33, 34, 35]]
    out = o.pba_substitute(A, 3, [1, 1, 2], lists)
    assert out.tolist() == [32, 11, 33, 34, 21]


def test_pba_single_block_is_serial_ba():
    for (n, m, n0, seed) in [(1000, 3, 4, 9), (777, 1, 2, 3), (64, 8, 9, 0)]:
        e1, cnt, fresh = o.pba(n, m, 1, n0, 1, 0.1, seed)
        assert np.array_equal(e1, o.ba(n, m, n0, seed))
        assert cnt.tolist() == [[n * m]] and fresh == 0


def test_pba_isolated_blocks_are_independent_ba():
    """W=1, f=0: every block only attaches to itself -> B serial BA runs."""
    n, m, B, n0, seed = 4 * 300, 3, 4, 5, 21
    e, cnt, fresh = o.pba(n, m, B, n0, 1, 0.0, seed)
    n_b, e0 = n // B, n0 * (n0 - 1) // 2
    assert fresh == 0 and np.array_equal(cnt, np.diag([n_b * m] * B).astype(np.uint64))
    span = n0 + n_b
    per = e0 + n_b * m
    for p in range(B):
        ref = o.ba(n_b, m, n0, seed, stream=p) + np.uint64(p * span)
        assert np.array_equal(e[p * per:(p + 1) * per], ref)


@pytest.mark.parametrize("B,W,f", [(8, 1, 0.1), (8, 2, 0.3), (6, 3, 1.0), (5, 5, 0.5)])
def test_pba_invariants(B, W, f):
    n, m, n0, seed = B * 400, 3, 4, 77
    e, cnt, fresh = o.pba(n, m, B, n0, W, f, seed)
    e = e.astype(np.int64)
    n_b, e0 = n // B, n0 * (n0 - 1) // 2
    span, per = n0 + n_b, e0 + n_b * m
    assert e.shape == (B * per, 2)
    assert cnt.sum(axis=1).tolist() == [n_b * m] * B
    R = cnt.sum(axis=0).astype(np.int64)
    assert R.sum() == n * m
    indeg = np.zeros(B, np.int64)
    for p in range(B):
        blk = e[p * per:(p + 1) * per]
        seedpart, gen = blk[:e0], blk[e0:]
        assert seedpart.tolist() == [[p * span + a, p * span + b]
                                     for a in range(n0) for b in range(a + 1, n0)]
        assert np.array_equal(gen[:, 0], p * span + n0 + np.arange(n_b * m) // m)
        q = gen[:, 1] // span
        assert (q < B).all()
        np.add.at(indeg, q, 1)
        if W == B or f == 0.0:
            phi = (p // W) * W
            assert ((q >= phi) & (q < phi + W)).all()
    # every block receives exactly the endpoints it was asked for
    assert indeg.tolist() == R.tolist()
    if W == B:
        assert fresh == 0


# Overlapping factions in the manner of Fig. 1: F0 = {0,1}, F1 = {1,2,3},
# F2 = {3,4}, F3 = {4,5,0}; a block's list concatenates the factions it is in.
FACTION_LISTS = [[0, 1, 4, 5, 0], [0, 1, 1, 2, 3], [1, 2, 3], [1, 2, 3, 3, 4], [3, 4, 4, 5, 0],
                 [4, 5, 0]]


def _received_by_target(edges, B, n_b, m, n0):
    """Local ids each target block q handed out, requester by requester in
    ascending block order and, within a requester, in entry order."""
    e0, N_e, span = n0 * (n0 - 1) // 2, n_b * m, n0 + n_b
    got = {q: [] for q in range(B)}
    for p in range(B):
        for dst in edges[p * (e0 + N_e) + e0:(p + 1) * (e0 + N_e), 1].astype(np.int64):
            got[int(dst // span)].append(int(dst % span))
    return got


@pytest.mark.parametrize("B,W,f,seed", [(4, 1, 0.5, 13), (6, 2, 0.3, 5), (3, 1, 1.0, 8)])
def test_pba_requesters_take_consecutive_slices_of_each_list(B, W, f, seed):
    """Reading R4 (Sec. 3, substitution; Fig. 1(b)): q's endpoint list T_q is
    split among its requesters in ascending block order, each consuming its
    slice in entry order. So the endpoints that blocks 0, 1, ... received from
    q, read in that order, are T_q from its start, with T_q computed on its
    own by phase 2."""
    n_b, m, n0 = 300, 3, 4
    edges, counts, _ = o.pba(B * n_b, m, B, n0, W, f, seed)
    R = counts.astype(np.int64).sum(axis=0)
    got = _received_by_target(edges, B, n_b, m, n0)
    for q in range(B):
        assert len(got[q]) == R[q]
        assert got[q] == [int(x) for x in o.pba_endpoints(q, int(R[q]), n_b, n0, seed)]
    # several requesters per target, or the split would not be exercised
    assert ((counts > 0).sum(axis=0) > 1).any()


def test_pba_factions_requesters_take_consecutive_slices():
    """The same split with overlapping faction lists in the manner of Fig. 1."""
    B, n_b, m, n0, seed = 3, 200, 2, 3, 4
    lists = [[1, 2, 0, 1], [1, 2, 1, 0], [2, 0, 1, 2]]
    edges, counts, _ = o.pba_factions(B * n_b, m, B, n0, lists, 0.2, seed)
    R = np.asarray(counts).astype(np.int64).sum(axis=0)
    got = _received_by_target(edges, B, n_b, m, n0)
    for q in range(B):
        assert got[q] == [int(x) for x in o.pba_endpoints(q, int(R[q]), n_b, n0, seed)]


def test_pba_factions_closure_without_inter_faction_picks():
    """f = 0: phase 1 only copies earlier entries, so block p's targets stay
    inside its own list (copies of the list itself)."""
    B, n_b, m, n0 = 6, 500, 3, 4
    e, cnt, fresh = o.pba_factions(B * n_b, m, B, n0, FACTION_LISTS, 0.0, seed=13)
    span, per, e0 = n0 + n_b, n0 * (n0 - 1) // 2 + n_b * m, n0 * (n0 - 1) // 2
    assert fresh == 0
    for p in range(B):
        q = e[p * per + e0:(p + 1) * per, 1].astype(np.int64) // span
        assert set(q.tolist()) <= set(FACTION_LISTS[p])
        assert set(np.nonzero(cnt[p])[0].tolist()) <= set(FACTION_LISTS[p])


def test_pba_factions_exact_counts_when_every_pick_is_fresh():
    """f = 1: entries below s_p copy the list, every later entry is a fresh
    pick outside the list, so the counts of listed blocks are their
    multiplicities in the list."""
    B, n_b, m, n0 = 6, 300, 2, 3
    _, cnt, fresh = o.pba_factions(B * n_b, m, B, n0, FACTION_LISTS, 1.0, seed=2)
    N_e = n_b * m
    assert fresh == sum(N_e - len(L) for L in FACTION_LISTS)
    for p, L in enumerate(FACTION_LISTS):
        listed = np.bincount(L, minlength=B)
        inside = np.isin(np.arange(B), L)
        assert np.array_equal(cnt[p][inside], listed[inside].astype(np.uint64))
        assert int(cnt[p][~inside].sum()) == N_e - len(L)


def test_pba_factions_invariants():
    B, n_b, m, n0 = 6, 400, 3, 4
    e, cnt, _ = o.pba_factions(B * n_b, m, B, n0, FACTION_LISTS, 0.3, seed=71)
    e = e.astype(np.int64)
    span, e0 = n0 + n_b, n0 * (n0 - 1) // 2
    per = e0 + n_b * m
    R = cnt.sum(axis=0).astype(np.int64)
    assert cnt.sum(axis=1).tolist() == [n_b * m] * B
    indeg = np.zeros(B, np.int64)
    for p in range(B):
        gen = e[p * per + e0:(p + 1) * per]
        assert np.array_equal(gen[:, 0], p * span + n0 + np.arange(n_b * m) // m)
        np.add.at(indeg, gen[:, 1] // span, 1)
        # the first entries copy the list
        L = FACTION_LISTS[p]
        assert (gen[:len(L), 1] // span).tolist() == L
    assert indeg.tolist() == R.tolist()


def test_pba_factions_duplicate_self_list_is_independent_ba():
    """Lists [p, p] and f = 0 keep every block on itself: the graph equals B
    independent serial BA runs, as with width-1 factions."""
    n, m, B, n0, seed = 4 * 250, 2, 4, 3, 5
    e, cnt, _ = o.pba_factions(n, m, B, n0, [[p, p] for p in range(B)], 0.0, seed)
    ref, rcnt, _ = o.pba(n, m, B, n0, 1, 0.0, seed)
    assert np.array_equal(e, ref) and np.array_equal(cnt, rcnt)


def test_pba_factions_rejects_empty_list():
    with pytest.raises(Exception):
        o.pba_factions(40, 2, 2, 3, [[0], []], 0.1, 1)


def test_pba_fresh_count_binomial():
    B, W, f, n_b, m = 16, 2, 0.1, 2000, 2
    total = 0
    for p in range(B):
        _, _, fr = o.pba_phase1(p, B, W, n_b * m, f, seed=5)
        total += fr
    trials = B * (n_b * m - W)
    pf = o.coin_threshold(f) / 2**32
    z = (total - trials * pf) / math.sqrt(trials * pf * (1 - pf))
    assert abs(z) < 4.5, z


def test_pba_fresh_targets_uniform_outside_faction():
    B, W, p = 8, 2, 5
    A, _, fresh = o.pba_phase1(p, B, W, 60000, 1.0, seed=8)
    assert A[:2].tolist() == [4, 5]
    tail = A[2:]
    assert fresh == len(tail)                 # f = 1: every later entry is fresh
    assert not np.isin(tail, [4, 5]).any()
    obs = np.bincount(tail, minlength=B)[[0, 1, 2, 3, 6, 7]]
    assert stats.chisquare(obs).pvalue > 1e-4


def test_pba_first_fresh_pick_uniform_at_small_f():
    """With f small the inter-faction pick must still be uniform over all
    blocks outside the factions, whatever the coin that chose it (Sec. 3).
    With W = 1 every entry before the first fresh pick copies A[0] = p, so
    the first entry other than p is that pick; pooled over blocks and seeds,
    its rank among the B - 1 outside blocks is uniform."""
    B, f = 16, 0.1
    ranks = []
    for seed in range(50):
        for p in range(B):
            A, _, _ = o.pba_phase1(p, B, 1, 300, f, seed=seed)
            other = A[A != p]
            assert len(other) > 0
            q = int(other[0])
            ranks.append(q if q < p else q - 1)
    obs = np.bincount(ranks, minlength=B - 1)
    assert len(obs) == B - 1
    assert stats.chisquare(obs).pvalue > 1e-4, obs


@pytest.mark.parametrize("W,f", [(1, 0.3), (2, 0.1)])
def test_pba_in_faction_count_mean_closed_form(W, f):
    """Sec. 3, phase 1 with inter-faction picks: the first s = W entries are
    the faction. A later entry j is a fresh pick (never in the faction) with
    probability f' = T_f/2^32, and otherwise a copy of a uniform earlier
    entry, in the faction with probability in_j/j. So the expected count
    after N entries is E[in_N] = s * prod_{j=s}^{N-1} (1 + (1 - f')/j), about
    N (s/N)^f: the realised share outside the faction is much larger than f.
    The sample mean over blocks and seeds is compared with it (z-test with
    the sample's own spread: the urn's limit is random)."""
    B, N = 16, 3000
    fp = o.coin_threshold(f) / 2**32
    expect = W * np.prod(1.0 + (1.0 - fp) / np.arange(W, N, dtype=np.float64))
    got = []
    for seed in range(40):
        for p in range(B):
            A, _, _ = o.pba_phase1(p, B, W, N, f, seed=seed)
            phi = (p // W) * W
            got.append(int(((A >= phi) & (A < phi + W)).sum()))
    got = np.asarray(got, dtype=np.float64)
    z = (got.mean() - expect) / (got.std(ddof=1) / math.sqrt(got.size))
    assert abs(z) < 4.5, (got.mean(), expect, z)
    assert expect / N < 1 - f          # far more than f of the entries are outside


def test_pba_phase1_polya_urn_law():
    """W=2, f=0: a two-colour Polya urn started with one ball of each colour.

    The number of first-colour draws among N draws is then exactly uniform on
    {0..N}, so the count of block phi in A_p is uniform on {1..N_e-1}.
    """
    B, W, N_e = 2, 2, 1000
    vals = []
    for s in range(1500):
        A, cnt, _ = o.pba_phase1(0, B, W, N_e, 0.0, seed=s)
        vals.append(int(cnt[0]))
    vals = np.array(vals)
    assert vals.min() >= 1 and vals.max() <= N_e - 1
    u = (vals - 1 + 0.5) / (N_e - 1)
    assert stats.kstest(u, "uniform").pvalue > 1e-4


def test_pba_endpoints_equal_ba_when_requests_match():
    """R_q = n_b*m gives sigma(i) = i div m: the local list is serial BA."""
    n_b, m, n0, q, seed = 500, 4, 5, 3, 4
    T = o.pba_endpoints(q, n_b * m, n_b, n0, seed)
    ref = o.ba(n_b, m, n0, seed, stream=q)[n0 * (n0 - 1) // 2:, 1]
    assert np.array_equal(T.astype(np.uint64), ref)


def test_pba_endpoints_growth_bound():
    n_b, n0 = 1000, 3
    for R_q in (1, 7, 999, 1000, 1001, 3333, 5000):
        T = o.pba_endpoints(2, R_q, n_b, n0, seed=12).astype(np.int64)
        sigma = (np.arange(R_q, dtype=np.int64) * n_b) // R_q
        assert (T < n0 + sigma).all()


def test_pba_endpoints_exact_small_law():
    """n_b=3, R_q=4: sigma = [0,0,1,2], earlier-edge counts E = [0,0,2,3]."""
    n_b, R_q, n0 = 3, 4, 2
    sigma = [0, 0, 1, 2]
    before = [0, 0, 2, 3]
    law = {(): 1.0}
    for i in range(R_q):
        new = {}
        for hist, pr in law.items():
            slots = [0, 1]
            for t in range(before[i]):
                slots += [n0 + sigma[t], hist[t]]
            for d in slots:
                key = hist + (d,)
                new[key] = new.get(key, 0.0) + pr / len(slots)
        law = new
    trials = 30000
    seen = Counter(tuple(int(x) for x in o.pba_endpoints(1, R_q, n_b, n0, seed=s))
                   for s in range(trials))
    assert set(seen) <= set(law)
    keys = sorted(law)
    obs = np.array([seen[k] for k in keys], float)
    exp = np.array([law[k] for k in keys]) * trials
    chi2 = ((obs - exp) ** 2 / exp).sum()
    assert chi2 < stats.chi2.ppf(1 - 1e-4, len(keys) - 1), chi2


def test_pba_invalid_arguments():
    with pytest.raises(ValueError):
        o.pba(10, 2, 3, 4, 1, 0.1, 1)         # B does not divide n
    with pytest.raises(ValueError):
        o.pba(12, 2, 4, 4, 3, 0.1, 1)         # W does not divide B
    with pytest.raises(ValueError):
        o.pba(12, 2, 4, 4, 1, 1.5, 1)         # f outside [0, 1]


# --------------------------------------------------------------------------
# Kronecker: quantiser, descent law, deterministic expansion (Fig. 2)
# --------------------------------------------------------------------------

def test_kron_thresholds_exact_cases():
    assert o.kron_thresholds([[1, 1], [1, 1]]).tolist() == [2**30, 2**31, 3 * 2**30]
    assert o.kron_thresholds([[0, 1], [0, 0]]).tolist() == [0, 2**32, 2**32]
    assert o.kron_thresholds([[2, 0], [0, 2]]).tolist() == [2**31, 2**31, 2**31]
    T = o.kron_thresholds([[0.57, 0.19], [0.19, 0.05]])
    assert (np.diff(T.astype(np.int64)) >= 0).all()
    for t, c in zip(T, np.cumsum([0.57, 0.19, 0.19])):
        assert abs(int(t) - c * 2**32) <= 1
    with pytest.raises(ValueError):
        o.kron_thresholds([[0, 0], [0, 0]])
    with pytest.raises(ValueError):
        o.kron_thresholds([[1, -1], [1, 1]])


@pytest.mark.parametrize("Pm", [
    [[1, 1], [1, 0]],
    [[3, 1, 2], [1, 5, 1], [2, 2, 4]],
    [[7, 3], [3, 1]],
    [[1, 2, 3, 4], [5, 6, 7, 8], [9, 10, 11, 12], [13, 14, 15, 17]],
])
def test_kron_thresholds_round_to_nearest(Pm):
    """Reading R8: each threshold is 2^32 times the cumulative share of the
    cells before it, rounded to the NEAREST integer. With integer initiator
    entries the exact value is a rational number, so the error is checked
    exactly: at most one half (a floor or a ceiling would reach up to 1)."""
    from fractions import Fraction
    flat = [int(x) for row in Pm for x in row]
    S = sum(flat)
    T = o.kron_thresholds(Pm)
    assert len(T) == len(flat) - 1
    cum = 0
    worst = Fraction(0)
    for c in range(len(flat) - 1):
        cum += flat[c]
        err = abs(Fraction(int(T[c])) - Fraction(cum * 2**32, S))
        worst = max(worst, err)
        assert err <= Fraction(1, 2) + Fraction(1, 10**6), (c, float(err))
    assert worst > Fraction(1, 4)      # the cases do exercise the rounding


def test_kron_pick_boundaries():
    T = o.kron_thresholds([[0.57, 0.19], [0.19, 0.05]])
    for c, t in enumerate(T.tolist()):
        assert o.kron_pick(T, t - 1) == c
        assert o.kron_pick(T, t) == c + 1
    assert o.kron_pick(T, 0) == 0
    assert o.kron_pick(T, 2**32 - 1) == 3
    # zero-probability cells are never picked
    Tz = o.kron_thresholds([[0, 1], [0, 0]])
    assert {o.kron_pick(Tz, w) for w in (0, 1, 2**31, 2**32 - 1)} == {1}


def _quantised(Pm):
    T = o.kron_thresholds(Pm).astype(np.float64)
    edges = np.concatenate([[0.0], T, [2.0**32]])
    return (np.diff(edges) / 2.0**32).reshape(np.asarray(Pm).shape)


@pytest.mark.parametrize("Pm,k", [
    ([[0.5, 0.3], [0.15, 0.05]], 4),
    ([[0.2, 0.5, 0.0], [0.1, 0.05, 0.05], [0.0, 0.02, 0.08]], 2),
])
def test_kron_cell_law_vs_kronecker_power(Pm, k):
    """Cell frequencies vs the brute-force k-th Kronecker power of the initiator."""
    Q = _quantised(Pm)
    Pk = Q
    for _ in range(k - 1):
        Pk = np.kron(Pk, Q)
    n = Pk.shape[0]
    M = 200000
    e = o.kron(Pm, k, M, seed=7).astype(np.int64)
    assert e.max() < n
    obs = np.bincount(e[:, 0] * n + e[:, 1], minlength=n * n).astype(float)
    exp = Pk.ravel() * M
    assert obs[exp == 0].sum() == 0
    keep = exp > 0
    chi2 = ((obs[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    assert chi2 < stats.chi2.ppf(1 - 1e-4, keep.sum() - 1), chi2


def test_kron_counter_layout():
    """Reading R8: level l of edge e (most significant first) reads word
    l mod 4 of the Philox block with counter (e_lo, e_hi, l div 4, 3). With
    the 2x2 initiator [[1, 1], [1, 1]] the thresholds are 2^30, 2^31 and
    3*2^30, so the cell of a level is the top two bits of its word: the row
    bit is bit 31 and the column bit is bit 30."""
    seed, k, M = 0x0F0E_0D0C_0B0A, 10, 48
    e_list = o.kron([[1, 1], [1, 1]], k, M, seed)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for e in range(M):
        row = col = 0
        for g in range((k + 3) // 4):
            w = o.philox4x32_10([e, 0, g, 3], key)
            for t in range(4):
                if 4 * g + t < k:
                    row = 2 * row + (int(w[t]) >> 31)
                    col = 2 * col + ((int(w[t]) >> 30) & 1)
        assert (int(e_list[e, 0]), int(e_list[e, 1])) == (row, col), e


def test_kron_row_popcount_binomial():
    """n0=2: #edges whose source has h one-digits ~ M C(k,h) p1^h p0^(k-h)."""
    Pm = [[0.57, 0.19], [0.19, 0.05]]
    Q = _quantised(Pm)
    p1 = Q[1].sum()
    k, M = 12, 300000
    e = o.kron(Pm, k, M, seed=3).astype(np.int64)
    for col in (0, 1):
        pc = (Q[1].sum() if col == 0 else Q[:, 1].sum())
        h = np.array([bin(int(v)).count("1") for v in e[:, col]])
        obs = np.bincount(h, minlength=k + 1).astype(float)
        exp = M * stats.binom.pmf(np.arange(k + 1), k, pc)
        keep = exp > 5
        chi2 = ((obs[keep] - exp[keep]) ** 2 / exp[keep]).sum()
        assert chi2 < stats.chi2.ppf(1 - 1e-4, keep.sum() - 1), (col, chi2)
    assert abs(p1 - 0.24) < 1e-9


def test_kron_expected_degrees_closed_form():
    """Expected degrees of the stochastic Kronecker model (Sec. 2, the model
    the PK method cites): a vertex whose base-n0 digits are a_0..a_{k-1} has
    expected out-degree M * prod_l sum_b Q[a_l][b] and expected in-degree
    M * prod_l sum_a Q[a][a_l], for Q the quantised initiator. Checked
    with a chi-square over all 3^7 rows and all 3^7 columns, at a depth where
    the full Kronecker power has 4.8e6 cells."""
    Pm = [[0.30, 0.15, 0.05], [0.10, 0.12, 0.08], [0.02, 0.08, 0.10]]
    Q = _quantised(Pm)
    n0, k, M = 3, 7, 600000
    e = o.kron(Pm, k, M, seed=21).astype(np.int64)
    digits = np.array([[(v // n0 ** (k - 1 - l)) % n0 for l in range(k)]
                       for v in range(n0 ** k)])
    for col, share in ((0, Q.sum(axis=1)), (1, Q.sum(axis=0))):
        exp = M * np.prod(share[digits], axis=1)
        assert abs(exp.sum() - M) < 1e-6 * M
        obs = np.bincount(e[:, col], minlength=n0 ** k).astype(float)
        assert len(obs) == n0 ** k
        assert exp.min() > 5
        chi2 = ((obs - exp) ** 2 / exp).sum()
        assert chi2 < stats.chi2.ppf(1 - 1e-4, n0 ** k - 1), (col, chi2)


def _fig2_seed(golden):
    return np.array([[float(x) for x in r] for r in golden("pk_fig2_seed.txt")])


def test_kron_det_fig2(golden):
    G1 = _fig2_seed(golden)
    assert int(G1.sum()) == 11
    for k in (1, 2, 3):
        e, peak = o.kron_det(G1, k)
        assert e.shape == (11 ** k, 2)
        Gk = G1
        for _ in range(k - 1):
            Gk = np.kron(Gk, G1)
        assert Gk.shape == (5 ** k, 5 ** k)
        dense = np.zeros_like(Gk)
        dense[e[:, 0].astype(np.int64), e[:, 1].astype(np.int64)] += 1
        assert np.array_equal(dense, Gk)          # same set, no duplicates
        assert peak <= k * (11 - 1) + 1
    # Fig. 2(c): the (0,0) block of G2 is G1 and the (1,2) block is zero
    e2, _ = o.kron_det(G1, 2)
    D = np.zeros((25, 25))
    D[e2[:, 0].astype(int), e2[:, 1].astype(int)] = 1
    assert np.array_equal(D[0:5, 0:5], G1)
    assert not D[5:10, 10:15].any()


def test_kron_det_order_is_seed_digit_order(golden):
    """Popping children in seed order yields edges in base-e0 digit order."""
    G1 = _fig2_seed(golden)
    sa, sb = np.nonzero(G1)
    e0, n0, k = len(sa), 5, 3
    e, _ = o.kron_det(G1, k)
    for idx in range(e0 ** k):
        digits = [(idx // e0 ** (k - 1 - l)) % e0 for l in range(k)]
        r = sum(int(sa[d]) * n0 ** (k - 1 - l) for l, d in enumerate(digits))
        c = sum(int(sb[d]) * n0 ** (k - 1 - l) for l, d in enumerate(digits))
        assert (int(e[idx, 0]), int(e[idx, 1])) == (r, c)


def test_kron_det_capacity():
    with pytest.raises(ValueError):
        o.kron_det([[1, 1], [1, 0]], 5, cap=3 ** 5 - 1)


# --------------------------------------------------------------------------
# CSR
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N,M", [(1, 0), (10, 50), (1000, 20000), (50, 3)])
def test_csr_matches_lexsort(N, M):
    rng = np.random.default_rng(N + M)
    e = np.stack([rng.integers(0, N, M), rng.integers(0, 3 * N, M)], 1).astype(np.uint64)
    rp, col = o.csr(e, N)
    order = np.lexsort((e[:, 1], e[:, 0]))
    assert np.array_equal(col, e[order, 1])
    assert rp[0] == 0 and rp[-1] == M
    assert (np.diff(rp.astype(np.int64)) >= 0).all()
    assert np.array_equal(np.diff(rp.astype(np.int64)),
                          np.bincount(e[:, 0].astype(np.int64), minlength=N))
    for v in range(min(N, 50)):
        row = col[rp[v]:rp[v + 1]]
        assert (np.diff(row.astype(np.int64)) >= 0).all()


def test_csr_rejects_out_of_range_source():
    with pytest.raises(ValueError):
        o.csr(np.array([[3, 0]], np.uint64), 3)


# --------------------------------------------------------------------------
# CSR options and the random graph used to randomise PK (reading R11)
# --------------------------------------------------------------------------

def _multigraph(seed, M, N, loops=True):
    rng = np.random.default_rng(seed)
    e = rng.integers(0, N, size=(M, 2), dtype=np.uint64)
    e[: M // 5] = e[M // 5: 2 * (M // 5)]            # many repeated pairs
    if loops:
        e[::11, 1] = e[::11, 0]                       # self-loops
    return e


def _rows(row_ptr, col):
    return [tuple(col[row_ptr[v]:row_ptr[v + 1]].tolist()) for v in range(len(row_ptr) - 1)]


def test_csr_dedup_equals_numpy_unique():
    e = _multigraph(1, 5000, 300)
    rp, col = o.csr_opts(e, 300, o.CSR_DEDUP)
    u = np.unique(e, axis=0)
    assert np.array_equal(col, u[:, 1])
    assert np.array_equal(rp, np.concatenate([[0], np.cumsum(np.bincount(u[:, 0].astype(np.int64),
                                                                         minlength=300))]))


def test_csr_symmetrize_is_symmetric_with_multiplicity():
    e = _multigraph(2, 3000, 100)
    rp, col = o.csr_opts(e, 100, o.CSR_SYMMETRIZE)
    assert col.size == 2 * e.shape[0]
    src = np.repeat(np.arange(100, dtype=np.uint64), np.diff(rp).astype(np.int64))
    fwd = Counter(zip(src.tolist(), col.tolist()))
    assert fwd == Counter((b, a) for (a, b) in fwd.elements())


def test_csr_odd_keeps_pairs_of_odd_multiplicity():
    e = _multigraph(3, 4000, 60)
    rp, col = o.csr_opts(e, 60, o.CSR_ODD)
    counts = Counter(map(tuple, e.tolist()))
    want = sorted(p for p, c in counts.items() if c % 2 == 1)
    src = np.repeat(np.arange(60), np.diff(rp).astype(np.int64))
    assert list(zip(src.tolist(), col.tolist())) == want
    # XOR identities: a list with itself cancels; disjoint sets give their union
    both = np.concatenate([e, e])
    _, c2 = o.csr_opts(both, 60, o.CSR_ODD)
    assert c2.size == 0
    a = np.array([[0, 1], [2, 3]], np.uint64)
    b = np.array([[1, 0], [3, 3]], np.uint64)
    _, c3 = o.csr_opts(np.concatenate([a, b]), 4, o.CSR_ODD)
    assert c3.tolist() == [1, 0, 3, 3]


def test_csr_no_loops_drops_exactly_the_loops():
    e = _multigraph(4, 2000, 50)
    rp, col = o.csr_opts(e, 50, o.CSR_NO_LOOPS)
    src = np.repeat(np.arange(50, dtype=np.uint64), np.diff(rp).astype(np.int64))
    assert not (src == col).any()
    assert col.size == int((e[:, 0] != e[:, 1]).sum())


def test_random_cells_counter_layout():
    """Edge e uses the draw with counter (e, 0, 0, 4); for N = 2^b the row is
    the top b bits of (w1:w0) and the column the top b bits of (w3:w2)."""
    seed, b = 0x1234_5678_9ABC, 10
    cells = o.random_cells(2**b, 64, seed)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for e in range(64):
        w = o.philox4x32_10([e, 0, 0, 4], key)
        assert int(cells[e, 0]) == ((int(w[1]) << 32 | int(w[0])) >> (64 - b))
        assert int(cells[e, 1]) == ((int(w[3]) << 32 | int(w[2])) >> (64 - b))


def test_random_cells_uniform():
    N, M = 37, 200_000
    cells = o.random_cells(N, M, seed=9).astype(np.int64)
    for axis in (0, 1):
        obs = np.bincount(cells[:, axis], minlength=N)
        assert stats.chisquare(obs).pvalue > 1e-4
    assert stats.chisquare(np.bincount(cells[:, 0] * N + cells[:, 1], minlength=N * N)).pvalue > 1e-4


# --------------------------------------------------------------------------
# Graph properties: degrees, histogram, BFS distances (Sec. 4's checks)
# --------------------------------------------------------------------------

def test_degrees_and_histogram_equal_bincount():
    rng = np.random.default_rng(12)
    N = 400
    e = rng.integers(0, N, size=(5000, 2), dtype=np.uint64)
    e[::7, 1] = e[::7, 0]
    for which, cols in ((o.DEG_OUT, [0]), (o.DEG_IN, [1]), (o.DEG_TOTAL, [0, 1])):
        deg = o.degrees(e, N, which)
        want = sum(np.bincount(e[:, c].astype(np.int64), minlength=N) for c in cols)
        assert np.array_equal(deg, want.astype(np.uint64))
        for max_deg in (5, 40, 10**4):
            h = o.degree_histogram(deg, max_deg)
            clamped = np.minimum(deg, max_deg + 1).astype(np.int64)
            assert np.array_equal(h, np.bincount(clamped, minlength=max_deg + 2).astype(np.uint64))


@pytest.mark.parametrize("symmetric", [False, True])
def test_bfs_equals_networkx_shortest_paths(symmetric):
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(5 + symmetric)
    N = 300
    e = rng.integers(0, N, size=(700, 2), dtype=np.uint64)
    flags = o.CSR_SYMMETRIZE if symmetric else 0
    rp, col = o.csr_opts(e, N, flags)
    G = nx.DiGraph()
    G.add_nodes_from(range(N))
    src = np.repeat(np.arange(N), np.diff(rp).astype(np.int64))
    G.add_edges_from(zip(src.tolist(), col.tolist()))
    for s in (0, 17, 299):
        dist, levels, scanned = o.bfs(rp, col, s)
        want = nx.single_source_shortest_path_length(G, s)
        got = {v: int(d) for v, d in enumerate(dist) if d != 0xFFFFFFFF}
        assert got == want
        assert levels == max(want.values()) + 1
        assert scanned == int(sum(rp[v + 1] - rp[v] for v in want))


def test_powerlaw_exponent_of_ba_is_three():
    """The BA model's degree law P(k) ~ k^-3 (Bollobas-Riordan): the discrete
    estimator on a 10^6-vertex oracle graph must recover an exponent near 3."""
    import paper_1003_3684_gb300 as pg
    e = o.ba(10**6, 4, 5, seed=3)
    deg = o.degrees(e, 10**6 + 5, o.DEG_TOTAL)
    h = o.degree_histogram(deg, 5000)
    gamma = pg.powerlaw_exponent(h, 12)
    assert 2.8 < gamma < 3.2, gamma

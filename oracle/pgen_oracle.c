/*
 * pgen oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU restatement of the two graph generators
 * of Yoo & Henderson, "Parallel Generation of Massive Scale-Free Graphs"
 * (arXiv 1003.3684): the parallel Barabasi-Albert method with two-phase
 * preferential attachment (Sec. 3, "Parallel Barabasi-Albert (PBA) method",
 * Fig. 1) and the Kronecker method (Sec. 3, "Parallel Kronecker (PK) method",
 * Fig. 2, and the stochastic-initiator model of Leskovec et al. it cites in
 * Sec. 2).
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library. The CUDA library shares no source, header, table or
 * helper with it; each side has its own Philox, its own quantiser and its own
 * index arithmetic. Every function computes the literal sequential algorithm
 * (an explicit endpoint array, an explicit urn, an explicit stack, a sort),
 * not the closed forms the GPU path uses.
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes, and implemented the same way on the GPU side):
 *  R1  n counts NEW vertices; every block also owns a seed clique K_{n0}
 *      whose e0 = n0(n0-1)/2 edges are part of the output.
 *  R2  a new vertex attaches only to edge slots of the seed and of strictly
 *      earlier vertices (no self-loops; repeated targets allowed).
 *  R3  phase 2 (ordinary preferential attachment over q's local vertices,
 *      as many endpoints as were requested) spreads the R_q local edges
 *      over the n_b local vertices: edge i has source time
 *      sigma(i) = floor(i*n_b/R_q) and may attach to the seed and to the
 *      E(sigma(i)) = ceil(sigma(i)*R_q/n_b) edges of earlier source times.
 *  R4  q's endpoint list is split among requesters in ascending block order;
 *      each requester consumes its slice in increasing edge order.
 *  R5  factions: by default aligned groups of W consecutive blocks (s = W);
 *      general lists give block p the member lists of every faction it
 *      belongs to, in order, and the first s_p entries of A_p copy them.
 *  R6  inter-faction picks: each entry j >= s is, with probability f
 *      (coin w2 < T_f, T_f = min(2^32 - 1, round_half_even(f * 2^32))), the
 *      x-th block outside p's list in ascending order, x = floor(w3 * n_out
 *      / 2^32); otherwise it copies a uniform earlier entry. No coin is
 *      drawn when no block lies outside the list.
 *  R7  random streams: Philox4x32-10 (Salmon et al., SC'11) with key
 *      (seed_lo, seed_hi) and counter (idx_lo, idx_hi, stream, tag);
 *      tag 1 = phase-1 entry, tag 2 = phase-2 local edge, tag 3 = Kronecker
 *      level group, tag 4 = random-graph cell. A uniform integer in [0, R)
 *      is the high 64 bits of ((w1 << 32) | w0) * R.
 *  R8  Kronecker: thresholds T_c = round_half_even(2^32 * cum_c / S) where
 *      cum_c is the left-to-right double sum of the initiator's first c+1
 *      row-major cells and S the sum of all of them; level l (most
 *      significant first) takes word (l mod 4) of the Philox block for
 *      counter (e_lo, e_hi, l div 4, 3) and picks cell #{c : w >= T_c}.
 *  R9  deterministic PK: a depth-first stack of meta-edges whose children
 *      are pushed in reverse, so that they pop in seed order.
 *  R10 CSR rows hold their destinations in ascending order, duplicates kept.
 *  R11 PK randomisation: exclusive-or with a G(N, M) random graph drawn
 *      with replacement; on multigraphs a cell is kept when its total
 *      multiplicity is odd.
 */
#include "pgen_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11, Sec. 3.2 (the Philox S-box: two 32x32->64       */
/* multiplies per round, the high halves XORed with the other two words     */
/* and the round key; the key is bumped by the Weyl constants each round).  */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint64_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += weyl0;
            k1 += weyl1;
        }
        uint64_t p0 = mult0 * (uint64_t)x0;
        uint64_t p1 = mult1 * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void draw(uint64_t seed, uint64_t idx, uint32_t stream, uint32_t tag, uint32_t w[4])
{
    uint32_t c[4] = {(uint32_t)idx, (uint32_t)(idx >> 32), stream, tag};
    uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox4x32_10(c, k, w);
}

/* Uniform integer in [0, R): high half of the 128-bit product (R7). */
uint64_t or_uniform(uint32_t w0, uint32_t w1, uint64_t R)
{
    unsigned __int128 x = ((unsigned __int128)(((uint64_t)w1 << 32) | w0)) * R;
    return (uint64_t)(x >> 64);
}

/* Inter-faction coin threshold T_f (R6). */
uint64_t or_coin_threshold(double f)
{
    double t = nearbyint(ldexp(f, 32));
    if (!(t > 0.0)) return 0;
    if (t > 4294967295.0) return 4294967295u;
    return (uint64_t)t;
}

/* Seed clique K_{n0}: its e0 edges in lexicographic order (a < b). */
static uint64_t seed_edge_count(uint32_t n0) { return (uint64_t)n0 * (n0 - 1) / 2; }

static void seed_clique(uint32_t n0, uint32_t* ea, uint32_t* eb)
{
    uint64_t e = 0;
    for (uint32_t a = 0; a < n0; ++a)
        for (uint32_t b = a + 1; b < n0; ++b) {
            ea[e] = a;
            eb[e] = b;
            ++e;
        }
}

/* ------------------------------------------------------------------------ */
/* Serial BA with copy-edge preferential attachment (Sec. 3, PBA method:    */
/* degree-proportional choice done in O(1) by taking a uniform existing     */
/* edge and then a uniform end of it). An explicit endpoint array M         */
/* holds both endpoints of every edge made so far; a new edge copies M[r].  */
/* Draws use stream `stream` of tag 2, so blocks = 1 of the two-phase       */
/* method (whose only endpoint list is T_0) reproduces it exactly.          */
/* ------------------------------------------------------------------------ */
int or_ba(uint64_t n, uint32_t m, uint32_t n0, uint64_t seed, uint32_t stream, uint64_t* out)
{
    if (m < 1 || n0 < 2) return 1;
    uint64_t e0 = seed_edge_count(n0);
    uint64_t n_edges = e0 + n * m;
    uint64_t* M = (uint64_t*)malloc(sizeof(uint64_t) * 2 * (n_edges ? n_edges : 1));
    uint32_t* ea = (uint32_t*)malloc(sizeof(uint32_t) * e0);
    uint32_t* eb = (uint32_t*)malloc(sizeof(uint32_t) * e0);
    if (!M || !ea || !eb) { free(M); free(ea); free(eb); return 2; }
    seed_clique(n0, ea, eb);
    for (uint64_t e = 0; e < e0; ++e) {
        M[2 * e] = ea[e];
        M[2 * e + 1] = eb[e];
    }
    for (uint64_t i = 0; i < n; ++i) {
        /* slots available to every edge of vertex i: seed + earlier vertices */
        uint64_t slots = 2 * (e0 + i * m);
        for (uint32_t t = 0; t < m; ++t) {
            uint64_t j = i * m + t;
            uint32_t w[4];
            draw(seed, j, stream, 2, w);
            uint64_t r = or_uniform(w[0], w[1], slots);
            M[2 * (e0 + j)] = n0 + i;
            M[2 * (e0 + j) + 1] = M[r];
        }
    }
    memcpy(out, M, sizeof(uint64_t) * 2 * n_edges);
    free(M); free(ea); free(eb);
    return 0;
}

/* Count message of Sec. 3 (PBA method): how often each block occurs in A. */
int or_pba_count(const uint32_t* A, uint64_t len, uint32_t B, uint64_t* counts)
{
    memset(counts, 0, sizeof(uint64_t) * B);
    for (uint64_t j = 0; j < len; ++j) {
        if (A[j] >= B) return 1;
        counts[A[j]]++;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* PBA phase 1 for one block p (Sec. 3, PBA method, and Fig. 1(a)).         */
/* `flist` lists, in order, the members of every faction p belongs to (s    */
/* entries, duplicates allowed); the first s entries of A copy it. Each     */
/* later entry is, with probability f, a uniformly random block outside     */
/* all of p's factions (the inter-faction edges of Sec. 3), and otherwise   */
/* a copy of a uniformly chosen earlier entry of A (preferential            */
/* attachment over blocks).                                                 */
/* counts[q] (B entries, zeroed here) receives #{j : A[j] = q}.             */
/* ------------------------------------------------------------------------ */
int or_pba_phase1_general(uint32_t p, uint32_t B, const uint32_t* flist, uint32_t s,
                          uint64_t n_entries, double f, uint64_t seed,
                          uint32_t* A, uint64_t* counts, uint64_t* fresh_out)
{
    uint8_t* inside = (uint8_t*)calloc(B, 1);
    uint32_t* outside = (uint32_t*)malloc(sizeof(uint32_t) * (B ? B : 1));
    if (!inside || !outside) { free(inside); free(outside); return 2; }
    for (uint32_t t = 0; t < s; ++t) {
        if (flist[t] >= B) { free(inside); free(outside); return 1; }
        inside[flist[t]] = 1;
    }
    uint32_t n_out = 0;
    for (uint32_t b = 0; b < B; ++b)
        if (!inside[b]) outside[n_out++] = b;
    uint64_t Tf = or_coin_threshold(f);
    uint64_t fresh = 0;
    for (uint64_t j = 0; j < n_entries; ++j) {
        if (j < s) {
            A[j] = flist[j];
            continue;
        }
        uint32_t w[4];
        draw(seed, j, p, 1, w);
        if (n_out > 0 && (uint64_t)w[2] < Tf) {
            uint64_t x = ((uint64_t)w[3] * n_out) >> 32;
            A[j] = outside[x];
            ++fresh;
        } else {
            A[j] = A[or_uniform(w[0], w[1], j)];
        }
    }
    if (counts) or_pba_count(A, n_entries, B, counts);
    if (fresh_out) *fresh_out = fresh;
    free(inside); free(outside);
    return 0;
}

/* Phase 1 with the aligned faction layout of reading R5. */
int or_pba_phase1(uint32_t p, uint32_t B, uint32_t W, uint64_t n_entries, double f,
                  uint64_t seed, uint32_t* A, uint64_t* counts, uint64_t* fresh_out)
{
    if (W == 0 || B % W != 0 || p >= B) return 1;
    uint32_t* flist = (uint32_t*)malloc(sizeof(uint32_t) * W);
    if (!flist) return 2;
    uint32_t phi = (p / W) * W;
    for (uint32_t t = 0; t < W; ++t) flist[t] = phi + t;
    int rc = or_pba_phase1_general(p, B, flist, W, n_entries, f, seed, A, counts, fresh_out);
    free(flist);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* PBA phase 2 endpoint list of block q (Sec. 3, PBA method: q picks the    */
/* requested endpoints among its own vertices by ordinary preferential      */
/* attachment; reading R3). A local endpoint array                          */
/* holds the local seed clique (ids 0..n0-1) and every local edge made so   */
/* far (source id n0 + sigma(i)); edge i copies a uniform slot among the    */
/* seed and the edges of strictly earlier source times. T[i] is that copied */
/* local id. Only the first `len` entries (len <= R_q) are produced.        */
/* ------------------------------------------------------------------------ */
int or_pba_endpoints(uint32_t q, uint64_t R_q, uint64_t n_b, uint32_t n0, uint64_t seed,
                     uint64_t len, uint32_t* T)
{
    if (n0 < 2 || len > R_q || (R_q > 0 && n_b == 0)) return 1;
    uint64_t e0 = seed_edge_count(n0);
    uint64_t* M = (uint64_t*)malloc(sizeof(uint64_t) * 2 * (e0 + len + 1));
    uint32_t* ea = (uint32_t*)malloc(sizeof(uint32_t) * e0);
    uint32_t* eb = (uint32_t*)malloc(sizeof(uint32_t) * e0);
    if (!M || !ea || !eb) { free(M); free(ea); free(eb); return 2; }
    seed_clique(n0, ea, eb);
    for (uint64_t e = 0; e < e0; ++e) {
        M[2 * e] = ea[e];
        M[2 * e + 1] = eb[e];
    }
    for (uint64_t i = 0; i < len; ++i) {
        uint64_t sigma = (uint64_t)(((unsigned __int128)i * n_b) / R_q);
        /* number of local edges whose source time is before sigma */
        unsigned __int128 num = (unsigned __int128)sigma * R_q;
        uint64_t before = (uint64_t)((num + n_b - 1) / n_b);
        uint32_t w[4];
        draw(seed, i, q, 2, w);
        uint64_t r = or_uniform(w[0], w[1], 2 * (e0 + before));
        M[2 * (e0 + i)] = n0 + sigma;
        M[2 * (e0 + i) + 1] = M[r];
        T[i] = (uint32_t)M[r];
    }
    free(M); free(ea); free(eb);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Substitution (Sec. 3, PBA method, Fig. 1(b)): each occurrence of block q */
/* in A, in index order, takes the next endpoint of the slice of q's list   */
/* that q sent to this requester. start[q] is where that slice begins in    */
/* T_q (reading R4). out[j] = T_{A[j]}[start[A[j]] + #earlier j' with the   */
/* same block].                                                             */
/* ------------------------------------------------------------------------ */
int or_pba_substitute(const uint32_t* A, uint64_t len, uint32_t B, const uint64_t* start,
                      const uint32_t* const* T, uint32_t* out)
{
    uint64_t* cursor = (uint64_t*)malloc(sizeof(uint64_t) * (B ? B : 1));
    if (!cursor) return 2;
    for (uint32_t q = 0; q < B; ++q) cursor[q] = start[q];
    for (uint64_t j = 0; j < len; ++j) {
        uint32_t q = A[j];
        if (q >= B) { free(cursor); return 1; }
        out[j] = T[q][cursor[q]++];
    }
    free(cursor);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Full two-phase PBA (Sec. 3, PBA method), blocks processed one after the  */
/* other exactly as the text orders the steps: phase 1 on every block, the  */
/* count exchange, phase 2 endpoint lists, then substitution. Output: for   */
/* each block p in turn, its e0 seed-clique edges then its n_b*m edges in  */
/* entry order, as (src, dst) uint64 pairs. Vertex ids: block b owns ids    */
/* b*(n0+n_b) .. b*(n0+n_b)+n0+n_b-1; its seed clique is the first n0.      */
/* counts_out (B*B, row p = requester) and fresh_out may be NULL.           */
/* ------------------------------------------------------------------------ */
/* Two-phase PBA with explicit faction lists (Sec. 3, PBA method; Fig. 1):   */
/* block p's list is flist[foff[p] .. foff[p+1]), the members of every       */
/* faction p belongs to, in order (at least one entry, each < B).            */
int or_pba_factions(uint64_t n, uint32_t m, uint32_t B, uint32_t n0, const uint32_t* foff,
                    const uint32_t* flist, double f, uint64_t seed, uint64_t* out,
                    uint64_t* counts_out, uint64_t* fresh_out)
{
    if (m < 1 || n0 < 2 || B < 1 || n % B != 0) return 1;
    if (!(f >= 0.0 && f <= 1.0)) return 1;
    for (uint32_t p = 0; p < B; ++p)
        if (foff[p + 1] <= foff[p]) return 1;
    uint64_t n_b = n / B;
    uint64_t N_e = n_b * m;
    uint64_t e0 = seed_edge_count(n0);
    uint64_t id_span = n0 + n_b;
    int rc = 0;

    uint32_t* A = (uint32_t*)malloc(sizeof(uint32_t) * (N_e * B + 1));
    uint64_t* c = (uint64_t*)calloc((size_t)B * B, sizeof(uint64_t));
    uint64_t* R = (uint64_t*)calloc(B, sizeof(uint64_t));
    uint64_t* start = (uint64_t*)malloc(sizeof(uint64_t) * B);
    uint32_t** T = (uint32_t**)calloc(B, sizeof(uint32_t*));
    uint32_t* dst = (uint32_t*)malloc(sizeof(uint32_t) * (N_e + 1));
    uint32_t* ea = (uint32_t*)malloc(sizeof(uint32_t) * e0);
    uint32_t* eb = (uint32_t*)malloc(sizeof(uint32_t) * e0);
    if (!A || !c || !R || !start || !T || !dst || !ea || !eb) { rc = 2; goto done; }
    seed_clique(n0, ea, eb);

    /* phase 1 on every block; p tells q how often q occurs in A_p */
    uint64_t fresh_total = 0;
    for (uint32_t p = 0; p < B; ++p) {
        uint64_t fr = 0;
        rc = or_pba_phase1_general(p, B, flist + foff[p], foff[p + 1] - foff[p], N_e, f, seed,
                                   A + (uint64_t)p * N_e, c + (uint64_t)p * B, &fr);
        if (rc) goto done;
        fresh_total += fr;
    }
    /* each q receives the counts and totals them */
    for (uint32_t p = 0; p < B; ++p)
        for (uint32_t q = 0; q < B; ++q) R[q] += c[(uint64_t)p * B + q];
    /* phase 2: each q builds its list of R_q local endpoints */
    for (uint32_t q = 0; q < B; ++q) {
        T[q] = (uint32_t*)malloc(sizeof(uint32_t) * (R[q] + 1));
        if (!T[q]) { rc = 2; goto done; }
        rc = or_pba_endpoints(q, R[q], n_b, n0, seed, R[q], T[q]);
        if (rc) goto done;
    }
    /* substitution on each requester p, slices handed out in ascending p */
    for (uint32_t q = 0; q < B; ++q) start[q] = 0;
    for (uint32_t p = 0; p < B; ++p) {
        const uint32_t* Ap = A + (uint64_t)p * N_e;
        rc = or_pba_substitute(Ap, N_e, B, start, (const uint32_t* const*)T, dst);
        if (rc) goto done;
        for (uint32_t q = 0; q < B; ++q) start[q] += c[(uint64_t)p * B + q];
        uint64_t base_p = (uint64_t)p * id_span;
        uint64_t* o = out + 2 * (uint64_t)p * (e0 + N_e);
        for (uint64_t e = 0; e < e0; ++e) {
            o[2 * e] = base_p + ea[e];
            o[2 * e + 1] = base_p + eb[e];
        }
        o += 2 * e0;
        for (uint64_t j = 0; j < N_e; ++j) {
            o[2 * j] = base_p + n0 + j / m;
            o[2 * j + 1] = (uint64_t)Ap[j] * id_span + dst[j];
        }
    }
    if (counts_out) memcpy(counts_out, c, sizeof(uint64_t) * B * B);
    if (fresh_out) *fresh_out = fresh_total;
done:
    if (T)
        for (uint32_t q = 0; q < B; ++q) free(T[q]);
    free(A); free(c); free(R); free(start); free(T); free(dst); free(ea); free(eb);
    return rc;
}

/* Aligned factions of width W (reading R5): block p's list is the W blocks */
/* of its group, phi = (p div W)*W, ..., phi + W - 1.                       */
int or_pba(uint64_t n, uint32_t m, uint32_t B, uint32_t n0, uint32_t W, double f,
           uint64_t seed, uint64_t* out, uint64_t* counts_out, uint64_t* fresh_out)
{
    if (B < 1 || W < 1 || B % W != 0) return 1;
    uint32_t* foff = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)B + 1));
    uint32_t* flist = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)B * W);
    if (!foff || !flist) { free(foff); free(flist); return 2; }
    for (uint32_t p = 0; p < B; ++p) {
        foff[p] = p * W;
        for (uint32_t t = 0; t < W; ++t) flist[(size_t)p * W + t] = (p / W) * W + t;
    }
    foff[B] = B * W;
    int rc = or_pba_factions(n, m, B, n0, foff, flist, f, seed, out, counts_out, fresh_out);
    free(foff); free(flist);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Kronecker initiator quantiser (reading R8). T has n0*n0 - 1 entries,     */
/* each in [0, 2^32]. Returns 1 on a bad initiator (negative, non-finite,   */
/* or zero sum).                                                            */
/* ------------------------------------------------------------------------ */
int or_kron_thresholds(const double* P, uint32_t n0, uint64_t* T)
{
    if (n0 < 1) return 1;
    uint32_t cells = n0 * n0;
    double S = 0.0;
    for (uint32_t c = 0; c < cells; ++c) {
        if (!(P[c] >= 0.0) || !isfinite(P[c])) return 1;
        S += P[c];
    }
    if (!(S > 0.0) || !isfinite(S)) return 1;
    double cum = 0.0;
    for (uint32_t c = 0; c + 1 < cells; ++c) {
        cum += P[c];
        T[c] = (uint64_t)nearbyint(ldexp(cum / S, 32));
    }
    return 0;
}

/* Cell picked by one 32-bit word: #{c : w >= T_c} (reading R8). */
uint32_t or_kron_pick(const uint64_t* T, uint32_t n_thr, uint32_t w)
{
    uint32_t cell = 0;
    for (uint32_t c = 0; c < n_thr; ++c)
        if ((uint64_t)w >= T[c]) cell++;
    return cell;
}

/* ------------------------------------------------------------------------ */
/* Stochastic Kronecker edges (Sec. 2 model of Leskovec et al., as cited in */
/* Sec. 3, PK method): every edge descends k levels; at each level it falls */
/* into one initiator cell (a, b) with the cell's probability, and the      */
/* vertex ids grow by one base-n0 digit (row a, column b) per level, most   */
/* significant first. Duplicates and self-loops are kept.                   */
/* ------------------------------------------------------------------------ */
int or_kron(const double* P, uint32_t n0, uint32_t k, uint64_t M, uint64_t seed, uint64_t* out)
{
    if (n0 < 1 || k < 1) return 1;
    uint32_t cells = n0 * n0;
    uint64_t* T = (uint64_t*)malloc(sizeof(uint64_t) * cells);
    if (!T) return 2;
    if (or_kron_thresholds(P, n0, T)) { free(T); return 1; }
    for (uint64_t e = 0; e < M; ++e) {
        uint64_t row = 0, col = 0;
        uint32_t w[4];
        for (uint32_t l = 0; l < k; ++l) {
            if (l % 4 == 0) draw(seed, e, l / 4, 3, w);
            uint32_t cell = or_kron_pick(T, cells - 1, w[l % 4]);
            row = row * n0 + cell / n0;
            col = col * n0 + cell % n0;
        }
        out[2 * e] = row;
        out[2 * e + 1] = col;
    }
    free(T);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Deterministic Kronecker graph by meta-edge expansion with a stack (Sec.  */
/* 3, PK method): the stack starts with the seed edges (the nonzero cells   */
/* of the initiator, row-major) as meta-edges of iteration 1; a popped      */
/* meta-edge of the final iteration k is output, any other one is replaced  */
/* by its n0 x n0 block copy of the seed (one child per seed edge). Children */
/* are pushed in reverse so that they pop in seed order. The stack never    */
/* holds more than k*(e0-1)+1 meta-edges; *max_depth_out reports the peak.  */
/* Returns 3 when e0^k exceeds cap.                                         */
/* ------------------------------------------------------------------------ */
int or_kron_det(const double* P, uint32_t n0, uint32_t k, uint64_t* out, uint64_t cap,
                uint64_t* n_out, uint64_t* max_depth_out)
{
    if (n0 < 1 || k < 1) return 1;
    uint32_t cells = n0 * n0;
    uint32_t* sa = (uint32_t*)malloc(sizeof(uint32_t) * cells);
    uint32_t* sb = (uint32_t*)malloc(sizeof(uint32_t) * cells);
    if (!sa || !sb) { free(sa); free(sb); return 2; }
    uint32_t e0 = 0;
    for (uint32_t c = 0; c < cells; ++c)
        if (P[c] > 0.0) {
            sa[e0] = c / n0;
            sb[e0] = c % n0;
            ++e0;
        }
    if (e0 == 0) { free(sa); free(sb); return 1; }
    uint64_t total = 1;
    for (uint32_t l = 0; l < k; ++l) {
        if (total > cap / e0) { free(sa); free(sb); return 3; }
        total *= e0;
    }

    uint64_t stack_cap = (uint64_t)k * e0 + 1;
    uint64_t* st_row = (uint64_t*)malloc(sizeof(uint64_t) * stack_cap);
    uint64_t* st_col = (uint64_t*)malloc(sizeof(uint64_t) * stack_cap);
    uint32_t* st_it = (uint32_t*)malloc(sizeof(uint32_t) * stack_cap);
    if (!st_row || !st_col || !st_it) {
        free(sa); free(sb); free(st_row); free(st_col); free(st_it);
        return 2;
    }
    uint64_t top = 0, peak = 0, emitted = 0;
    for (uint32_t t = e0; t-- > 0;) {
        st_row[top] = sa[t];
        st_col[top] = sb[t];
        st_it[top] = 1;
        ++top;
    }
    peak = top;
    while (top > 0) {
        --top;
        uint64_t r = st_row[top], c = st_col[top];
        uint32_t it = st_it[top];
        if (it == k) {
            out[2 * emitted] = r;
            out[2 * emitted + 1] = c;
            ++emitted;
            continue;
        }
        for (uint32_t t = e0; t-- > 0;) {
            st_row[top] = r * n0 + sa[t];
            st_col[top] = c * n0 + sb[t];
            st_it[top] = it + 1;
            ++top;
        }
        if (top > peak) peak = top;
    }
    *n_out = emitted;
    if (max_depth_out) *max_depth_out = peak;
    free(sa); free(sb); free(st_row); free(st_col); free(st_it);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* CSR of an edge list (not in the paper; reading R10): sort the (src, dst) */
/* pairs, then row_ptr[v] = number of edges with src < v.                   */
/* ------------------------------------------------------------------------ */
static int cmp_pair(const void* a, const void* b)
{
    const uint64_t* x = (const uint64_t*)a;
    const uint64_t* y = (const uint64_t*)b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    if (x[1] != y[1]) return x[1] < y[1] ? -1 : 1;
    return 0;
}

/* CSR with options (not in the paper; reading R11). The list is the M pairs,
 * plus (dst, src) for each when OR_CSR_SYMMETRIZE; self-loops are dropped
 * when OR_CSR_NO_LOOPS; after sorting, OR_CSR_DEDUP keeps one copy of each
 * distinct pair and OR_CSR_ODD keeps one copy of each pair that occurs an
 * odd number of times (the exclusive-or of adjacency matrices, Sec. 3 PK
 * randomisation). *M_out receives the number of col entries.             */
#define OR_CSR_SYMMETRIZE 1u
#define OR_CSR_DEDUP 2u
#define OR_CSR_NO_LOOPS 4u
#define OR_CSR_ODD 8u

int or_csr_opts(const uint64_t* pairs, uint64_t M, uint64_t N, uint32_t flags, uint64_t* row_ptr,
                uint64_t* col, uint64_t* M_out)
{
    uint64_t cap = (flags & OR_CSR_SYMMETRIZE) ? 2 * M : M;
    uint64_t* s = (uint64_t*)malloc(sizeof(uint64_t) * 2 * (cap ? cap : 1));
    if (!s) return 2;
    uint64_t n = 0;
    for (uint64_t e = 0; e < M; ++e) {
        uint64_t a = pairs[2 * e], b = pairs[2 * e + 1];
        if (a >= N || b >= N) { free(s); return 1; }
        if ((flags & OR_CSR_NO_LOOPS) && a == b) continue;
        s[2 * n] = a; s[2 * n + 1] = b; ++n;
        if (flags & OR_CSR_SYMMETRIZE) { s[2 * n] = b; s[2 * n + 1] = a; ++n; }
    }
    qsort(s, n, 2 * sizeof(uint64_t), cmp_pair);
    uint64_t k = 0;
    for (uint64_t i = 0; i < n;) {
        uint64_t j = i + 1;
        while (j < n && s[2 * j] == s[2 * i] && s[2 * j + 1] == s[2 * i + 1]) ++j;
        uint64_t copies = j - i;
        if (flags & OR_CSR_ODD) copies = (j - i) & 1;
        else if (flags & OR_CSR_DEDUP) copies = 1;
        for (uint64_t c = 0; c < copies; ++c) {
            s[2 * k] = s[2 * i]; s[2 * k + 1] = s[2 * i + 1]; ++k;
        }
        i = j;
    }
    for (uint64_t v = 0; v <= N; ++v) row_ptr[v] = 0;
    for (uint64_t e = 0; e < k; ++e) row_ptr[s[2 * e] + 1]++;
    for (uint64_t v = 0; v < N; ++v) row_ptr[v + 1] += row_ptr[v];
    for (uint64_t e = 0; e < k; ++e) col[e] = s[2 * e + 1];
    *M_out = k;
    free(s);
    return 0;
}

/* Random graph G(N, M) with replacement (reading R11): edge e is the cell */
/* (uniform over N from (w1:w0), uniform over N from (w3:w2)) of the draw  */
/* with counter (e_lo, e_hi, 0, 4).                                        */
int or_random_cells(uint64_t N, uint64_t M, uint64_t seed, uint64_t* out)
{
    if (N == 0 && M > 0) return 1;
    for (uint64_t e = 0; e < M; ++e) {
        uint32_t w[4];
        draw(seed, e, 0, 4, w);
        out[2 * e] = or_uniform(w[0], w[1], N);
        out[2 * e + 1] = or_uniform(w[2], w[3], N);
    }
    return 0;
}

int or_csr(const uint64_t* pairs, uint64_t M, uint64_t N, uint64_t* row_ptr, uint64_t* col)
{
    uint64_t* s = (uint64_t*)malloc(sizeof(uint64_t) * 2 * (M ? M : 1));
    if (!s) return 2;
    memcpy(s, pairs, sizeof(uint64_t) * 2 * M);
    for (uint64_t e = 0; e < M; ++e)
        if (s[2 * e] >= N) { free(s); return 1; }
    qsort(s, M, 2 * sizeof(uint64_t), cmp_pair);
    for (uint64_t v = 0; v <= N; ++v) row_ptr[v] = 0;
    for (uint64_t e = 0; e < M; ++e) row_ptr[s[2 * e] + 1]++;
    for (uint64_t v = 0; v < N; ++v) row_ptr[v + 1] += row_ptr[v];
    for (uint64_t e = 0; e < M; ++e) col[e] = s[2 * e + 1];
    free(s);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Graph properties (Sec. 4 examines degree distributions and path lengths). */
/* which: 0 = out (src), 1 = in (dst), 2 = both ends counted.               */
/* ------------------------------------------------------------------------ */
int or_degrees(const uint64_t* pairs, uint64_t M, uint64_t N, int which, uint64_t* deg)
{
    if (which < 0 || which > 2) return 1;
    for (uint64_t v = 0; v < N; ++v) deg[v] = 0;
    for (uint64_t e = 0; e < M; ++e) {
        uint64_t a = pairs[2 * e], b = pairs[2 * e + 1];
        if (which != 1 && a < N) deg[a]++;
        if (which != 0 && b < N) deg[b]++;
    }
    return 0;
}

int or_degree_histogram(const uint64_t* deg, uint64_t N, uint64_t max_deg, uint64_t* hist)
{
    for (uint64_t d = 0; d < max_deg + 2; ++d) hist[d] = 0;
    for (uint64_t v = 0; v < N; ++v) hist[deg[v] <= max_deg ? deg[v] : max_deg + 1]++;
    return 0;
}

/* Breadth-first search with an explicit FIFO queue; dist = UINT32_MAX where */
/* unreached. *levels = 1 + the largest distance; *scanned = the sum of the  */
/* row lengths of the reached vertices.                                      */
int or_bfs(const uint64_t* row_ptr, const uint64_t* col, uint64_t N, uint64_t source,
           uint32_t* dist, uint32_t* levels, uint64_t* scanned)
{
    if (source >= N) return 1;
    uint64_t* queue = (uint64_t*)malloc(sizeof(uint64_t) * (N ? N : 1));
    if (!queue) return 2;
    for (uint64_t v = 0; v < N; ++v) dist[v] = 0xFFFFFFFFu;
    uint64_t head = 0, tail = 0, sc = 0;
    uint32_t deepest = 0;
    dist[source] = 0;
    queue[tail++] = source;
    while (head < tail) {
        uint64_t v = queue[head++];
        sc += row_ptr[v + 1] - row_ptr[v];
        if (dist[v] > deepest) deepest = dist[v];
        for (uint64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            uint64_t u = col[e];
            if (u < N && dist[u] == 0xFFFFFFFFu) {
                dist[u] = dist[v] + 1;
                queue[tail++] = u;
            }
        }
    }
    *levels = deepest + 1;
    *scanned = sc;
    free(queue);
    return 0;
}

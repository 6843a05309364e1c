/*
 * pgen -- GB300-native generation of massive scale-free graphs.
 *
 * C ABI of the CUDA library libpgen.so (sm_103a). It implements the two
 * generators of Yoo & Henderson, "Parallel Generation of Massive Scale-Free
 * Graphs" (arXiv 1003.3684): the parallel Barabasi-Albert method with
 * two-phase preferential attachment (Sec. 3, PBA method, Fig. 1) and the
 * Kronecker method (Sec. 3, PK method, Fig. 2; stochastic initiator of the
 * Kronecker model cited in Sec. 2, and its randomisation by exclusive-or with
 * a random graph), with general faction lists and generation in parts; plus
 * CSR assembly, batched launch and the graph checks of Sec. 4 (degrees,
 * degree histogram, breadth-first distances).
 *
 * Conventions shared by every entry point:
 *  - Pointers named d_* are DEVICE pointers on the current CUDA device; h_*
 *    are host pointers. The caller owns every buffer; the library allocates
 *    no device memory (scratch comes from the caller's workspace d_ws; the
 *    one exception, gen_pba_noalloc, uses a fixed array compiled into the
 *    library).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Calls only enqueue work and do not synchronise the stream,
 *    except pg_bfs, which waits once per search level (see there). Outputs
 *    written through h_* pointers are computed from the arguments on the
 *    host before any launch and are valid on return.
 *  - Arguments are validated on the host before anything is launched; an
 *    invalid call launches nothing and returns PG_EINVAL (bad value),
 *    PG_ENOSPC (output capacity too small) or PG_ENOMEM (workspace too
 *    small). PG_ECUDA reports a failed launch (cudaGetLastError).
 *  - Vertex ids are written as (src, dst) pairs, interleaved: uint32 pairs
 *    for PG_ID32, uint64 pairs for PG_ID64. Output edge buffers must be
 *    16-byte aligned (inputs to edges_to_csr: aligned to one pair).
 *  - Every random draw is Philox4x32-10 (Salmon et al., SC'11) with key
 *    (seed & 0xffffffff, seed >> 32) and a counter that names the draw, so
 *    the output is a pure function of the arguments.
 */
#ifndef PGEN_H
#define PGEN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PG_OK = 0,
    PG_EINVAL = 1,   /* invalid argument (nothing launched) */
    PG_ENOSPC = 2,   /* output capacity smaller than the edge count */
    PG_ECUDA = 3,    /* a CUDA launch or API call failed */
    PG_ETIMEOUT = 4, /* a bounded device-side wait gave up */
    PG_ENOMEM = 5    /* workspace smaller than the size the library asks for */
} pg_status;

typedef enum { PG_ID32 = 0, PG_ID64 = 1 } pg_idwidth;

typedef enum { PG_KRON_STOCHASTIC = 0, PG_KRON_DETERMINISTIC = 1 } pg_kron_mode;

/* Human-readable name of a status code (static string; library plumbing, not
 * part of the method). */
const char* pg_status_string(pg_status s);

/* Number of SMs and library version, for logging (not part of the method). */
int pg_device_sm_count(void);
const char* pg_version(void);

/* Test hook (not part of the method): with on != 0, gen_pba, gen_pba_factions,
 * pg_pba_prepare / gen_pba_blocks, gen_pba_to_host and gen_pba_noalloc use the
 * 64-bit-index variants of their kernels for every input. Those variants
 * otherwise run only when a block's phase-2 list plus its seed edges reach
 * 2^32 entries (or, for blocks = 1, n*m + e0 >= 2^32). The output is the same
 * either way; the switch lets parity tests check the 64-bit arithmetic on
 * graphs small enough for the oracle. Process-wide and read at each launch;
 * a prepared workspace keeps the choice made when it was prepared (after the
 * switch has once been on, emits also launch the 64-bit variant, which exits
 * at once for workspaces prepared without it). Default off; cannot fail. */
void pg_force_wide_path(int on);

/* Test hook (not part of the method; host only, no GPU needed): exercises the
 * bookkeeping that sets kernel attributes once per device. `threads` host
 * threads (1..64) each run the device ids devs[0..n) in order through one
 * shared instance, whose set-up step counts its calls per device and fails
 * for device fail_dev (-1: never). Writes calls[d] (64 ints) = number of
 * set-up calls for device d, and status[i] (n ints) = the cudaError_t that
 * thread 0 got for devs[i] (ids outside 0..63 fail). Returns PG_EINVAL for
 * bad arguments, else PG_OK. */
int pg_test_per_device_once(const int* devs, int n, int threads, int fail_dev, int* calls,
                            int* status);

/* Throughput probe (not part of the method): launches one kernel in which
 * each of pg_philox_probe_threads() threads (8 CTAs of 256 per SM) makes
 * calls_per_thread Philox4x32-10 calls and writes one folded word to
 * d_out[thread] (out_words >= pg_philox_probe_threads()). Time it with
 * events on `stream`: threads * calls / seconds is the device's Philox rate,
 * the measured ceiling of the integer-bound kernels. */
size_t pg_philox_probe_threads(void);
pg_status pg_philox_probe(uint32_t calls_per_thread, uint32_t* d_out, size_t out_words,
                          void* stream);
/* Integer pipe probe: same launch shape; each thread runs 8 independent
 * chains of `iters` operations of one kind (op 0: 32x32->64 multiply, 1:
 * 32-bit multiply-add, 2: three-input logic x ^ (y & z), 3: three-input add), so
 * threads * 8 * iters / seconds is the device's rate for that operation. */
pg_status pg_int_probe(int op, uint32_t iters, uint32_t* d_out, size_t out_words, void* stream);

/* ------------------------------------------------------------------------
 * Parallel Barabasi-Albert generator (Sec. 3, PBA method; Fig. 1).
 *
 * n              new vertices in total (n % blocks == 0); n_b = n / blocks.
 * m              edges added per new vertex (>= 1).
 * blocks         B, the number of vertex blocks (the paper's processors),
 *                1 <= B <= 1024.
 * n0             size of each block's seed clique K_{n0} (>= 2).
 * faction_width  W: blocks form aligned factions of W consecutive blocks
 *                (B % W == 0); the first W entries of a block's phase-1
 *                list are its faction's blocks, in order.
 * inter_frac     f in [0, 1]: per later phase-1 entry, the probability of
 *                an inter-faction pick (uniform over blocks outside the
 *                faction); otherwise the entry copies a uniform earlier
 *                entry (preferential attachment over blocks).
 * seed           Philox key.
 *
 * Phase 1 draws use counter (j_lo, j_hi, p, 1) for entry j of block p;
 * phase 2 draws use (i_lo, i_hi, q, 2) for local edge i of block q. Block q
 * builds its R_q requested endpoints by preferential attachment over its
 * own vertices, the i-th edge standing at source time floor(i*n_b/R_q);
 * requesters receive slices of that list in ascending block order and
 * substitute them in entry order.
 *
 * Vertex ids: block b owns ids b*(n0+n_b) .. b*(n0+n_b)+n0+n_b-1; the first
 * n0 are its seed clique. Output: for each block p in order, its
 * e0 = n0(n0-1)/2 seed edges (lexicographic) then its n_b*m new edges in
 * entry order (src = the new vertex, dst = the attached vertex).
 * Edge count = B*(e0 + n_b*m); blocks = 1 is serial BA on ids 0..n0+n-1.
 *
 * d_edges/cap_edges  output buffer and its capacity in edges.
 * n_edges_out        (host, may be NULL) receives the edge count.
 * d_ws/ws_bytes      device workspace of at least pg_pba_workspace_size()
 *                    bytes, 256-byte aligned (unused when blocks == 1).
 * ---------------------------------------------------------------------- */
uint64_t pg_pba_edge_count(uint64_t n, uint32_t m, uint32_t blocks, uint32_t n0);
size_t pg_pba_workspace_size(uint64_t n, uint32_t m, uint32_t blocks);
pg_status gen_pba(uint64_t n, uint32_t m, uint32_t blocks, uint32_t n0, uint32_t faction_width,
                  double inter_frac, uint64_t seed, pg_idwidth w, void* d_edges,
                  uint64_t cap_edges, uint64_t* n_edges_out, void* d_ws, size_t ws_bytes,
                  void* stream);

/* gen_pba (Sec. 3, PBA method), and a copy of the edge list into host memory
 * h_edges (pinned, B*(e0+n_b*m) pairs; the paper has no counterpart, as it
 * excludes writing the graph out from its timings). The copy of each range
 * of blocks starts on a second, library-owned stream as soon as that range
 * is written, so the transfer overlaps generation. `stream` waits for the
 * last copy, so synchronising `stream` covers both. d_edges still receives
 * the full edge list. */
pg_status gen_pba_to_host(uint64_t n, uint32_t m, uint32_t blocks, uint32_t n0,
                          uint32_t faction_width, double inter_frac, uint64_t seed, pg_idwidth w,
                          void* h_edges, void* d_edges, uint64_t cap_edges, uint64_t* n_edges_out,
                          void* d_ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * PBA with general faction lists (Sec. 3, PBA method: a block's factions
 * need not be aligned groups and may overlap, as F0..F2 of Fig. 1).
 *
 * pg_pba_faction_table (host only, no CUDA call) packs the lists into the
 * device layout: block p's list is h_members[h_offsets[p] .. h_offsets[p+1])
 * (blocks + 1 offsets), the members of every faction p belongs to, in
 * order: 1 to 1024 entries, each < blocks, repeats allowed. h_table
 * receives pg_pba_faction_table_size(blocks) bytes (one 4112-byte record
 * per block: list size, size of the complement, the list, and the blocks
 * outside the list in ascending order). PG_EINVAL for a bad list, PG_ENOSPC
 * when table_bytes is too small. The caller copies the table to device
 * memory (16-byte aligned) by any means it likes.
 *
 * gen_pba_factions is gen_pba with that table in place of faction_width:
 * entry t < s_p of block p's phase-1 list is the t-th entry of p's list;
 * a later entry is, with probability inter_frac, the x-th block outside
 * p's list (x = floor(w3 * (blocks outside) / 2^32)), otherwise a copy of
 * a uniform earlier entry. A block whose list names every block makes no
 * inter-faction picks. Aligned width-W lists give gen_pba's output exactly.
 * Same workspace, output layout and vertex ids as gen_pba; blocks = 1 is
 * serial BA (the only possible list names block 0).
 * ---------------------------------------------------------------------- */
size_t pg_pba_faction_table_size(uint32_t blocks);
pg_status pg_pba_faction_table(uint32_t blocks, const uint32_t* h_offsets,
                               const uint32_t* h_members, void* h_table, size_t table_bytes);
pg_status gen_pba_factions(uint64_t n, uint32_t m, uint32_t blocks, uint32_t n0,
                           const void* d_faction_table, double inter_frac, uint64_t seed,
                           pg_idwidth w, void* d_edges, uint64_t cap_edges,
                           uint64_t* n_edges_out, void* d_ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * PBA in parts: the edges of any range of blocks, on demand (the paper has
 * no counterpart; it excludes writing the graph out from its timings).
 *
 * pg_pba_prepare runs phase 1, the count exchange and its scan, and leaves
 * their results in d_ws (pg_pba_workspace_size bytes). Factions: aligned
 * width faction_width, or the device table of gen_pba_factions when
 * d_faction_table is not NULL (faction_width is then ignored).
 * gen_pba_blocks then writes the edges of blocks [b_begin, b_end), block
 * b_begin's first edge at d_edges[0]: (b_end - b_begin) * (e0 + n_b*m)
 * edges, each equal to the same edge of gen_pba / gen_pba_factions with
 * the same arguments. It reads the workspace only, so any number of ranges
 * may follow one prepare -- in any order, into buffers much smaller than
 * the whole graph (stream a graph to host or disk range by range, or
 * regenerate a lost range after a restart from the arguments alone). The
 * workspace must not change between the two calls; n, m, blocks, n0 and
 * seed must match. blocks = 1 (serial BA) needs no prepare: the only range
 * is [0, 1).
 * ---------------------------------------------------------------------- */
pg_status pg_pba_prepare(uint64_t n, uint32_t m, uint32_t blocks, uint32_t n0,
                         uint32_t faction_width, const void* d_faction_table, double inter_frac,
                         uint64_t seed, void* d_ws, size_t ws_bytes, void* stream);
pg_status gen_pba_blocks(uint64_t n, uint32_t m, uint32_t blocks, uint32_t n0, uint64_t seed,
                         pg_idwidth w, uint32_t b_begin, uint32_t b_end, void* d_edges,
                         uint64_t cap_edges, uint64_t* n_edges_out, const void* d_ws,
                         size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * gen_pba without a caller-supplied workspace (the paper has no
 * counterpart; this is a library convenience).
 *
 * For callers that cannot allocate device memory: code inside a host
 * application whose allocator owns the whole device and forbids outside
 * cudaMalloc calls, plugins handed device buffers but no allocation API, and
 * latency-critical paths that must avoid cudaMalloc/cudaFree and the
 * device-wide synchronisation they cause. Same arguments and output as
 * gen_pba, minus d_ws/ws_bytes; the library allocates nothing.
 *
 * Scratch: a fixed device array of pg_pba_noalloc_scratch_bytes() (32 MiB)
 * compiled into the library, held by every GPU that loads it until the
 * process exits. A graph whose workspace (pg_pba_workspace_size) exceeds it
 * is rejected with PG_ENOMEM before anything is launched; blocks = 1 needs
 * no scratch. The first call on each device looks up the array's device
 * address (once per device, with that device current); make that first call
 * before any stream capture. All calls share the one array: calls whose work
 * overlaps on the GPU (other streams, or other host threads) race and give
 * wrong results, so order them on one stream. Each call clears what must
 * start at zero.
 * ---------------------------------------------------------------------- */
size_t pg_pba_noalloc_scratch_bytes(void);
pg_status gen_pba_noalloc(uint64_t n, uint32_t m, uint32_t blocks, uint32_t n0,
                          uint32_t faction_width, double inter_frac, uint64_t seed, pg_idwidth w,
                          void* d_edges, uint64_t cap_edges, uint64_t* n_edges_out, void* stream);

/* ------------------------------------------------------------------------
 * Kronecker generator (Sec. 3, PK method; Fig. 2).
 *
 * h_initiator  host, n0*n0 doubles, row-major, all >= 0 with a positive sum.
 * n0           initiator order: 1 <= n0 <= 16 (stochastic) or 1 <= n0 <= 256
 *              with at most 8192 nonzero cells (deterministic). The graph
 *              has n0^k vertices.
 * k            number of Kronecker levels, 1 <= k <= 64.
 * mode PG_KRON_STOCHASTIC: n_edges edges, each drawn independently by a
 *   k-level descent (most significant level first). Cell c of the
 *   initiator is chosen at a level when the level's 32-bit word w
 *   satisfies T_{c-1} <= w < T_c, where T_c = round_half_even(2^32 *
 *   (sum of cells 0..c) / (sum of all cells)), sums taken left to right in
 *   double. Level l uses word (l mod 4) of the draw with counter
 *   (e_lo, e_hi, l div 4, 3). Duplicates and self-loops are kept.
 * mode PG_KRON_DETERMINISTIC: the nonzero cells are the seed graph's e0
 *   edges (row-major); the output is all e0^k edges of the k-th Kronecker
 *   power in meta-edge stack order (edge index written in base e0, most
 *   significant digit = the seed edge chosen at the first expansion).
 *   n_edges is ignored.
 * Ids must fit the id width (n0^k <= 2^32 for PG_ID32).
 * ---------------------------------------------------------------------- */
uint64_t pg_kron_edge_count(const double* h_initiator, uint32_t n0, uint32_t k,
                            uint64_t n_edges, pg_kron_mode mode);
pg_status gen_kronecker(const double* h_initiator, uint32_t n0, uint32_t k, uint64_t n_edges,
                        uint64_t seed, pg_kron_mode mode, pg_idwidth w, void* d_edges,
                        uint64_t cap_edges, uint64_t* n_edges_out, void* stream);

/* Edges [e_begin, e_end) of the graph gen_kronecker (Sec. 3, PK method)
 * makes with the same arguments (ranges are not in the paper): e_end <=
 * n_edges, or <= e0^k when deterministic; written to
 * d_edges[0 .. e_end - e_begin). Every edge depends only on its index, so
 * ranges may be generated in any order, on any device, and concatenate to
 * the whole list. */
pg_status gen_kronecker_range(const double* h_initiator, uint32_t n0, uint32_t k,
                              uint64_t n_edges, uint64_t seed, pg_kron_mode mode, pg_idwidth w,
                              uint64_t e_begin, uint64_t e_end, void* d_edges,
                              uint64_t cap_edges, void* stream);

/* ------------------------------------------------------------------------
 * CSR assembly (not in the paper; the usual input format of the graph
 * algorithms the generated graphs feed).
 *
 * d_edges      n_edges (src, dst) pairs of width w, aligned to one pair (8
 *              bytes for PG_ID32, 16 for PG_ID64); every src and every dst
 *              is < n_vertices (rows are sorted on the bits of that range).
 *              A list already grouped by source (non-decreasing src) whose
 *              rows have at most 32 edges -- what gen_pba writes -- takes a
 *              path without sorting; the result is the same.
 * d_row_ptr    n_vertices + 1 uint64: row_ptr[v] = #edges with src < v.
 * d_col        n_edges ids of width w: the destinations grouped by source,
 *              ascending within each row (duplicates kept). The result does
 *              not depend on scheduling.
 * d_ws         workspace of pg_csr_workspace_size() bytes, 256-byte aligned
 *              (two copies of the list plus a status word per tile and
 *              digit).
 * Every id must be < n_vertices (the generators above always satisfy it).
 * The device does not report a violation, but it never indexes memory with
 * such an id: an edge whose src is out of range is dropped, and the rows
 * and col entries it would have touched are unspecified.
 * ---------------------------------------------------------------------- */
size_t pg_csr_workspace_size(uint64_t n_edges, uint64_t n_vertices);
pg_status edges_to_csr(const void* d_edges, uint64_t n_edges, uint64_t n_vertices,
                       pg_idwidth w, uint64_t* d_row_ptr, void* d_col, void* d_ws,
                       size_t ws_bytes, void* stream);

/* CSR with options (not in the paper, except PG_CSR_ODD below). flags:
 *   PG_CSR_SYMMETRIZE  the list plus (dst, src) of every pair (an undirected
 *                      graph's both directions); col then holds up to
 *                      2*n_edges entries.
 *   PG_CSR_DEDUP       one entry per distinct (src, dst).
 *   PG_CSR_NO_LOOPS    pairs with src == dst are dropped.
 *   PG_CSR_ODD         one entry per pair that occurs an odd number of times:
 *                      the exclusive-or of adjacency matrices. A PK list
 *                      concatenated with gen_random_cells' list gives the
 *                      randomisation of Sec. 3 (PK method) that combines the
 *                      Kronecker adjacency with a random graph's by XOR.
 * Rows are sorted ascending as in edges_to_csr. The number of col entries
 * written is row_ptr[n_vertices], on the device (read it after the stream
 * work is done). cap_col: capacity of d_col in entries; it must cover the
 * list (n_edges, or 2*n_edges with PG_CSR_SYMMETRIZE). flags = 0 is
 * edges_to_csr. Workspace: pg_csr_opts_workspace_size() bytes, 256-byte
 * aligned. */
#define PG_CSR_SYMMETRIZE 1u
#define PG_CSR_DEDUP 2u
#define PG_CSR_NO_LOOPS 4u
#define PG_CSR_ODD 8u
size_t pg_csr_opts_workspace_size(uint64_t n_edges, uint64_t n_vertices, uint32_t flags);
pg_status edges_to_csr_opts(const void* d_edges, uint64_t n_edges, uint64_t n_vertices,
                            pg_idwidth w, uint32_t flags, uint64_t* d_row_ptr, void* d_col,
                            uint64_t cap_col, void* d_ws, size_t ws_bytes, void* stream);

/* The sort's wait status (not in the paper; host only, no device call). The
 * digit pass of the sort finds where each tile's run of a digit starts by
 * reading counts that earlier tiles publish. Tiles are handed out in order, so every count it
 * waits for is written by a CTA already running. Each wait still gives up
 * after a fixed number of polls and then sets a uint32 word of the
 * workspace to nonzero. That word is zeroed by every edges_to_csr or
 * edges_to_csr_opts call that sorts, which is any call with n_edges > 0 and
 * n_vertices > 1. When the word is nonzero after such a call, the CSR it
 * wrote is unspecified.
 * Returns the byte offset of the word within the workspace of a call with
 * these arguments (flags = 0: edges_to_csr), 4-byte aligned and inside
 * the workspace size that the call requires. Read it after the stream has
 * finished the call. Returns SIZE_MAX when such a call does not sort (then
 * nothing is waited for) or when w or flags are invalid. */
size_t pg_csr_wait_error_offset(uint64_t n_edges, uint64_t n_vertices, pg_idwidth w,
                                uint32_t flags);

/* Checked completion of an edges_to_csr / edges_to_csr_opts call (not in the
 * paper). Waits for `stream` (the call's stream), then reads the wait word
 * described above from d_ws (the call's workspace; the other arguments are
 * the call's). Returns PG_OK when no wait gave up (or the call had nothing
 * to sort), PG_ETIMEOUT when one did, so that the CSR the call wrote must not
 * be used, PG_EINVAL for invalid w or flags, PG_ECUDA when the copy or the
 * synchronisation fails. After a wait gives up, the call's remaining sort
 * passes do nothing and every write stays inside its output buffers. */
pg_status pg_csr_check(const void* d_ws, uint64_t n_edges, uint64_t n_vertices, pg_idwidth w,
                       uint32_t flags, void* stream);

/* Test hook (not part of the method): spin_limit (0 = the default, 2^18)
 * is the number of polls after which a wait of the sort gives up, and tile
 * withhold_tile (0xffffffff = none) of every digit pass never publishes its
 * counts, so that the tiles after it wait in vain. Lets a test make the
 * bounded wait run out on purpose and check pg_csr_check's PG_ETIMEOUT.
 * Process-wide, read at each call; cannot fail. */
void pg_csr_test_wait_hook(uint32_t spin_limit, uint32_t withhold_tile);

/* ------------------------------------------------------------------------
 * Checked build (a debugging aid, not part of the method). The same sources
 * compiled with -DPGEN_CHECKED give libpgen_checked.so, with the same entry
 * points. There every kernel access whose index comes from data -- a random
 * draw, a block id read from the phase-1 lists, a vertex id, a position from
 * a scan -- and every store of a result element is compared with the bound
 * of its buffer first. A failed comparison skips the access (a skipped load
 * reads as 0) and is counted in a device record of the kernel's source file;
 * nothing traps, so the CUDA context stays usable.
 * ---------------------------------------------------------------------- */

/* 1 in the checked build, 0 in the default one. */
int pg_checked_build(void);

/* Waits for `stream`, then reports the failed bounds comparisons since the
 * last reset on the current device: *count their number (saturating at
 * 2^32 - 1); *unit the source file of the first one found, in the order
 * 1 Kronecker, 2 PBA, 3 CSR, 4 batch, 5 graph checks (0 when count is 0);
 * *line its source line, *index and *bound the compared values. Files are
 * read in that order, so with failures in several files the lowest number
 * is reported. reset != 0 zeroes every record after reading it. Any output
 * pointer may be NULL. The default build has no checks: it reports count 0
 * and returns PG_OK. PG_ECUDA when a copy or the synchronisation fails. */
pg_status pg_check_read(int reset, uint32_t* count, uint32_t* unit, uint32_t* line,
                        uint64_t* index, uint64_t* bound, void* stream);

/* Test hook of the checked build: from the next launch on, every bound that
 * a store of a result element (an edge, a col entry) is compared with is
 * taken as bound >> shift (0 restores the real bounds). The shortened bound
 * lies inside the real buffer, so the stores it skips were in bounds: a test
 * sees real kernels report and skip stores without any access outside a
 * buffer. Stream-ordered on `stream`, and waits for it. PG_EINVAL for
 * shift > 63 or in the default build. */
pg_status pg_check_test_out_shift(uint32_t shift, void* stream);

/* Random graph G(N, M) with replacement, for the exclusive-or randomisation
 * of PK graphs (Sec. 3, PK method): edge e (e < n_edges) is the cell
 * (row, col) = (floor((w1:w0) * N / 2^64), floor((w3:w2) * N / 2^64)) of the
 * Philox draw with counter (e_lo, e_hi, 0, 4); N = n_vertices. Written as
 * pairs of width w to d_edges (16-byte aligned, cap_edges >= n_edges). */
pg_status gen_random_cells(uint64_t n_vertices, uint64_t n_edges, uint64_t seed, pg_idwidth w,
                           void* d_edges, uint64_t cap_edges, void* stream);

/* ------------------------------------------------------------------------
 * Graph-property checks (Sec. 4 studies the degree distribution and the path
 * lengths of the generated graphs). Exact integer results.
 *
 * pg_degrees: d_deg[v] (n_vertices uint64, cleared by the call) = number of
 *   edges with src == v (PG_DEG_OUT), dst == v (PG_DEG_IN), or both counted
 *   (PG_DEG_TOTAL; a self-loop counts twice). Ids >= n_vertices are skipped.
 * pg_degree_histogram: d_hist (max_degree + 2 uint64, cleared by the call)
 *   [d] = number of vertices of degree d for d <= max_degree, and
 *   [max_degree + 1] = the number of vertices of larger degree.
 * pg_bfs: breadth-first search over a CSR graph (row_ptr, col as
 *   edges_to_csr writes them; for undirected distances pass the CSR of
 *   edges_to_csr_opts with PG_CSR_SYMMETRIZE) from `source`:
 *   d_dist[v] (n_vertices uint32) = hops from source, 0xFFFFFFFF where
 *   unreached. n_vertices < 2^32 - 1. Workspace: pg_bfs_workspace_size()
 *   bytes, 256-byte aligned. Unlike the generators, this call waits for the
 *   stream once per BFS level (to read the next frontier's size);
 *   *levels_out (host) = number of levels run (the source's eccentricity + 1
 *   within its component), *scanned_out (host) = the sum of the reached
 *   vertices' row lengths (the adjacency entries a top-down search reads).
 *   flags: PG_BFS_UNDIRECTED declares the CSR symmetric (every (u, v) has a
 *   (v, u)); wide levels may then run bottom-up, each unvisited vertex
 *   looking for a parent in the frontier (Beamer, Asanovic and Patterson,
 *   "Direction-Optimizing Breadth-First Search", SC'12). The results are the
 *   same either way; on a CSR that is not symmetric the flag gives wrong
 *   distances. 0: every level top-down.
 * ---------------------------------------------------------------------- */
#define PG_DEG_OUT 0
#define PG_DEG_IN 1
#define PG_DEG_TOTAL 2
pg_status pg_degrees(const void* d_edges, uint64_t n_edges, uint64_t n_vertices, pg_idwidth w,
                     int which, uint64_t* d_deg, void* stream);
pg_status pg_degree_histogram(const uint64_t* d_deg, uint64_t n_vertices, uint32_t max_degree,
                              uint64_t* d_hist, void* stream);
#define PG_BFS_UNDIRECTED 1u
size_t pg_bfs_workspace_size(uint64_t n_vertices);
pg_status pg_bfs(const uint64_t* d_row_ptr, const void* d_col, uint64_t n_vertices, pg_idwidth w,
                 uint64_t source, uint32_t flags, uint32_t* d_dist, void* d_ws, size_t ws_bytes,
                 uint32_t* levels_out, uint64_t* scanned_out, void* stream);

/* ------------------------------------------------------------------------
 * Batched generation: many independent graphs in one persistent launch. The
 * batching is not in the paper; each job is one of its generators (Sec. 3,
 * the O(1) preferential attachment of the PBA method, or the stochastic
 * Kronecker model that the PK method cites in Sec. 2).
 *
 * A job is a BA graph (as gen_pba: n new vertices, m edges each, seed
 * clique K_{n0}; blocks <= 1 is the serial model, blocks > 1 the two-phase
 * PBA method with inter_frac and faction_width as in gen_pba) or a
 * stochastic Kronecker graph (as gen_kronecker with PG_KRON_STOCHASTIC).
 * Job i's edges are exactly those the single-graph call with the same
 * arguments writes, placed at h_edge_offsets[i] in one shared output arena.
 * Jobs follow one another in the arena, except that with PG_ID32 a
 * two-phase job starts at an even edge, so one unused arena edge may
 * precede it.
 *
 * pg_batch_plan (host only) validates the jobs and writes a plan of
 * pg_batch_plan_size() bytes into h_plan: per-job records (parameters,
 * Philox round keys, thresholds, arena offset), a work-item table that cuts
 * every serial-BA and Kronecker job into tiles of tile_edges edges (64 <=
 * tile_edges <= 8192, a multiple of 64), and the launch geometry of the
 * two-phase jobs. h_edge_offsets (n_jobs + 1 entries, may be NULL) receives
 * each job's first edge and the arena length; h_n_items the number of work
 * items. 32-bit chain arithmetic is used, so serial BA jobs need
 * n*m + e0 < 2^32. At most 8192 jobs.
 *
 * gen_batch launches one persistent kernel over a copy of the plan in
 * device memory (d_plan, 16-byte aligned): resident CTAs claim work items
 * from a counter in d_ws until none are left. grid_ctas = 0 picks one wave
 * of resident CTAs. Then each two-phase job runs the single-graph PBA
 * kernels (phase 1, the count exchange, the emission) in d_ws after the
 * counter. h_plan is the host plan d_plan was copied from (its two-phase
 * geometry is read there). d_ws: pg_batch_workspace_size(h_plan) bytes,
 * 256-byte aligned. The call is stream-ordered with no host
 * synchronisation and can be captured in a CUDA graph; a replay regenerates
 * the same edges.
 *
 * gen_batch_csr builds, after gen_batch on the same stream, the CSR (as
 * edges_to_csr) of every job with want_csr: job i's row_ptr (its vertex
 * count + 1 entries, starting at 0) at d_row_ptr[row_offset_i], and its
 * col entries (its edge count) at d_col[col_offset_i], the offsets given
 * by pg_batch_csr_layout (UINT64_MAX for a job without want_csr). All of
 * them come from one CSR of the jobs' union graph, in a fixed number of
 * launches whatever the number of jobs: each job's sources are shifted by
 * the vertices of the CSR jobs before it, the union is sorted once, and
 * every job's row_ptr is rebased to 0. With PG_ID32 the CSR jobs' vertices
 * together must be at most 2^32. d_ws: pg_batch_csr_workspace_size(h_plan)
 * bytes, 256-byte aligned; its wait word (see pg_csr_wait_error_offset) is
 * at pg_batch_csr_wait_error_offset(h_plan) (SIZE_MAX when the call sorts
 * nothing). PG_ENOSPC when cap_row_ptr or cap_col is smaller than the
 * totals of pg_batch_csr_layout.
 * ---------------------------------------------------------------------- */
typedef enum { PG_JOB_BA = 0, PG_JOB_KRON = 1 } pg_job_kind;

typedef struct {
    uint32_t kind;            /* pg_job_kind */
    uint32_t m;               /* BA: edges per new vertex */
    uint32_t n0;              /* BA: seed clique size; KRON: initiator order (<= 16) */
    uint32_t k;               /* KRON: levels */
    uint64_t n;               /* BA: new vertices; KRON: edge count */
    uint64_t seed;            /* Philox key */
    const double* initiator;  /* KRON: host, n0*n0 doubles, row-major */
    uint32_t blocks;          /* BA: vertex blocks (0 or 1: serial BA) */
    uint32_t faction_width;   /* BA with blocks > 1: faction width (0: 1) */
    double inter_frac;        /* BA with blocks > 1: inter-block fraction */
    uint32_t want_csr;        /* 1: gen_batch_csr builds this job's CSR */
    uint32_t reserved;        /* 0 */
} pg_job;

size_t pg_batch_plan_size(const pg_job* jobs, uint32_t n_jobs);
size_t pg_batch_workspace_size(const void* h_plan);
pg_status pg_batch_plan(const pg_job* jobs, uint32_t n_jobs, uint32_t tile_edges, pg_idwidth w,
                        void* h_plan, size_t plan_size, uint64_t* h_edge_offsets,
                        uint64_t* h_n_items);
pg_status gen_batch(const void* h_plan, const void* d_plan, uint32_t n_jobs, pg_idwidth w,
                    void* d_arena, uint64_t cap_edges, uint64_t total_edges, uint32_t grid_ctas,
                    void* d_ws, size_t ws_bytes, void* stream);
pg_status pg_batch_csr_layout(const void* h_plan, uint32_t n_jobs, uint64_t* h_row_offsets,
                              uint64_t* h_col_offsets, uint64_t* rows_total, uint64_t* cols_total);
size_t pg_batch_csr_workspace_size(const void* h_plan);
size_t pg_batch_csr_wait_error_offset(const void* h_plan);
pg_status gen_batch_csr(const void* h_plan, const void* d_plan, uint32_t n_jobs, pg_idwidth w,
                        const void* d_arena, uint64_t* d_row_ptr, uint64_t cap_row_ptr,
                        void* d_col, uint64_t cap_col, void* d_ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * Kernel timing trace (profiling aid, not part of the method).
 * pg_trace_enable(1): from then on every kernel the library launches is
 * bracketed by two CUDA events recorded on the launch's stream.
 * pg_trace_dump(buf, len): waits for the recorded events and returns the
 * size (with the NUL) of a JSON object {"kernel_name": [launches, total_ms],
 * ...}. When buf holds at least that many bytes the object is written there
 * and the record is cleared; otherwise (buf NULL or too small) nothing is
 * written and the record is kept, so the call doubles as a size query.
 * ---------------------------------------------------------------------- */
void pg_trace_enable(int on);
size_t pg_trace_dump(char* buf, size_t len);

/* Number of kernels the library has launched in this process, on every
 * device and stream, since it was loaded (accounting, not part of the
 * method): a caller reads it before and after a region of work. Counting is
 * always on and costs one relaxed atomic add per launch. */
uint64_t pg_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* PGEN_H */

// CSR assembly of a generated edge list.
//
// Rows hold their destinations in ascending order (duplicates kept), so the
// result is unique for a given multiset of edges.
//
// Grouped lists (non-decreasing src, as gen_pba and serial BA write them,
// rows of at most kGroupedMaxRow edges): csr_check finds the list grouped and
// csr_grouped places each destination at its rank within its own row and
// marks each row's end in row_ptr.
//
// Any other list: least-significant-digit radix sort of the (src, dst) keys,
// from the low bits of dst to the high bits of src, up to 8 bits per pass:
//   radix_hist_all one read of the list counts the digits of every pass
//                  (the totals do not depend on the order a pass leaves);
//   radix_dstart   per pass, where each digit's run starts in the output;
//   radix_scatter  per pass: stable rank of each element within its tile
//                  among equal digits (shared-memory peer words + per-warp
//                  counters + cross-warp scan), a reorder in shared memory, the tile's
//                  start in each digit's run by decoupled look-back over the
//                  earlier tiles' published counts, and coalesced writes.
// Ranks come from counts in entry order, never from atomics racing for a
// slot, so the result does not depend on the schedule, and a power-law row
// (a hub with 10^5 edges) costs no more than any other key. The last pass
// writes the destinations to col itself and raises row_ptr[src + 1] at the
// last pair of each source in each tile. Both paths then take a parallel
// prefix maximum over row_ptr, which fills the rows without edges. The sort kernels
// read the sortedness flag and return at once when the grouped path applied,
// so no host round trip decides the path.
//
// Ids at or above n_vertices are never used as an index (such edges are
// dropped), so a bad list cannot make a kernel write out of bounds.
#include <atomic>
#include <cstring>

#include "pg_internal.h"
#include "pg_trace.h"

namespace pgen {
namespace {

constexpr int kSortWarps = 16;
constexpr int kSortThreads = kSortWarps * 32;
constexpr int kMaxDigitBits = 8;
constexpr uint32_t kMaxBuckets = 1u << kMaxDigitBits;
constexpr uint32_t kScanTile = 4096;
constexpr uint32_t kGroupedMaxRow = 32;
constexpr uint32_t kHistCopies = 8;   // copies of each digit counter in the histogram kernel

template <typename Id>
struct PairOf;
template <>
struct PairOf<uint32_t> {
    using T = uint2;
};
template <>
struct PairOf<uint64_t> {
    using T = ulonglong2;
};

// The digit of a pass: field 0 = dst and field 1 = src take `mask` bits at
// `shift` of that id; field 2 is a digit of the key (src << nd) | dst that
// starts in dst (shift < nd) and ends in src.
template <typename P>
__device__ __forceinline__ uint32_t digit_of(const P& e, int field, int shift, uint32_t mask,
                                             int nd)
{
    if (field == 2)
        return (uint32_t)(((uint64_t)e.y >> shift) | ((uint64_t)e.x << (nd - shift))) & mask;
    const uint64_t v = field ? (uint64_t)e.x : (uint64_t)e.y;
    return (uint32_t)(v >> shift) & mask;
}

// Elements per thread of a sort tile: 16 pairs of 32-bit ids or 8 of 64-bit.
template <typename Id>
struct SortShape {
    static constexpr int items = sizeof(Id) == 4 ? 16 : 8;
    static constexpr uint32_t tile = kSortThreads * items;
};

// The digits of every LSD pass, from the host: pass k sorts by `bits[k]`
// bits of the destination (field 0) or source (field 1) at `shift[k]`, or
// (field 2) by the bits [shift[k], shift[k] + bits[k]) of the key
// (src << nd) | dst, which straddle the two ids.
constexpr int kMaxPasses = 16;   // 64-bit ids: 128 key bits in digits of 8
struct PassList {
    uint32_t n;
    int nd;   // bits of the dst field
    int field[kMaxPasses], shift[kMaxPasses], bits[kMaxPasses];
};
// Digit totals of every pass in one read of the list: tot[k][d] = number of
// pairs whose pass-k digit is d. Each CTA counts into shared memory
// (n passes x kMaxBuckets counters, kHistCopies copies of each) and adds its
// counts once.
template <typename Id>
__global__ void __launch_bounds__(256) radix_hist_all_kernel(
    const typename PairOf<Id>::T* __restrict__ in, uint64_t M, const __grid_constant__ PassList pl,
    unsigned long long* __restrict__ tot, const uint32_t* __restrict__ sort_needed)
{
    extern __shared__ uint32_t h[];
    if (*sort_needed == 0) return;
    // kHistCopies copies of every counter, interleaved, lane l adding to copy
    // l mod kHistCopies: lanes whose digits agree (the skewed digits of a
    // power-law graph) mostly hit different words
    const uint32_t cells = pl.n * kMaxBuckets;
    for (uint32_t t = threadIdx.x; t < cells * kHistCopies; t += blockDim.x) h[t] = 0;
    __syncthreads();
    const uint32_t copy = threadIdx.x & (kHistCopies - 1);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    constexpr int kU = 4;
    for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < M; i0 += kU * stride) {
        typename PairOf<Id>::T e[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (i0 + u * stride < M) e[u] = in[i0 + u * stride];
        // pass by pass, so that each pass's digit rule is read once for the
        // kU elements
        for (uint32_t k = 0; k < pl.n; ++k) {
            const int field = pl.field[k], shift = pl.shift[k];
            const uint32_t mask = (1u << pl.bits[k]) - 1;
            uint32_t* hk = h + (k * kMaxBuckets) * kHistCopies + copy;
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (i0 + u * stride < M)
                    atomicAdd(&hk[digit_of(e[u], field, shift, mask, pl.nd) * kHistCopies], 1u);
        }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < cells; t += blockDim.x) {
        uint32_t c = 0;
#pragma unroll
        for (uint32_t r = 0; r < kHistCopies; ++r) c += h[t * kHistCopies + r];
        if (c) atomicAdd(&tot[t], (unsigned long long)c);
    }
}

// Tile status words, one per (tile, digit): bits 63..59 the pass (1 + its
// index, so the words of an earlier pass read as not ready), bits 58..57 the
// kind, a pair count below. kAgg: the tile's own count of the digit; kInc: the
// count of the digit in this tile and every earlier one. The array is zeroed
// once per call.
constexpr int kPassShift = 59;
constexpr unsigned long long kAgg = 1ull << 57, kInc = 2ull << 57;
constexpr unsigned long long kCountMask = (1ull << 57) - 1;
static_assert(kMaxPasses < 32, "the pass tag fits bits 63..59");
constexpr uint32_t kSpinLimit = 1u << 18;   // polls of one status word
constexpr int kLookWindow = 8;              // earlier tiles read per round trip

// Test hook (host-set, off by default): a shorter poll limit, and one tile
// per pass that never publishes its counts, so that the tiles after it give
// up waiting and set the error word. The values are passed to each launch.
struct CsrWaitHook {
    uint32_t spin_limit, withhold;
};
std::atomic<uint32_t> g_hook_spin{kSpinLimit};
std::atomic<uint32_t> g_hook_withhold{0xFFFFFFFFu};
CsrWaitHook csr_wait_hook() { return CsrWaitHook{g_hook_spin.load(), g_hook_withhold.load()}; }

// One LSD pass over a tile: load once, rank stably (per warp by match, then
// across warps), reorder the tile by digit in shared memory, and write each
// digit's run to its place in the output with consecutive threads on
// consecutive elements. Where a tile's run of digit d starts is dstart[d]
// (from the pass's digit totals) plus the count of d in earlier tiles, found
// by decoupled look-back over the status words. A CTA takes its tile index
// from a ticket, so every earlier tile belongs to a CTA already running or
// done. It publishes its own counts before it waits on anything, and it sums
// earlier tiles' counts, kLookWindow at a time, until it meets an inclusive
// one. The look-back runs after the reorder, when the tile's pairs no longer
// occupy registers. Every poll loop is bounded: after spin_limit polls of
// one word (kSpinLimit unless a test hook shortened it) it sets *err and
// goes on with the partial sum, which can only be too small, so every write
// stays inside the output.
template <typename Id>
__global__ void __launch_bounds__(kSortThreads, 2) radix_scatter_kernel(
    const typename PairOf<Id>::T* __restrict__ in, typename PairOf<Id>::T* __restrict__ out,
    uint64_t M, int field, int shift, int bits, int nd, unsigned long long* __restrict__ status,
    uint32_t pass, const uint64_t* __restrict__ dstart, uint32_t* __restrict__ ticket,
    uint32_t* __restrict__ err, const uint32_t* __restrict__ sort_needed, uint32_t spin_limit,
    uint32_t withhold, Id* __restrict__ col_out, uint64_t* __restrict__ row_ptr, uint64_t N)
{
    using P = typename PairOf<Id>::T;
    constexpr int kItems = SortShape<Id>::items;
    constexpr uint32_t kTile = SortShape<Id>::tile;
    extern __shared__ __align__(16) unsigned char smem[];
    uint16_t (*wcnt)[kMaxBuckets] = reinterpret_cast<uint16_t (*)[kMaxBuckets]>(smem);   // 8 KB
    uint64_t* tbase = reinterpret_cast<uint64_t*>(smem + kSortWarps * kMaxBuckets * 2);   // 2 KB
    uint32_t* loff = reinterpret_cast<uint32_t*>(tbase + kMaxBuckets);                  // 1 KB
    P* buf = reinterpret_cast<P*>(loff + kMaxBuckets);                                  // tile
    __shared__ uint32_t s_part[kSortWarps + 1];
    __shared__ uint32_t s_tile;
    // after a wait that gave up in an earlier pass the list this pass reads
    // no longer has the digit totals dstart was made from, so a scatter
    // could leave the output: the remaining passes do nothing
    if (*sort_needed == 0 || *(volatile const uint32_t*)err != 0) return;
    const uint32_t nb = 1u << bits, mask = nb - 1;
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
    for (uint32_t d = threadIdx.x; d < nb; d += blockDim.x)
        for (int w = 0; w < kSortWarps; ++w) wcnt[w][d] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t tile0 = (uint64_t)tile * kTile;
    const uint32_t n = (uint32_t)((M - tile0 < kTile) ? M - tile0 : kTile);
    const uint32_t wbase = wid * (32 * kItems);
    P e[kItems];
    // ranks within the warp (< 32 * kItems <= 512), two per register; the
    // digits are recomputed from e[] where needed, so no array holds them
    uint32_t rk[kItems / 2];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const uint32_t t = wbase + r * 32 + lane;
        if (t < n) e[r] = in[tile0 + t];
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    // item r of every lane, in lane order: the lanes holding equal digits
    // find each other through a word per digit (each ORs in its lane bit,
    // then all read the word back and clear it; the word table is the
    // reorder buffer, unused until the ranks are done, one kMaxBuckets-word
    // slab per warp); the lowest lane of each group reads and advances the
    // warp's counter, the group gets the old value by shuffle; the counter
    // is touched by one thread per group and the syncwarp orders it before
    // the next item's read
    uint32_t* pmask = reinterpret_cast<uint32_t*>(buf) + wid * kMaxBuckets;
    for (uint32_t d = lane; d < nb; d += 32) pmask[d] = 0;
    __syncwarp();
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const uint32_t t = wbase + r * 32 + lane;
        const bool valid = t < n;
        const uint32_t d = valid ? digit_of(e[r], field, shift, mask, nd) : 0xFFFFFFFFu;
        if (valid) atomicOr(&pmask[d], 1u << lane);
        __syncwarp();
        const uint32_t peers = valid ? pmask[d] : 0u;
        __syncwarp();
        if (valid) pmask[d] = 0;
        const uint32_t leader = __ffs(peers) - 1;
        uint32_t prev = 0;
        if (lane == leader && d != 0xFFFFFFFFu) {
            prev = wcnt[wid][d];
            wcnt[wid][d] = (uint16_t)(prev + __popc(peers));
        }
        prev = __shfl_sync(0xFFFFFFFFu, prev, leader);
        __syncwarp();
        const uint32_t rank = prev + __popc(peers & lt);
        if (r & 1) rk[r >> 1] |= rank << 16;
        else rk[r >> 1] = rank;
    }
    __syncthreads();
    // per digit: prefix over warps (in wcnt) and the tile total (in loff),
    // published at once so that later tiles can sum it
    const unsigned long long tag = (unsigned long long)(pass + 1) << kPassShift;
    volatile unsigned long long* st = status + (uint64_t)tile * nb;
    for (uint32_t d = threadIdx.x; d < nb; d += blockDim.x) {
        uint32_t acc = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = wcnt[w][d];
            wcnt[w][d] = (uint16_t)acc;
            acc += c;
        }
        loff[d] = acc;
        if (tile != withhold) st[d] = tag | (tile == 0 ? kInc : kAgg) | acc;
    }
    __syncthreads();
    // exclusive scan of the tile totals over digits (each thread a run of digits)
    {
        const uint32_t per = (nb + blockDim.x - 1) / blockDim.x;
        const uint32_t d0 = threadIdx.x * per;
        uint32_t sum = 0;
        for (uint32_t d = d0; d < d0 + per && d < nb; ++d) sum += loff[d];
        // warp inclusive scan of the run sums, then across warps
        uint32_t x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= (uint32_t)o) x += y;
        }
        if (lane == 31) s_part[wid] = x;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t acc = 0;
            for (int w = 0; w < kSortWarps; ++w) {
                const uint32_t c = s_part[w];
                s_part[w] = acc;
                acc += c;
            }
        }
        __syncthreads();
        uint32_t run = s_part[wid] + x - sum;
        for (uint32_t d = d0; d < d0 + per && d < nb; ++d) {
            const uint32_t c = loff[d];
            loff[d] = run;
            run += c;
        }
    }
    __syncthreads();
    // reorder the tile by digit in shared memory
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const uint32_t t = wbase + r * 32 + lane;
        if (t < n) {
            const uint32_t d = digit_of(e[r], field, shift, mask, nd);
            const uint32_t rank = (rk[r >> 1] >> ((r & 1) * 16)) & 0xFFFFu;
            const uint32_t at = loff[d] + wcnt[wid][d] + rank;
            if (PG_CHECK(at, n)) buf[at] = e[r];
        }
    }
    // look back through up to kLookWindow earlier tiles per round trip
    for (uint32_t d = threadIdx.x; d < nb; d += blockDim.x) {
        unsigned long long excl = 0;
        if (tile > 0) {
            uint32_t next = tile - 1;   // nearest tile not yet summed (tile 0 is inclusive)
            uint32_t polls = 0;
            bool found = false;
            while (!found) {
                unsigned long long w[kLookWindow];
#pragma unroll
                for (int u = 0; u < kLookWindow; ++u)
                    w[u] = (next >= (uint32_t)u)
                               ? *((volatile const unsigned long long*)status +
                                   (uint64_t)(next - u) * nb + d)
                               : 0ull;
                int used = 0;
                bool stalled = false;
#pragma unroll
                for (int u = 0; u < kLookWindow; ++u) {
                    if (found || stalled) continue;
                    const unsigned long long flag =
                        (w[u] >> kPassShift) == pass + 1 ? w[u] & (3ull << 57) : 0;
                    if (flag == 0) {
                        stalled = true;
                        continue;
                    }
                    excl += w[u] & kCountMask;
                    ++used;
                    if (flag == kInc) found = true;
                }
                if (found) break;
                next -= used;
                if (stalled) {
                    if (++polls > spin_limit) {
                        atomicOr(err, 1u);
                        break;
                    }
                    __nanosleep(32);
                } else {
                    polls = 0;
                }
            }
            const uint32_t cnt_d = (d + 1 < nb ? loff[d + 1] : n) - loff[d];
            if (tile != withhold) st[d] = tag | kInc | (excl + cnt_d);
        }
        // where the tile's run of d starts in the output, less its start in
        // the sorted tile (never negative: the tile's counts of the lower
        // digits, loff[d], are at most their totals, which dstart[d] sums)
        tbase[d] = dstart[d] + excl - loff[d];
    }
    __syncthreads();
    // write runs: sorted position p goes to tbase[d] + p (one table read per pair)
    if (col_out == nullptr) {
        for (uint32_t p = threadIdx.x; p < n; p += blockDim.x) {
            const P v = buf[p];
            const uint32_t d = digit_of(v, field, shift, mask, nd);
            if (PG_CHECK(tbase[d] + p, M)) out[tbase[d] + p] = v;
        }
        return;
    }
    // the last pass of a CSR: the tile is in (src, dst) order, so each
    // destination goes straight to col, and the last pair of each source
    // in the tile raises row_ptr[src + 1] to its end (the source's last pair
    // overall gives the maximum; the prefix maximum fills empty rows)
    for (uint32_t p = threadIdx.x; p < n; p += blockDim.x) {
        const P v = buf[p];
        const uint32_t d = digit_of(v, field, shift, mask, nd);
        const uint64_t o = tbase[d] + p;
        if (PG_CHECK_OUT(o, M)) col_out[o] = (Id)v.y;
        const uint64_t src = v.x;
        if (src < N && (p + 1 == n || (uint64_t)buf[p + 1].x != src))
            atomicMax(reinterpret_cast<unsigned long long*>(row_ptr) + src + 1,
                      (unsigned long long)(o + 1));
    }
}

static_assert(SortShape<uint32_t>::tile * sizeof(uint2) >= kSortWarps * kMaxBuckets * 4 &&
                  SortShape<uint64_t>::tile * sizeof(ulonglong2) >= kSortWarps * kMaxBuckets * 4,
              "the reorder buffer holds every warp's digit words");

template <typename Id>
size_t scatter_smem_bytes()
{
    return (size_t)kSortWarps * kMaxBuckets * 2 + kMaxBuckets * 8 + kMaxBuckets * 4 +
           (size_t)SortShape<Id>::tile * sizeof(typename PairOf<Id>::T);
}

// ---- exclusive scan of uint32 counts into uint64 offsets ------------------
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t* s_warp,
                                                         uint64_t& total)
{
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t nw = blockDim.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint64_t w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= (uint32_t)o) w += y;
        }
        if (lane < nw) s_warp[lane] = w;   // inclusive warp totals
    }
    __syncthreads();
    total = s_warp[nw - 1];
    const uint64_t before = wid ? s_warp[wid - 1] : 0;
    __syncthreads();
    return before + x - v;
}

// Zeroes the tile status words once per call (nothing when no sort runs).
__global__ void __launch_bounds__(256) zero_status_kernel(uint4* __restrict__ p, uint64_t n16,
                                                          const uint32_t* __restrict__ sort_needed)
{
    if (*sort_needed == 0) return;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride)
        p[i] = make_uint4(0u, 0u, 0u, 0u);
}
// Where each digit's run starts in pass k's output: the exclusive scan of
// that pass's digit totals. grid = passes, block = kMaxBuckets threads.
__global__ void __launch_bounds__(kMaxBuckets) radix_dstart_kernel(
    const unsigned long long* __restrict__ tot, const __grid_constant__ PassList pl,
    uint64_t* __restrict__ dstart, const uint32_t* __restrict__ sort_needed)
{
    __shared__ uint64_t s_warp[32];
    if (*sort_needed == 0) return;
    const uint32_t k = blockIdx.x, nb = 1u << pl.bits[k], d = threadIdx.x;
    const uint64_t c = d < nb ? tot[(size_t)k * kMaxBuckets + d] : 0;
    uint64_t total;
    const uint64_t ex = block_exclusive_scan(c, s_warp, total);
    if (d < nb) dstart[(size_t)k * kMaxBuckets + d] = ex;
}

// exclusive scan of n_parts sums in place, one CTA looping over chunks
__global__ void __launch_bounds__(1024) scan_parts_kernel(uint64_t* __restrict__ part,
                                                          uint64_t n_parts,
                                                          const uint32_t* __restrict__ sort_needed)
{
    __shared__ uint64_t s_warp[32];
    if (*sort_needed == 0) return;
    uint64_t carry = 0;
    for (uint64_t base = 0; base < n_parts; base += blockDim.x) {
        const uint64_t i = base + threadIdx.x;
        const uint64_t v = i < n_parts ? part[i] : 0;
        uint64_t total;
        const uint64_t ex = block_exclusive_scan(v, s_warp, total);
        if (i < n_parts) part[i] = carry + ex;
        carry += total;
    }
}

// ---- final pass: col and row_ptr from the sorted pairs ---------------------
// Flags (sort_needed = 1) a list that is not grouped by source, or that has
// a row longer than kGroupedMaxRow.
template <typename Id>
__global__ void __launch_bounds__(256) csr_check_kernel(const typename PairOf<Id>::T* __restrict__ s,
                                                        uint64_t M, uint32_t* __restrict__ sort_needed)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    // A warp that finds a violation sets the flag (one atomic per warp) and
    // stops; every few rounds the warps also read the flag and stop once any
    // warp has set it, so an unsorted list costs about one round, not a full
    // read. The trip count is uniform across the warp (i0 steps by the grid).
    const volatile uint32_t* flag = sort_needed;
    const uint32_t lane = threadIdx.x & 31;
    uint32_t round = 0;
    for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < M;
         i0 += stride, ++round) {
        const uint64_t i = i0 + lane;
        bool bad = false;
        if (i < M) {
            const uint64_t src = s[i].x;
            const bool starts = (i == 0) || s[i - 1].x != src;
            bad = i > 0 && (uint64_t)s[i - 1].x > src;
            bad |= starts && i + kGroupedMaxRow < M && (uint64_t)s[i + kGroupedMaxRow].x == src;
        }
        if (__any_sync(0xFFFFFFFFu, bad)) {
            if (lane == 0) atomicOr(sort_needed, 1u);
            return;
        }
        if ((round & 7) == 7 && *flag != 0) return;
    }
}

// Row ends of a list sorted (or grouped) by source: the last edge i of row v
// writes row_ptr[v + 1] = i + 1. A prefix maximum over row_ptr then fills the
// rows without edges (row_ptr starts zeroed).
template <typename P>
__device__ __forceinline__ void mark_row_end(const P* s, uint64_t M, uint64_t N, uint64_t i,
                                             uint64_t* row_ptr)
{
    const uint64_t v = s[i].x;
    if (v < N && (i + 1 == M || s[i + 1].x != s[i].x)) row_ptr[v + 1] = i + 1;
}

// Grouped list: destination of edge i goes to its row start + its rank among
// the row's destinations (ties broken by position, so equal values keep
// their multiplicity).
template <typename Id>
__global__ void __launch_bounds__(256) csr_grouped_kernel(const typename PairOf<Id>::T* __restrict__ s,
                                                          uint64_t M, uint64_t N, Id* __restrict__ col,
                                                          uint64_t* __restrict__ row_ptr,
                                                          const uint32_t* __restrict__ sort_needed)
{
    if (*sort_needed != 0) return;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
        const uint64_t src = s[i].x, d = s[i].y;
        uint64_t a = i, b = i + 1;
        while (a > 0 && (uint64_t)s[a - 1].x == src) --a;
        while (b < M && (uint64_t)s[b].x == src) ++b;
        uint64_t rank = 0;
        for (uint64_t j = a; j < b; ++j) {
            const uint64_t dj = s[j].y;
            rank += (dj < d) || (dj == d && j < i);
        }
        if (PG_CHECK_OUT(a + rank, M)) col[a + rank] = (Id)d;
        mark_row_end(s, M, N, i, row_ptr);
    }
}

// In-place inclusive prefix maximum over n uint64 (three kernels, as the sums).
__device__ __forceinline__ uint64_t block_inclusive_max(uint64_t v, uint64_t* s_warp, uint64_t& total)
{
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t nw = blockDim.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (uint32_t)o && y > x) x = y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint64_t w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= (uint32_t)o && y > w) w = y;
        }
        if (lane < nw) s_warp[lane] = w;
    }
    __syncthreads();
    total = s_warp[nw - 1];
    const uint64_t before = wid ? s_warp[wid - 1] : 0;
    __syncthreads();
    return x > before ? x : before;
}

__global__ void __launch_bounds__(256) max_reduce_kernel(const uint64_t* __restrict__ in, uint64_t n,
                                                         uint64_t* __restrict__ part)
{
    __shared__ uint64_t s_warp[32];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    uint64_t m = 0;
    for (uint32_t t = threadIdx.x; t < kScanTile; t += blockDim.x)
        if (base + t < n && in[base + t] > m) m = in[base + t];
    uint64_t total;
    block_inclusive_max(m, s_warp, total);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// exclusive prefix maximum of the tile maxima, one CTA looping over chunks
__global__ void __launch_bounds__(1024) max_parts_kernel(uint64_t* __restrict__ part, uint64_t n_parts)
{
    __shared__ uint64_t s_warp[32];
    __shared__ uint64_t s_inc[1024];
    uint64_t carry = 0;
    for (uint64_t base = 0; base < n_parts; base += blockDim.x) {
        const uint64_t i = base + threadIdx.x;
        const uint64_t v = i < n_parts ? part[i] : 0;
        uint64_t total;
        s_inc[threadIdx.x] = block_inclusive_max(v, s_warp, total);
        __syncthreads();
        uint64_t ex = threadIdx.x ? s_inc[threadIdx.x - 1] : 0;
        if (ex < carry) ex = carry;
        if (i < n_parts) part[i] = ex;
        if (total > carry) carry = total;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) max_apply_kernel(uint64_t* __restrict__ data, uint64_t n,
                                                        const uint64_t* __restrict__ part)
{
    __shared__ uint64_t s_warp[32];
    __shared__ uint64_t s_inc[256];
    constexpr int per = kScanTile / 256;
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile + threadIdx.x * per;
    uint64_t v[per];
    uint64_t m = 0;
#pragma unroll
    for (int t = 0; t < per; ++t) {
        v[t] = (base + t < n) ? data[base + t] : 0;
        if (v[t] > m) m = v[t];
    }
    uint64_t total;
    s_inc[threadIdx.x] = block_inclusive_max(m, s_warp, total);
    __syncthreads();
    uint64_t run = threadIdx.x ? s_inc[threadIdx.x - 1] : 0;   // previous threads' runs
    const uint64_t carry = part[blockIdx.x];                    // previous tiles
    if (run < carry) run = carry;
#pragma unroll
    for (int t = 0; t < per; ++t) {
        if (v[t] > run) run = v[t];
        if (base + t < n) data[base + t] = run;
    }
}

template <typename Id>
__global__ void __launch_bounds__(256) csr_finish_kernel(const typename PairOf<Id>::T* __restrict__ s,
                                                         uint64_t M, uint64_t N, uint64_t* __restrict__ row_ptr,
                                                         Id* __restrict__ col,
                                                         const uint32_t* __restrict__ sort_needed)
{
    if (*sort_needed == 0) return;
    // four grid strides per trip, so each thread has four independent loads
    // in flight
    constexpr int kU = 4;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < M; i0 += kU * stride) {
        typename PairOf<Id>::T e[kU];
        uint64_t nx[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const uint64_t i = i0 + u * stride;
            if (i < M) {
                e[u] = s[i];
                nx[u] = (i + 1 < M) ? (uint64_t)s[i + 1].x : ~(uint64_t)0;
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const uint64_t i = i0 + u * stride;
            if (i < M) {
                if (PG_CHECK_OUT(i, M)) col[i] = (Id)e[u].y;
                const uint64_t v = e[u].x;
                if (v < N && nx[u] != v) row_ptr[v + 1] = i + 1;
            }
        }
    }
}

// ---- CSR options (symmetrise, dedup, drop loops, odd multiplicity) ---------
// All options act on the list sorted by (src, dst): the sort always runs,
// then a compaction keeps the wanted positions of the sorted pairs, writes
// their destinations to col in order and marks row ends for the prefix max.
constexpr uint32_t kOptSym = 1, kOptDedup = 2, kOptNoLoops = 4, kOptOdd = 8;

template <typename Id>
__global__ void __launch_bounds__(256) csr_sym_kernel(const typename PairOf<Id>::T* __restrict__ in,
                                                      uint64_t M,
                                                      typename PairOf<Id>::T* __restrict__ x)
{
    using P = typename PairOf<Id>::T;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
        const P e = in[i];
        P r;
        r.x = e.y;
        r.y = e.x;
        x[2 * i] = e;
        x[2 * i + 1] = r;
    }
}

template <typename P>
__device__ __forceinline__ bool same_pair(const P& a, const P& b)
{
    return a.x == b.x && a.y == b.y;
}

template <typename P>
__device__ __forceinline__ bool pair_less(const P& a, const P& b)
{
    return a.x < b.x || (a.x == b.x && a.y < b.y);
}

// Where the run of pairs equal to e = s[i] starts. Runs are short in
// practice, so the first steps go back one pair at a time; a longer run is
// found by binary search of the sorted list below. (With ids outside the
// vertex range the list need not be in lexicographic order there, and the
// search only stays within [0, i].)
template <typename P>
__device__ __forceinline__ uint64_t run_start(const P* s, uint64_t i, const P& e)
{
    uint64_t j = i;
    for (int t = 0; t < 8 && j > 0 && same_pair(s[j - 1], e); ++t) --j;
    if (j == 0 || !same_pair(s[j - 1], e)) return j;
    uint64_t lo = 0, hi = j;   // s[hi] == e: the first index of e lies in [lo, hi]
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (pair_less(s[mid], e)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Whether sorted position i survives the options.
template <typename P>
__device__ __forceinline__ bool keep_at(const P* s, uint64_t M, uint64_t i, uint32_t flags)
{
    const P e = s[i];
    if ((flags & kOptNoLoops) && e.x == e.y) return false;
    if (flags & kOptOdd) {
        // the last pair of each run is kept when the run's length is odd
        const bool end = (i + 1 == M) || !same_pair(s[i + 1], e);
        return end && (((i + 1 - run_start(s, i, e)) & 1) != 0);
    }
    if (flags & kOptDedup) return i == 0 || !same_pair(s[i - 1], e);
    return true;
}

template <typename Id>
__global__ void __launch_bounds__(256) csr_keep_count_kernel(const typename PairOf<Id>::T* __restrict__ s,
                                                             uint64_t M, uint32_t flags,
                                                             uint64_t* __restrict__ part)
{
    __shared__ uint64_t s_warp[32];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    uint64_t cnt = 0;
    for (uint32_t t = threadIdx.x; t < kScanTile; t += blockDim.x)
        if (base + t < M) cnt += keep_at(s, M, base + t, flags) ? 1 : 0;
    uint64_t total;
    block_exclusive_scan(cnt, s_warp, total);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// Each warp takes kScanTile/8 consecutive positions of its tile, 32 at a
// time (consecutive lanes on consecutive pairs, so the reads coalesce): one
// ballot per round gives every kept position its place among the warp's,
// the warps' counts are scanned across the block, and the kept destinations
// are written in sorted order. The last position of every row writes
// row_ptr[src + 1] = kept entries up to and including it.
template <typename Id>
__global__ void __launch_bounds__(256, 4) csr_keep_apply_kernel(const typename PairOf<Id>::T* __restrict__ s,
                                                             uint64_t M, uint64_t N, uint32_t flags,
                                                             const uint64_t* __restrict__ part,
                                                             Id* __restrict__ col,
                                                             uint64_t* __restrict__ row_ptr)
{
    using P = typename PairOf<Id>::T;
    __shared__ uint64_t s_warp[32];
    constexpr int kRounds = kScanTile / 256;   // rounds of 32 positions per warp
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const uint64_t wbase = (uint64_t)blockIdx.x * kScanTile + (uint64_t)wid * (32 * kRounds);
    uint32_t m[kRounds];
    uint32_t cnt = 0;
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const uint64_t i = wbase + r * 32 + lane;
        m[r] = __ballot_sync(0xFFFFFFFFu, i < M && keep_at(s, M, i, flags));
        cnt += __popc(m[r]);
    }
    // the warps before this one in the tile, from lane 0's exclusive prefix
    uint64_t total;
    const uint64_t ex = block_exclusive_scan(lane == 0 ? (uint64_t)cnt : 0, s_warp, total);
    uint64_t e = part[blockIdx.x] + __shfl_sync(0xFFFFFFFFu, ex, 0);
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const uint64_t i = wbase + r * 32 + lane;
        const bool keep = (m[r] >> lane) & 1u;
        const uint64_t at = e + __popc(m[r] & lt);   // this position's place if kept
        if (i < M) {
            const P pv = s[i];
            if (keep && PG_CHECK_OUT(at, M)) col[at] = (Id)pv.y;
            const uint64_t v = pv.x;
            if (v < N && (i + 1 == M || (uint64_t)s[i + 1].x != v))
                row_ptr[v + 1] = at + (keep ? 1 : 0);
        }
        e += __popc(m[r]);
    }
}

}  // namespace

PG_CHECK_UNIT(csr)

namespace {

int bit_length(uint64_t x)
{
    int b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

struct CsrLayout {
    size_t off_a, off_b, off_status, off_flag, off_dig, off_rpart, total;
    uint32_t n_tiles, max_nb;
    uint64_t n_status, n_rparts;
};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// The LSD passes that sort pairs by (src, dst): the key (src << nd) | dst,
// nd = the bits of n_dst - 1 and ns those of n_src - 1, cut from its low end
// into ceil((nd + ns) / kMaxDigitBits) digits whose widths differ by at most
// one (the wider ones first). A digit inside one id reads that id alone; the
// one that contains the boundary reads both.
PassList make_passes(uint64_t n_src, uint64_t n_dst)
{
    PassList pl;
    std::memset(&pl, 0, sizeof(pl));
    const int nd = bit_length(n_dst > 0 ? n_dst - 1 : 0);
    const int ns = bit_length(n_src > 0 ? n_src - 1 : 0);
    const int total = nd + ns;
    const int n = (total + kMaxDigitBits - 1) / kMaxDigitBits;
    pl.nd = nd;
    int shift = 0;
    for (int k = 0; k < n; ++k) {
        const int b = total / n + (k < total % n ? 1 : 0);
        if (shift + b <= nd) {
            pl.field[k] = 0;
            pl.shift[k] = shift;
        } else if (shift >= nd) {
            pl.field[k] = 1;
            pl.shift[k] = shift - nd;
        } else {
            pl.field[k] = 2;
            pl.shift[k] = shift;
        }
        pl.bits[k] = b;
        shift += b;
    }
    pl.n = (uint32_t)n;
    return pl;
}

CsrLayout csr_layout(uint64_t M, uint64_t N, size_t pair_bytes, uint64_t N_dst = 0)
{
    CsrLayout L;
    const PassList pl = make_passes(N, N_dst ? N_dst : N);
    int dbits = 0;
    for (uint32_t k = 0; k < pl.n; ++k) dbits = pl.bits[k] > dbits ? pl.bits[k] : dbits;
    const uint32_t tile = pair_bytes == 8 ? SortShape<uint32_t>::tile : SortShape<uint64_t>::tile;
    L.max_nb = 1u << dbits;
    L.n_tiles = (uint32_t)((M + tile - 1) / tile);
    L.n_status = (uint64_t)L.max_nb * L.n_tiles;
    size_t o = 0;
    L.off_a = o;
    o += a256(M * pair_bytes);
    L.off_b = o;
    o += a256(M * pair_bytes);
    L.off_status = o;   // tile status words of the pass being sorted
    o += a256(L.n_status * 8);
    L.off_flag = o;     // +0: sort-needed flag, +64: one ticket per pass, +128: look-back error
    o += 256;
    L.off_dig = o;      // digit totals, then digit starts, of every pass
    o += a256(2 * (size_t)kMaxPasses * kMaxBuckets * 8);
    L.n_rparts = (N + 1 + kScanTile - 1) / kScanTile;
    L.off_rpart = o;
    o += a256((L.n_rparts + 1) * 8);
    L.total = o;
    return L;
}

// The opt-in shared-memory sizes of the sort kernels, set once per device
// for each id width.
PerDeviceOnce g_csr_attrs[2];
template <typename Id>
cudaError_t set_csr_attributes()
{
    return g_csr_attrs[sizeof(Id) == 8].run_current([] {
        return first_error({
            cudaFuncSetAttribute(radix_scatter_kernel<Id>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)scatter_smem_bytes<Id>()),
            cudaFuncSetAttribute(radix_hist_all_kernel<Id>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kMaxPasses * 4 * kMaxBuckets * kHistCopies))});
    });
}

// LSD radix passes over M pairs starting at `in` (the digits of the key
// (src << nd) | dst from its low end). *sorted receives the sorted list (in
// itself when there is no digit to sort), *spare a ping-pong buffer the
// result does not occupy. With col_final set, the last pass writes the CSR
// directly instead of the sorted pairs: destinations to col_final, row ends
// raised into row_ptr (zeroed by the caller); *sorted is then not a list.
int sort_grid(uint64_t work);

template <typename Id>
cudaError_t radix_passes(const typename PairOf<Id>::T* in, uint64_t M, uint64_t N, uint64_t N_dst,
                         const CsrLayout& L, unsigned char* ws, const uint32_t* sort_needed,
                         cudaStream_t s, const typename PairOf<Id>::T** sorted,
                         typename PairOf<Id>::T** spare, Id* col_final = nullptr,
                         uint64_t* row_ptr = nullptr)
{
    using P = typename PairOf<Id>::T;
    P* buf[2] = {(P*)(ws + L.off_a), (P*)(ws + L.off_b)};
    unsigned long long* status = (unsigned long long*)(ws + L.off_status);
    unsigned long long* tot = (unsigned long long*)(ws + L.off_dig);
    uint64_t* dstart = (uint64_t*)(ws + L.off_dig) + (size_t)kMaxPasses * kMaxBuckets;
    uint32_t* tickets = (uint32_t*)(ws + L.off_flag + 64);
    uint32_t* err = (uint32_t*)(ws + L.off_flag + 128);
    // the passes: digits of the key (src << nd) | dst, at most kMaxDigitBits each
    const PassList pl = make_passes(N, N_dst);
    const P* cur = in;
    int which = 0;
    cudaError_t err_c;
    const CsrWaitHook hk = csr_wait_hook();
    // the tickets and the wait error word start at zero on every call that
    // has edges (a call without edges has nothing to sort and no wait)
    if (M > 0 && cudaMemsetAsync(ws + L.off_flag + 64, 0, 128, s) != cudaSuccess)
        return cudaErrorUnknown;
    if (M > 0 && pl.n > 0) {
        if (cudaMemsetAsync(tot, 0, (size_t)pl.n * kMaxBuckets * 8, s) != cudaSuccess)
            return cudaErrorUnknown;
        {
            TraceScope trace("csr_radix_hist", s);
            { zero_status_kernel<<<sort_grid(L.n_status / 2 + 1), 256, 0, s>>>(
                (uint4*)status, (L.n_status * 8 + 15) / 16, sort_needed); note_launch(); }
            { radix_hist_all_kernel<Id><<<sort_grid(M), 256, (size_t)pl.n * kMaxBuckets * 4 * kHistCopies, s>>>(
                cur, M, pl, tot, sort_needed); note_launch(); }
        }
        {
            TraceScope trace("csr_scan", s);
            { radix_dstart_kernel<<<pl.n, kMaxBuckets, 0, s>>>(tot, pl, dstart, sort_needed); note_launch(); }
        }
        for (uint32_t k = 0; k < pl.n; ++k) {
            TraceScope trace("csr_radix_scatter", s);
            { radix_scatter_kernel<Id><<<L.n_tiles, kSortThreads, scatter_smem_bytes<Id>(), s>>>(
                cur, buf[which], M, pl.field[k], pl.shift[k], pl.bits[k], pl.nd, status, k,
                dstart + (size_t)k * kMaxBuckets, tickets + k, err, sort_needed, hk.spin_limit,
                hk.withhold, k + 1 == pl.n ? col_final : nullptr, row_ptr, N); note_launch(); }
            if ((err_c = cudaGetLastError()) != cudaSuccess) return err_c;
            cur = buf[which];
            which ^= 1;
        }
    }
    *sorted = cur;
    *spare = buf[which];
    return cudaSuccess;
}

// In-place prefix maximum over n uint64 (three kernels).
cudaError_t prefix_max(uint64_t* data, uint64_t n, uint64_t* parts, cudaStream_t s)
{
    const uint64_t n_parts = (n + kScanTile - 1) / kScanTile;
    if (n_parts == 0) return cudaSuccess;
    { max_reduce_kernel<<<(unsigned)n_parts, 256, 0, s>>>(data, n, parts); note_launch(); }
    { max_parts_kernel<<<1, 1024, 0, s>>>(parts, n_parts); note_launch(); }
    { max_apply_kernel<<<(unsigned)n_parts, 256, 0, s>>>(data, n, parts); note_launch(); }
    return cudaGetLastError();
}

int sort_grid(uint64_t work)
{
    int grid = (int)((work + 255) / 256);
    const int cap = device_sm_count() * 8;
    if (grid > cap) grid = cap;
    return grid < 1 ? 1 : grid;
}

template <typename Id>
cudaError_t csr_impl(const void* d_edges, uint64_t M, uint64_t N, uint64_t N_dst,
                     uint64_t* d_row_ptr, void* d_col, void* d_ws, cudaStream_t s)
{
    using P = typename PairOf<Id>::T;
    const CsrLayout L = csr_layout(M, N, sizeof(P), N_dst);
    cudaError_t err;
    if ((err = set_csr_attributes<Id>()) != cudaSuccess) return err;
    unsigned char* ws = (unsigned char*)d_ws;
    uint32_t* sort_needed = (uint32_t*)(ws + L.off_flag);
    const int grid = sort_grid(M + 1);
    if (cudaMemsetAsync(sort_needed, 0, 4, s) != cudaSuccess) return cudaErrorUnknown;
    if (cudaMemsetAsync(d_row_ptr, 0, (N + 1) * 8, s) != cudaSuccess) return cudaErrorUnknown;
    {
        TraceScope trace("csr_check", s);
        { csr_check_kernel<Id><<<grid, 256, 0, s>>>((const P*)d_edges, M, sort_needed); note_launch(); }
        { csr_grouped_kernel<Id><<<grid, 256, 0, s>>>((const P*)d_edges, M, N, (Id*)d_col, d_row_ptr,
                                                   sort_needed); note_launch(); }
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    const P* cur;
    P* spare;
    // with at least one digit to sort, the last pass writes col and the row
    // ends itself; a key without digits (one vertex) leaves the list as it is
    const bool in_sort = M > 0 && make_passes(N, N_dst).n > 0;
    if ((err = radix_passes<Id>((const P*)d_edges, M, N, N_dst, L, ws, sort_needed, s, &cur,
                                &spare, in_sort ? (Id*)d_col : nullptr, d_row_ptr)) !=
        cudaSuccess)
        return err;
    if (!in_sort) {
        TraceScope trace("csr_finish", s);
        { csr_finish_kernel<Id><<<grid, 256, 0, s>>>(cur, M, N, d_row_ptr, (Id*)d_col, sort_needed); note_launch(); }
    }
    TraceScope trace("csr_rows", s);   // rows without edges take the previous row's end
    return prefix_max(d_row_ptr, N + 1, (uint64_t*)(ws + L.off_rpart), s);
}

// Workspace of the options path: the sort's layout for the (possibly
// doubled) list, then the doubled list, and the parts of two scans.
struct OptsLayout {
    CsrLayout L;
    size_t off_x, off_cpart, total;
    uint64_t M2, n_cparts;
};

OptsLayout opts_layout(uint64_t M, uint64_t N, uint32_t flags, size_t pair_bytes)
{
    OptsLayout O;
    O.M2 = (flags & kOptSym) ? 2 * M : M;
    O.L = csr_layout(O.M2, N, pair_bytes);
    size_t o = a256(O.L.total);
    O.off_x = o;
    if (flags & kOptSym) o += a256(O.M2 * pair_bytes);
    O.n_cparts = (O.M2 + kScanTile - 1) / kScanTile;
    O.off_cpart = o;
    o += a256((O.n_cparts + 1) * 8);
    O.total = o;
    return O;
}

template <typename Id>
cudaError_t csr_opts_impl(const void* d_edges, uint64_t M, uint64_t N, uint32_t flags,
                          uint64_t* d_row_ptr, void* d_col, void* d_ws, cudaStream_t s)
{
    using P = typename PairOf<Id>::T;
    const OptsLayout O = opts_layout(M, N, flags, sizeof(P));
    cudaError_t err;
    if ((err = set_csr_attributes<Id>()) != cudaSuccess) return err;
    unsigned char* ws = (unsigned char*)d_ws;
    uint32_t* sort_needed = (uint32_t*)(ws + O.L.off_flag);
    const uint64_t M2 = O.M2;
    // every option needs the sorted list: the sort kernels run unconditionally
    if (cudaMemsetAsync(sort_needed, 1, 4, s) != cudaSuccess) return cudaErrorUnknown;
    if (cudaMemsetAsync(d_row_ptr, 0, (N + 1) * 8, s) != cudaSuccess) return cudaErrorUnknown;
    const P* in = (const P*)d_edges;
    if ((flags & kOptSym) && M > 0) {
        P* x = (P*)(ws + O.off_x);
        { csr_sym_kernel<Id><<<sort_grid(M), 256, 0, s>>>(in, M, x); note_launch(); }
        in = x;
    }
    const P* cur;
    P* spare;
    if ((err = radix_passes<Id>(in, M2, N, N, O.L, ws, sort_needed, s, &cur, &spare)) !=
        cudaSuccess)
        return err;
    TraceScope trace("csr_compact", s);
    if (M2 > 0) {
        uint64_t* cpart = (uint64_t*)(ws + O.off_cpart);
        { csr_keep_count_kernel<Id><<<(unsigned)O.n_cparts, 256, 0, s>>>(cur, M2, flags, cpart); note_launch(); }
        { scan_parts_kernel<<<1, 1024, 0, s>>>(cpart, O.n_cparts, sort_needed); note_launch(); }
        { csr_keep_apply_kernel<Id><<<(unsigned)O.n_cparts, 256, 0, s>>>(cur, M2, N, flags, cpart,
                                                                        (Id*)d_col, d_row_ptr); note_launch(); }
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    return prefix_max(d_row_ptr, N + 1, (uint64_t*)(ws + O.L.off_rpart), s);
}

}  // namespace

void set_csr_wait_hook(uint32_t spin_limit, uint32_t withhold_tile)
{
    g_hook_spin.store(spin_limit ? spin_limit : kSpinLimit);
    g_hook_withhold.store(withhold_tile);
}

size_t csr_workspace_bytes(uint64_t n_edges, uint64_t n_vertices, uint64_t n_dst)
{
    // one size that fits either id width
    const size_t a = csr_layout(n_edges, n_vertices, 16, n_dst).total;
    const size_t b = csr_layout(n_edges, n_vertices, 8, n_dst).total;
    return a > b ? a : b;
}

size_t csr_opts_workspace_bytes(uint64_t n_edges, uint64_t n_vertices, uint32_t flags)
{
    const size_t a = opts_layout(n_edges, n_vertices, flags, 16).total;
    const size_t b = opts_layout(n_edges, n_vertices, flags, 8).total;
    return a > b ? a : b;
}

// Byte offset of the look-back error word in the workspace of a call with
// these arguments (the layout the call itself uses).
size_t csr_wait_error_offset(uint64_t n_edges, uint64_t n_vertices, uint32_t flags, int id64,
                             uint64_t n_dst)
{
    const size_t pair_bytes = id64 ? 16 : 8;
    const CsrLayout L = flags ? opts_layout(n_edges, n_vertices, flags, pair_bytes).L
                              : csr_layout(n_edges, n_vertices, pair_bytes, n_dst);
    return L.off_flag + 128;
}

cudaError_t launch_csr_opts(const void* d_edges, uint64_t n_edges, uint64_t n_vertices, int id64,
                            uint32_t flags, uint64_t* d_row_ptr, void* d_col, void* d_ws,
                            cudaStream_t s)
{
    return id64 ? csr_opts_impl<uint64_t>(d_edges, n_edges, n_vertices, flags, d_row_ptr, d_col,
                                          d_ws, s)
                : csr_opts_impl<uint32_t>(d_edges, n_edges, n_vertices, flags, d_row_ptr, d_col,
                                          d_ws, s);
}

cudaError_t launch_csr(const void* d_edges, uint64_t n_edges, uint64_t n_vertices, int id64,
                       uint64_t* d_row_ptr, void* d_col, void* d_ws, size_t ws_bytes,
                       cudaStream_t s, uint64_t n_dst)
{
    (void)ws_bytes;
    const uint64_t nd = n_dst ? n_dst : n_vertices;
    return id64 ? csr_impl<uint64_t>(d_edges, n_edges, n_vertices, nd, d_row_ptr, d_col, d_ws, s)
                : csr_impl<uint32_t>(d_edges, n_edges, n_vertices, nd, d_row_ptr, d_col, d_ws, s);
}

}  // namespace pgen

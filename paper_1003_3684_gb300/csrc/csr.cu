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
// first the digits of dst, then those of src, up to 10 bits per pass. Each
// pass is three kernels:
//   radix_hist     per-tile digit counts, stored digit-major H[d][tile];
//   scan_rows      per digit, the exclusive scan of its counts over tiles,
//                  and (by the last CTA to finish) the scan of the digit
//                  totals: together, where each tile's run of each digit
//                  starts in the output;
//   radix_scatter  stable rank of each element within its tile among equal
//                  digits (warp match + per-warp counters + cross-warp scan)
//                  and a scattered write of the (src, dst) pair.
// No atomics decide any position, so the result does not depend on the
// schedule, and a power-law row (a hub with 10^5 edges) costs no more than
// any other key. A final pass writes col and marks row ends. Both paths then
// take a parallel prefix maximum over row_ptr, which fills the rows without
// edges. The sort kernels read the sortedness flag and return at once when
// the grouped path applied, so no host round trip decides the path.
//
// Ids at or above n_vertices are never used as an index (such edges are
// dropped), so a bad list cannot make a kernel write out of bounds.
#include "pg_internal.h"
#include "pg_trace.h"

namespace pgen {
namespace {

constexpr int kSortWarps = 16;
constexpr int kSortThreads = kSortWarps * 32;
constexpr int kMaxDigitBits = 10;
constexpr uint32_t kMaxBuckets = 1u << kMaxDigitBits;
constexpr uint32_t kScanTile = 4096;
constexpr uint32_t kGroupedMaxRow = 32;

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

template <typename P>
__device__ __forceinline__ uint32_t digit_of(const P& e, int field, int shift, uint32_t mask)
{
    const uint64_t v = field ? (uint64_t)e.x : (uint64_t)e.y;   // field 1 = src, 0 = dst
    return (uint32_t)(v >> shift) & mask;
}

// Elements per thread of a sort tile: 16 pairs of 32-bit ids or 8 of 64-bit.
template <typename Id>
struct SortShape {
    static constexpr int items = sizeof(Id) == 4 ? 16 : 8;
    static constexpr uint32_t tile = kSortThreads * items;
};

// Per-tile digit counts. Each warp counts into its own shared-memory
// histogram with plain atomic increments (no cross-warp contention; a skewed
// digit only meets the other lanes of its warp), then the warps' counts are
// summed per digit. Dynamic shared memory: kSortWarps << bits counters.
template <typename Id>
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(
    const typename PairOf<Id>::T* __restrict__ in, uint64_t M, int field, int shift, int bits,
    uint32_t* __restrict__ H, uint32_t n_tiles, const uint32_t* __restrict__ sort_needed)
{
    extern __shared__ uint32_t wh[];
    if (*sort_needed == 0) return;
    const uint32_t nb = 1u << bits, mask = nb - 1;
    const uint32_t wid = threadIdx.x >> 5;
    for (uint32_t t = threadIdx.x; t < kSortWarps * nb; t += blockDim.x) wh[t] = 0;
    __syncthreads();
    constexpr uint32_t kTile = SortShape<Id>::tile;
    const uint64_t base = (uint64_t)blockIdx.x * kTile;
    const uint64_t end = (base + kTile < M) ? base + kTile : M;
    uint32_t* mine = wh + wid * nb;
    constexpr int kUnroll = 4;
    for (uint64_t i0 = base + threadIdx.x; i0 < end; i0 += (uint64_t)kUnroll * blockDim.x) {
        uint32_t d[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint64_t i = i0 + (uint64_t)u * blockDim.x;
            d[u] = (i < end) ? digit_of(in[i], field, shift, mask) : 0xFFFFFFFFu;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (d[u] != 0xFFFFFFFFu) atomicAdd(&mine[d[u]], 1u);
    }
    __syncthreads();
    for (uint32_t dd = threadIdx.x; dd < nb; dd += blockDim.x) {
        uint32_t sum = 0;
#pragma unroll 4
        for (int w = 0; w < kSortWarps; ++w) sum += wh[w * nb + dd];
        H[(uint64_t)dd * n_tiles + blockIdx.x] = sum;
    }
}

// One LSD pass over a tile: load once, rank stably (per warp by match, then
// across warps), reorder the tile by digit in shared memory, and write each
// digit's run to its place in the output with consecutive threads on
// consecutive elements.
template <typename Id>
__global__ void __launch_bounds__(kSortThreads, 2) radix_scatter_kernel(
    const typename PairOf<Id>::T* __restrict__ in, typename PairOf<Id>::T* __restrict__ out,
    uint64_t M, int field, int shift, int bits, const uint64_t* __restrict__ Hs,
    const uint64_t* __restrict__ dstart, uint32_t n_tiles, const uint32_t* __restrict__ sort_needed)
{
    using P = typename PairOf<Id>::T;
    constexpr int kItems = SortShape<Id>::items;
    constexpr uint32_t kTile = SortShape<Id>::tile;
    extern __shared__ __align__(16) unsigned char smem[];
    uint16_t (*wcnt)[kMaxBuckets] = reinterpret_cast<uint16_t (*)[kMaxBuckets]>(smem);   // 32 KB
    uint64_t* tbase = reinterpret_cast<uint64_t*>(smem + kSortWarps * kMaxBuckets * 2);   // 8 KB
    uint32_t* loff = reinterpret_cast<uint32_t*>(tbase + kMaxBuckets);                  // 4 KB
    P* buf = reinterpret_cast<P*>(loff + kMaxBuckets);                                  // tile
    __shared__ uint32_t s_part[kSortWarps + 1];
    if (*sort_needed == 0) return;
    const uint32_t nb = 1u << bits, mask = nb - 1;
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t tile = blockIdx.x;
    for (uint32_t d = threadIdx.x; d < nb; d += blockDim.x) {
        for (int w = 0; w < kSortWarps; ++w) wcnt[w][d] = 0;
        tbase[d] = dstart[d] + Hs[(uint64_t)d * n_tiles + tile];
    }
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
    // item r of every lane, in lane order: the lowest lane of each group of
    // equal digits reads and advances the warp's counter, the group gets the
    // old value by shuffle; the counter is touched by one thread per group
    // and the syncwarp orders it before the next item's read
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const uint32_t t = wbase + r * 32 + lane;
        const uint32_t d = (t < n) ? digit_of(e[r], field, shift, mask) : 0xFFFFFFFFu;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
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
    // per digit: prefix over warps (in wcnt) and the tile total (in loff)
    for (uint32_t d = threadIdx.x; d < nb; d += blockDim.x) {
        uint32_t acc = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = wcnt[w][d];
            wcnt[w][d] = (uint16_t)acc;
            acc += c;
        }
        loff[d] = acc;
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
            const uint32_t d = digit_of(e[r], field, shift, mask);
            const uint32_t rank = (rk[r >> 1] >> ((r & 1) * 16)) & 0xFFFFu;
            buf[loff[d] + wcnt[wid][d] + rank] = e[r];
        }
    }
    __syncthreads();
    // write runs: sorted position p goes to tbase[d] + (p - loff[d])
    for (uint32_t p = threadIdx.x; p < n; p += blockDim.x) {
        const P v = buf[p];
        const uint32_t d = digit_of(v, field, shift, mask);
        out[tbase[d] + (p - loff[d])] = v;
    }
}

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

// Offsets of one LSD pass in one launch. H is digit-major: n_tiles counts
// per digit. CTA d scans its row into Hs[d][t] = sum of H[d][t'] over t' < t
// and writes the row total to tot[d]. The CTA that finishes last (it draws the
// last ticket; no CTA waits on another) scans the totals into dstart[d], the
// first output position of digit d, and puts the ticket back to zero. The
// scatter adds dstart[d] and Hs[d][t].
constexpr uint32_t kRowPer = 4;
__global__ void __launch_bounds__(1024) scan_rows_kernel(const uint32_t* __restrict__ H,
                                                         uint32_t n_tiles, uint32_t nb,
                                                         uint64_t* __restrict__ Hs,
                                                         uint64_t* __restrict__ tot,
                                                         uint64_t* __restrict__ dstart,
                                                         uint32_t* __restrict__ ticket,
                                                         const uint32_t* __restrict__ sort_needed)
{
    __shared__ uint64_t s_warp[32];
    __shared__ uint32_t s_last;
    if (*sort_needed == 0) return;
    const uint32_t d = blockIdx.x;
    const uint32_t* row = H + (uint64_t)d * n_tiles;
    uint64_t* out = Hs + (uint64_t)d * n_tiles;
    uint64_t carry = 0;
    for (uint32_t t0 = 0; t0 < n_tiles; t0 += blockDim.x * kRowPer) {
        const uint32_t tb = t0 + threadIdx.x * kRowPer;
        uint32_t v[kRowPer];
        uint64_t sum = 0;
#pragma unroll
        for (uint32_t k = 0; k < kRowPer; ++k) {
            v[k] = (tb + k < n_tiles) ? row[tb + k] : 0;
            sum += v[k];
        }
        uint64_t total;
        uint64_t run = carry + block_exclusive_scan(sum, s_warp, total);
#pragma unroll
        for (uint32_t k = 0; k < kRowPer; ++k) {
            if (tb + k < n_tiles) out[tb + k] = run;
            run += v[k];
        }
        carry += total;
    }
    if (threadIdx.x == 0) {
        tot[d] = carry;
        __threadfence();
        s_last = (atomicAdd(ticket, 1u) == nb - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (s_last == 0) return;
    __threadfence();
    const unsigned long long* tot_l2 = reinterpret_cast<const unsigned long long*>(tot);
    uint64_t start = 0;
    for (uint32_t d0 = 0; d0 < nb; d0 += blockDim.x) {
        const uint32_t i = d0 + threadIdx.x;
        const uint64_t c = i < nb ? (uint64_t)__ldcg(tot_l2 + i) : 0;   // not from L1
        uint64_t total;
        const uint64_t ex = block_exclusive_scan(c, s_warp, total);
        if (i < nb) dstart[i] = start + ex;
        start += total;
    }
    if (threadIdx.x == 0) *ticket = 0;
}

// Threads per CTA of scan_rows: enough for one trip over a row, 32 to 1024.
uint32_t scan_rows_threads(uint32_t n_tiles)
{
    const uint32_t want = (n_tiles + kRowPer - 1) / kRowPer;
    const uint32_t t = (want + 31) & ~31u;
    return t < 32 ? 32 : (t > 1024 ? 1024 : t);
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
        col[a + rank] = (Id)d;
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
                col[i] = (Id)e[u].y;
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

// S[i] = i where a run of equal pairs starts, else 0 (a prefix max then
// gives every position the start of its run).
template <typename Id>
__global__ void __launch_bounds__(256) csr_runstart_kernel(const typename PairOf<Id>::T* __restrict__ s,
                                                           uint64_t M, uint64_t* __restrict__ S)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride)
        S[i] = (i == 0 || !same_pair(s[i], s[i - 1])) ? i : 0;
}

// Whether sorted position i survives the options.
template <typename P>
__device__ __forceinline__ bool keep_at(const P* s, uint64_t M, uint64_t i, uint32_t flags,
                                        const uint64_t* S)
{
    const P e = s[i];
    if ((flags & kOptNoLoops) && e.x == e.y) return false;
    if (flags & kOptOdd) {
        const bool end = (i + 1 == M) || !same_pair(s[i + 1], e);
        return end && (((i + 1 - S[i]) & 1) != 0);
    }
    if (flags & kOptDedup) return i == 0 || !same_pair(s[i - 1], e);
    return true;
}

template <typename Id>
__global__ void __launch_bounds__(256) csr_keep_count_kernel(const typename PairOf<Id>::T* __restrict__ s,
                                                             uint64_t M, uint32_t flags,
                                                             const uint64_t* __restrict__ S,
                                                             uint64_t* __restrict__ part)
{
    __shared__ uint64_t s_warp[32];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    uint64_t cnt = 0;
    for (uint32_t t = threadIdx.x; t < kScanTile; t += blockDim.x)
        if (base + t < M) cnt += keep_at(s, M, base + t, flags, S) ? 1 : 0;
    uint64_t total;
    block_exclusive_scan(cnt, s_warp, total);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// Each thread takes kScanTile/256 consecutive positions of its tile, so the
// kept destinations are written in sorted order; the last position of every
// row writes row_ptr[src + 1] = kept entries up to and including it.
template <typename Id>
__global__ void __launch_bounds__(256) csr_keep_apply_kernel(const typename PairOf<Id>::T* __restrict__ s,
                                                             uint64_t M, uint64_t N, uint32_t flags,
                                                             const uint64_t* __restrict__ S,
                                                             const uint64_t* __restrict__ part,
                                                             Id* __restrict__ col,
                                                             uint64_t* __restrict__ row_ptr)
{
    __shared__ uint64_t s_warp[32];
    constexpr int per = kScanTile / 256;
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile + threadIdx.x * per;
    uint32_t keep = 0;
#pragma unroll
    for (int t = 0; t < per; ++t)
        if (base + t < M && keep_at(s, M, base + t, flags, S)) keep |= 1u << t;
    uint64_t total;
    uint64_t e = part[blockIdx.x] + block_exclusive_scan((uint64_t)__popc(keep), s_warp, total);
#pragma unroll
    for (int t = 0; t < per; ++t) {
        const uint64_t i = base + t;
        if (i >= M) break;
        const uint64_t v = s[i].x;
        if (keep & (1u << t)) col[e++] = (Id)s[i].y;
        if (v < N && (i + 1 == M || (uint64_t)s[i + 1].x != v)) row_ptr[v + 1] = e;
    }
}

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
    size_t off_a, off_b, off_h, off_hs, off_flag, off_dig, off_rpart, total;
    uint32_t n_tiles, max_nb;
    uint64_t n_h, n_rparts;
};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

CsrLayout csr_layout(uint64_t M, uint64_t N, size_t pair_bytes)
{
    CsrLayout L;
    const int bits = bit_length(N > 0 ? N - 1 : 0);
    const int passes = (bits + kMaxDigitBits - 1) / kMaxDigitBits;
    const int dbits = passes ? (bits + passes - 1) / passes : 0;
    const uint32_t tile = pair_bytes == 8 ? SortShape<uint32_t>::tile : SortShape<uint64_t>::tile;
    L.max_nb = 1u << dbits;
    L.n_tiles = (uint32_t)((M + tile - 1) / tile);
    L.n_h = (uint64_t)L.max_nb * L.n_tiles;
    size_t o = 0;
    L.off_a = o;
    o += a256(M * pair_bytes);
    L.off_b = o;
    o += a256(M * pair_bytes);
    L.off_h = o;
    o += a256(L.n_h * 4);
    L.off_hs = o;
    o += a256(L.n_h * 8);
    L.off_flag = o;   // +0: sort-needed flag, +64: the row scan's ticket
    o += 256;
    L.off_dig = o;    // digit totals, then digit starts (kMaxBuckets each)
    o += a256(2 * (size_t)kMaxBuckets * 8);
    L.n_rparts = (N + 1 + kScanTile - 1) / kScanTile;
    L.off_rpart = o;
    o += a256((L.n_rparts + 1) * 8);
    L.total = o;
    return L;
}

template <typename Id>
void set_csr_attributes()
{
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(radix_scatter_kernel<Id>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)scatter_smem_bytes<Id>());
        cudaFuncSetAttribute(radix_hist_kernel<Id>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kSortWarps * 4 * kMaxBuckets));
        attr = true;
    }
}

// LSD radix passes over M pairs starting at `in` (dst digits, then src
// digits). *sorted receives the sorted list (in itself when there is no
// digit to sort), *spare a ping-pong buffer the result does not occupy.
template <typename Id>
cudaError_t radix_passes(const typename PairOf<Id>::T* in, uint64_t M, uint64_t N, const CsrLayout& L,
                         unsigned char* ws, const uint32_t* sort_needed, cudaStream_t s,
                         const typename PairOf<Id>::T** sorted, typename PairOf<Id>::T** spare)
{
    using P = typename PairOf<Id>::T;
    P* buf[2] = {(P*)(ws + L.off_a), (P*)(ws + L.off_b)};
    uint32_t* H = (uint32_t*)(ws + L.off_h);
    uint64_t* Hs = (uint64_t*)(ws + L.off_hs);
    uint64_t* tot = (uint64_t*)(ws + L.off_dig);
    uint64_t* dstart = tot + kMaxBuckets;
    uint32_t* ticket = (uint32_t*)(ws + L.off_flag + 64);
    cudaError_t err;
    if (cudaMemsetAsync(ticket, 0, 4, s) != cudaSuccess) return cudaErrorUnknown;
    const int bits = bit_length(N > 0 ? N - 1 : 0);
    const int passes = (bits + kMaxDigitBits - 1) / kMaxDigitBits;
    const P* cur = in;
    int which = 0;
    if (M > 0) {
        for (int field = 0; field < 2; ++field) {      // dst digits, then src digits
            int shift = 0;
            for (int ps = 0; ps < passes; ++ps) {
                const int b = (bits - shift < (bits + passes - 1) / passes)
                                  ? bits - shift
                                  : (bits + passes - 1) / passes;
                if (b <= 0) break;
                {
                    TraceScope trace("csr_radix_hist", s);
                    radix_hist_kernel<Id><<<L.n_tiles, kSortThreads,
                                            (size_t)kSortWarps * 4 << b, s>>>(
                        cur, M, field, shift, b, H, L.n_tiles, sort_needed);
                }
                {
                    TraceScope trace("csr_scan", s);
                    scan_rows_kernel<<<1u << b, scan_rows_threads(L.n_tiles), 0, s>>>(
                        H, L.n_tiles, 1u << b, Hs, tot, dstart, ticket, sort_needed);
                }
                {
                    TraceScope trace("csr_radix_scatter", s);
                    radix_scatter_kernel<Id><<<L.n_tiles, kSortThreads, scatter_smem_bytes<Id>(), s>>>(
                        cur, buf[which], M, field, shift, b, Hs, dstart, L.n_tiles,
                        sort_needed);
                }
                if ((err = cudaGetLastError()) != cudaSuccess) return err;
                cur = buf[which];
                which ^= 1;
                shift += b;
            }
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
    max_reduce_kernel<<<(unsigned)n_parts, 256, 0, s>>>(data, n, parts);
    max_parts_kernel<<<1, 1024, 0, s>>>(parts, n_parts);
    max_apply_kernel<<<(unsigned)n_parts, 256, 0, s>>>(data, n, parts);
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
cudaError_t csr_impl(const void* d_edges, uint64_t M, uint64_t N, uint64_t* d_row_ptr, void* d_col,
                     void* d_ws, cudaStream_t s)
{
    using P = typename PairOf<Id>::T;
    const CsrLayout L = csr_layout(M, N, sizeof(P));
    set_csr_attributes<Id>();
    unsigned char* ws = (unsigned char*)d_ws;
    uint32_t* sort_needed = (uint32_t*)(ws + L.off_flag);
    cudaError_t err;
    const int grid = sort_grid(M + 1);
    if (cudaMemsetAsync(sort_needed, 0, 4, s) != cudaSuccess) return cudaErrorUnknown;
    if (cudaMemsetAsync(d_row_ptr, 0, (N + 1) * 8, s) != cudaSuccess) return cudaErrorUnknown;
    {
        TraceScope trace("csr_check", s);
        csr_check_kernel<Id><<<grid, 256, 0, s>>>((const P*)d_edges, M, sort_needed);
        csr_grouped_kernel<Id><<<grid, 256, 0, s>>>((const P*)d_edges, M, N, (Id*)d_col, d_row_ptr,
                                                   sort_needed);
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    const P* cur;
    P* spare;
    if ((err = radix_passes<Id>((const P*)d_edges, M, N, L, ws, sort_needed, s, &cur, &spare)) !=
        cudaSuccess)
        return err;
    TraceScope trace("csr_finish", s);
    csr_finish_kernel<Id><<<grid, 256, 0, s>>>(cur, M, N, d_row_ptr, (Id*)d_col, sort_needed);
    return prefix_max(d_row_ptr, N + 1, (uint64_t*)(ws + L.off_rpart), s);
}

// Workspace of the options path: the sort's layout for the (possibly
// doubled) list, then the doubled list, and the parts of two scans.
struct OptsLayout {
    CsrLayout L;
    size_t off_x, off_cpart, off_spart, total;
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
    O.off_spart = o;
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
    set_csr_attributes<Id>();
    unsigned char* ws = (unsigned char*)d_ws;
    uint32_t* sort_needed = (uint32_t*)(ws + O.L.off_flag);
    cudaError_t err;
    const uint64_t M2 = O.M2;
    // every option needs the sorted list: the sort kernels run unconditionally
    if (cudaMemsetAsync(sort_needed, 1, 4, s) != cudaSuccess) return cudaErrorUnknown;
    if (cudaMemsetAsync(d_row_ptr, 0, (N + 1) * 8, s) != cudaSuccess) return cudaErrorUnknown;
    const P* in = (const P*)d_edges;
    if ((flags & kOptSym) && M > 0) {
        P* x = (P*)(ws + O.off_x);
        csr_sym_kernel<Id><<<sort_grid(M), 256, 0, s>>>(in, M, x);
        in = x;
    }
    const P* cur;
    P* spare;
    if ((err = radix_passes<Id>(in, M2, N, O.L, ws, sort_needed, s, &cur, &spare)) != cudaSuccess)
        return err;
    TraceScope trace("csr_compact", s);
    if (M2 > 0) {
        uint64_t* S = nullptr;
        if (flags & kOptOdd) {
            S = reinterpret_cast<uint64_t*>(spare);    // M2 words fit: a pair is >= 8 bytes
            csr_runstart_kernel<Id><<<sort_grid(M2), 256, 0, s>>>(cur, M2, S);
            if ((err = prefix_max(S, M2, (uint64_t*)(ws + O.off_spart), s)) != cudaSuccess)
                return err;
        }
        uint64_t* cpart = (uint64_t*)(ws + O.off_cpart);
        csr_keep_count_kernel<Id><<<(unsigned)O.n_cparts, 256, 0, s>>>(cur, M2, flags, S, cpart);
        scan_parts_kernel<<<1, 1024, 0, s>>>(cpart, O.n_cparts, sort_needed);
        csr_keep_apply_kernel<Id><<<(unsigned)O.n_cparts, 256, 0, s>>>(cur, M2, N, flags, S, cpart,
                                                                        (Id*)d_col, d_row_ptr);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    return prefix_max(d_row_ptr, N + 1, (uint64_t*)(ws + O.L.off_rpart), s);
}

}  // namespace

size_t csr_workspace_bytes(uint64_t n_edges, uint64_t n_vertices)
{
    // one size that fits either id width
    const size_t a = csr_layout(n_edges, n_vertices, 16).total;
    const size_t b = csr_layout(n_edges, n_vertices, 8).total;
    return a > b ? a : b;
}

size_t csr_opts_workspace_bytes(uint64_t n_edges, uint64_t n_vertices, uint32_t flags)
{
    const size_t a = opts_layout(n_edges, n_vertices, flags, 16).total;
    const size_t b = opts_layout(n_edges, n_vertices, flags, 8).total;
    return a > b ? a : b;
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
                       cudaStream_t s)
{
    (void)ws_bytes;
    return id64 ? csr_impl<uint64_t>(d_edges, n_edges, n_vertices, d_row_ptr, d_col, d_ws, s)
                : csr_impl<uint32_t>(d_edges, n_edges, n_vertices, d_row_ptr, d_col, d_ws, s);
}

}  // namespace pgen

// Graph-property checks on generated graphs (Sec. 4 examines the degree
// distribution and path lengths of the generated graphs): vertex degrees,
// their histogram, and breadth-first search distances from a source.
//
// Every result is exact integer work. Degrees and histogram counts are sums
// (atomic order does not change them); BFS distances are unique even though
// the order in which a level's vertices are found depends on the schedule.
#include <cstring>

#include "../../include/pgen.h"
#include "pg_internal.h"
#include "pg_trace.h"

namespace pgen {
namespace {

constexpr uint32_t kBfsWarps = 8;          // warps per CTA of the BFS level kernel
constexpr uint32_t kHistSmem = 8192;   // histograms up to this many buckets count in smem

template <typename Id>
__global__ void __launch_bounds__(256) degree_kernel(const Id* __restrict__ e, uint64_t M,
                                                     uint64_t N, int which,
                                                     unsigned long long* __restrict__ deg)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
        const uint64_t s = e[2 * i], d = e[2 * i + 1];
        if (which != PG_DEG_IN && s < N) atomicAdd(&deg[s], 1ull);
        if (which != PG_DEG_OUT && d < N) atomicAdd(&deg[d], 1ull);
    }
}

// hist[d] = #{v : deg[v] = d} for d <= max_deg, hist[max_deg + 1] = the rest.
__global__ void __launch_bounds__(256) histogram_kernel(const uint64_t* __restrict__ deg, uint64_t N,
                                                        uint32_t max_deg,
                                                        unsigned long long* __restrict__ hist)
{
    __shared__ uint32_t h[kHistSmem];
    const uint32_t nb = max_deg + 2;
    const bool in_smem = nb <= kHistSmem;
    if (in_smem) {
        for (uint32_t t = threadIdx.x; t < nb; t += blockDim.x) h[t] = 0;
        __syncthreads();
    }
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += stride) {
        const uint64_t d = deg[v];
        const uint32_t b = d <= max_deg ? (uint32_t)d : max_deg + 1;
        if (in_smem) atomicAdd(&h[b], 1u);
        else atomicAdd(&hist[b], 1ull);
    }
    if (in_smem) {
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < nb; t += blockDim.x)
            if (h[t]) atomicAdd(&hist[t], (unsigned long long)h[t]);
    }
}

// Adjacency entries are read once per search: streaming loads, so that they
// do not push the visited bitmap out of L2.
__device__ __forceinline__ uint64_t load_streaming(const uint32_t* p) { return __ldcs(p); }
__device__ __forceinline__ uint64_t load_streaming(const uint64_t* p)
{
    return __ldcs(reinterpret_cast<const unsigned long long*>(p));
}

// Claims for one step of 32 adjacency entries: lane l holds neighbour u when
// `have`. A neighbour whose bit in the visited bitmap (N bits, small enough
// to stay in L2) is clear is claimed by an atomic OR of that bit; the claimer
// writes its distance. Claimed vertices collect in the warp's buffer (64
// slots, fewer than 32 held between steps) and leave for the next frontier
// 32 at a time, so the frontier's counter takes one atomic per 32 claims (the
// frontier's order is not part of the result).
struct BfsQueue {
    uint32_t* buf;       // this warp's 64 shared-memory slots
    uint32_t held;       // warp-uniform, < 32 between steps
    uint32_t* next;
    uint32_t* nsize;
    uint32_t* dist;
    uint32_t* vis;
    uint32_t level;
    uint64_t N;

    __device__ __forceinline__ void step(bool have, uint32_t u, uint32_t lane, uint32_t lt)
    {
        bool claim = false;
        if (have) {
            const uint32_t bit = 1u << (u & 31);
            // a stale cached word only costs an atomic that finds the bit set
            if ((vis[u >> 5] & bit) == 0) claim = (atomicOr(&vis[u >> 5], bit) & bit) == 0;
        }
        if (claim) dist[u] = level + 1;
        push(claim, u, lane, lt);
    }

    // appends u (where `take`) to the next frontier
    __device__ __forceinline__ void push(bool take, uint32_t u, uint32_t lane, uint32_t lt)
    {
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, take);
        if (take) buf[held + __popc(m & lt)] = u;
        held += __popc(m);
        if (held >= 32) {
            __syncwarp();
            uint32_t at = 0;
            if (lane == 0) at = atomicAdd(nsize, 32u);
            at = __shfl_sync(0xFFFFFFFFu, at, 0);
            if (PG_CHECK(at + lane, N)) next[at + lane] = buf[lane];
            const uint32_t rest = held - 32;
            const uint32_t x = lane < rest ? buf[32 + lane] : 0;
            __syncwarp();
            if (lane < rest) buf[lane] = x;
            __syncwarp();
            held = rest;
        }
    }

    __device__ __forceinline__ void flush(uint32_t lane)
    {
        __syncwarp();
        if (held) {
            uint32_t at = 0;
            if (lane == 0) at = atomicAdd(nsize, held);
            at = __shfl_sync(0xFFFFFFFFu, at, 0);
            if (lane < held && PG_CHECK(at + lane, N)) next[at + lane] = buf[lane];
        }
    }
};

// Rows of kLongRow or more entries leave the level kernel for the slice
// kernel, which cuts them into slices of kSlice entries spread over all warps.
constexpr uint64_t kLongRow = 64;
constexpr uint32_t kSlice = 512;

// One BFS level, short rows. Each warp takes 32 frontier vertices at a time
// and walks their short rows as one concatenated range, 32 adjacency entries
// per step: lane k of a step finds the vertex owning entry base + k by a
// binary search over the 32 rows' starts (a warp scan of their degrees, kept
// in shared memory), so short rows (most rows of a power-law graph) do not
// leave lanes idle. A long row is appended to the long-row list instead:
// one 64-bit atomic on long_ctr adds 1 to the row count (high word) and its
// slice count to the slice total (low word), so the slice bases of the list
// ascend with its index. scanned += the short rows' lengths.
template <typename Id>
__global__ void __launch_bounds__(kBfsWarps * 32) bfs_level_kernel(const uint64_t* __restrict__ row_ptr,
                                                        const Id* __restrict__ col,
                                                        const uint32_t* __restrict__ frontier,
                                                        uint32_t fsize, uint32_t* __restrict__ next,
                                                        uint32_t* __restrict__ nsize,
                                                        uint32_t* __restrict__ dist,
                                                        uint32_t* __restrict__ vis, uint32_t level,
                                                        uint64_t N,
                                                        unsigned long long* __restrict__ long_ctr,
                                                        uint32_t* __restrict__ long_v,
                                                        uint32_t* __restrict__ long_base)
{
    __shared__ uint32_t wbuf[kBfsWarps][64];
    __shared__ uint64_t wstart[kBfsWarps][32];   // the 32 rows' starts in the concatenation
    __shared__ uint64_t wrow[kBfsWarps][32];     // and in col
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    BfsQueue Q{wbuf[wid], 0, next, nsize, dist, vis, level, N};
    uint64_t* st = wstart[wid];
    uint64_t* rw = wrow[wid];
    const uint64_t first = (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32;
    for (uint64_t c = first; c < fsize; c += warps * 32) {
        uint64_t a = 0, d = 0;
        if (c + lane < fsize && PG_CHECK(frontier[c + lane], N)) {
            const uint32_t v = frontier[c + lane];
            a = row_ptr[v];
            d = row_ptr[v + 1] - a;
            if (d >= kLongRow) {
                const uint64_t ns = (d + kSlice - 1) / kSlice;
                const unsigned long long old = atomicAdd(long_ctr, (1ull << 32) | ns);
                const uint32_t r = (uint32_t)(old >> 32);
                if (PG_CHECK(r, N)) {
                    long_v[r] = v;
                    long_base[r] = (uint32_t)old;
                }
                d = 0;
            }
        }
        // inclusive scan of the short rows' lengths over the warp
        uint64_t incl = d;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        const uint64_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        st[lane] = incl - d;
        rw[lane] = a;
        __syncwarp();
        for (uint64_t base = 0; base < total; base += 32) {
            const uint64_t k = base + lane;
            bool have = false;
            uint32_t u = 0;
            if (k < total) {
                // the last row whose start is at or below k owns entry k (an
                // empty row starts where the next one does)
                uint32_t o = 0;
#pragma unroll
                for (uint32_t step = 16; step > 0; step >>= 1)
                    if (st[o + step] <= k) o += step;
                const uint64_t u64 = load_streaming(col + rw[o] + (k - st[o]));
                have = u64 < N;
                u = (uint32_t)u64;
            }
            Q.step(have, u, lane, lt);
        }
        __syncwarp();   // the next chunk rewrites the row tables
    }
    Q.flush(lane);
}

// One BFS level, long rows: slice t of the level's long rows is entries
// [t - long_base[r]) * kSlice, ...) of row r, the last row whose base is at
// or below t. Warps take slices t = warp, warp + warps, ...; a warp finds r
// by a 32-way search (each round the lanes test 32 evenly spaced bases and
// a ballot keeps the interval below the first base above t), then walks the
// slice 32 entries per step with the same claims as the level kernel.
template <typename Id>
__global__ void __launch_bounds__(kBfsWarps * 32) bfs_long_kernel(const uint64_t* __restrict__ row_ptr,
                                                       const Id* __restrict__ col,
                                                       uint32_t* __restrict__ next,
                                                       uint32_t* __restrict__ nsize,
                                                       uint32_t* __restrict__ dist,
                                                       uint32_t* __restrict__ vis, uint32_t level,
                                                       uint64_t N,
                                                       const unsigned long long* __restrict__ long_ctr,
                                                       const uint32_t* __restrict__ long_v,
                                                       const uint32_t* __restrict__ long_base)
{
    __shared__ uint32_t wbuf[kBfsWarps][64];
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const unsigned long long ctr = *long_ctr;   // written by the level kernel before
    const uint32_t rows = (uint32_t)(ctr >> 32), slices = (uint32_t)ctr;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    BfsQueue Q{wbuf[wid], 0, next, nsize, dist, vis, level, N};
    for (uint32_t t = blockIdx.x * (blockDim.x >> 5) + wid; t < slices; t += warps) {
        uint32_t lo = 0, n = rows;   // r lies in [lo, lo + n); long_base[lo] <= t
        while (n > 1) {
            const uint32_t step = (n + 31) / 32;
            const uint32_t off = lane * step;
            const bool le = off < n && PG_CHECK(lo + off, rows) && long_base[lo + off] <= t;
            const uint32_t m = __ballot_sync(0xFFFFFFFFu, le);   // lane 0 always set
            const uint32_t k = 31 - __clz(m);
            lo += k * step;
            n = (n - k * step < step) ? n - k * step : step;
        }
        uint64_t e0 = 0, e1 = 0;
        if (PG_CHECK(lo, rows) && PG_CHECK(long_v[lo], N)) {
            const uint32_t v = long_v[lo];
            const uint64_t a = row_ptr[v], end = row_ptr[v + 1];
            e0 = a + (uint64_t)(t - long_base[lo]) * kSlice;
            e1 = (e0 + kSlice < end) ? e0 + kSlice : end;
            if (e0 > e1) e0 = e1;
        }
        for (uint64_t e = e0; e < e1; e += 32) {
            bool have = false;
            uint32_t u = 0;
            if (e + lane < e1) {
                const uint64_t u64 = load_streaming(col + e + lane);
                have = u64 < N;
                u = (uint32_t)u64;
            }
            Q.step(have, u, lane, lt);
        }
    }
    Q.flush(lane);
}

// One BFS level bottom-up (Beamer, Asanovic and Patterson, "Direction-
// Optimizing Breadth-First Search", SC'12), for a symmetric CSR: every vertex
// not yet visited looks through its row for a neighbour at distance `level`
// and, at the first one, takes distance level + 1. A warp owns 32 consecutive
// vertices, one visited word, and sets their new bits with one plain store:
// no other warp writes that word during the level. A neighbour claimed in
// the same level already reads level + 1, so it is never taken for a parent.
template <typename Id>
__global__ void __launch_bounds__(kBfsWarps * 32) bfs_bottom_up_kernel(
    const uint64_t* __restrict__ row_ptr, const Id* __restrict__ col, uint32_t* __restrict__ next,
    uint32_t* __restrict__ nsize, uint32_t* __restrict__ dist, uint32_t* __restrict__ vis,
    uint32_t level, uint64_t N)
{
    __shared__ uint32_t wbuf[kBfsWarps][64];
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    BfsQueue Q{wbuf[wid], 0, next, nsize, dist, vis, level, N};
    for (uint64_t base = (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < N;
         base += warps * 32) {
        const uint64_t v = base + lane;
        const uint32_t word = vis[base >> 5];
        bool found = false;
        if (v < N && ((word >> lane) & 1u) == 0) {
            const uint64_t b = row_ptr[v + 1];
            for (uint64_t e = row_ptr[v]; e < b; ++e) {
                const uint64_t u = load_streaming(col + e);
                if (u < N && dist[u] == level) {
                    found = true;
                    break;
                }
            }
        }
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, found);
        if (found) dist[v] = level + 1;
        if (lane == 0 && m) vis[base >> 5] = word | m;
        Q.push(found, (uint32_t)v, lane, lt);
    }
    Q.flush(lane);
}

// scanned = the sum of the reached vertices' row lengths (what a top-down
// search reads, whichever direction each level ran).
__global__ void __launch_bounds__(256) bfs_reach_kernel(const uint64_t* __restrict__ row_ptr,
                                                        const uint32_t* __restrict__ dist,
                                                        uint64_t N,
                                                        unsigned long long* __restrict__ scanned)
{
    unsigned long long sum = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += stride)
        if (dist[v] != 0xFFFFFFFFu) sum += row_ptr[v + 1] - row_ptr[v];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xFFFFFFFFu, sum, o);
    if ((threadIdx.x & 31) == 0 && sum) atomicAdd(scanned, sum);
}

__global__ void bfs_seed_kernel(uint32_t* dist, uint32_t* vis, uint32_t* frontier, uint32_t source)
{
    dist[source] = 0;
    vis[source >> 5] = 1u << (source & 31);
    frontier[0] = source;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

int grid_cap(uint64_t items)
{
    const uint64_t full = (uint64_t)device_sm_count() * 8;
    const uint64_t need = (items + 255) / 256;
    return (int)(need < 1 ? 1 : (need < full ? need : full));
}

}  // namespace

PG_CHECK_UNIT(analyze)

}  // namespace pgen

using namespace pgen;

extern "C" {

pg_status pg_degrees(const void* d_edges, uint64_t n_edges, uint64_t n_vertices, pg_idwidth w,
                     int which, uint64_t* d_deg, void* stream)
{
    if (w != PG_ID32 && w != PG_ID64) return PG_EINVAL;
    if (which != PG_DEG_OUT && which != PG_DEG_IN && which != PG_DEG_TOTAL) return PG_EINVAL;
    if (n_vertices > 0 && !d_deg) return PG_EINVAL;
    if (n_edges > 0 && !d_edges) return PG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (n_vertices > 0 && cudaMemsetAsync(d_deg, 0, n_vertices * 8, s) != cudaSuccess) return PG_ECUDA;
    if (n_edges == 0) return PG_OK;
    TraceScope trace("degrees", s);
    const int grid = grid_cap(n_edges);
    if (w == PG_ID64)
        { degree_kernel<uint64_t><<<grid, 256, 0, s>>>((const uint64_t*)d_edges, n_edges, n_vertices,
                                                    which, (unsigned long long*)d_deg); note_launch(); }
    else
        { degree_kernel<uint32_t><<<grid, 256, 0, s>>>((const uint32_t*)d_edges, n_edges, n_vertices,
                                                    which, (unsigned long long*)d_deg); note_launch(); }
    return cudaGetLastError() == cudaSuccess ? PG_OK : PG_ECUDA;
}

pg_status pg_degree_histogram(const uint64_t* d_deg, uint64_t n_vertices, uint32_t max_degree,
                              uint64_t* d_hist, void* stream)
{
    if (!d_hist || (n_vertices > 0 && !d_deg) || max_degree > 0xFFFFFFF0u) return PG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(d_hist, 0, ((size_t)max_degree + 2) * 8, s) != cudaSuccess) return PG_ECUDA;
    if (n_vertices == 0) return PG_OK;
    TraceScope trace("degree_histogram", s);
    { histogram_kernel<<<grid_cap(n_vertices), 256, 0, s>>>(d_deg, n_vertices, max_degree,
                                                         (unsigned long long*)d_hist); note_launch(); }
    return cudaGetLastError() == cudaSuccess ? PG_OK : PG_ECUDA;
}

size_t pg_bfs_workspace_size(uint64_t n_vertices)
{
    // two frontiers of n_vertices uint32, the counters, the visited bitmap,
    // and the long-row list (a vertex and a slice base per row)
    return 4 * (((size_t)n_vertices * 4 + 255) & ~(size_t)255) + 256 +
           ((((size_t)n_vertices + 31) / 32 * 4 + 255) & ~(size_t)255);
}

pg_status pg_bfs(const uint64_t* d_row_ptr, const void* d_col, uint64_t n_vertices, pg_idwidth w,
                 uint64_t source, uint32_t flags, uint32_t* d_dist, void* d_ws, size_t ws_bytes,
                 uint32_t* levels_out, uint64_t* scanned_out, void* stream)
{
    if (w != PG_ID32 && w != PG_ID64) return PG_EINVAL;
    if (flags & ~(uint32_t)PG_BFS_UNDIRECTED) return PG_EINVAL;
    if (n_vertices == 0 || n_vertices >= 0xFFFFFFFFull || source >= n_vertices) return PG_EINVAL;
    if (!d_row_ptr || !d_col || !d_dist || !d_ws || !aligned(d_ws, 256)) return PG_EINVAL;
    if (ws_bytes < pg_bfs_workspace_size(n_vertices)) return PG_ENOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t fbytes = ((size_t)n_vertices * 4 + 255) & ~(size_t)255;
    unsigned char* ws = (unsigned char*)d_ws;
    uint32_t* fr[2] = {(uint32_t*)ws, (uint32_t*)(ws + fbytes)};
    // counters: the next frontier's size and the long-row list's counts,
    // zeroed every level, then the scanned total
    uint32_t* nsize = (uint32_t*)(ws + 2 * fbytes);
    unsigned long long* long_ctr = (unsigned long long*)(ws + 2 * fbytes + 8);
    unsigned long long* scanned = (unsigned long long*)(ws + 2 * fbytes + 16);
    uint32_t* vis = (uint32_t*)(ws + 2 * fbytes + 256);
    const size_t vbytes = ((size_t)n_vertices + 31) / 32 * 4;
    unsigned char* lists = ws + 2 * fbytes + 256 + ((vbytes + 255) & ~(size_t)255);
    uint32_t* long_v = (uint32_t*)lists;
    uint32_t* long_base = (uint32_t*)(lists + fbytes);
    if (cudaMemsetAsync(d_dist, 0xFF, n_vertices * 4, s) != cudaSuccess) return PG_ECUDA;
    if (cudaMemsetAsync(ws + 2 * fbytes, 0, 256, s) != cudaSuccess) return PG_ECUDA;
    if (cudaMemsetAsync(vis, 0, vbytes, s) != cudaSuccess) return PG_ECUDA;
    { bfs_seed_kernel<<<1, 1, 0, s>>>(d_dist, vis, fr[0], (uint32_t)source); note_launch(); }
    uint32_t fsize = 1, level = 0, cur = 0;
    uint64_t visited = 1;
    bool bottom_up = false;
    TraceScope trace("bfs", s);
    // the slice kernel's grid: every warp of a full wave takes slices
    const int long_grid = device_sm_count() * 8;
    const bool undirected = (flags & PG_BFS_UNDIRECTED) != 0;
    while (fsize > 0) {
        // direction of this level (Beamer et al.'s rule with vertex counts
        // standing in for edge counts): bottom-up once the frontier is more
        // than 1/30 of the vertices not yet visited, top-down again once it
        // is under 1/24 of all vertices
        if (undirected) {
            if (!bottom_up && (uint64_t)fsize * 30 > n_vertices - visited) bottom_up = true;
            else if (bottom_up && (uint64_t)fsize * 24 < n_vertices) bottom_up = false;
        }
        if (cudaMemsetAsync(nsize, 0, 16, s) != cudaSuccess) return PG_ECUDA;
        if (bottom_up) {
            TraceScope bu_trace("bfs_bottom_up", s);
            const int grid = grid_cap(n_vertices);
            if (w == PG_ID64)
                { bfs_bottom_up_kernel<uint64_t><<<grid, kBfsWarps * 32, 0, s>>>(
                    d_row_ptr, (const uint64_t*)d_col, fr[cur ^ 1], nsize, d_dist, vis, level,
                    n_vertices); note_launch(); }
            else
                { bfs_bottom_up_kernel<uint32_t><<<grid, kBfsWarps * 32, 0, s>>>(
                    d_row_ptr, (const uint32_t*)d_col, fr[cur ^ 1], nsize, d_dist, vis, level,
                    n_vertices); note_launch(); }
        } else {
            const int grid = grid_cap(fsize);
            if (w == PG_ID64) {
                { bfs_level_kernel<uint64_t><<<grid, kBfsWarps * 32, 0, s>>>(
                    d_row_ptr, (const uint64_t*)d_col, fr[cur], fsize, fr[cur ^ 1], nsize, d_dist,
                    vis, level, n_vertices, long_ctr, long_v, long_base); note_launch(); }
                { bfs_long_kernel<uint64_t><<<long_grid, kBfsWarps * 32, 0, s>>>(
                    d_row_ptr, (const uint64_t*)d_col, fr[cur ^ 1], nsize, d_dist, vis, level,
                    n_vertices, long_ctr, long_v, long_base); note_launch(); }
            } else {
                { bfs_level_kernel<uint32_t><<<grid, kBfsWarps * 32, 0, s>>>(
                    d_row_ptr, (const uint32_t*)d_col, fr[cur], fsize, fr[cur ^ 1], nsize, d_dist,
                    vis, level, n_vertices, long_ctr, long_v, long_base); note_launch(); }
                { bfs_long_kernel<uint32_t><<<long_grid, kBfsWarps * 32, 0, s>>>(
                    d_row_ptr, (const uint32_t*)d_col, fr[cur ^ 1], nsize, d_dist, vis, level,
                    n_vertices, long_ctr, long_v, long_base); note_launch(); }
            }
        }
        if (cudaGetLastError() != cudaSuccess) return PG_ECUDA;
        // the next frontier's size decides whether another level runs
        if (cudaMemcpyAsync(&fsize, nsize, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return PG_ECUDA;
        visited += fsize;
        cur ^= 1;
        ++level;
    }
    { bfs_reach_kernel<<<grid_cap(n_vertices), 256, 0, s>>>(d_row_ptr, d_dist, n_vertices, scanned); note_launch(); }
    uint64_t sc = 0;
    if (cudaMemcpyAsync(&sc, scanned, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return PG_ECUDA;
    if (levels_out) *levels_out = level;
    if (scanned_out) *scanned_out = sc;
    return PG_OK;
}

}  // extern "C"

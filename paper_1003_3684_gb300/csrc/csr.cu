// CSR assembly of a generated edge list.
//
// The rows must hold their destinations in ascending order, so the edge list
// is sorted by the key (src, dst) with a least-significant-digit radix sort:
// first the digits of dst, then those of src, up to 10 bits per pass. Each
// pass is three kernels:
//   radix_hist     per-tile digit counts, stored digit-major H[d][tile];
//   scan_*         one exclusive scan over H gives, for every (digit, tile),
//                  where that tile's run of the digit starts in the output;
//   radix_scatter  stable rank of each element within its tile among equal
//                  digits (warp match + per-warp counters + cross-warp scan)
//                  and a scattered write of the (src, dst) pair.
// No atomics decide any position, so the result does not depend on the
// schedule, and a power-law row (a hub with 10^5 edges) costs no more than
// any other key. A final pass writes col and fills row_ptr from the row
// boundaries of the sorted list (row_ptr[v] = first index with src >= v).
#include "pg_internal.h"
#include "pg_trace.h"

namespace pgen {
namespace {

constexpr int kSortWarps = 16;
constexpr int kSortThreads = kSortWarps * 32;
constexpr int kSortItems = 16;
constexpr uint32_t kSortTile = kSortThreads * kSortItems;   // 8192
constexpr int kMaxDigitBits = 10;
constexpr uint32_t kMaxBuckets = 1u << kMaxDigitBits;
constexpr uint32_t kScanTile = 4096;

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

template <typename Id>
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(
    const typename PairOf<Id>::T* __restrict__ in, uint64_t M, int field, int shift, int bits,
    uint32_t* __restrict__ H, uint32_t n_tiles)
{
    __shared__ uint32_t h[kMaxBuckets];
    const uint32_t nb = 1u << bits, mask = nb - 1;
    for (uint32_t d = threadIdx.x; d < nb; d += blockDim.x) h[d] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * kSortTile;
    const uint64_t end = (base + kSortTile < M) ? base + kSortTile : M;
    for (uint64_t i = base + threadIdx.x; i < end; i += blockDim.x)
        atomicAdd(&h[digit_of(in[i], field, shift, mask)], 1u);
    __syncthreads();
    for (uint32_t d = threadIdx.x; d < nb; d += blockDim.x)
        H[(uint64_t)d * n_tiles + blockIdx.x] = h[d];
}

template <typename Id>
__global__ void __launch_bounds__(kSortThreads, 2) radix_scatter_kernel(
    const typename PairOf<Id>::T* __restrict__ in, typename PairOf<Id>::T* __restrict__ out,
    uint64_t M, int field, int shift, int bits, const uint64_t* __restrict__ Hs, uint32_t n_tiles)
{
    using P = typename PairOf<Id>::T;
    __shared__ uint16_t wcnt[kSortWarps][kMaxBuckets];   // 32 KB
    __shared__ uint64_t tbase[kMaxBuckets];               // 8 KB
    const uint32_t nb = 1u << bits, mask = nb - 1;
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t tile = blockIdx.x;
    for (uint32_t d = threadIdx.x; d < nb; d += blockDim.x) {
        for (int w = 0; w < kSortWarps; ++w) wcnt[w][d] = 0;
        tbase[d] = Hs[(uint64_t)d * n_tiles + tile];
    }
    __syncthreads();
    const uint64_t base = (uint64_t)tile * kSortTile + wid * (32 * kSortItems);
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t dig[kSortItems], rnk[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint64_t i = base + r * 32 + lane;
        const uint32_t d = (i < M) ? digit_of(in[i], field, shift, mask) : 0xFFFFFFFFu;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        uint32_t prev = 0;
        if (d != 0xFFFFFFFFu) prev = wcnt[wid][d];
        __syncwarp();
        if (d != 0xFFFFFFFFu && (peers & lt) == 0) wcnt[wid][d] = (uint16_t)(prev + __popc(peers));
        __syncwarp();
        dig[r] = d;
        rnk[r] = prev + __popc(peers & lt);
    }
    __syncthreads();
    for (uint32_t d = threadIdx.x; d < nb; d += blockDim.x) {
        uint32_t acc = 0;
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = wcnt[w][d];
            wcnt[w][d] = (uint16_t)acc;
            acc += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint64_t i = base + r * 32 + lane;
        if (dig[r] != 0xFFFFFFFFu) {
            const P e = in[i];
            out[tbase[dig[r]] + wcnt[wid][dig[r]] + rnk[r]] = e;
        }
    }
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

// per-tile sums (tile = kScanTile counts, 256 threads x 16)
__global__ void __launch_bounds__(256) scan_reduce_kernel(const uint32_t* __restrict__ in,
                                                          uint64_t n, uint64_t* __restrict__ part)
{
    __shared__ uint64_t s_warp[32];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    uint64_t sum = 0;
    for (uint32_t t = threadIdx.x; t < kScanTile; t += blockDim.x)
        if (base + t < n) sum += in[base + t];
    uint64_t total;
    block_exclusive_scan(sum, s_warp, total);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// exclusive scan of the tile sums, one CTA looping over chunks
__global__ void __launch_bounds__(1024) scan_parts_kernel(uint64_t* __restrict__ part,
                                                          uint64_t n_parts)
{
    __shared__ uint64_t s_warp[32];
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

__global__ void __launch_bounds__(256) scan_apply_kernel(const uint32_t* __restrict__ in,
                                                         uint64_t n,
                                                         const uint64_t* __restrict__ part,
                                                         uint64_t* __restrict__ out)
{
    __shared__ uint64_t s_warp[32];
    constexpr int per = kScanTile / 256;
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile + threadIdx.x * per;
    uint32_t v[per];
    uint64_t sum = 0;
#pragma unroll
    for (int t = 0; t < per; ++t) {
        v[t] = (base + t < n) ? in[base + t] : 0;
        sum += v[t];
    }
    uint64_t total;
    uint64_t run = part[blockIdx.x] + block_exclusive_scan(sum, s_warp, total);
#pragma unroll
    for (int t = 0; t < per; ++t) {
        if (base + t < n) out[base + t] = run;
        run += v[t];
    }
}

// ---- final pass: col and row_ptr from the sorted pairs ---------------------
template <typename Id>
__global__ void __launch_bounds__(256) csr_finish_kernel(const typename PairOf<Id>::T* __restrict__ s,
                                                         uint64_t M, uint64_t N,
                                                         uint64_t* __restrict__ row_ptr,
                                                         Id* __restrict__ col)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= M; i += stride) {
        // rows (prev_src, cur_src] start at index i
        const uint64_t lo = (i == 0) ? 0 : (uint64_t)s[i - 1].x + 1;
        const uint64_t hi = (i == M) ? N : (uint64_t)s[i].x;
        for (uint64_t v = lo; v <= hi && v <= N; ++v) row_ptr[v] = i;
        if (i < M) col[i] = (Id)s[i].y;
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
    size_t off_a, off_b, off_h, off_hs, off_part, total;
    uint32_t n_tiles, max_nb;
    uint64_t n_h, n_parts;
};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

CsrLayout csr_layout(uint64_t M, uint64_t N, size_t pair_bytes)
{
    CsrLayout L;
    const int bits = bit_length(N > 0 ? N - 1 : 0);
    const int passes = (bits + kMaxDigitBits - 1) / kMaxDigitBits;
    const int dbits = passes ? (bits + passes - 1) / passes : 0;
    L.max_nb = 1u << dbits;
    L.n_tiles = (uint32_t)((M + kSortTile - 1) / kSortTile);
    L.n_h = (uint64_t)L.max_nb * L.n_tiles;
    L.n_parts = (L.n_h + kScanTile - 1) / kScanTile;
    size_t o = 0;
    L.off_a = o;
    o += a256(M * pair_bytes);
    L.off_b = o;
    o += a256(M * pair_bytes);
    L.off_h = o;
    o += a256(L.n_h * 4);
    L.off_hs = o;
    o += a256(L.n_h * 8);
    L.off_part = o;
    o += a256((L.n_parts + 1) * 8);
    L.total = o;
    return L;
}

template <typename Id>
cudaError_t csr_impl(const void* d_edges, uint64_t M, uint64_t N, uint64_t* d_row_ptr, void* d_col,
                     void* d_ws, cudaStream_t s)
{
    using P = typename PairOf<Id>::T;
    const CsrLayout L = csr_layout(M, N, sizeof(P));
    unsigned char* ws = (unsigned char*)d_ws;
    P* buf[2] = {(P*)(ws + L.off_a), (P*)(ws + L.off_b)};
    uint32_t* H = (uint32_t*)(ws + L.off_h);
    uint64_t* Hs = (uint64_t*)(ws + L.off_hs);
    uint64_t* part = (uint64_t*)(ws + L.off_part);
    cudaError_t err;

    const int bits = bit_length(N > 0 ? N - 1 : 0);
    const int passes = (bits + kMaxDigitBits - 1) / kMaxDigitBits;
    const P* cur = (const P*)d_edges;
    int which = 0;
    if (M > 0) {
        for (int field = 0; field < 2; ++field) {      // dst digits, then src digits
            int shift = 0;
            for (int ps = 0; ps < passes; ++ps) {
                const int b = (bits - shift < (bits + passes - 1) / passes)
                                  ? bits - shift
                                  : (bits + passes - 1) / passes;
                if (b <= 0) break;
                const uint64_t nh = ((uint64_t)1 << b) * L.n_tiles;
                {
                    TraceScope trace("csr_radix_hist", s);
                    radix_hist_kernel<Id><<<L.n_tiles, kSortThreads, 0, s>>>(cur, M, field, shift,
                                                                             b, H, L.n_tiles);
                }
                const uint64_t n_parts = (nh + kScanTile - 1) / kScanTile;
                {
                    TraceScope trace("csr_scan", s);
                    scan_reduce_kernel<<<(unsigned)n_parts, 256, 0, s>>>(H, nh, part);
                    scan_parts_kernel<<<1, 1024, 0, s>>>(part, n_parts);
                    scan_apply_kernel<<<(unsigned)n_parts, 256, 0, s>>>(H, nh, part, Hs);
                }
                {
                    TraceScope trace("csr_radix_scatter", s);
                    radix_scatter_kernel<Id><<<L.n_tiles, kSortThreads, 0, s>>>(
                        cur, buf[which], M, field, shift, b, Hs, L.n_tiles);
                }
                if ((err = cudaGetLastError()) != cudaSuccess) return err;
                cur = buf[which];
                which ^= 1;
                shift += b;
            }
        }
    }
    const uint64_t work = M + 1;
    int grid = (int)((work + 255) / 256);
    const int cap = device_sm_count() * 8;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    TraceScope trace("csr_finish", s);
    csr_finish_kernel<Id><<<grid, 256, 0, s>>>(cur, M, N, d_row_ptr, (Id*)d_col);
    return cudaGetLastError();
}

}  // namespace

size_t csr_workspace_bytes(uint64_t n_edges, uint64_t n_vertices)
{
    // sized for 16-byte pairs so that one size fits either id width
    return csr_layout(n_edges, n_vertices, 16).total;
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

// Parallel Barabasi-Albert generator (arXiv 1003.3684, Sec. 3, PBA method).
//
// The paper runs one processor per vertex block and exchanges messages
// between phases. Here a block's phases run as data-parallel kernels over
// (block, segment) pairs on one GPU, and every message becomes HBM traffic:
//
//   pba_prefix   phase 1, first P entries of every block's list A_p, built
//                in shared memory level by level (entries [L, 2L) only copy
//                from [0, 2L)); written to A_p.
//   pba_phase1   phase 1, the rest of A_p. Entry j copies a uniform earlier
//                entry r < j, or is an inter-faction pick. Instead of walking
//                A_p in order, each entry follows its own chain of copy
//                pointers (one Philox per link, recomputed from the counter)
//                until it reaches a pick or the shared-memory prefix. Writes
//                A_p (uint16) and a per-(block, segment) count of each
//                target block -- the paper's count message.
//   pba_scan     exclusive scan of the counts over (requester, segment) per
//                target block: R_q (how many endpoints q must produce) and
//                the start of each requester segment's slice of q's list.
//   pba_emit     phase 2 and substitution. The stable rank of entry j among
//                the entries of its segment that name the same block (warp
//                match + per-warp counters + cross-warp scan) gives index i
//                into q's endpoint list T_q; T_q[i] is resolved by its own
//                copy chain through q's local preferential attachment
//                (recomputed, never materialised), and the finished (src,
//                dst) pairs leave through a shared-memory staging tile as
//                coalesced vector stores.
//
// blocks = 1 is serial BA: ba_kernel resolves edge j's chain directly.
//
// Copy chains are geometric in length, so each thread owns ITEMS entries and
// advances whichever one it is working on by one link per loop trip; a warp
// then waits for the slowest lane's sum of ITEMS chains rather than for the
// longest single chain.
#include "pg_internal.h"
#include "pg_trace.h"

namespace pgen {
namespace {

constexpr uint32_t kPrefixMax = 65536;    // phase-1 prefix held in smem (uint16)
constexpr int kP1Threads = 1024;
constexpr int kP1Items = 16;
constexpr uint64_t kP1Tile = (uint64_t)kP1Threads * kP1Items;   // 16384
constexpr int kEmitWarps = 16;
constexpr int kEmitThreads = kEmitWarps * 32;
constexpr int kEmitItems = 16;
constexpr uint32_t kEmitTile = kEmitThreads * kEmitItems;        // 8192
constexpr uint32_t kMaxBlocks = 1024;
constexpr int kBaThreads = 256;
constexpr int kBaItems = 16;
constexpr uint32_t kBaTile = kBaThreads * kBaItems;              // 4096

static_assert(kP1Tile % kEmitTile == 0, "segment length must suit both tiles");

// Inter-faction pick: uniform over the B - W blocks outside [phi, phi + W).
__device__ __forceinline__ uint32_t fresh_block(uint32_t w3, uint32_t B, uint32_t W,
                                                uint32_t phi)
{
    const uint32_t x = __umulhi(w3, B - W);
    return x < phi ? x : x + W;
}

// ---------------------------------------------------------------------------
// Phase 1, prefix [0, P) of each block, built in shared memory.
// grid = B, block = kP1Threads, dynamic smem = P * 2 bytes.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kP1Threads) pba_prefix_kernel(const __grid_constant__ PbaGeom g,
                                                                uint16_t* __restrict__ A)
{
    extern __shared__ uint16_t sA[];
    const uint32_t p = blockIdx.x;
    const uint32_t phi = (p / g.W) * g.W;
    const uint32_t P = g.P;
    const uint32_t s = g.W < P ? g.W : P;
    for (uint32_t t = threadIdx.x; t < s; t += blockDim.x) sA[t] = (uint16_t)(phi + t);
    __syncthreads();
    for (uint32_t L = s; L < P;) {
        const uint32_t hi = (2 * L < P) ? 2 * L : P;
        for (uint32_t j = L + threadIdx.x; j < hi; j += blockDim.x) {
            uint64_t cur = j;
            uint32_t v;
            for (;;) {
                const uint4 w = draw(cur, p, 1, g.key);
                if (g.coin_on && w.z < g.coin_thr) {
                    v = fresh_block(w.w, g.B, g.W, phi);
                    break;
                }
                const uint64_t r = uniform64(w.x, w.y, cur);
                if (r < L) {
                    v = sA[r];
                    break;
                }
                cur = r;   // r lies in [L, j): follow its chain too
            }
            sA[j] = (uint16_t)v;
        }
        __syncthreads();
        L = hi;
    }
    uint16_t* Ap = A + (uint64_t)p * g.A_stride;
    for (uint32_t t = threadIdx.x; t < P; t += blockDim.x) Ap[t] = sA[t];
}

// ---------------------------------------------------------------------------
// Phase 1, entries of one (block, segment); grid = (S, B).
// dynamic smem: prefix P*2 | histogram B*4 | staging kP1Tile*2
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kP1Threads, 1) pba_phase1_kernel(const __grid_constant__ PbaGeom g,
                                                                   uint16_t* __restrict__ A,
                                                                   uint32_t* __restrict__ cnt)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint16_t* sA = reinterpret_cast<uint16_t*>(smem);
    uint32_t* hist = reinterpret_cast<uint32_t*>(smem + ((g.P * 2 + 15) & ~15u));
    uint16_t* sOut = reinterpret_cast<uint16_t*>(reinterpret_cast<unsigned char*>(hist) +
                                                 (((size_t)g.B * 4 + 15) & ~(size_t)15));
    const uint32_t p = blockIdx.y, sgm = blockIdx.x;
    const uint32_t phi = (p / g.W) * g.W;
    const uint32_t P = g.P;
    uint16_t* Ap = A + (uint64_t)p * g.A_stride;   // 16-byte aligned row
    const uint64_t lo = (uint64_t)sgm * g.seg_len;
    const uint64_t hi = (lo + g.seg_len < g.N_e) ? lo + g.seg_len : g.N_e;

    for (uint32_t t = threadIdx.x; t < P / 8; t += blockDim.x)
        reinterpret_cast<uint4*>(sA)[t] = reinterpret_cast<const uint4*>(Ap)[t];
    for (uint32_t t = (P & ~7u) + threadIdx.x; t < P; t += blockDim.x) sA[t] = Ap[t];
    for (uint32_t t = threadIdx.x; t < g.B; t += blockDim.x) hist[t] = 0;
    __syncthreads();

    for (uint64_t base = lo; base < hi; base += kP1Tile) {
        int k = 0;
        uint64_t j = base + threadIdx.x;
        uint64_t cur = j;
        while (k < kP1Items) {
            bool done = true;
            uint32_t v = 0;
            if (j < hi) {
                if (cur < P) {
                    v = sA[cur];
                } else {
                    const uint4 w = draw(cur, p, 1, g.key);
                    if (g.coin_on && w.z < g.coin_thr) {
                        v = fresh_block(w.w, g.B, g.W, phi);
                    } else {
                        cur = uniform64(w.x, w.y, cur);
                        done = false;
                    }
                }
            }
            if (done) {
                if (j < hi) {
                    sOut[k * kP1Threads + threadIdx.x] = (uint16_t)v;
                    atomicAdd(&hist[v], 1u);
                }
                ++k;
                j += kP1Threads;
                cur = j;
            }
        }
        __syncthreads();
        // coalesced store of the tile (entries [base, min(base + tile, hi)))
        const uint64_t n = (hi - base < kP1Tile) ? hi - base : kP1Tile;
        if (n == kP1Tile) {   // base is a multiple of the tile: aligned
            const uint4* src = reinterpret_cast<const uint4*>(sOut);
            uint4* dst = reinterpret_cast<uint4*>(Ap + base);
            for (uint32_t t = threadIdx.x; t < kP1Tile / 8; t += blockDim.x) dst[t] = src[t];
        } else {
            for (uint32_t t = threadIdx.x; t < n; t += blockDim.x) Ap[base + t] = sOut[t];
        }
        __syncthreads();
    }
    uint32_t* row = cnt + ((uint64_t)p * g.S + sgm) * g.B;
    for (uint32_t t = threadIdx.x; t < g.B; t += blockDim.x) row[t] = hist[t];
}

// ---------------------------------------------------------------------------
// Count exchange: per target block q, exclusive scan over rows (p, segment)
// of cnt[row][q]; writes off[row][q], R[q] and the divisor for R[q].
// grid = ceil(B / 32), block = 1024 (warp w scans a slab of rows, lane = q).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) pba_scan_kernel(const uint32_t* __restrict__ cnt,
                                                        uint64_t* __restrict__ off,
                                                        uint64_t* __restrict__ R,
                                                        FastDiv* __restrict__ divR, uint32_t B,
                                                        uint32_t rows)
{
    __shared__ uint64_t part[32][33];
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t q = blockIdx.x * 32 + lane;
    const uint32_t per = (rows + 31) / 32;
    const uint32_t r0 = w * per;
    const uint32_t r1 = (r0 + per < rows) ? r0 + per : rows;
    uint64_t sum = 0;
    if (q < B)
        for (uint32_t r = r0; r < r1; ++r) sum += cnt[(uint64_t)r * B + q];
    part[w][lane] = sum;
    __syncthreads();
    if (w == 0) {
        uint64_t acc = 0;
        for (int x = 0; x < 32; ++x) {
            const uint64_t c = part[x][lane];
            part[x][lane] = acc;
            acc += c;
        }
        if (q < B) {
            R[q] = acc;
            divR[q] = make_fastdiv(acc > 0 ? acc : 1);
        }
    }
    __syncthreads();
    if (q < B) {
        uint64_t acc = part[w][lane];
        for (uint32_t r = r0; r < r1; ++r) {
            const uint64_t c = cnt[(uint64_t)r * B + q];
            off[(uint64_t)r * B + q] = acc;
            acc += c;
        }
    }
}

// ---------------------------------------------------------------------------
// Phase 2 endpoint T_q[i] (local id in block q) by its copy chain through q's
// local preferential attachment: local edge i stands at source time
// sigma(i) = floor(i*n_b/R_q) and copies a uniform slot among the seed clique
// and the E(sigma(i)) = ceil(sigma(i)*R_q/n_b) edges of earlier source times.
// One Philox per link; returns after the link that lands on a seed slot or on
// the source end of an earlier edge.
// ---------------------------------------------------------------------------
struct QDiv {
    uint64_t R;
    FastDiv d;
};

__device__ __forceinline__ uint16_t pack_shifts(const FastDiv& f)
{
    return (uint16_t)(f.s1 | (f.s2 << 8));
}

// one link of the chain; returns true and sets v when finished
__device__ __forceinline__ bool t_step(uint64_t& cur, uint32_t q, const QDiv& qd,
                                       const PbaGeom& g, uint32_t& v)
{
    const uint64_t sig = fdiv(cur * g.n_b, qd.d);
    const uint64_t before = fdiv(sig * qd.R + (g.n_b - 1), g.div_nb);
    const uint4 w = draw(cur, q, 2, g.key);
    const uint64_t r = uniform64(w.x, w.y, 2 * (g.e0 + before));
    uint64_t e = r >> 1;
    if (e < g.e0) {
        v = seed_endpoint(e, (uint32_t)(r & 1), g.n0);
        return true;
    }
    e -= g.e0;
    if ((r & 1) == 0) {
        v = g.n0 + (uint32_t)fdiv(e * g.n_b, qd.d);
        return true;
    }
    cur = e;
    return false;
}

// Serial BA (blocks = 1): sigma(i) = i div m, E = sigma * m.
__device__ __forceinline__ bool ba_step(uint64_t& cur, const PbaGeom& g, uint64_t& v)
{
    const uint64_t sig = fdiv(cur, g.div_m);
    const uint4 w = draw(cur, 0, 2, g.key);
    const uint64_t r = uniform64(w.x, w.y, 2 * (g.e0 + sig * g.m));
    uint64_t e = r >> 1;
    if (e < g.e0) {
        v = seed_endpoint(e, (uint32_t)(r & 1), g.n0);
        return true;
    }
    e -= g.e0;
    if ((r & 1) == 0) {
        v = g.n0 + fdiv(e, g.div_m);
        return true;
    }
    cur = e;
    return false;
}

template <typename Id>
__device__ __forceinline__ void store_pair(Id* out, uint64_t e, uint64_t s, uint64_t d)
{
    out[2 * e] = (Id)s;
    out[2 * e + 1] = (Id)d;
}

template <typename Id>
__device__ __forceinline__ void store_two(Id* out, uint64_t e, uint64_t s0, uint64_t d0,
                                          uint64_t s1, uint64_t d1)
{
    if constexpr (sizeof(Id) == 4) {
        *reinterpret_cast<uint4*>(out + 2 * e) =
            make_uint4((uint32_t)s0, (uint32_t)d0, (uint32_t)s1, (uint32_t)d1);
    } else {
        ulonglong2* o = reinterpret_cast<ulonglong2*>(out + 2 * e);
        o[0] = make_ulonglong2(s0, d0);
        o[1] = make_ulonglong2(s1, d1);
    }
}

// Writes n consecutive edges starting at global edge index e_first; edge t
// comes from edge_at(t, src, dst). Pairs of edges whose first index is even
// go out as one 16-byte (uint32 ids) or two 16-byte (uint64 ids) stores; an
// odd first index is written alone first so that the rest stay aligned.
template <typename Id, typename F>
__device__ __forceinline__ void emit_tile(Id* out, uint64_t e_first, uint32_t n, F&& edge_at)
{
    const uint32_t head = (uint32_t)(e_first & 1) < n ? (uint32_t)(e_first & 1) : n;
    if (head && threadIdx.x == 0) {
        uint64_t s0, d0;
        edge_at(0, s0, d0);
        store_pair(out, e_first, s0, d0);
    }
    for (uint32_t t2 = head + 2 * threadIdx.x; t2 < n; t2 += 2 * blockDim.x) {
        uint64_t s0, d0;
        edge_at(t2, s0, d0);
        if (t2 + 1 < n) {
            uint64_t s1, d1;
            edge_at(t2 + 1, s1, d1);
            store_two(out, e_first + t2, s0, d0, s1, d1);
        } else {
            store_pair(out, e_first + t2, s0, d0);
        }
    }
}

// Seed clique of one block (e0 edges, lexicographic) at out[e_first...].
template <typename Id>
__device__ void write_seed_edges(Id* out, uint64_t e_first, uint64_t base, uint32_t n0)
{
    const uint64_t e0 = (uint64_t)n0 * (n0 - 1) / 2;
    for (uint64_t e = threadIdx.x; e < e0; e += blockDim.x)
        store_pair(out, e_first + e, base + seed_endpoint(e, 0, n0),
                   base + seed_endpoint(e, 1, n0));
}

// ---------------------------------------------------------------------------
// Phase 2 + substitution + emission for one (block, segment); grid = (S, B).
// ---------------------------------------------------------------------------
struct EmitSmem {   // 108 KB: two CTAs per SM
    uint64_t cur[kMaxBlocks];                   // next unused index into T_q
    uint64_t R[kMaxBlocks];                     // R_q
    uint64_t mul[kMaxBlocks];                   // divisor multiplier for R_q
    uint16_t sh[kMaxBlocks];                    // divisor shifts (s1 | s2 << 8)
    uint16_t wcnt[kEmitWarps + 1][kMaxBlocks];  // per-warp counts / prefixes; last row = tile total
    uint32_t item[kEmitTile];                   // local rank, then resolved local id
    uint16_t qs[kEmitTile];                     // target block of each entry
};

template <typename Id>
__global__ void __launch_bounds__(kEmitThreads, 2) pba_emit_kernel(
    const __grid_constant__ PbaGeom g, const uint16_t* __restrict__ A,
    const uint64_t* __restrict__ off, const uint64_t* __restrict__ R,
    const FastDiv* __restrict__ divR, Id* __restrict__ out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    EmitSmem& sm = *reinterpret_cast<EmitSmem*>(smem_raw);
    const uint32_t p = blockIdx.y, sgm = blockIdx.x;
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t B = g.B;
    const uint16_t* Ap = A + (uint64_t)p * g.A_stride;
    const uint64_t lo = (uint64_t)sgm * g.seg_len;
    const uint64_t hi = (lo + g.seg_len < g.N_e) ? lo + g.seg_len : g.N_e;
    const uint64_t out_block = (uint64_t)p * (g.e0 + g.N_e);
    const uint64_t src_base = (uint64_t)p * g.span + g.n0;

    const uint64_t* offrow = off + ((uint64_t)p * g.S + sgm) * B;
    for (uint32_t q = threadIdx.x; q < B; q += blockDim.x) {
        sm.cur[q] = offrow[q];
        sm.R[q] = R[q];
        const FastDiv d = divR[q];
        sm.mul[q] = d.mul;
        sm.sh[q] = pack_shifts(d);
        for (int x = 0; x <= kEmitWarps; ++x) sm.wcnt[x][q] = 0;
    }
    if (sgm == 0) write_seed_edges(out, out_block, (uint64_t)p * g.span, g.n0);
    __syncthreads();

    const uint32_t lt_mask = (1u << lane) - 1u;
    for (uint64_t base = lo; base < hi; base += kEmitTile) {
        // 1. stable rank within each warp's contiguous run of 32*ITEMS entries
        for (int r = 0; r < kEmitItems; ++r) {
            const uint32_t t = wid * (32 * kEmitItems) + r * 32 + lane;
            const uint64_t j = base + t;
            const uint32_t q = (j < hi) ? Ap[j] : 0xFFFFu;
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, q);
            uint32_t prev = 0;
            if (q != 0xFFFFu) prev = sm.wcnt[wid][q];
            __syncwarp();
            if (q != 0xFFFFu && (peers & lt_mask) == 0) sm.wcnt[wid][q] = (uint16_t)(prev + __popc(peers));
            __syncwarp();
            sm.item[t] = prev + __popc(peers & lt_mask);
            sm.qs[t] = (uint16_t)q;
        }
        __syncthreads();
        // 2. exclusive scan of the per-warp counts, per target block
        for (uint32_t q = threadIdx.x; q < B; q += blockDim.x) {
            uint32_t acc = 0;
            for (int x = 0; x < kEmitWarps; ++x) {
                const uint32_t c = sm.wcnt[x][q];
                sm.wcnt[x][q] = (uint16_t)acc;
                acc += c;
            }
            sm.wcnt[kEmitWarps][q] = (uint16_t)acc;
        }
        __syncthreads();
        // 3. resolve T_q[i] for every entry the thread owns
        {
            int k = 0;
            uint32_t t = wid * (32 * kEmitItems) + lane;
            uint64_t cur = 0;
            uint32_t q = 0;
            QDiv qd;
            bool fresh = true;
            while (k < kEmitItems) {
                if (fresh) {
                    q = sm.qs[t];
                    if (q == 0xFFFFu) {
                        ++k;
                        t += 32;
                        continue;
                    }
                    cur = sm.cur[q] + sm.wcnt[wid][q] + sm.item[t];
                    qd.R = sm.R[q];
                    qd.d.mul = sm.mul[q];
                    qd.d.s1 = sm.sh[q] & 0xFFu;
                    qd.d.s2 = sm.sh[q] >> 8;
                    fresh = false;
                }
                uint32_t v;
                if (t_step(cur, q, qd, g, v)) {
                    sm.item[t] = v;
                    ++k;
                    t += 32;
                    fresh = true;
                }
            }
        }
        __syncthreads();
        // 4. advance the per-block cursors; emit the tile
        for (uint32_t q = threadIdx.x; q < B; q += blockDim.x) {
            sm.cur[q] += sm.wcnt[kEmitWarps][q];
            for (int x = 0; x <= kEmitWarps; ++x) sm.wcnt[x][q] = 0;
        }
        const uint32_t n = (uint32_t)((hi - base < kEmitTile) ? hi - base : kEmitTile);
        const uint64_t e_first = out_block + g.e0 + base;
        auto edge_at = [&](uint32_t t2, uint64_t& s_, uint64_t& d_) {
            s_ = src_base + fdiv(base + t2, g.div_m);
            d_ = (uint64_t)sm.qs[t2] * g.span + sm.item[t2];
        };
        emit_tile(out, e_first, n, edge_at);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Serial BA (blocks = 1): edge j's target by its own copy chain.
// grid-stride over tiles of kBaTile edges; block = kBaThreads.
// ---------------------------------------------------------------------------
template <typename Id>
__global__ void __launch_bounds__(kBaThreads) ba_kernel(const __grid_constant__ PbaGeom g,
                                                        Id* __restrict__ out)
{
    __shared__ __align__(16) Id sDst[kBaTile];
    if (blockIdx.x == 0) write_seed_edges(out, 0, 0, g.n0);
    const uint64_t N = g.N_e;
    for (uint64_t base = (uint64_t)blockIdx.x * kBaTile; base < N;
         base += (uint64_t)gridDim.x * kBaTile) {
        int k = 0;
        uint64_t j = base + threadIdx.x;
        uint64_t cur = j;
        while (k < kBaItems) {
            uint64_t v = 0;
            if (j >= N || ba_step(cur, g, v)) {
                sDst[k * kBaThreads + threadIdx.x] = (Id)v;
                ++k;
                j += kBaThreads;
                cur = j;
            }
        }
        __syncthreads();
        const uint32_t n = (uint32_t)((N - base < kBaTile) ? N - base : kBaTile);
        auto edge_at = [&](uint32_t t2, uint64_t& s_, uint64_t& d_) {
            s_ = g.n0 + fdiv(base + t2, g.div_m);
            d_ = (uint64_t)sDst[t2];
        };
        emit_tile(out, g.e0 + base, n, edge_at);
        __syncthreads();
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t p1_smem_bytes(const PbaGeom& g)
{
    return ((g.P * 2 + 15) & ~15u) + (((size_t)g.B * 4 + 15) & ~(size_t)15) + kP1Tile * 2;
}

}  // namespace

uint32_t pba_segments(uint64_t N_e, uint32_t B, int sm_count)
{
    const uint64_t target = 8ull * (uint64_t)(sm_count > 0 ? sm_count : 1);
    uint64_t S = (target + B - 1) / B;
    const uint64_t max_s = (N_e + kP1Tile - 1) / kP1Tile;
    if (S > max_s) S = max_s;
    if (S < 1) S = 1;
    const uint64_t len = pba_segment_length(N_e, (uint32_t)S);
    const uint64_t used = (N_e + len - 1) / len;
    return (uint32_t)(used > 0 ? used : 1);
}

uint64_t pba_segment_length(uint64_t N_e, uint32_t S)
{
    const uint64_t per = (N_e + S - 1) / (S ? S : 1);
    uint64_t len = (per + kP1Tile - 1) / kP1Tile * kP1Tile;
    return len ? len : kP1Tile;
}

PbaWorkspace pba_workspace_layout(uint64_t A_stride, uint32_t B, uint32_t S)
{
    PbaWorkspace w;
    size_t o = 0;
    w.off_A = o;
    o += align256((size_t)B * A_stride * 2);
    w.off_cnt = o;
    o += align256((size_t)B * S * B * 4);
    w.off_off = o;
    o += align256((size_t)B * S * B * 8);
    w.off_R = o;
    o += align256((size_t)B * 8);
    w.off_magic = o;
    o += align256((size_t)B * sizeof(FastDiv));
    w.total = o;
    return w;
}

cudaError_t launch_ba(const PbaGeom& g, int id64, void* d_out, cudaStream_t s)
{
    const int sms = device_sm_count();
    const uint64_t tiles = (g.N_e + kBaTile - 1) / kBaTile;
    const uint64_t full = (uint64_t)sms * (id64 ? 6 : 8);
    const int grid = (int)(tiles < full ? (tiles > 0 ? tiles : 1) : full);
    TraceScope trace("ba_chain", s);
    if (id64)
        ba_kernel<uint64_t><<<grid, kBaThreads, 0, s>>>(g, (uint64_t*)d_out);
    else
        ba_kernel<uint32_t><<<grid, kBaThreads, 0, s>>>(g, (uint32_t*)d_out);
    return cudaGetLastError();
}

cudaError_t launch_pba(const PbaGeom& g, int id64, void* d_out, void* d_ws, cudaStream_t s)
{
    if (g.B > kMaxBlocks) return cudaErrorInvalidValue;
    const PbaWorkspace L = pba_workspace_layout(g.A_stride, g.B, g.S);
    unsigned char* ws = (unsigned char*)d_ws;
    uint16_t* A = (uint16_t*)(ws + L.off_A);
    uint32_t* cnt = (uint32_t*)(ws + L.off_cnt);
    uint64_t* off = (uint64_t*)(ws + L.off_off);
    uint64_t* R = (uint64_t*)(ws + L.off_R);
    FastDiv* divR = (FastDiv*)(ws + L.off_magic);
    cudaError_t err;

    static bool attrs_set = false;
    if (!attrs_set) {
        cudaFuncSetAttribute(pba_prefix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kPrefixMax * 2));
        cudaFuncSetAttribute(pba_phase1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kPrefixMax * 2 + kMaxBlocks * 4 + kP1Tile * 2 + 64));
        cudaFuncSetAttribute(pba_emit_kernel<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(EmitSmem));
        cudaFuncSetAttribute(pba_emit_kernel<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(EmitSmem));
        attrs_set = true;
    }
    if (g.N_e > 0) {
        {
            TraceScope trace("pba_prefix", s);
            pba_prefix_kernel<<<g.B, kP1Threads, g.P * 2, s>>>(g, A);
        }
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        {
            TraceScope trace("pba_phase1", s);
            pba_phase1_kernel<<<dim3(g.S, g.B), kP1Threads, p1_smem_bytes(g), s>>>(g, A, cnt);
        }
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    } else {
        cudaMemsetAsync(cnt, 0, (size_t)g.B * g.S * g.B * 4, s);
    }
    {
        TraceScope trace("pba_scan", s);
        pba_scan_kernel<<<(g.B + 31) / 32, 1024, 0, s>>>(cnt, off, R, divR, g.B, g.B * g.S);
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    const dim3 grid(g.S, g.B);
    TraceScope trace("pba_emit", s);
    if (id64)
        pba_emit_kernel<uint64_t><<<grid, kEmitThreads, sizeof(EmitSmem), s>>>(g, A, off, R, divR,
                                                                              (uint64_t*)d_out);
    else
        pba_emit_kernel<uint32_t><<<grid, kEmitThreads, sizeof(EmitSmem), s>>>(g, A, off, R, divR,
                                                                              (uint32_t*)d_out);
    return cudaGetLastError();
}

}  // namespace pgen

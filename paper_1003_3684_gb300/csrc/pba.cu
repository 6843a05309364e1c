// Parallel Barabasi-Albert generator (arXiv 1003.3684, Sec. 3, PBA method).
//
// The paper runs one processor per vertex block and exchanges messages
// between phases. Here the phases of all blocks run as data-parallel kernels
// on one GPU, and every message becomes HBM traffic:
//
//   pba_prefix   phase 1, first P entries of every block's list A_p, built in
//                shared memory level by level: entries [L, 2L) copy from
//                [0, L) (already final) or follow their own chain inside
//                [L, 2L). Writes A_p[0, P) and counts it.
//   pba_pass     phase 1, one level [L, hi) of every block per launch, with
//                hi = L + L/kLevelDiv rounded up to whole granules (levels
//                grow 1.5x: more copies land in the finished part than with
//                doubling, so fewer chain links, and few enough launches that
//                their partial last waves stay cheap). Entry j draws once
//                (Philox, counter (j, p, 1)):
//                an inter-faction pick, or a copy of entry r < j. A copy with
//                r < L reads the finished A_p[r] from global memory (the
//                grid is block-major, so the few blocks in flight keep their
//                A_p in L2); a copy with r >= L follows r's own draw. Adds
//                the counts of each (block, segment) -- the paper's count
//                message -- into cnt.
//   pba_scan     exclusive scan of the counts over (requester, segment) per
//                target block: R_q (how many endpoints q must produce) and
//                where each requester segment's slice of q's list starts.
//   pba_emit     phase 2 and substitution. The stable rank of entry j among
//                the earlier entries of its segment naming the same block
//                (warp match + per-warp counters + cross-warp scan) gives its
//                index i in q's endpoint list T_q; T_q[i] is resolved by its
//                own copy chain through q's local preferential attachment
//                (recomputed, never stored), and the (src, dst) pairs leave
//                through a shared-memory tile as coalesced vector stores.
//
// blocks = 1 is serial BA: ba_kernel resolves edge j's chain directly.
//
// Copy chains have geometric lengths. A warp works on a run of consecutive
// entries; each lane follows one chain, one Philox per loop trip, and a lane
// whose entry is finished takes the next unclaimed entry of the run (ballot),
// so lanes stay busy until the run is exhausted.
#include <atomic>
#include <type_traits>

#include "pg_internal.h"
#include "pg_trace.h"

namespace pgen {
namespace {

constexpr uint32_t kGranule = 16384;        // segment lengths are multiples of this
constexpr uint32_t kPrefixMax = 6 * kGranule;   // phase-1 prefix built in smem (192 KB)
constexpr int kPrefixThreads = 1024;
constexpr int kPassThreads = 512;
constexpr uint32_t kPassRun = 1024;             // entries per warp run in a pass
constexpr uint32_t kPassChunk = (kPassThreads / 32) * kPassRun;   // 16384 per CTA
constexpr int kEmitWarps = 8;
constexpr int kEmitThreads = kEmitWarps * 32;
constexpr uint64_t kLevelDiv = 2;   // phase-1 level [L, L + L/kLevelDiv)
constexpr int kEmitItems = 8;
constexpr uint32_t kEmitRun = 32 * kEmitItems;                   // 256 entries per warp run
constexpr uint32_t kMaxBlocks = 1024;
constexpr uint32_t kSeedTab = 256;   // seed clique edges in the lean links' table: n0 <= 23
constexpr int kBaThreads = 256;
template <typename Id>
struct BaShape {   // 32 KB of staging for either id width
    static constexpr uint32_t run = sizeof(Id) == 4 ? 1024 : 512;
    static constexpr uint32_t tile = (kBaThreads / 32) * run;
};

static_assert(kPassChunk == kGranule, "a pass CTA covers one granule");
static_assert(kGranule % kEmitRun == 0, "segments hold whole emit runs");

// Inter-faction pick: uniform over the B - W blocks outside [phi, phi + W).
__device__ __forceinline__ uint32_t fresh_block(uint32_t w3, uint32_t B, uint32_t W,
                                                uint32_t phi)
{
    const uint32_t x = __umulhi(w3, B - W);
    return x < phi ? x : x + W;
}

// The factions of block p: an aligned group of W blocks starting at phi, or
// (kTable) the block's record of the faction table. An inter-faction pick
// takes the x-th block outside the list, x uniform below the number of such
// blocks; for an aligned group that is fresh_block.
template <bool kTable>
struct Faction {
    const uint16_t* rec;
    uint32_t s, n_out, phi;
    bool coin;
    __device__ __forceinline__ Faction(const PbaGeom& g, uint32_t p)
    {
        if constexpr (kTable) {
            rec = g.ftab + (size_t)p * kFacStride;
            s = rec[0];
            n_out = rec[1];
            phi = 0;
            coin = g.coin_thr > 0 && n_out > 0;
        } else {
            rec = nullptr;
            s = g.W;
            n_out = g.B - g.W;
            phi = (p / g.W) * g.W;
            coin = g.coin_on != 0;
        }
    }
    __device__ __forceinline__ uint32_t member(uint32_t t) const
    {
        if constexpr (kTable) return PG_CHECK(t, kFacSlots) ? rec[kFacHeader + t] : 0u;
        else return phi + t;
    }
    __device__ __forceinline__ uint32_t fresh(uint32_t w3, const PbaGeom& g) const
    {
        if constexpr (kTable) {
            const uint32_t x = __umulhi(w3, n_out);
            return PG_CHECK(x, kFacSlots) ? rec[kFacHeader + kFacSlots + x] : 0u;
        } else {
            return fresh_block(w3, g.B, g.W, phi);
        }
    }
};

// Adds a smem histogram of B counters to cnt row (p, sgm), skipping zeros.
__device__ __forceinline__ void flush_counts(const uint32_t* hist, uint32_t* cnt,
                                             const PbaGeom& g, uint32_t p, uint32_t sgm)
{
    if (!PG_CHECK(sgm, g.S)) return;
    uint32_t* row = cnt + ((uint64_t)p * g.S + sgm) * g.B;
    for (uint32_t t = threadIdx.x; t < g.B; t += blockDim.x)
        if (hist[t]) atomicAdd(&row[t], hist[t]);
}

// ---------------------------------------------------------------------------
// Phase 1, prefix [0, P) of each block, built in shared memory.
// grid = B, block = kPrefixThreads, dynamic smem = P*2 (rounded to 16) + B*4.
// ---------------------------------------------------------------------------
template <bool kTable>
__global__ void __launch_bounds__(kPrefixThreads) pba_prefix_kernel(
    const __grid_constant__ PbaGeom g, uint16_t* __restrict__ A, uint32_t* __restrict__ cnt)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint16_t* sA = reinterpret_cast<uint16_t*>(smem);
    uint32_t* hist = reinterpret_cast<uint32_t*>(smem + ((g.P * 2 + 15) & ~15u));
    const uint32_t p = blockIdx.x;
    const Faction<kTable> F(g, p);
    const PhiloxHead ph = philox_head(0u, p, 1u, g.key);   // counters (j, 0, p, 1)
    const uint32_t P = g.P;
    const uint32_t s = F.s < P ? F.s : P;
    for (uint32_t t = threadIdx.x; t < s; t += blockDim.x) sA[t] = (uint16_t)F.member(t);
    __syncthreads();
    for (uint32_t L = s; L < P;) {
        const uint32_t hi = (2 * L < P) ? 2 * L : P;
        for (uint32_t j = L + threadIdx.x; j < hi; j += blockDim.x) {
            uint32_t cur = j, v;
            for (;;) {
                const uint4 w = philox_headed(cur, ph, g.key);
                if (F.coin && w.z < g.coin_thr) {
                    v = F.fresh(w.w, g);
                    break;
                }
                const uint32_t r = uniform32(w.x, w.y, cur);
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
    // counts of the prefix, per segment it overlaps
    for (uint32_t sgm = 0; (uint64_t)sgm * g.seg_len < P; ++sgm) {
        const uint32_t a = (uint32_t)((uint64_t)sgm * g.seg_len);
        const uint32_t b = (uint32_t)((a + g.seg_len < P) ? a + g.seg_len : P);
        for (uint32_t t = threadIdx.x; t < g.B; t += blockDim.x) hist[t] = 0;
        __syncthreads();
        for (uint32_t t = a + threadIdx.x; t < b; t += blockDim.x)
            if (PG_CHECK(sA[t], g.B)) atomicAdd(&hist[sA[t]], 1u);
        __syncthreads();
        flush_counts(hist, cnt, g, p, sgm);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Phase 1, one level [L, hi) of every block; grid = (chunks, B),
// chunk c = [L + c*kPassChunk, ...). dynamic smem = B*4 (histogram) + one
// staged run of kPassRun entries per warp.
// A copy that lands below L loads A_p[r]; the load is consumed one loop trip
// later (after the next Philox), so its latency overlaps arithmetic.
// ---------------------------------------------------------------------------
template <bool kTable>
__global__ void __launch_bounds__(kPassThreads) pba_pass_kernel(const __grid_constant__ PbaGeom g,
                                                                uint32_t L, uint32_t hi,
                                                                uint16_t* __restrict__ A,
                                                                uint32_t* __restrict__ cnt)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* hist = reinterpret_cast<uint32_t*>(smem);                              // B
    uint16_t* stage = reinterpret_cast<uint16_t*>(smem + (((size_t)g.B * 4 + 15) & ~(size_t)15));
    const uint32_t p = blockIdx.y;
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const Faction<kTable> F(g, p);
    const PhiloxHead ph = philox_head(0u, p, 1u, g.key);   // counters (j, 0, p, 1)
    uint16_t* Ap = A + (uint64_t)p * g.A_stride;
    uint16_t* my = stage + wid * kPassRun;              // this warp's run, staged
    const uint32_t chunk = L + blockIdx.x * kPassChunk;   // a granule: one segment
    for (uint32_t t = threadIdx.x; t < g.B; t += blockDim.x) hist[t] = 0;
    __syncthreads();

    const uint32_t run = chunk + wid * kPassRun;
    const uint32_t n_items = run < hi ? ((hi - run < kPassRun) ? hi - run : kPassRun) : 0;
    const bool coin_on = F.coin;
    uint32_t next = 32, item = lane;
    uint32_t cur = run + item;
    bool active = item < n_items;
    bool pend = false, pend_load = false;
    uint32_t pend_k = 0, pend_v = 0, lv = 0;
    uint32_t own = 0;   // entries equal to p (the most frequent value) counted here
    // every lane draws (an idle lane's draw is discarded), so the trip is
    // straight-line code apart from the deferred store. A copy of the
    // finished prefix is loaded into lv and first read one trip later, by
    // that store, so the load's latency overlaps a whole trip.
    auto trip = [&]() {
        const uint4 w = philox_headed(cur, ph, g.key);
        if (pend) my[pend_k] = (uint16_t)(pend_load ? lv : pend_v);
        const bool coin = coin_on && w.z < g.coin_thr;
        const uint32_t r = uniform32(w.x, w.y, cur);
        const bool hit = !coin && r < L;
        const bool done = active && (coin || hit);
        if constexpr (kTable) {
            if (active && coin) pend_v = F.fresh(w.w, g);   // a table read only for a pick
        } else {
            pend_v = F.fresh(w.w, g);
        }
        if (active && hit) lv = __ldg(Ap + r);
        pend_load = hit;
        pend_k = done ? item : pend_k;
        pend = done;
        cur = (active && !done) ? r : cur;
        const uint32_t dm = __ballot_sync(0xFFFFFFFFu, done);
        const uint32_t nit = next + __popc(dm & lt);
        next += __popc(dm);
        item = done ? nit : item;
        cur = done ? run + nit : cur;
        active = done ? nit < n_items : active;
    };
    // trips while unclaimed entries remain (`next` is the same in every
    // lane), then until every lane's chain and deferred store are done
    while (next < n_items) trip();
    while (__any_sync(0xFFFFFFFFu, active || pend)) trip();
    __syncwarp();
    // counts of the finished run, outside the pooled loop (converged lanes)
    for (uint32_t t = lane; t < n_items; t += 32) {
        const uint32_t v = my[t];
        if (v == p) ++own;
        else if (PG_CHECK(v, g.B)) atomicAdd(&hist[v], 1u);
    }
    // the run back to A: 16-byte stores when the run is whole (run is a
    // multiple of 8 entries and rows are 16-byte aligned), marked streaming
    // so that they do not evict the finished prefixes the copies read
    const bool in_row = n_items == 0 || PG_CHECK(run + n_items - 1, g.N_e);
    if (in_row && n_items == kPassRun) {
        const uint4* src = reinterpret_cast<const uint4*>(my);
        uint4* dst = reinterpret_cast<uint4*>(Ap + run);
        for (uint32_t t = lane; t < kPassRun / 8; t += 32) __stcs(dst + t, src[t]);
    } else if (in_row) {
        for (uint32_t t = lane; t < n_items; t += 32) Ap[run + t] = my[t];
    }
    if (own) atomicAdd(&hist[p], own);
    __syncthreads();
    flush_counts(hist, cnt, g, p, (uint32_t)(chunk / g.seg_len));
}

// ---------------------------------------------------------------------------
// Count exchange: per target block q, exclusive scan over rows (p, segment)
// of cnt[row][q]; writes off[row][q], R[q] and the divisor for R[q].
// grid = ceil(B / 32), block = 1024 (warp w scans a slab of rows, lane = q).
// ---------------------------------------------------------------------------
// Exact reciprocal of R for sigma(x) = floor(x * n_b / R), x < R < 2^32:
// C = ceil(n_b * 2^64 / R) as three 32-bit words (C2 = n_b div R). Then
// x*C/2^64 = x*n_b/R + x*d/2^64 with 0 <= d < 1, and x/2^64 < 1/R because
// R^2 < 2^64; the fractional part of x*n_b/R is a multiple of 1/R below 1, so
// adding less than 1/R never carries: floor(x*C/2^64) = sigma(x) exactly.
struct __align__(16) QRecip {
    uint32_t R, C2, C1, C0;
};

__device__ inline QRecip make_recip(uint64_t R, uint32_t nb)
{
    QRecip c{0, 0, 0, 0};
    if (R == 0 || R >= ((uint64_t)1 << 32)) return c;
    c.R = (uint32_t)R;
    c.C2 = (uint32_t)(nb / R);
    const uint64_t rem = nb % R;                     // < R < 2^32
    const uint64_t a = rem << 32;
    const uint64_t q_hi = a / R, r1 = a % R;
    const uint64_t b = r1 << 32;
    const uint64_t q_lo = b / R, r2 = b % R;
    const uint64_t frac = (q_hi << 32) + q_lo + (r2 != 0 ? 1 : 0);
    c.C1 = (uint32_t)(frac >> 32);
    c.C0 = (uint32_t)frac;
    return c;
}

__device__ __forceinline__ uint32_t sigma32(uint32_t x, const QRecip& c)
{
    const uint64_t t0 = (uint64_t)x * c.C0;
    const uint64_t t1 = (uint64_t)x * c.C1 + (t0 >> 32);
    return (uint32_t)(t1 >> 32) + x * c.C2;
}

__global__ void __launch_bounds__(1024) pba_scan_kernel(const uint32_t* __restrict__ cnt,
                                                        uint64_t* __restrict__ off,
                                                        uint64_t* __restrict__ R,
                                                        FastDiv* __restrict__ divR,
                                                        QRecip* __restrict__ recip, uint32_t nb,
                                                        uint32_t B, uint32_t rows, uint64_t e0,
                                                        uint32_t force_wide,
                                                        uint32_t* __restrict__ wide_flag,
                                                        uint32_t n0, uint32_t* __restrict__ stab)
{
    // the seed clique's edges for the emit's lean links (a | b << 16)
    if (blockIdx.x == 0)
        for (uint32_t e = threadIdx.x; e < kSeedTab; e += blockDim.x)
            stab[e] = e < e0 ? seed_endpoint(e, 0, n0) | (seed_endpoint(e, 1, n0) << 16) : 0u;
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
            recip[q] = make_recip(acc, nb);
            if (force_wide || acc + e0 >= ((uint64_t)1 << 32)) atomicOr(wide_flag, 1u);
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
// One Philox per link; a link ends the chain when it lands on a seed slot or
// on the source end of an earlier edge.
// ---------------------------------------------------------------------------
struct QDiv {
    uint64_t R;
    FastDiv d;
};

// 64-bit link (any R_q).
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

// 32-bit link (R_q + e0 < 2^32), the same values as t_step: with W = (w1:w0)
// and X = e0 + before < 2^32, the slot r = floor(W * 2X / 2^64) has
// e = r >> 1 = the high word of s = w1*X + (w0*X >> 32) and side = bit 31 of
// s's low word. One rarely taken branch (a seed slot): the side-0 value is
// computed on every link and selected, so lanes of a warp that stop and
// lanes that continue run the same instructions.
__device__ __forceinline__ bool t_link32(uint32_t& cur, uint32_t q, const QRecip& c,
                                         const PbaGeom& g, uint32_t& v)
{
    const uint32_t nb = (uint32_t)g.n_b;
    const uint32_t sig = sigma32(cur, c);
    uint32_t before;
    if (g.nb_shift != 0xFFFFFFFFu)
        before = (uint32_t)(((uint64_t)sig * c.R + (nb - 1)) >> g.nb_shift);
    else
        before = (uint32_t)fdiv((uint64_t)sig * c.R + (nb - 1), g.div_nb);
    const uint4 w = philox(make_uint4(cur, 0u, q, 2u), g.key);
    const uint32_t e0 = (uint32_t)g.e0;
    const uint32_t X = e0 + before;
    const uint64_t s = (uint64_t)w.y * X + (((uint64_t)w.x * X) >> 32);
    const uint32_t e = (uint32_t)(s >> 32);
    const uint32_t side = ((uint32_t)s) >> 31;
    const uint32_t e2 = e - e0;
    const bool seed = e < e0;
    uint32_t vs = 0;
    if (seed) vs = seed_endpoint(e, side, g.n0);
    v = seed ? vs : g.n0 + sigma32(e2, c);
    const bool fin = seed || side == 0;
    cur = fin ? cur : e2;
    return fin;
}

// The same link for n_b a power of two, with sigma(cur) carried in from the
// previous link (the side-0 value of a link is sigma of the edge the chain
// moves to, so a continuing chain computes one sigma per link instead of
// two) and the seed clique's edges read from a table in the workspace
// (stab[e] = a | b << 16; every lane reads entry 0 unless it hit a seed
// slot, so the load is a broadcast from L1) instead of a branch: the link is
// straight-line code.
__device__ __forceinline__ bool t_link_lean(uint32_t& cur, uint32_t& sig, bool& fresh, uint32_t q,
                                            const QRecip& c, const PbaGeom& g,
                                            const uint32_t* __restrict__ stab, uint32_t& v)
{
    const uint4 w = philox(make_uint4(cur, 0u, q, 2u), g.key);
    // a newly claimed entry's sigma, computed after the draw so that the
    // load of the target's reciprocal has the draw's time to land
    if (fresh) sig = sigma32(cur, c);
    fresh = false;
    // X = e0 + ceil(sig*R / n_b) = (sig*R + (n_b - 1) + e0*n_b) >> log2(n_b):
    // e0*n_b is a multiple of n_b, and the sum stays below n_b*(R + e0 + 1) <= 2^64
    const uint32_t X = (uint32_t)(((uint64_t)sig * c.R + g.lean_add) >> g.nb_shift);
    const uint32_t e0 = (uint32_t)g.e0;
    const uint64_t s = (uint64_t)w.y * X + (((uint64_t)w.x * X) >> 32);
    const uint32_t e = (uint32_t)(s >> 32);
    const uint32_t side = ((uint32_t)s) >> 31;
    const uint32_t e2 = e - e0;
    const uint32_t sig2 = sigma32(e2, c);
    const bool seed = e < e0;
    const uint32_t ti = seed ? e : 0u;
    const uint32_t ab = PG_CHECK(ti, kSeedTab) ? __ldg(stab + ti) : 0u;
    const uint32_t vs = side ? (ab >> 16) : (ab & 0xFFFFu);
    v = seed ? vs : g.n0 + sig2;
    // a continuing chain moves to e2; an ended one is replaced by the caller's
    // next claim (which sets cur and marks sig fresh) or goes idle
    cur = e2;
    sig = sig2;
    return seed || side == 0;
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

// 32-bit serial BA link (n*m + e0 < 2^32).
__device__ __forceinline__ bool ba_step32(uint32_t& cur, const PbaGeom& g, const PhiloxHead& ph,
                                          uint32_t& v)
{
    const uint32_t sig = fdiv32(cur, g.div_m32);
    const uint4 w = philox_headed(cur, ph, g.key);   // counter (cur, 0, 0, 2)
    const uint32_t X = (uint32_t)g.e0 + sig * g.m;
    const uint64_t hi = (uint64_t)w.y * X, lo = (uint64_t)w.x * X;
    const uint64_t r = (hi + (lo >> 32)) >> 31;
    const uint32_t e = (uint32_t)(r >> 1);
    if (e < (uint32_t)g.e0) {
        v = seed_endpoint(e, (uint32_t)(r & 1), g.n0);
        return true;
    }
    const uint32_t e2 = e - (uint32_t)g.e0;
    if ((r & 1) == 0) {
        v = g.n0 + fdiv32(e2, g.div_m32);
        return true;
    }
    cur = e2;
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

// Writes n consecutive edges starting at global edge index e_first of an
// output of `cap` edges; edge t comes from edge_at(t, src, dst). Pairs of
// edges whose first index is even go out as one 16-byte (uint32 ids) or two
// 16-byte (uint64 ids) stores; an odd first index is written alone first so
// that the rest stay aligned.
template <typename Id, typename F>
__device__ __forceinline__ void emit_tile(Id* out, uint64_t cap, uint64_t e_first, uint32_t n,
                                          F&& edge_at)
{
    const uint32_t head = (uint32_t)(e_first & 1) < n ? (uint32_t)(e_first & 1) : n;
    if (head && threadIdx.x == 0) {
        uint64_t s0, d0;
        edge_at(0, s0, d0);
        if (PG_CHECK_OUT(e_first, cap)) store_pair(out, e_first, s0, d0);
    }
    for (uint32_t t2 = head + 2 * threadIdx.x; t2 < n; t2 += 2 * blockDim.x) {
        uint64_t s0, d0;
        edge_at(t2, s0, d0);
        if (t2 + 1 < n) {
            uint64_t s1, d1;
            edge_at(t2 + 1, s1, d1);
            if (PG_CHECK_OUT(e_first + t2 + 1, cap)) store_two(out, e_first + t2, s0, d0, s1, d1);
        } else {
            if (PG_CHECK_OUT(e_first + t2, cap)) store_pair(out, e_first + t2, s0, d0);
        }
    }
}

// Seed clique of one block (e0 edges, lexicographic) at out[e_first...].
template <typename Id>
__device__ void write_seed_edges(Id* out, uint64_t cap, uint64_t e_first, uint64_t base,
                                 uint32_t n0)
{
    const uint64_t e0 = (uint64_t)n0 * (n0 - 1) / 2;
    for (uint64_t e = threadIdx.x; e < e0; e += blockDim.x)
        if (PG_CHECK_OUT(e_first + e, cap))
            store_pair(out, e_first + e, base + seed_endpoint(e, 0, n0),
                       base + seed_endpoint(e, 1, n0));
}

// Warp-scoped version of emit_tile: lanes of one warp write n edges.
template <typename Id, typename F>
__device__ __forceinline__ void emit_run(Id* out, uint64_t cap, uint64_t e_first, uint32_t n,
                                         uint32_t lane, F&& edge_at)
{
    const uint32_t head = (uint32_t)(e_first & 1) < n ? (uint32_t)(e_first & 1) : n;
    if (head && lane == 0) {
        uint64_t s0, d0;
        edge_at(0, s0, d0);
        if (PG_CHECK_OUT(e_first, cap)) store_pair(out, e_first, s0, d0);
    }
    for (uint32_t t2 = head + 2 * lane; t2 < n; t2 += 64) {
        uint64_t s0, d0;
        edge_at(t2, s0, d0);
        if (t2 + 1 < n) {
            uint64_t s1, d1;
            edge_at(t2 + 1, s1, d1);
            if (PG_CHECK_OUT(e_first + t2 + 1, cap)) store_two(out, e_first + t2, s0, d0, s1, d1);
        } else {
            if (PG_CHECK_OUT(e_first + t2, cap)) store_pair(out, e_first + t2, s0, d0);
        }
    }
}

// ---------------------------------------------------------------------------
// Phase 2 + substitution + emission. Every warp owns one segment of one block
// (grid = (ceil(S / kEmitWarps), B)) and walks it in runs of kEmitRun entries:
//   rank   entry j gets i = (next unused slot of T_{A[j]} for this segment),
//          by a warp match over 32 entries and per-warp cursors in smem;
//   chain  the lanes resolve T_q[i] for the run's entries, pooled;
//   emit   the run's (src, dst) pairs leave as vector stores.
// kFast (32-bit arithmetic, valid when every R_q + e0 < 2^32; the scan's flag
// says which variant does the work) keeps two runs ranked at a time, in two
// buffers: a lane that finishes an entry of run r takes the next unclaimed
// entry of run r or r+1, so the pool drains once per segment rather than at
// the end of every run. Run r is emitted as soon as all its entries are
// resolved, and run r+2 is ranked into its buffer. Warps never wait on each
// other.
// ---------------------------------------------------------------------------
template <typename CurT>
struct EmitWarpSmem {
    CurT cur[kMaxBlocks];      // next unused index into T_q, per target block
    CurT item[2][kEmitRun];    // slot index i, then the resolved local id
    uint16_t qs[2][kEmitRun];  // target block of each entry of the run
};

// kMode 0: 64-bit links (some R_q + e0 >= 2^32); 1: 32-bit links; 2: 32-bit
// lean links (n_b a power of two, n0 <= 23).
template <typename Id, int kMode>
__global__ void __launch_bounds__(kEmitThreads) pba_emit_kernel(
    const __grid_constant__ PbaGeom g, const uint16_t* __restrict__ A,
    const uint64_t* __restrict__ off, const uint64_t* __restrict__ R,
    const FastDiv* __restrict__ divR, const QRecip* __restrict__ recip,
    const uint32_t* __restrict__ wide_flag, const uint32_t* __restrict__ stab,
    Id* __restrict__ out, uint32_t block_off, uint32_t out_block0, uint64_t out_cap)
{
    constexpr bool kFast = kMode != 0;
    using CurT = typename std::conditional<kFast, uint32_t, uint64_t>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if ((*wide_flag == 0) != kFast) return;   // the other variant does the work
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t p = blockIdx.y + block_off;
    const uint32_t sw = blockIdx.x * kEmitWarps + wid;
    if (sw >= g.S) return;                   // no block-wide barrier follows
    EmitWarpSmem<CurT>& ws = reinterpret_cast<EmitWarpSmem<CurT>*>(smem_raw)[wid];
    const uint32_t B = g.B;
    const uint32_t lt = (1u << lane) - 1u;
    const uint16_t* Ap = A + (uint64_t)p * g.A_stride;
    const uint64_t lo = (uint64_t)sw * g.seg_len;
    const uint64_t hi = (lo + g.seg_len < g.N_e) ? lo + g.seg_len : g.N_e;
    const uint64_t out_block = (uint64_t)(p - out_block0) * (g.e0 + g.N_e);
    const uint64_t src_base = (uint64_t)p * g.span + g.n0;

    const uint64_t* offrow = off + ((uint64_t)p * g.S + sw) * B;
    for (uint32_t q = lane; q < B; q += 32) ws.cur[q] = (CurT)offrow[q];
    if (sw == 0) {
        const uint64_t e0 = g.e0, base_id = (uint64_t)p * g.span;
        for (uint64_t e = lane; e < e0; e += 32)
            if (PG_CHECK_OUT(out_block + e, out_cap))
                store_pair(out, out_block + e, base_id + seed_endpoint(e, 0, g.n0),
                           base_id + seed_endpoint(e, 1, g.n0));
    }
    __syncwarp();

    // block ids of run `run` of the segment (0xFFFF past its end)
    auto load_run = [&](uint32_t run, uint32_t (&qv)[kEmitItems]) {
#pragma unroll
        for (int r = 0; r < kEmitItems; ++r) {
            const uint64_t j = lo + (uint64_t)run * kEmitRun + r * 32 + lane;
            qv[r] = (j < hi) ? Ap[j] : 0xFFFFu;
        }
    };
    // rank: slot index of each entry in its target's list, in entry order
    auto rank_run = [&](const uint32_t (&qv)[kEmitItems], CurT* item, uint16_t* qs) {
#pragma unroll
        for (int r = 0; r < kEmitItems; ++r) {
            const uint32_t q = qv[r];
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, q);
            CurT prev = 0;
            const bool named = q != 0xFFFFu && PG_CHECK(q, B);
            if (named) prev = ws.cur[q];
            __syncwarp();
            if (named && (peers & lt) == 0) ws.cur[q] = prev + __popc(peers);
            __syncwarp();
            item[r * 32 + lane] = prev + __popc(peers & lt);
            qs[r * 32 + lane] = (uint16_t)q;
        }
        __syncwarp();
    };
    // emit: the run's n resolved entries, entry t at segment position base + t
    auto emit_buf = [&](uint64_t base, uint32_t n, const CurT* item, const uint16_t* qs) {
        auto edge_at = [&](uint32_t t2, uint64_t& s_, uint64_t& d_) {
            s_ = src_base + fdiv32((uint32_t)(base + t2), g.div_m32);
            d_ = (uint64_t)qs[t2] * g.span + (uint32_t)item[t2];
            (void)PG_CHECK(item[t2], g.span);   // a local id of block qs[t2]
        };
        emit_run(out, out_cap, out_block + g.e0 + base, n, lane, edge_at);
        __syncwarp();
    };

    const uint32_t total = (uint32_t)(hi - lo);   // entries of the segment
    const uint32_t runs = (total + kEmitRun - 1) / kEmitRun;
    uint32_t qv[kEmitItems];
    if constexpr (kFast) {
        load_run(0, qv);
        rank_run(qv, ws.item[0], ws.qs[0]);
        if (runs > 1) {
            load_run(1, qv);
            rank_run(qv, ws.item[1], ws.qs[1]);
        }
        if (runs > 2) load_run(2, qv);   // in flight during run 0's chains
        // pooled chains over the segment: entry gk of the segment lives in
        // buffer (gk / kEmitRun) & 1, at flat index gk % (2 * kEmitRun);
        // claims are handed out in entry order
        CurT* item_all = &ws.item[0][0];
        const uint16_t* qs_all = &ws.qs[0][0];
        uint32_t gk = lane, next = 32, q = 0, cur = 0, sig = 0, k = 0;
        bool active = false, fresh = false;
        QRecip c{0, 0, 0, 0};
        auto take = [&](uint32_t pos) {
            k = pos % (2 * kEmitRun);
            q = qs_all[k];
            cur = (uint32_t)item_all[k];
            c = PG_CHECK(q, B) ? recip[q] : QRecip{0, 0, 0, 0};
            fresh = true;
        };
        // one link for every lane; a lane whose chain ended stores its value
        // and takes the next unclaimed entry (below `limit`)
        auto trip = [&](uint32_t limit) {
            uint32_t v;
            bool fin;
            if constexpr (kMode == 2) fin = t_link_lean(cur, sig, fresh, q, c, g, stab, v);
            else fin = t_link32(cur, q, c, g, v);
            const bool done = fin && active;
            if (done) item_all[k] = v;
            const uint32_t dm = __ballot_sync(0xFFFFFFFFu, done);
            const uint32_t pos = next + __popc(dm & lt);
            next += __popc(dm);
            const bool tk = done && pos < limit;
            if (done) {
                gk = pos;
                active = tk;
            }
            if (tk) take(pos);
        };
        for (uint32_t r = 0; r < runs; ++r) {
            const uint32_t n_r = (total - r * kEmitRun < kEmitRun) ? total - r * kEmitRun : kEmitRun;
            const uint32_t limit = (total - r * kEmitRun < 2 * kEmitRun) ? total
                                                                        : (r + 2) * kEmitRun;
            const uint32_t r_end = r * kEmitRun + n_r;
            if (!active && gk < limit) {      // a claim in the newly ranked run
                active = true;
                take(gk);
            }
            // run r is resolved once every entry before r_end has been claimed
            // (claims go in entry order) and no active lane still holds one:
            // trips while entries of run r remain unclaimed (`next` is the same
            // in every lane), then trips until the lanes holding its last
            // entries are done
            while (next < r_end) trip(limit);
            while (__any_sync(0xFFFFFFFFu, active && gk < r_end)) trip(limit);
            __syncwarp();
            emit_buf(lo + (uint64_t)r * kEmitRun, n_r, ws.item[r & 1], ws.qs[r & 1]);
            if (r + 2 < runs) {
                rank_run(qv, ws.item[r & 1], ws.qs[r & 1]);
                if (r + 3 < runs) load_run(r + 3, qv);
            }
        }
    } else {
        // one run at a time in buffer 0, 64-bit links
        load_run(0, qv);
        for (uint32_t r = 0; r < runs; ++r) {
            const uint32_t n = (total - r * kEmitRun < kEmitRun) ? total - r * kEmitRun : kEmitRun;
            rank_run(qv, ws.item[0], ws.qs[0]);
            if (r + 1 < runs) load_run(r + 1, qv);
            uint32_t k = lane, next = 32, q = 0xFFFFu;
            bool active = true, fresh = true;
            CurT cur = 0;
            QDiv qd;
            qd.R = 0;
            qd.d = FastDiv{0, 0, 0};
            while (__any_sync(0xFFFFFFFFu, active)) {
                if (active && fresh) {
                    q = ws.qs[0][k];
                    cur = ws.item[0][k];
                    if (q != 0xFFFFu && PG_CHECK(q, B)) {
                        qd.R = R[q];
                        qd.d = divR[q];
                    }
                    fresh = false;
                }
                __syncwarp();
                const bool live = active && q != 0xFFFFu;   // 0xFFFF: past the segment end
                uint32_t v = 0;
                bool fin = false;
                uint64_t c64 = cur;
                if (live) fin = t_step(c64, q, qd, g, v);
                cur = c64;
                if (fin) ws.item[0][k] = v;
                const bool done = active && (fin || !live);
                const uint32_t dm = __ballot_sync(0xFFFFFFFFu, done);
                if (done) {
                    k = next + __popc(dm & lt);
                    active = k < kEmitRun;
                    fresh = true;
                }
                next += __popc(dm);
            }
            __syncwarp();
            emit_buf(lo + (uint64_t)r * kEmitRun, n, ws.item[0], ws.qs[0]);
        }
    }
}

// ---------------------------------------------------------------------------
// Serial BA (blocks = 1): edge j's target by its own copy chain.
// Each CTA takes tiles of kBaTile edges; each warp a run of kBaRun edges
// with pooled chains; targets are staged in smem and leave as vector stores.
// ---------------------------------------------------------------------------
template <typename Id, bool kFast>
__global__ void __launch_bounds__(kBaThreads) ba_kernel(const __grid_constant__ PbaGeom g,
                                                        Id* __restrict__ out)
{
    constexpr uint32_t kBaRun = BaShape<Id>::run, kBaTile = BaShape<Id>::tile;
    __shared__ __align__(16) Id sDst[kBaTile];
    const uint64_t cap = g.e0 + g.N_e;   // edges of the output
    if (blockIdx.x == 0) write_seed_edges(out, cap, 0, 0, g.n0);
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const uint64_t N = g.N_e;
    const PhiloxHead ph = philox_head(0u, 0u, 2u, g.key);
    for (uint64_t base = (uint64_t)blockIdx.x * kBaTile; base < N;
         base += (uint64_t)gridDim.x * kBaTile) {
        const uint64_t run = base + wid * kBaRun;
        const uint32_t n_items = run < N ? (uint32_t)((N - run < kBaRun) ? N - run : kBaRun) : 0;
        uint32_t next = 32, item = lane;
        uint64_t cur = run + item;
        uint32_t cur32 = (uint32_t)cur;
        bool active = item < n_items;
        while (__any_sync(0xFFFFFFFFu, active)) {
            bool done = false;
            if (active) {
                if (kFast) {
                    uint32_t v;
                    done = ba_step32(cur32, g, ph, v);
                    if (done) sDst[wid * kBaRun + item] = (Id)v;
                } else {
                    uint64_t v;
                    done = ba_step(cur, g, v);
                    if (done) sDst[wid * kBaRun + item] = (Id)v;
                }
            }
            const uint32_t dm = __ballot_sync(0xFFFFFFFFu, done);
            if (done) {
                item = next + __popc(dm & lt);
                cur = run + item;
                cur32 = (uint32_t)cur;
                active = item < n_items;
            }
            next += __popc(dm);
        }
        __syncthreads();
        const uint32_t n = (uint32_t)((N - base < kBaTile) ? N - base : kBaTile);
        auto edge_at = [&](uint32_t t2, uint64_t& s_, uint64_t& d_) {
            s_ = g.n0 + (kFast ? fdiv32((uint32_t)(base + t2), g.div_m32) : fdiv(base + t2, g.div_m));
            d_ = (uint64_t)sDst[t2];
            (void)PG_CHECK(d_, g.span);   // an id below the graph's vertex count
        };
        emit_tile(out, cap, g.e0 + base, n, edge_at);
        __syncthreads();
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

PG_CHECK_UNIT(pba)

uint32_t pba_prefix_len(uint64_t N_e) { return (uint32_t)(N_e < kPrefixMax ? N_e : kPrefixMax); }

uint32_t pba_segments(uint64_t N_e, uint32_t B, int sm_count)
{
    // about eight waves of warps (32 resident per SM), each warp one segment;
    // a multiple of kEmitWarps segments per block when the entries allow
    const uint64_t target = 8ull * 32ull * (uint64_t)(sm_count > 0 ? sm_count : 1);
    uint64_t S = (target + B - 1) / B;
    S = (S + kEmitWarps - 1) / kEmitWarps * kEmitWarps;
    const uint64_t max_s = (N_e + kGranule - 1) / kGranule;
    if (S > max_s) S = max_s;
    if (S < 1) S = 1;
    const uint64_t len = pba_segment_length(N_e, (uint32_t)S);
    const uint64_t used = (N_e + len - 1) / len;
    return (uint32_t)(used > 0 ? used : 1);
}

uint64_t pba_segment_length(uint64_t N_e, uint32_t S)
{
    const uint64_t per = (N_e + S - 1) / (S ? S : 1);
    uint64_t len = (per + kGranule - 1) / kGranule * kGranule;
    return len ? len : kGranule;
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
    w.off_recip = o;
    o += align256((size_t)B * sizeof(QRecip));
    w.off_flag = o;
    o += 256;
    w.off_stab = o;
    o += align256(kSeedTab * 4);
    w.total = o;
    return w;
}

// When set, the serial and two-phase kernels take their 64-bit-index
// variants for every input (the same output); a test hook that lets the
// parity tests check those variants on graphs small enough for the oracle.
// A workspace records the choice when it is prepared, so once the switch has
// been on, every later emit also launches the 64-bit variant (which returns
// at once unless the workspace's flag asks for it).
namespace {
std::atomic<bool> g_force_wide{false};
std::atomic<bool> g_ever_forced{false};
}
void set_wide_path_forced(bool on)
{
    if (on) g_ever_forced.store(true);
    g_force_wide.store(on);
}
bool wide_path_forced() { return g_force_wide.load(); }

cudaError_t launch_ba(const PbaGeom& g, int id64, void* d_out, cudaStream_t s)
{
    const int sms = device_sm_count();
    const uint64_t tile = id64 ? BaShape<uint64_t>::tile : BaShape<uint32_t>::tile;
    const uint64_t tiles = (g.N_e + tile - 1) / tile;
    const uint64_t full = (uint64_t)sms * 8;
    const int grid = (int)(tiles < full ? (tiles > 0 ? tiles : 1) : full);
    const bool fast = !wide_path_forced() && g.N_e + g.e0 < ((uint64_t)1 << 32);
    TraceScope trace("ba_chain", s);
    if (id64) {
        if (fast) { ba_kernel<uint64_t, true><<<grid, kBaThreads, 0, s>>>(g, (uint64_t*)d_out); note_launch(); }
        else { ba_kernel<uint64_t, false><<<grid, kBaThreads, 0, s>>>(g, (uint64_t*)d_out); note_launch(); }
    } else {
        if (fast) { ba_kernel<uint32_t, true><<<grid, kBaThreads, 0, s>>>(g, (uint32_t*)d_out); note_launch(); }
        else { ba_kernel<uint32_t, false><<<grid, kBaThreads, 0, s>>>(g, (uint32_t*)d_out); note_launch(); }
    }
    return cudaGetLastError();
}

namespace {

struct PbaBuffers {
    uint16_t* A;
    uint32_t* cnt;
    uint64_t *off, *R;
    FastDiv* divR;
    QRecip* recip;
    uint32_t* wide;
    uint32_t* stab;
};

PbaBuffers pba_buffers(const PbaGeom& g, void* d_ws)
{
    const PbaWorkspace L = pba_workspace_layout(g.A_stride, g.B, g.S);
    unsigned char* ws = (unsigned char*)d_ws;
    return PbaBuffers{(uint16_t*)(ws + L.off_A), (uint32_t*)(ws + L.off_cnt),
                      (uint64_t*)(ws + L.off_off), (uint64_t*)(ws + L.off_R),
                      (FastDiv*)(ws + L.off_magic), (QRecip*)(ws + L.off_recip),
                      (uint32_t*)(ws + L.off_flag), (uint32_t*)(ws + L.off_stab)};
}

constexpr size_t kSmemFast = kEmitWarps * sizeof(EmitWarpSmem<uint32_t>);
constexpr size_t kSmemWide = kEmitWarps * sizeof(EmitWarpSmem<uint64_t>);

// the 32-bit emit variant for this geometry: lean links when n_b is a power
// of two and the seed clique's edges fit the table
bool lean_links(const PbaGeom& g)
{
    return g.nb_shift != 0xFFFFFFFFu && g.e0 <= kSeedTab;
}

// The opt-in shared-memory sizes of the kernels that need more than the
// default, set once per device.
PerDeviceOnce g_pba_attrs;
cudaError_t set_pba_attributes()
{
    return g_pba_attrs.run_current([] {
        const int prefix = (int)(kPrefixMax * 2 + kMaxBlocks * 4);
        return first_error({
            cudaFuncSetAttribute(pba_prefix_kernel<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, prefix),
            cudaFuncSetAttribute(pba_prefix_kernel<true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, prefix),
            cudaFuncSetAttribute(pba_emit_kernel<uint32_t, 2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemFast),
            cudaFuncSetAttribute(pba_emit_kernel<uint64_t, 2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemFast),
            cudaFuncSetAttribute(pba_emit_kernel<uint32_t, 1>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemFast),
            cudaFuncSetAttribute(pba_emit_kernel<uint64_t, 1>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemFast),
            cudaFuncSetAttribute(pba_emit_kernel<uint32_t, 0>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemWide),
            cudaFuncSetAttribute(pba_emit_kernel<uint64_t, 0>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemWide)});
    });
}

}  // namespace

// Phase 1, counts and their scan: everything the emission of any block
// range reads, left in the workspace.
cudaError_t launch_pba_phase1(const PbaGeom& g, void* d_ws, cudaStream_t s)
{
    if (g.B > kMaxBlocks) return cudaErrorInvalidValue;
    cudaError_t err;
    if ((err = set_pba_attributes()) != cudaSuccess) return err;
    const PbaBuffers W = pba_buffers(g, d_ws);
    if ((err = cudaMemsetAsync(W.cnt, 0, (size_t)g.B * g.S * g.B * 4, s)) != cudaSuccess) return err;
    if ((err = cudaMemsetAsync(W.wide, 0, 4, s)) != cudaSuccess) return err;
    if (g.N_e > 0) {
        {
            TraceScope trace("pba_prefix", s);
            const size_t smem = ((size_t)g.P * 2 + 15) / 16 * 16 + (size_t)g.B * 4;
            if (g.ftab)
                { pba_prefix_kernel<true><<<g.B, kPrefixThreads, smem, s>>>(g, W.A, W.cnt); note_launch(); }
            else
                { pba_prefix_kernel<false><<<g.B, kPrefixThreads, smem, s>>>(g, W.A, W.cnt); note_launch(); }
        }
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        TraceScope trace("pba_phase1", s);
        for (uint64_t lvl = g.P; lvl < g.N_e;) {
            // level [lvl, hi): lvl / kLevelDiv more entries, in whole granules
            const uint64_t grow = (lvl / kLevelDiv + kPassChunk - 1) / kPassChunk * kPassChunk;
            const uint64_t hi = (lvl + grow < g.N_e) ? lvl + grow : g.N_e;
            const uint32_t chunks = (uint32_t)((hi - lvl + kPassChunk - 1) / kPassChunk);
            const size_t smem = (((size_t)g.B * 4 + 15) & ~(size_t)15) +
                                (size_t)(kPassThreads / 32) * kPassRun * 2;
            if (g.ftab)
                { pba_pass_kernel<true><<<dim3(chunks, g.B), kPassThreads, smem, s>>>(
                    g, (uint32_t)lvl, (uint32_t)hi, W.A, W.cnt); note_launch(); }
            else
                { pba_pass_kernel<false><<<dim3(chunks, g.B), kPassThreads, smem, s>>>(
                    g, (uint32_t)lvl, (uint32_t)hi, W.A, W.cnt); note_launch(); }
            if ((err = cudaGetLastError()) != cudaSuccess) return err;
            lvl = hi;
        }
    }
    {
        TraceScope trace("pba_scan", s);
        { pba_scan_kernel<<<(g.B + 31) / 32, 1024, 0, s>>>(W.cnt, W.off, W.R, W.divR, W.recip,
                                                          (uint32_t)g.n_b, g.B, g.B * g.S, g.e0,
                                                          wide_path_forced() ? 1u : 0u, W.wide,
                                                          g.n0, W.stab); note_launch(); }
    }
    return cudaGetLastError();
}

// Edges of blocks [b_begin, b_end), block b_begin's first edge at d_out[0].
cudaError_t launch_pba_emit(const PbaGeom& g, int id64, void* d_out, const void* d_ws,
                            uint32_t b_begin, uint32_t b_end, cudaStream_t s, const HostCopy* hc)
{
    if (g.B > kMaxBlocks || b_begin > b_end || b_end > g.B) return cudaErrorInvalidValue;
    if (b_begin == b_end) return cudaSuccess;
    cudaError_t err;
    if ((err = set_pba_attributes()) != cudaSuccess) return err;
    const PbaBuffers W = pba_buffers(g, const_cast<void*>(d_ws));
    // every R_q + e0 < 2^32 is certain when all entries together are fewer
    const bool surely_fast =
        !g_ever_forced.load() && (uint64_t)g.B * g.N_e + g.e0 < ((uint64_t)1 << 32);
    const uint32_t nblk = b_end - b_begin;
    const bool lean = lean_links(g);
    const uint32_t chunks = hc ? hc->chunks : 1;
    const uint32_t per = (nblk + chunks - 1) / chunks;
    const uint64_t edges_per_block = g.e0 + g.N_e;
    const uint64_t out_cap = (uint64_t)nblk * edges_per_block;   // edges at d_out
    const size_t pair = id64 ? 16 : 8;
    for (uint32_t b0 = b_begin, c = 0; b0 < b_end; b0 += per, ++c) {
        const uint32_t nb = (b_end - b0 < per) ? b_end - b0 : per;
        const dim3 grid((g.S + kEmitWarps - 1) / kEmitWarps, nb);
        {
            TraceScope trace("pba_emit", s);
            if (id64) {
                if (lean)
                    { pba_emit_kernel<uint64_t, 2><<<grid, kEmitThreads, kSmemFast, s>>>(
                        g, W.A, W.off, W.R, W.divR, W.recip, W.wide, W.stab, (uint64_t*)d_out, b0, b_begin,
                        out_cap); note_launch(); }
                else
                    { pba_emit_kernel<uint64_t, 1><<<grid, kEmitThreads, kSmemFast, s>>>(
                        g, W.A, W.off, W.R, W.divR, W.recip, W.wide, W.stab, (uint64_t*)d_out, b0, b_begin,
                        out_cap); note_launch(); }
                if (!surely_fast)
                    { pba_emit_kernel<uint64_t, 0><<<grid, kEmitThreads, kSmemWide, s>>>(
                        g, W.A, W.off, W.R, W.divR, W.recip, W.wide, W.stab, (uint64_t*)d_out, b0, b_begin,
                        out_cap); note_launch(); }
            } else {
                if (lean)
                    { pba_emit_kernel<uint32_t, 2><<<grid, kEmitThreads, kSmemFast, s>>>(
                        g, W.A, W.off, W.R, W.divR, W.recip, W.wide, W.stab, (uint32_t*)d_out, b0, b_begin,
                        out_cap); note_launch(); }
                else
                    { pba_emit_kernel<uint32_t, 1><<<grid, kEmitThreads, kSmemFast, s>>>(
                        g, W.A, W.off, W.R, W.divR, W.recip, W.wide, W.stab, (uint32_t*)d_out, b0, b_begin,
                        out_cap); note_launch(); }
                if (!surely_fast)
                    { pba_emit_kernel<uint32_t, 0><<<grid, kEmitThreads, kSmemWide, s>>>(
                        g, W.A, W.off, W.R, W.divR, W.recip, W.wide, W.stab, (uint32_t*)d_out, b0, b_begin,
                        out_cap); note_launch(); }
            }
        }
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        if (hc) {
            // this chunk's edges go to the host while the next chunk is made
            const size_t off_b = (size_t)(b0 - b_begin) * edges_per_block * pair;
            const size_t len = (size_t)nb * edges_per_block * pair;
            if ((err = cudaEventRecord(hc->done[c], s)) != cudaSuccess) return err;
            if ((err = cudaStreamWaitEvent(hc->copy_stream, hc->done[c], 0)) != cudaSuccess) return err;
            if ((err = cudaMemcpyAsync((char*)hc->h_edges + off_b, (const char*)d_out + off_b, len,
                                       cudaMemcpyDeviceToHost, hc->copy_stream)) != cudaSuccess)
                return err;
        }
    }
    if (hc) {
        // the caller's stream waits for the last copy
        if ((err = cudaEventRecord(hc->copied, hc->copy_stream)) != cudaSuccess) return err;
        if ((err = cudaStreamWaitEvent(s, hc->copied, 0)) != cudaSuccess) return err;
    }
    return cudaGetLastError();
}

cudaError_t launch_pba(const PbaGeom& g, int id64, void* d_out, void* d_ws, cudaStream_t s,
                       const HostCopy* hc)
{
    cudaError_t err = launch_pba_phase1(g, d_ws, s);
    if (err != cudaSuccess) return err;
    return launch_pba_emit(g, id64, d_out, d_ws, 0, g.B, s, hc);
}

}  // namespace pgen

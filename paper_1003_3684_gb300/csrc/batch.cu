// Batched generation: many independent graphs in one persistent launch.
//
// The host turns a list of jobs (serial BA or stochastic Kronecker graphs of
// any size) into a plan: one record per job with its parameters, its Philox
// round keys, its Kronecker thresholds, where its edges start in a shared
// output arena, and how many work items (tiles of `tile` edges) it has. The
// kernel's CTAs stay resident; each repeatedly claims the next work item from
// a device counter (one atomicAdd, never a wait), finds the item's job by a
// binary search over the per-job first-item table in shared memory, and runs
// the job's tile with the same arithmetic as the single-graph kernels: pooled
// copy chains for BA, k-level descent for Kronecker. Small and large jobs
// thus share the GPU without a launch per graph. The whole call (counter reset
// + kernel) is stream-ordered and contains no host synchronisation, so it can
// be captured in a CUDA graph and replayed.
#include <cmath>
#include <type_traits>
#include <cstring>

#include "../../include/pgen.h"
#include "pg_internal.h"
#include "pg_trace.h"

namespace pgen {
namespace {

constexpr int kBatchThreads = 256;
constexpr uint32_t kBatchWarps = kBatchThreads / 32;
constexpr uint32_t kMaxTile = 8192;        // staging limit (edges per work item)
constexpr uint32_t kMaxBatchJobs = 8192;   // first-item table held in smem

// A job's kind in the plan: PG_JOB_BA (serial BA, tiles of the persistent
// kernel), PG_JOB_KRON, or a two-phase PBA job (blocks > 1), which has no
// work items: gen_batch runs it with the single-graph PBA kernels.
constexpr uint32_t kKindTwoPhase = 2;

struct BatchJob {              // 256 bytes, one per job
    uint32_t kind, m, n0, k;
    uint64_t n_units;          // BA: n*m generated edges; KRON: edges
    uint64_t out_edge;         // first edge of the job in the arena
    uint64_t e0;               // BA: seed-clique edges (written by tile 0)
    uint32_t tile;             // edges per work item
    uint32_t n_zero, n_u;      // KRON thresholds (see KronParams)
    uint32_t u_off;            // KRON: offset of u[] in the threshold pool (n0 > 2)
    uint32_t u0, u1, u2, pad;  // KRON n0 = 2 thresholds
    FastDiv32 div_m;
    uint32_t want_csr;         // 0: no CSR; 1 + g: gen_batch_csr builds it in group g
    Key key;                   // 80 bytes
    uint64_t n_vertices;       // ids of the job's graph: 0 .. n_vertices - 1
    uint64_t vbase;            // want_csr: first row of the job in its group's union graph
    uint64_t csr_edge;         // want_csr: first col entry of the job (and its union slot)
    uint64_t rbase;            // want_csr: first row_ptr entry of the job
    uint64_t edges;            // the job's edges: [out_edge, out_edge + edges) of the arena
    uint8_t reserved[256 - 80 - 88 - 40];
};
static_assert(sizeof(BatchJob) == 256, "job record is 256 bytes");

// A two-phase PBA job's launch geometry, read by the host in gen_batch.
struct TwoPhaseJob {
    uint32_t job, pad;
    uint64_t ws_bytes;         // its PBA workspace
    PbaGeom g;
};

struct PlanHeader {
    uint32_t n_jobs, n_pool;
    uint64_t n_items, total_edges;
    uint64_t off_jobs, off_first, off_pool;
    uint64_t off_starts;       // n_jobs + 1 uint64: every job's first edge, then the total
    uint64_t off_rstart[2];    // per CSR group g: csr_jobs[g] + 1 uint64, each CSR job's
                               // first row_ptr entry, then the group's end
    uint64_t off_two;          // n_two TwoPhaseJob records (host only)
    uint32_t n_two, id64;
    uint64_t two_ws;           // the largest two-phase job's workspace
    // The CSR jobs form two groups, each with its own union graph: 0, the BA
    // jobs (their lists are grouped by source, so their union needs no
    // sort), and 1, the Kronecker jobs. Group 0's row_ptr and col entries
    // come first in the output arenas.
    uint64_t csr_jobs[2], csr_vertices[2], csr_edges[2];
    uint64_t csr_max_vertices[2];   // the largest job of the group: bounds its col ids
};

size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

size_t plan_bytes(uint32_t n_jobs, uint32_t n_pool, uint32_t n_two, uint32_t n_csr)
{
    return a16(sizeof(PlanHeader)) + a16((size_t)n_jobs * sizeof(BatchJob)) +
           a16((size_t)(n_jobs + 1) * 4) + a16((size_t)n_pool * 4) +
           a16((size_t)(n_jobs + 1) * 8) + 2 * a16((size_t)(n_csr + 1) * 8) +
           a16((size_t)n_two * sizeof(TwoPhaseJob));
}

// Edge e (and e + 1) of an arena of `cap` edges.
template <typename Id>
__device__ __forceinline__ void put_pair(Id* out, uint64_t cap, uint64_t e, uint64_t s, uint64_t d)
{
    if (!PG_CHECK_OUT(e, cap)) return;
    out[2 * e] = (Id)s;
    out[2 * e + 1] = (Id)d;
}

template <typename Id>
__device__ __forceinline__ void put_two(Id* out, uint64_t cap, uint64_t e, uint64_t s0,
                                        uint64_t d0, uint64_t s1, uint64_t d1)
{
    if (!PG_CHECK_OUT(e + 1, cap)) return;
    if constexpr (sizeof(Id) == 4) {
        *reinterpret_cast<uint4*>(out + 2 * e) =
            make_uint4((uint32_t)s0, (uint32_t)d0, (uint32_t)s1, (uint32_t)d1);
    } else {
        ulonglong2* o = reinterpret_cast<ulonglong2*>(out + 2 * e);
        o[0] = make_ulonglong2(s0, d0);
        o[1] = make_ulonglong2(s1, d1);
    }
}

// One serial-BA link with 32-bit indices (as in the single-graph kernel).
__device__ __forceinline__ bool ba_link(uint32_t& cur, const BatchJob& J, const Key& key,
                                        const PhiloxHead& ph, uint32_t& v)
{
    const uint32_t sig = fdiv32(cur, J.div_m);
    const uint4 w = philox_headed(cur, ph, key);   // counter (cur, 0, 0, 2)
    const uint32_t X = (uint32_t)J.e0 + sig * J.m;
    const uint64_t s = (uint64_t)w.y * X + (((uint64_t)w.x * X) >> 32);
    const uint32_t e = (uint32_t)(s >> 32);
    const uint32_t side = ((uint32_t)s) >> 31;
    if (e < (uint32_t)J.e0) {
        v = seed_endpoint(e, side, J.n0);
        return true;
    }
    const uint32_t e2 = e - (uint32_t)J.e0;
    if (side == 0) {
        v = J.n0 + fdiv32(e2, J.div_m);
        return true;
    }
    cur = e2;
    return false;
}

__device__ __forceinline__ void kron_level(uint32_t w, uint32_t base, uint32_t u0, uint32_t u1,
                                           uint32_t u2, uint64_t& row, uint64_t& col)
{
    const uint32_t cell = base + (w > u0) + (w > u1) + (w > u2);
    row = (row << 1) | (cell >> 1);
    col = (col << 1) | (cell & 1);
}

// The same pick for a 2x2 initiator whose four cells are all positive
// (n_zero = 0, three real thresholds u0 <= u1 <= u2): the row bit is
// a = (w > u1), the column bit (w > u2) when a is set, else (w > u0).
__device__ __forceinline__ void kron_level_full(uint32_t w, uint32_t u0, uint32_t u1, uint32_t u2,
                                                uint64_t& row, uint64_t& col)
{
    const uint32_t a = w > u1 ? 1u : 0u;
    const uint32_t b = w > (a ? u2 : u0) ? 1u : 0u;
    row = row * 2 + a;
    col = col * 2 + b;
}

// The full-initiator 2x2 pick for a job whose ids and edge indices fit 32
// bits (k <= 32 levels, fewer than 2^32 edges): the same values with 32-bit
// rows, columns and counters (e, 0, g, 3), the thresholds and k in registers
// for the whole tile, whole groups of four levels unrolled.
__device__ __forceinline__ void kron_edge_full32(const Key& key, uint32_t k, uint32_t u0,
                                                 uint32_t u1, uint32_t u2, uint32_t e,
                                                 uint32_t& row, uint32_t& col)
{
    row = 0;
    col = 0;
    uint32_t l = 0;
    auto level = [&](uint32_t w) {
        const uint32_t a = w > u1 ? 1u : 0u;
        const uint32_t b = w > (a ? u2 : u0) ? 1u : 0u;
        row = row * 2 + a;
        col = col * 2 + b;
    };
    for (uint32_t g = 0; l + 4 <= k; ++g, l += 4) {
        const uint4 w = philox(make_uint4(e, 0u, g, 3u), key);
        level(w.x);
        level(w.y);
        level(w.z);
        level(w.w);
    }
    if (l < k) {
        const uint4 w = philox(make_uint4(e, 0u, l >> 2, 3u), key);
        level(w.x);
        if (l + 1 < k) level(w.y);
        if (l + 2 < k) level(w.z);
    }
}

__device__ __forceinline__ void kron_edge(const BatchJob& J, const Key& key,
                                          const uint32_t* pool, uint32_t n_pool, uint64_t e,
                                          uint64_t& row, uint64_t& col)
{
    row = 0;
    col = 0;
    if (J.n0 == 2 && J.n_zero == 0 && J.n_u == 3) {
        uint32_t l = 0;
        for (uint32_t g = 0; l < J.k; ++g, l += 4) {
            const uint4 w = philox(make_uint4((uint32_t)e, (uint32_t)(e >> 32), g, 3u), key);
            kron_level_full(w.x, J.u0, J.u1, J.u2, row, col);
            if (l + 1 < J.k) kron_level_full(w.y, J.u0, J.u1, J.u2, row, col);
            if (l + 2 < J.k) kron_level_full(w.z, J.u0, J.u1, J.u2, row, col);
            if (l + 3 < J.k) kron_level_full(w.w, J.u0, J.u1, J.u2, row, col);
        }
        return;
    }
    if (J.n0 == 2) {
        uint32_t l = 0;
        for (uint32_t g = 0; l < J.k; ++g, l += 4) {
            const uint4 w = philox(make_uint4((uint32_t)e, (uint32_t)(e >> 32), g, 3u), key);
            kron_level(w.x, J.n_zero, J.u0, J.u1, J.u2, row, col);
            if (l + 1 < J.k) kron_level(w.y, J.n_zero, J.u0, J.u1, J.u2, row, col);
            if (l + 2 < J.k) kron_level(w.z, J.n_zero, J.u0, J.u1, J.u2, row, col);
            if (l + 3 < J.k) kron_level(w.w, J.n_zero, J.u0, J.u1, J.u2, row, col);
        }
        return;
    }
    if (J.n_u > 0 && !PG_CHECK((uint64_t)J.u_off + J.n_u - 1, n_pool)) return;
    const uint32_t* u = pool + J.u_off;
    uint4 w = make_uint4(0, 0, 0, 0);
    for (uint32_t l = 0; l < J.k; ++l) {
        if ((l & 3) == 0)
            w = philox(make_uint4((uint32_t)e, (uint32_t)(e >> 32), l >> 2, 3u), key);
        const uint32_t x = (l & 3) == 0 ? w.x : (l & 3) == 1 ? w.y : (l & 3) == 2 ? w.z : w.w;
        uint32_t lo = 0, hi = J.n_u;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (u[mid] < x) lo = mid + 1;
            else hi = mid;
        }
        const uint32_t cell = J.n_zero + lo;
        row = row * J.n0 + cell / J.n0;
        col = col * J.n0 + cell % J.n0;
    }
}

template <typename Id>
__global__ void __launch_bounds__(kBatchThreads) batch_kernel(const unsigned char* __restrict__ plan,
                                                              Id* __restrict__ arena,
                                                              unsigned long long* __restrict__ counter,
                                                              uint64_t cap, uint32_t n_jobs_smem)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const PlanHeader& H = *reinterpret_cast<const PlanHeader*>(plan);
    const BatchJob* jobs = reinterpret_cast<const BatchJob*>(plan + H.off_jobs);
    const uint32_t* first_g = reinterpret_cast<const uint32_t*>(plan + H.off_first);
    const uint32_t* pool = reinterpret_cast<const uint32_t*>(plan + H.off_pool);
    const uint32_t n_jobs = H.n_jobs;
    const uint64_t n_items = H.n_items;
    // the first-item table in smem was sized for n_jobs_smem jobs (uniform exit)
    if (!PG_CHECK(n_jobs, n_jobs_smem + 1)) return;

    Id* sDst = reinterpret_cast<Id*>(smem);                                    // kMaxTile ids
    uint32_t* first = reinterpret_cast<uint32_t*>(smem + kMaxTile * sizeof(Id));   // n_jobs + 1
    __shared__ uint32_t s_item, s_job;
    __shared__ BatchJob sJ;

    for (uint32_t t = threadIdx.x; t <= n_jobs; t += blockDim.x) first[t] = first_g[t];
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    for (;;) {
        __syncthreads();   // previous item finished with s_item / sJ / sDst
        if (threadIdx.x == 0) {
            const unsigned long long it = atomicAdd(counter, 1ull);
            s_item = it < n_items ? (uint32_t)it : 0xFFFFFFFFu;
            if (it < n_items) {
                uint32_t lo = 0, hi = n_jobs;   // last job with first[job] <= it
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (first[mid] <= (uint32_t)it) lo = mid;
                    else hi = mid;
                }
                s_job = lo;
            }
        }
        __syncthreads();
        if (s_item == 0xFFFFFFFFu) break;
        for (uint32_t t = threadIdx.x; t < sizeof(BatchJob) / 4; t += blockDim.x)
            reinterpret_cast<uint32_t*>(&sJ)[t] = reinterpret_cast<const uint32_t*>(&jobs[s_job])[t];
        __syncthreads();
        const BatchJob& J = sJ;
        const Key key = J.key;
        const uint64_t t0 = (uint64_t)(s_item - first[s_job]) * J.tile;
        const uint32_t n = (uint32_t)((J.n_units - t0 < J.tile) ? J.n_units - t0 : J.tile);

        if (J.kind == PG_JOB_BA) {
            if (t0 == 0)
                for (uint64_t e = threadIdx.x; e < J.e0; e += blockDim.x)
                    put_pair(arena, cap, J.out_edge + e, seed_endpoint(e, 0, J.n0),
                             seed_endpoint(e, 1, J.n0));
            // warps take runs of the tile; lanes pool their chains
            const uint32_t per = (n + kBatchWarps - 1) / kBatchWarps;
            const uint32_t r0 = wid * per < n ? wid * per : n;
            const uint32_t r1 = r0 + per < n ? r0 + per : n;
            const uint32_t n_items_w = r1 - r0;
            uint32_t next = 32, item = lane;
            uint32_t cur = (uint32_t)(t0 + r0 + item);
            bool active = item < n_items_w;
            const PhiloxHead ph = philox_head(0u, 0u, 2u, key);
            while (__any_sync(0xFFFFFFFFu, active)) {
                bool done = false;
                if (active) {
                    uint32_t v;
                    done = ba_link(cur, J, key, ph, v);
                    if (done && PG_CHECK(r0 + item, kMaxTile)) sDst[r0 + item] = (Id)v;
                }
                const uint32_t dm = __ballot_sync(0xFFFFFFFFu, done);
                if (done) {
                    item = next + __popc(dm & lt);
                    cur = (uint32_t)(t0 + r0 + item);
                    active = item < n_items_w;
                }
                next += __popc(dm);
            }
            __syncthreads();
            const uint64_t e_first = J.out_edge + J.e0 + t0;
            const uint32_t head = (uint32_t)(e_first & 1) < n ? (uint32_t)(e_first & 1) : n;
            if (head && threadIdx.x == 0)
                put_pair(arena, cap, e_first, J.n0 + fdiv32((uint32_t)t0, J.div_m), (uint64_t)sDst[0]);
            for (uint32_t t2 = head + 2 * threadIdx.x; t2 < n; t2 += 2 * blockDim.x) {
                const uint64_t s0 = J.n0 + fdiv32((uint32_t)(t0 + t2), J.div_m);
                if (t2 + 1 < n)
                    put_two(arena, cap, e_first + t2, s0, (uint64_t)sDst[t2],
                            J.n0 + fdiv32((uint32_t)(t0 + t2 + 1), J.div_m), (uint64_t)sDst[t2 + 1]);
                else
                    put_pair(arena, cap, e_first + t2, s0, (uint64_t)sDst[t2]);
            }
        } else if (J.n0 == 2 && J.n_zero == 0 && J.n_u == 3 && J.k <= 32 &&
                   J.n_units <= 0xFFFFFFFFull) {
            // 32-bit full-initiator descent (the kron2 kernel's arithmetic)
            const uint32_t k = J.k, u0 = J.u0, u1 = J.u1, u2 = J.u2;
            const uint64_t e_first = J.out_edge + t0;
            const uint32_t head = (uint32_t)(e_first & 1) < n ? (uint32_t)(e_first & 1) : n;
            if (head && threadIdx.x == 0) {
                uint32_t r, c;
                kron_edge_full32(key, k, u0, u1, u2, (uint32_t)t0, r, c);
                put_pair(arena, cap, e_first, r, c);
            }
            for (uint32_t t2 = head + 2 * threadIdx.x; t2 < n; t2 += 2 * blockDim.x) {
                uint32_t r0, c0;
                kron_edge_full32(key, k, u0, u1, u2, (uint32_t)(t0 + t2), r0, c0);
                if (t2 + 1 < n) {
                    uint32_t r1, c1;
                    kron_edge_full32(key, k, u0, u1, u2, (uint32_t)(t0 + t2 + 1), r1, c1);
                    put_two(arena, cap, e_first + t2, r0, c0, r1, c1);
                } else {
                    put_pair(arena, cap, e_first + t2, r0, c0);
                }
            }
        } else {
            const uint64_t e_first = J.out_edge + t0;
            const uint32_t head = (uint32_t)(e_first & 1) < n ? (uint32_t)(e_first & 1) : n;
            if (head && threadIdx.x == 0) {
                uint64_t r, c;
                kron_edge(J, key, pool, H.n_pool, t0, r, c);
                put_pair(arena, cap, e_first, r, c);
            }
            for (uint32_t t2 = head + 2 * threadIdx.x; t2 < n; t2 += 2 * blockDim.x) {
                uint64_t r0, c0;
                kron_edge(J, key, pool, H.n_pool, t0 + t2, r0, c0);
                if (t2 + 1 < n) {
                    uint64_t r1, c1;
                    kron_edge(J, key, pool, H.n_pool, t0 + t2 + 1, r1, c1);
                    put_two(arena, cap, e_first + t2, r0, c0, r1, c1);
                } else {
                    put_pair(arena, cap, e_first + t2, r0, c0);
                }
            }
        }
    }
}

// Rewrites the edges of every want_csr job into its group's union list of
// (vbase + src, dst) pairs, at the job's csr_edge: the union graph of the
// group, whose CSR is its jobs' CSRs one after another (rows of job t are
// vbase_t .. vbase_t + n_vertices_t - 1, and its col entries keep their
// local ids). One pair per thread, moved as one vector load and store; lane
// 0 of a warp finds the job of the warp's first edge by a binary search over
// the job starts, and each lane steps from there to its own.
template <typename Id>
__global__ void __launch_bounds__(256) batch_union_kernel(const unsigned char* __restrict__ plan,
                                                          const Id* __restrict__ arena,
                                                          Id* __restrict__ uni)
{
    using P = typename std::conditional<sizeof(Id) == 4, uint2, ulonglong2>::type;
    const PlanHeader& H = *reinterpret_cast<const PlanHeader*>(plan);
    const BatchJob* jobs = reinterpret_cast<const BatchJob*>(plan + H.off_jobs);
    const uint64_t* starts = reinterpret_cast<const uint64_t*>(plan + H.off_starts);
    const uint32_t n_jobs = H.n_jobs;
    const uint64_t E = H.total_edges;
    const P* in = reinterpret_cast<const P*>(arena);
    P* out = reinterpret_cast<P*>(uni);
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t base = (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < E;
         base += warps * 32) {
        uint32_t job = 0;
        if (lane == 0) {
            uint32_t lo = 0, hi = n_jobs;   // the last job starting at or before base
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (starts[mid] <= base) lo = mid;
                else hi = mid;
            }
            job = lo;
        }
        job = __shfl_sync(0xFFFFFFFFu, job, 0);
        const uint64_t e = base + lane;
        if (e >= E) continue;
        while (job + 1 < n_jobs && starts[job + 1] <= e) ++job;
        const BatchJob& J = jobs[job];
        const uint64_t local = e - J.out_edge;   // past the job's edges: an alignment gap
        if (!J.want_csr || local >= J.edges) continue;
        const uint64_t at = J.csr_edge + local;
        if (PG_CHECK(at, H.csr_edges[0] + H.csr_edges[1])) {
            P p = in[e];
            p.x += (decltype(p.x))J.vbase;
            out[at] = p;
        }
    }
}

// Row pointers of the CSR jobs of one group from its union's (rp_u,
// vertices + 1 entries): job t of the group owns output entries rstart[t] ..
// rstart[t] + n_vertices_t, and entry v there is rp_u[vbase_t + v] -
// rp_u[vbase_t], with vbase_t = rstart[t] - rstart[0] - t.
__global__ void __launch_bounds__(256) batch_rebase_kernel(const uint64_t* __restrict__ rstart,
                                                           uint64_t jobs, uint64_t vertices,
                                                           const uint64_t* __restrict__ rp_u,
                                                           uint64_t* __restrict__ out)
{
    const uint64_t r0 = rstart[0], R = rstart[jobs] - r0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += stride) {
        uint64_t lo = 0, hi = jobs;   // the last job whose entries start at or before r
        while (hi - lo > 1) {
            const uint64_t mid = (lo + hi) >> 1;
            if (rstart[mid] - r0 <= r) lo = mid;
            else hi = mid;
        }
        const uint64_t vbase = rstart[lo] - r0 - lo;
        const uint64_t v = vbase + (r - (rstart[lo] - r0));
        if (PG_CHECK(v, vertices + 1)) out[r0 + r] = rp_u[v] - rp_u[vbase];
    }
}

__global__ void or_word_kernel(uint32_t* __restrict__ dst, const uint32_t* __restrict__ src)
{
    *dst |= *src;
}

}  // namespace

PG_CHECK_UNIT(batch)

namespace {

bool kron_thresholds_host(const double* P, uint32_t n0, uint64_t* T)
{
    const uint32_t cells = n0 * n0;
    double S = 0.0;
    for (uint32_t c = 0; c < cells; ++c) {
        if (!(P[c] >= 0.0) || !std::isfinite(P[c])) return false;
        S += P[c];
    }
    if (!(S > 0.0) || !std::isfinite(S)) return false;
    double cum = 0.0;
    for (uint32_t c = 0; c + 1 < cells; ++c) {
        cum += P[c];
        T[c] = (uint64_t)std::nearbyint(std::ldexp(cum / S, 32));
    }
    return true;
}

}  // namespace

}  // namespace pgen

using namespace pgen;

extern "C" {

size_t pg_batch_plan_size(const pg_job* jobs, uint32_t n_jobs)
{
    uint64_t pool = 0;
    uint32_t two = 0, csr = 0;
    for (uint32_t i = 0; jobs && i < n_jobs; ++i) {
        if (jobs[i].kind == PG_JOB_KRON && jobs[i].n0 > 2 && jobs[i].n0 <= 16)
            pool += (uint64_t)jobs[i].n0 * jobs[i].n0;
        if (jobs[i].kind == PG_JOB_BA && jobs[i].blocks > 1) ++two;
        if (jobs[i].want_csr) ++csr;
    }
    return plan_bytes(n_jobs, (uint32_t)pool, two, csr);
}

size_t pg_batch_workspace_size(const void* h_plan)
{
    // the persistent kernel's work counter, then the two-phase jobs' PBA
    // workspace (they run one after another, so one region serves all)
    if (!h_plan) return 256;
    const PlanHeader& H = *(const PlanHeader*)h_plan;
    return 256 + (H.n_two ? ((H.two_ws + 255) & ~(uint64_t)255) : 0);
}

pg_status pg_batch_plan(const pg_job* jobs, uint32_t n_jobs, uint32_t tile_edges, pg_idwidth w,
                        void* h_plan, size_t plan_size, uint64_t* h_edge_offsets,
                        uint64_t* h_n_items)
{
    if (!jobs || n_jobs == 0 || n_jobs > kMaxBatchJobs || !h_plan) return PG_EINVAL;
    if (tile_edges < 64 || tile_edges > kMaxTile || tile_edges % 64 != 0) return PG_EINVAL;
    if (w != PG_ID32 && w != PG_ID64) return PG_EINVAL;
    if (plan_size < pg_batch_plan_size(jobs, n_jobs)) return PG_ENOMEM;
    std::memset(h_plan, 0, plan_size);
    uint32_t n_two = 0, n_csr = 0;
    for (uint32_t i = 0; i < n_jobs; ++i) {
        if (jobs[i].kind == PG_JOB_BA && jobs[i].blocks > 1) ++n_two;
        if (jobs[i].want_csr) ++n_csr;
    }
    unsigned char* base = (unsigned char*)h_plan;
    PlanHeader& H = *(PlanHeader*)base;
    H.n_jobs = n_jobs;
    H.id64 = w == PG_ID64;
    H.off_jobs = a16(sizeof(PlanHeader));
    H.off_first = H.off_jobs + a16((size_t)n_jobs * sizeof(BatchJob));
    H.off_pool = H.off_first + a16((size_t)(n_jobs + 1) * 4);
    BatchJob* J = (BatchJob*)(base + H.off_jobs);
    uint32_t* first = (uint32_t*)(base + H.off_first);
    uint32_t* pool = (uint32_t*)(base + H.off_pool);
    uint32_t pool_entries = 0;
    for (uint32_t i = 0; i < n_jobs; ++i)
        if (jobs[i].kind == PG_JOB_KRON && jobs[i].n0 > 2 && jobs[i].n0 <= 16)
            pool_entries += jobs[i].n0 * jobs[i].n0;
    H.off_starts = H.off_pool + a16((size_t)pool_entries * 4);
    H.off_rstart[0] = H.off_starts + a16((size_t)(n_jobs + 1) * 8);
    H.off_rstart[1] = H.off_rstart[0] + a16((size_t)(n_csr + 1) * 8);
    H.off_two = H.off_rstart[1] + a16((size_t)(n_csr + 1) * 8);
    uint64_t* starts = (uint64_t*)(base + H.off_starts);
    TwoPhaseJob* two = (TwoPhaseJob*)(base + H.off_two);
    uint64_t edges = 0, items = 0;
    uint32_t n_pool = 0;
    const uint64_t id_limit = w == PG_ID32 ? ((uint64_t)1 << 32) : ~(uint64_t)0;
    for (uint32_t i = 0; i < n_jobs; ++i) {
        const pg_job& q = jobs[i];
        BatchJob& b = J[i];
        b.kind = q.kind;
        b.tile = tile_edges;
        b.key = make_key(q.seed);
        uint64_t job_items = 0;
        if (q.kind == PG_JOB_BA && q.blocks > 1) {
            // two-phase PBA: the single-graph kernels write it, from an even
            // edge so that their 16-byte stores stay aligned
            TwoPhaseJob& tp = two[H.n_two];
            uint64_t ne = 0;
            const int st = pba_setup(q.n, q.m, q.blocks, q.n0, q.faction_width ? q.faction_width : 1,
                                     q.inter_frac, q.seed, w == PG_ID64, &tp.g, &ne);
            if (st != PG_OK) return (pg_status)st;
            if (w == PG_ID32) edges += edges & 1;
            tp.job = i;
            tp.ws_bytes = pba_workspace_layout(tp.g.A_stride, tp.g.B, tp.g.S).total;
            if (tp.ws_bytes > H.two_ws) H.two_ws = tp.ws_bytes;
            ++H.n_two;
            b.kind = kKindTwoPhase;
            b.m = q.m;
            b.n0 = q.n0;
            b.edges = ne;
            b.n_vertices = (uint64_t)tp.g.B * tp.g.span;
        } else if (q.kind == PG_JOB_BA) {
            if (q.m < 1 || q.n0 < 2 || q.n0 > 65536) return PG_EINVAL;
            const unsigned __int128 ne = (unsigned __int128)q.n * q.m;
            b.e0 = (uint64_t)q.n0 * (q.n0 - 1) / 2;
            if (ne + b.e0 >= ((unsigned __int128)1 << 32)) return PG_EINVAL;   // 32-bit links
            if ((uint64_t)q.n0 + q.n > id_limit) return PG_EINVAL;
            b.m = q.m;
            b.n0 = q.n0;
            b.n_units = (uint64_t)ne;
            b.div_m = make_fastdiv32(q.m);
            b.edges = b.e0 + b.n_units;
            b.n_vertices = (uint64_t)q.n0 + q.n;
            job_items = (b.n_units + tile_edges - 1) / tile_edges;
            if (job_items == 0) job_items = 1;   // its seed clique
        } else if (q.kind == PG_JOB_KRON) {
            if (!q.initiator || q.n0 < 1 || q.n0 > 16 || q.k < 1 || q.k > 64) return PG_EINVAL;
            unsigned __int128 nv = 1;
            for (uint32_t l = 0; l < q.k && nv <= id_limit; ++l) nv *= q.n0;
            if (nv > id_limit) return PG_EINVAL;
            uint64_t T[255];
            if (!kron_thresholds_host(q.initiator, q.n0, T)) return PG_EINVAL;
            const uint32_t cells = q.n0 * q.n0;
            uint32_t c = 0;
            while (c + 1 < cells && T[c] == 0) ++c;
            b.n_zero = c;
            uint32_t u[255];
            uint32_t nu = 0;
            for (; c + 1 < cells && T[c] < ((uint64_t)1 << 32); ++c) u[nu++] = (uint32_t)(T[c] - 1);
            b.n_u = nu;
            b.n0 = q.n0;
            b.k = q.k;
            b.n_units = q.n;
            if (q.n0 == 2) {
                b.u0 = nu > 0 ? u[0] : 0xFFFFFFFFu;
                b.u1 = nu > 1 ? u[1] : 0xFFFFFFFFu;
                b.u2 = nu > 2 ? u[2] : 0xFFFFFFFFu;
            } else {
                b.u_off = n_pool;
                for (uint32_t t = 0; t < nu; ++t) pool[n_pool++] = u[t];
            }
            b.edges = b.n_units;
            b.n_vertices = (uint64_t)nv;
            job_items = (b.n_units + tile_edges - 1) / tile_edges;
        } else {
            return PG_EINVAL;
        }
        b.out_edge = edges;
        starts[i] = edges;
        edges += b.edges;
        if (q.want_csr) b.want_csr = 1 + (q.kind == PG_JOB_KRON ? 1u : 0u);
        first[i] = (uint32_t)items;
        items += job_items;
        if (items >= 0xFFFFFFFFull) return PG_EINVAL;
        if (h_edge_offsets) h_edge_offsets[i] = b.out_edge;
    }
    first[n_jobs] = (uint32_t)items;
    starts[n_jobs] = edges;
    // the CSR groups: each job's rows in its group's union graph, then its
    // places in the output arenas (group 0's jobs first, in job order)
    for (uint32_t i = 0; i < n_jobs; ++i) {
        if (!J[i].want_csr) continue;
        const uint32_t g = J[i].want_csr - 1;
        J[i].vbase = H.csr_vertices[g];
        H.csr_vertices[g] += J[i].n_vertices;
        H.csr_edges[g] += J[i].edges;
        ++H.csr_jobs[g];
        if (J[i].n_vertices > H.csr_max_vertices[g]) H.csr_max_vertices[g] = J[i].n_vertices;
        if (H.csr_vertices[g] > id_limit || H.csr_vertices[g] >= ((uint64_t)1 << 62))
            return PG_EINVAL;   // the union's row ids must fit the id width
    }
    const uint64_t row_base[2] = {0, H.csr_vertices[0] + H.csr_jobs[0]};
    const uint64_t col_base[2] = {0, H.csr_edges[0]};
    uint64_t t_g[2] = {0, 0}, e_g[2] = {0, 0};
    for (uint32_t i = 0; i < n_jobs; ++i) {
        if (!J[i].want_csr) continue;
        const uint32_t g = J[i].want_csr - 1;
        uint64_t* rstart = (uint64_t*)(base + H.off_rstart[g]);
        J[i].csr_edge = col_base[g] + e_g[g];
        J[i].rbase = row_base[g] + J[i].vbase + t_g[g];
        rstart[t_g[g]++] = J[i].rbase;
        e_g[g] += J[i].edges;
    }
    for (uint32_t g = 0; g < 2; ++g)
        ((uint64_t*)(base + H.off_rstart[g]))[H.csr_jobs[g]] =
            row_base[g] + H.csr_vertices[g] + H.csr_jobs[g];
    H.n_items = items;
    H.total_edges = edges;
    H.n_pool = n_pool;
    if (h_edge_offsets) h_edge_offsets[n_jobs] = edges;
    if (h_n_items) *h_n_items = items;
    return PG_OK;
}

namespace {
// The host plan's header, if it describes a plan of n_jobs jobs of width w.
const PlanHeader* plan_header(const void* h_plan, uint32_t n_jobs, pg_idwidth w)
{
    if (!h_plan) return nullptr;
    const PlanHeader* H = (const PlanHeader*)h_plan;
    if (H->n_jobs != n_jobs || H->id64 != (w == PG_ID64 ? 1u : 0u)) return nullptr;
    return H;
}
}  // namespace

pg_status gen_batch(const void* h_plan, const void* d_plan, uint32_t n_jobs, pg_idwidth w,
                    void* d_arena, uint64_t cap_edges, uint64_t total_edges, uint32_t grid_ctas,
                    void* d_ws, size_t ws_bytes, void* stream)
{
    if (!d_plan || n_jobs == 0 || n_jobs > kMaxBatchJobs) return PG_EINVAL;
    if (w != PG_ID32 && w != PG_ID64) return PG_EINVAL;
    const PlanHeader* HP = plan_header(h_plan, n_jobs, w);
    if (!HP || HP->total_edges != total_edges) return PG_EINVAL;
    if (cap_edges < total_edges) return PG_ENOSPC;
    if (total_edges > 0 && (!d_arena || ((uintptr_t)d_arena & 15))) return PG_EINVAL;
    if (!d_ws || ws_bytes < pg_batch_workspace_size(h_plan) || ((uintptr_t)d_ws & 255))
        return PG_ENOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t id_bytes = w == PG_ID64 ? 8 : 4;
    const size_t smem = kMaxTile * id_bytes + (size_t)(n_jobs + 1) * 4;
    // the opt-in shared-memory sizes, set once per device
    static PerDeviceOnce attrs;
    const cudaError_t ae = attrs.run_current([] {
        return first_error({
            cudaFuncSetAttribute(batch_kernel<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kMaxTile * 4 + (kMaxBatchJobs + 1) * 4)),
            cudaFuncSetAttribute(batch_kernel<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kMaxTile * 8 + (kMaxBatchJobs + 1) * 4))});
    });
    if (ae != cudaSuccess) return PG_ECUDA;
    if (HP->n_items > 0) {
        int per_sm = 0;
        if (w == PG_ID64)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<uint64_t>, kBatchThreads, smem);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<uint32_t>, kBatchThreads, smem);
        if (per_sm < 1) per_sm = 1;
        const uint32_t full = (uint32_t)(device_sm_count() * per_sm);
        const uint32_t grid = grid_ctas == 0 || grid_ctas > full ? full : grid_ctas;
        if (cudaMemsetAsync(d_ws, 0, 8, s) != cudaSuccess) return PG_ECUDA;
        TraceScope trace("batch_persistent", s);
        if (w == PG_ID64)
            { batch_kernel<uint64_t><<<grid, kBatchThreads, smem, s>>>(
                (const unsigned char*)d_plan, (uint64_t*)d_arena, (unsigned long long*)d_ws, cap_edges,
                n_jobs); note_launch(); }
        else
            { batch_kernel<uint32_t><<<grid, kBatchThreads, smem, s>>>(
                (const unsigned char*)d_plan, (uint32_t*)d_arena, (unsigned long long*)d_ws, cap_edges,
                n_jobs); note_launch(); }
        if (cudaGetLastError() != cudaSuccess) return PG_ECUDA;
    }
    // two-phase PBA jobs: phase 1, the count exchange and the emission of
    // each, in the shared workspace region after the counter
    const TwoPhaseJob* two = (const TwoPhaseJob*)((const unsigned char*)h_plan + HP->off_two);
    const BatchJob* J = (const BatchJob*)((const unsigned char*)h_plan + HP->off_jobs);
    for (uint32_t t = 0; t < HP->n_two; ++t) {
        const uint64_t at = J[two[t].job].out_edge;
        if (launch_pba(two[t].g, w == PG_ID64, (unsigned char*)d_arena + at * 2 * id_bytes,
                       (unsigned char*)d_ws + 256, s) != cudaSuccess)
            return PG_ECUDA;
    }
    return PG_OK;
}

pg_status pg_batch_csr_layout(const void* h_plan, uint32_t n_jobs, uint64_t* h_row_offsets,
                              uint64_t* h_col_offsets, uint64_t* rows_total, uint64_t* cols_total)
{
    if (!h_plan || ((const PlanHeader*)h_plan)->n_jobs != n_jobs) return PG_EINVAL;
    const PlanHeader& H = *(const PlanHeader*)h_plan;
    const BatchJob* J = (const BatchJob*)((const unsigned char*)h_plan + H.off_jobs);
    for (uint32_t i = 0; i < n_jobs; ++i) {
        if (h_row_offsets) h_row_offsets[i] = J[i].want_csr ? J[i].rbase : UINT64_MAX;
        if (h_col_offsets) h_col_offsets[i] = J[i].want_csr ? J[i].csr_edge : UINT64_MAX;
    }
    if (rows_total)
        *rows_total = H.csr_vertices[0] + H.csr_jobs[0] + H.csr_vertices[1] + H.csr_jobs[1];
    if (cols_total) *cols_total = H.csr_edges[0] + H.csr_edges[1];
    return PG_OK;
}

namespace {
// gen_batch_csr's workspace: the union lists of both groups, each group's
// union row pointers, the call's wait word, then one CSR workspace that the
// two groups' CSR calls use in turn.
struct BatchCsrLayout {
    size_t off_rp[2], off_wait, off_csr, total;
};
BatchCsrLayout batch_csr_layout(const PlanHeader& H)
{
    BatchCsrLayout L;
    const size_t pair = H.id64 ? 16 : 8;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t o = up((size_t)(H.csr_edges[0] + H.csr_edges[1]) * pair);
    size_t ws = 0;
    for (int g = 0; g < 2; ++g) {
        L.off_rp[g] = o;
        o += up(((size_t)H.csr_vertices[g] + 1) * 8);
        if (H.csr_jobs[g]) {
            const size_t w = csr_workspace_bytes(H.csr_edges[g], H.csr_vertices[g],
                                                 H.csr_max_vertices[g]);
            ws = w > ws ? w : ws;
        }
    }
    L.off_wait = o;
    o += 256;
    L.off_csr = o;
    L.total = o + ws;
    return L;
}
bool csr_jobs_any(const PlanHeader& H) { return H.csr_jobs[0] + H.csr_jobs[1] > 0; }
}  // namespace

size_t pg_batch_csr_workspace_size(const void* h_plan)
{
    if (!h_plan) return 0;
    const PlanHeader& H = *(const PlanHeader*)h_plan;
    return csr_jobs_any(H) ? batch_csr_layout(H).total : 0;
}

size_t pg_batch_csr_wait_error_offset(const void* h_plan)
{
    if (!h_plan) return SIZE_MAX;
    const PlanHeader& H = *(const PlanHeader*)h_plan;
    return csr_jobs_any(H) ? batch_csr_layout(H).off_wait : SIZE_MAX;
}

pg_status gen_batch_csr(const void* h_plan, const void* d_plan, uint32_t n_jobs, pg_idwidth w,
                        const void* d_arena, uint64_t* d_row_ptr, uint64_t cap_row_ptr,
                        void* d_col, uint64_t cap_col, void* d_ws, size_t ws_bytes, void* stream)
{
    if (!d_plan || n_jobs == 0 || n_jobs > kMaxBatchJobs) return PG_EINVAL;
    if (w != PG_ID32 && w != PG_ID64) return PG_EINVAL;
    const PlanHeader* HP = plan_header(h_plan, n_jobs, w);
    if (!HP) return PG_EINVAL;
    const PlanHeader& H = *HP;
    if (!csr_jobs_any(H)) return PG_OK;
    uint64_t rows = 0, cols = 0;
    pg_batch_csr_layout(h_plan, n_jobs, nullptr, nullptr, &rows, &cols);
    if (cap_row_ptr < rows || cap_col < cols) return PG_ENOSPC;
    if (!d_row_ptr || ((uintptr_t)d_row_ptr & 7)) return PG_EINVAL;
    if (cols > 0 && (!d_arena || !d_col || ((uintptr_t)d_arena & 15))) return PG_EINVAL;
    const BatchCsrLayout L = batch_csr_layout(H);
    if (!d_ws || ws_bytes < L.total || ((uintptr_t)d_ws & 255)) return PG_ENOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* ws = (unsigned char*)d_ws;
    const size_t pair = H.id64 ? 16 : 8, id_bytes = pair / 2;
    uint32_t* wait = (uint32_t*)(ws + L.off_wait);
    if (cudaMemsetAsync(wait, 0, 4, s) != cudaSuccess) return PG_ECUDA;
    if (cols > 0) {
        TraceScope trace("batch_csr_union", s);
        const uint64_t warps = (H.total_edges + 31) / 32;
        const uint64_t full = (uint64_t)device_sm_count() * 8;
        const int grid = (int)(warps / 8 + 1 < full ? warps / 8 + 1 : full);
        if (w == PG_ID64)
            { batch_union_kernel<uint64_t><<<grid, 256, 0, s>>>(
                (const unsigned char*)d_plan, (const uint64_t*)d_arena, (uint64_t*)ws); note_launch(); }
        else
            { batch_union_kernel<uint32_t><<<grid, 256, 0, s>>>(
                (const unsigned char*)d_plan, (const uint32_t*)d_arena, (uint32_t*)ws); note_launch(); }
        if (cudaGetLastError() != cudaSuccess) return PG_ECUDA;
    }
    const uint64_t col_base[2] = {0, H.csr_edges[0]};
    for (int g = 0; g < 2; ++g) {
        if (!H.csr_jobs[g]) continue;
        const uint64_t E = H.csr_edges[g], V = H.csr_vertices[g], nd = H.csr_max_vertices[g];
        uint64_t* rp_u = (uint64_t*)(ws + L.off_rp[g]);
        if (launch_csr(ws + col_base[g] * pair, E, V, (int)H.id64, rp_u,
                       (unsigned char*)d_col + col_base[g] * id_bytes, ws + L.off_csr,
                       L.total - L.off_csr, s, nd) != cudaSuccess)
            return PG_ECUDA;
        if (E > 0 && V >= 2)   // the group's sort had a wait word: fold it into the call's
            { or_word_kernel<<<1, 1, 0, s>>>(
                wait, (const uint32_t*)(ws + L.off_csr + csr_wait_error_offset(E, V, 0, (int)H.id64,
                                                                               nd))); note_launch(); }
        TraceScope trace("batch_csr_rebase", s);
        const uint64_t R = V + H.csr_jobs[g];
        const uint64_t full = (uint64_t)device_sm_count() * 8;
        const int grid = (int)(R / 256 + 1 < full ? R / 256 + 1 : full);
        { batch_rebase_kernel<<<grid, 256, 0, s>>>(
            (const uint64_t*)((const unsigned char*)d_plan + H.off_rstart[g]), H.csr_jobs[g], V,
            rp_u, d_row_ptr); note_launch(); }
        if (cudaGetLastError() != cudaSuccess) return PG_ECUDA;
    }
    return PG_OK;
}

}  // extern "C"

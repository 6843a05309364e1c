// Kronecker graph kernels (arXiv 1003.3684, Sec. 3, PK method).
//
// Stochastic mode: every edge is independent -- one thread derives an edge
// from its index alone by a k-level descent through the initiator (the
// stochastic Kronecker model of Leskovec et al. that Sec. 2 cites), most
// significant level first. Level l consumes word (l mod 4) of the Philox
// block for counter (e_lo, e_hi, l div 4, 3), so ceil(k/4) Philox calls
// give all k levels. A level picks cell c when T_{c-1} <= w < T_c with
// 32-bit fixed-point thresholds T prepared on the host.
//
// Deterministic mode: the stack expansion of Sec. 3 visits meta-edges
// depth first with children in seed order, so the e-th emitted edge is the
// one whose base-e0 digits (most significant first) name the seed edge taken
// at each expansion. Each thread decodes its own edge index, several digits
// per lookup in a shared-memory table of digit groups; the order is the
// stack's without running a stack.
//
// The stochastic kernels are integer-ALU bound (Philox and the descent); the
// deterministic one is bound by its output. Both write their output once, as
// coalesced 16-byte vector stores of two edges.
#include <type_traits>

#include "pg_internal.h"
#include "pg_trace.h"

namespace pgen {
namespace {

template <typename Id>
struct Pair2;
template <>
struct Pair2<uint32_t> {
    __device__ static void store(uint32_t* out, uint64_t e, uint64_t r0, uint64_t c0,
                                 uint64_t r1, uint64_t c1)
    {
        *reinterpret_cast<uint4*>(out + 2 * e) =
            make_uint4((uint32_t)r0, (uint32_t)c0, (uint32_t)r1, (uint32_t)c1);
    }
    __device__ static void store1(uint32_t* out, uint64_t e, uint64_t r0, uint64_t c0)
    {
        *reinterpret_cast<uint2*>(out + 2 * e) = make_uint2((uint32_t)r0, (uint32_t)c0);
    }
};
template <>
struct Pair2<uint64_t> {
    __device__ static void store(uint64_t* out, uint64_t e, uint64_t r0, uint64_t c0,
                                 uint64_t r1, uint64_t c1)
    {
        ulonglong2* o = reinterpret_cast<ulonglong2*>(out + 2 * e);
        o[0] = make_ulonglong2(r0, c0);
        o[1] = make_ulonglong2(r1, c1);
    }
    __device__ static void store1(uint64_t* out, uint64_t e, uint64_t r0, uint64_t c0)
    {
        *reinterpret_cast<ulonglong2*>(out + 2 * e) = make_ulonglong2(r0, c0);
    }
};

// ---- stochastic descent, initiator order 2 (branch-free 3-threshold pick) --
// T is uint32_t when k <= 32 (ids fit 32 bits), else uint64_t.
template <typename T>
__device__ __forceinline__ void descend2(uint32_t w, uint32_t u0, uint32_t u1, uint32_t u2,
                                         uint32_t base, T& row, T& col)
{
    const uint32_t cell = base + (w > u0) + (w > u1) + (w > u2);
    row = (row << 1) | (T)(cell >> 1);
    col = (col << 1) | (T)(cell & 1);
}

// The same pick when cell 0 has positive weight and all three thresholds
// are real (n_zero = 0, n_u = 3): with u0 <= u1 <= u2 the row bit of the
// cell is a = (w > u1), and its column bit is (w > u2) when a is set (cells
// 2, 3), else (w > u0) (cells 0, 1): two compares instead of three and a
// parity. row = 2*row + a runs on the multiply-add pipe, not the ALU pipe.
template <typename T>
__device__ __forceinline__ void descend2_full(uint32_t w, uint32_t u0, uint32_t u1, uint32_t u2,
                                              T& row, T& col)
{
    const uint32_t a = w > u1 ? 1u : 0u;
    const uint32_t b = w > (a ? u2 : u0) ? 1u : 0u;
    row = row * 2 + (T)a;
    col = col * 2 + (T)b;
}

template <typename T>
__device__ __forceinline__ void kron2_edge_full(const KronParams& p, uint64_t e, uint32_t u0,
                                                uint32_t u1, uint32_t u2, T& row, T& col)
{
    row = 0;
    col = 0;
    const uint32_t k = p.k;
    uint32_t l = 0;
    for (uint32_t g = 0; l + 4 <= k; ++g, l += 4) {
        const uint4 w = draw(e, g, 3, p.key);
        descend2_full(w.x, u0, u1, u2, row, col);
        descend2_full(w.y, u0, u1, u2, row, col);
        descend2_full(w.z, u0, u1, u2, row, col);
        descend2_full(w.w, u0, u1, u2, row, col);
    }
    if (l < k) {
        const uint4 w = draw(e, l >> 2, 3, p.key);
        descend2_full(w.x, u0, u1, u2, row, col);
        if (l + 1 < k) descend2_full(w.y, u0, u1, u2, row, col);
        if (l + 2 < k) descend2_full(w.z, u0, u1, u2, row, col);
    }
}

template <typename T>
__device__ __forceinline__ void kron2_edge(const KronParams& p, uint64_t e, uint32_t u0,
                                           uint32_t u1, uint32_t u2, T& row, T& col)
{
    row = 0;
    col = 0;
    const uint32_t k = p.k;
    uint32_t l = 0;
    for (uint32_t g = 0; l + 4 <= k; ++g, l += 4) {
        const uint4 w = draw(e, g, 3, p.key);
        descend2(w.x, u0, u1, u2, p.n_zero, row, col);
        descend2(w.y, u0, u1, u2, p.n_zero, row, col);
        descend2(w.z, u0, u1, u2, p.n_zero, row, col);
        descend2(w.w, u0, u1, u2, p.n_zero, row, col);
    }
    if (l < k) {
        const uint4 w = draw(e, l >> 2, 3, p.key);
        descend2(w.x, u0, u1, u2, p.n_zero, row, col);
        if (l + 1 < k) descend2(w.y, u0, u1, u2, p.n_zero, row, col);
        if (l + 2 < k) descend2(w.z, u0, u1, u2, p.n_zero, row, col);
    }
}

template <typename Id, typename T, bool kFull>
__global__ void __launch_bounds__(256) kron2_kernel(const __grid_constant__ KronParams p,
                                                    Id* __restrict__ out, uint64_t e_begin,
                                                    uint64_t n_edges)
{
    const uint32_t u0 = p.u[0], u1 = p.u[1], u2 = p.u[2];   // padded to three
    const uint64_t n_pairs = (n_edges + 1) >> 1;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    auto edge = [&](uint64_t ee, T& r, T& c) {
        if constexpr (kFull) kron2_edge_full(p, ee, u0, u1, u2, r, c);
        else kron2_edge(p, ee, u0, u1, u2, r, c);
    };
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_pairs; t += stride) {
        const uint64_t e = 2 * t;
        T r0, c0;
        edge(e_begin + e, r0, c0);
        if (e + 1 < n_edges) {
            T r1, c1;
            edge(e_begin + e + 1, r1, c1);
            if (PG_CHECK_OUT(e + 1, n_edges)) Pair2<Id>::store(out, e, r0, c0, r1, c1);
        } else {
            if (PG_CHECK_OUT(e, n_edges)) Pair2<Id>::store1(out, e, r0, c0);
        }
    }
}

// The same descent with 32-bit edge indices, counters (e, 0, g, 3), ids and
// loop arithmetic, for launches whose edge indices all lie below 2^32 and
// whose ids fit 32 bits (k <= 32): the same values, less index arithmetic.
template <bool kFull>
__device__ __forceinline__ void kron2_edge32(const KronParams& p, uint32_t e, uint32_t u0,
                                             uint32_t u1, uint32_t u2, uint32_t& row,
                                             uint32_t& col)
{
    row = 0;
    col = 0;
    const uint32_t k = p.k;
    auto level = [&](uint32_t w) {
        if constexpr (kFull) descend2_full(w, u0, u1, u2, row, col);
        else descend2(w, u0, u1, u2, p.n_zero, row, col);
    };
    uint32_t l = 0;
    for (uint32_t g = 0; l + 4 <= k; ++g, l += 4) {
        const uint4 w = philox(make_uint4(e, 0u, g, 3u), p.key);
        level(w.x);
        level(w.y);
        level(w.z);
        level(w.w);
    }
    if (l < k) {
        const uint4 w = philox(make_uint4(e, 0u, l >> 2, 3u), p.key);
        level(w.x);
        if (l + 1 < k) level(w.y);
        if (l + 2 < k) level(w.z);
    }
}

template <typename Id, bool kFull>
__global__ void __launch_bounds__(256) kron2_kernel32(const __grid_constant__ KronParams p,
                                                      Id* __restrict__ out, uint32_t e_begin,
                                                      uint32_t n_edges)
{
    const uint32_t u0 = p.u[0], u1 = p.u[1], u2 = p.u[2];   // padded to three
    const uint32_t n_pairs = (n_edges >> 1) + (n_edges & 1);
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n_pairs; t += stride) {
        const uint32_t e = 2 * t;
        uint32_t r0, c0;
        kron2_edge32<kFull>(p, e_begin + e, u0, u1, u2, r0, c0);
        if (e + 1 < n_edges) {
            uint32_t r1, c1;
            kron2_edge32<kFull>(p, e_begin + e + 1, u0, u1, u2, r1, c1);
            if (PG_CHECK_OUT(e + 1, n_edges)) Pair2<Id>::store(out, e, r0, c0, r1, c1);
        } else {
            if (PG_CHECK_OUT(e, n_edges)) Pair2<Id>::store1(out, e, r0, c0);
        }
    }
}

// ---- stochastic descent, any order n0 <= 16 (binary search in smem) -------
__device__ __forceinline__ void kron_edge_generic(const KronParams& p, const uint32_t* u,
                                                  uint32_t n_u, uint64_t e, uint64_t& row,
                                                  uint64_t& col)
{
    row = 0;
    col = 0;
    uint4 w = make_uint4(0, 0, 0, 0);
    for (uint32_t l = 0; l < p.k; ++l) {
        if ((l & 3) == 0) w = draw(e, l >> 2, 3, p.key);
        const uint32_t x = (l & 3) == 0 ? w.x : (l & 3) == 1 ? w.y : (l & 3) == 2 ? w.z : w.w;
        // count of u[t] < x (u ascending): first index with u[t] >= x
        uint32_t lo = 0, hi = n_u;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (u[mid] < x) lo = mid + 1;
            else hi = mid;
        }
        const uint32_t cell = p.n_zero + lo;
        row = row * p.n0 + cell / p.n0;
        col = col * p.n0 + cell % p.n0;
    }
}

template <typename Id>
__global__ void __launch_bounds__(256) kron_generic_kernel(const __grid_constant__ KronParams p,
                                                           Id* __restrict__ out, uint64_t e_begin,
                                                           uint64_t n_edges)
{
    __shared__ uint32_t u[kMaxKronThr];
    const uint32_t n_u = p.n_u;
    for (uint32_t t = threadIdx.x; t < n_u; t += blockDim.x) u[t] = p.u[t];
    __syncthreads();
    const uint64_t n_pairs = (n_edges + 1) >> 1;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_pairs; t += stride) {
        const uint64_t e = 2 * t;
        uint64_t r0, c0;
        kron_edge_generic(p, u, n_u, e_begin + e, r0, c0);
        if (e + 1 < n_edges) {
            uint64_t r1, c1;
            kron_edge_generic(p, u, n_u, e_begin + e + 1, r1, c1);
            if (PG_CHECK_OUT(e + 1, n_edges)) Pair2<Id>::store(out, e, r0, c0, r1, c1);
        } else {
            if (PG_CHECK_OUT(e, n_edges)) Pair2<Id>::store1(out, e, r0, c0);
        }
    }
}

// ---- deterministic expansion: base-e0 digits of the edge index ------------
// Edge e's digits d_0 (most significant) ... d_{k-1} select seed edges
// (a_d, b_d); row = sum a_{d_l} n0^(k-1-l), col likewise. Taken from the
// least significant end, g digits at a time: tab[c] holds the row and column
// parts (16 bits each) of the group of g digits whose base-e0 value is c, so
// a group costs one division by e0^g and one lookup; the n_rest most
// significant digits, if any, go one at a time through the seed table.
// Digits and groups are clamped to their tables, so a lookup stays inside
// them whatever the arithmetic gives.
template <typename T, typename Div>
__device__ __forceinline__ T div_by(T x, const Div& f);
template <>
__device__ __forceinline__ uint32_t div_by(uint32_t x, const FastDiv32& f)
{
    return fdiv32(x, f);
}
template <>
__device__ __forceinline__ uint64_t div_by(uint64_t x, const FastDiv& f)
{
    return fdiv(x, f);
}

template <typename T>
__device__ __forceinline__ void kron_det_edge(const KronDetParams& p, const uint32_t* tab,
                                              const uint16_t* ab, T e, T& row, T& col)
{
    row = 0;
    col = 0;
    T mul = 1;
    for (uint32_t i = 0; i < p.n_groups; ++i) {
        T q;
        if constexpr (sizeof(T) == 4) q = div_by(e, p.div_E32);
        else q = div_by(e, p.div_E);
        const T c = e - q * p.E;
        e = q;
        const uint32_t v = tab[(PG_CHECK(c, p.E) && c < p.E) ? (uint32_t)c : p.E - 1];
        row += (T)(v & 0xFFFFu) * mul;
        col += (T)(v >> 16) * mul;
        mul *= (T)p.n0g;
    }
    for (uint32_t l = 0; l < p.n_rest; ++l) {
        T q;
        if constexpr (sizeof(T) == 4) q = div_by(e, p.div_e0_32);
        else q = div_by(e, p.div_e0);
        const T r = e - q * p.e0;
        e = q;
        const uint32_t v = ab[(PG_CHECK(r, p.e0) && r < p.e0) ? (uint32_t)r : p.e0 - 1];
        row += (T)(v & 0xFFu) * mul;
        col += (T)(v >> 8) * mul;
        mul *= p.n0;
    }
}

// The contribution of every digit above the lowest group, given q = e div
// e0^g: the remaining groups, then the single digits, at weights from n0^g.
template <typename T>
__device__ __forceinline__ void kron_det_upper(const KronDetParams& p, const uint32_t* tab,
                                               const uint16_t* ab, T e, T& row, T& col)
{
    row = 0;
    col = 0;
    T mul = (T)p.n0g;
    for (uint32_t i = 1; i < p.n_groups; ++i) {
        T q;
        if constexpr (sizeof(T) == 4) q = div_by(e, p.div_E32);
        else q = div_by(e, p.div_E);
        const T c = e - q * p.E;
        e = q;
        const uint32_t v = tab[(PG_CHECK(c, p.E) && c < p.E) ? (uint32_t)c : p.E - 1];
        row += (T)(v & 0xFFFFu) * mul;
        col += (T)(v >> 16) * mul;
        mul *= (T)p.n0g;
    }
    for (uint32_t l = 0; l < p.n_rest; ++l) {
        T q;
        if constexpr (sizeof(T) == 4) q = div_by(e, p.div_e0_32);
        else q = div_by(e, p.div_e0);
        const T r = e - q * p.e0;
        e = q;
        const uint32_t v = ab[(PG_CHECK(r, p.e0) && r < p.e0) ? (uint32_t)r : p.e0 - 1];
        row += (T)(v & 0xFFu) * mul;
        col += (T)(v >> 8) * mul;
        mul *= p.n0;
    }
}

// One CTA of kDetThreads threads per table copy: the table is built once per
// CTA, and two CTAs (2 x 64 KB at most) fill an SM's warp slots.
constexpr int kDetThreads = 1024;

// Dynamic shared memory: the group table (E words), then the seed table.
size_t kron_det_smem(const KronDetParams& p)
{
    return (size_t)p.E * 4 + ((size_t)p.e0 * 2 + 15) / 16 * 16;
}

// kNarrow: every edge index of the launch and every id below 2^32, so the
// digits, ids and weights are 32-bit.
template <typename Id, bool kNarrow>
__global__ void __launch_bounds__(kDetThreads) kron_det_kernel(const __grid_constant__ KronDetParams p,
                                                       Id* __restrict__ out, uint64_t e_begin,
                                                       uint64_t n_edges)
{
    using T = typename std::conditional<kNarrow, uint32_t, uint64_t>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* tab = reinterpret_cast<uint32_t*>(smem);
    uint16_t* ab = reinterpret_cast<uint16_t*>(smem + (size_t)p.E * 4);
    for (uint32_t t = threadIdx.x; t < p.e0; t += blockDim.x) ab[t] = p.ab[t];
    __syncthreads();
    // the table of digit groups, least significant digit first
    for (uint32_t c = threadIdx.x; c < p.E; c += blockDim.x) {
        uint32_t x = c, rr = 0, cc = 0, mul = 1;
        for (uint32_t j = 0; j < p.g; ++j) {
            const uint32_t q = fdiv32(x, p.div_e0_32);
            const uint32_t d = x - q * p.e0;
            x = q;
            const uint32_t v = ab[(PG_CHECK(d, p.e0) && d < p.e0) ? d : p.e0 - 1];
            rr += (v & 0xFFu) * mul;
            cc += (v >> 8) * mul;
            mul *= p.n0;
        }
        tab[c] = rr | (cc << 16);
    }
    __syncthreads();
    // each warp owns a contiguous range of pairs, lane l taking pairs l,
    // l + 32, ... of it, so a lane's edge index grows by 64 per step: its
    // lowest digit group advances by 64 and the part above it is decoded
    // again only when that group wraps
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t n_pairs = (n_edges + 1) >> 1;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t per_warp = ((n_pairs + warps - 1) / warps + 31) / 32 * 32;
    const uint64_t p_end0 = (gw + 1) * per_warp;
    const uint64_t p_end = p_end0 < n_pairs ? p_end0 : n_pairs;
    uint64_t pi = gw * per_warp + lane;
    if (pi >= p_end) return;
    T q, lo, ur, uc;
    {
        const T ea = (T)(e_begin + 2 * pi);
        if constexpr (sizeof(T) == 4) q = div_by(ea, p.div_E32);
        else q = div_by(ea, p.div_E);
        lo = ea - q * p.E;
        if (!(PG_CHECK(lo, p.E) && lo < p.E)) lo = p.E - 1;
        kron_det_upper<T>(p, tab, ab, q, ur, uc);
    }
    for (; pi < p_end; pi += 32) {
        const uint64_t e = 2 * pi;
        const bool two = e + 1 < n_edges;
        const uint32_t l0 = (uint32_t)lo;
        const uint32_t v0 = tab[l0];
        const T r0 = (T)(v0 & 0xFFFFu) + ur, c0 = (T)(v0 >> 16) + uc;
        T r1 = 0, c1 = 0;
        if (two) {
            if (l0 + 1 < p.E) {
                const uint32_t v1 = tab[l0 + 1];
                r1 = (T)(v1 & 0xFFFFu) + ur;
                c1 = (T)(v1 >> 16) + uc;
            } else {
                kron_det_edge<T>(p, tab, ab, (T)(e_begin + e + 1), r1, c1);
            }
            if (PG_CHECK_OUT(e + 1, n_edges)) Pair2<Id>::store(out, e, r0, c0, r1, c1);
        } else {
            if (PG_CHECK_OUT(e, n_edges)) Pair2<Id>::store1(out, e, r0, c0);
        }
        lo += 64;
        if (lo >= p.E) {
            // the group wrapped (several times when e0^g < 64)
            do {
                lo -= p.E;
                ++q;
            } while (lo >= p.E);
            kron_det_upper<T>(p, tab, ab, q, ur, uc);
        }
    }
}

// ---- random graph G(N, M) with replacement (the exclusive-or randomisation
// of Sec. 3's PK method): edge e is the cell (uniform over N from (w1:w0),
// uniform over N from (w3:w2)) of the draw with counter (e_lo, e_hi, 0, 4).
template <typename Id>
__global__ void __launch_bounds__(256) random_cells_kernel(const Key key, uint64_t N,
                                                           Id* __restrict__ out, uint64_t e_begin,
                                                           uint64_t n_edges)
{
    const uint64_t n_pairs = (n_edges + 1) >> 1;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_pairs; t += stride) {
        const uint64_t e = 2 * t;
        const uint4 a = draw(e_begin + e, 0, 4, key);
        if (e + 1 < n_edges) {
            const uint4 b = draw(e_begin + e + 1, 0, 4, key);
            if (PG_CHECK_OUT(e + 1, n_edges))
                Pair2<Id>::store(out, e, uniform64(a.x, a.y, N), uniform64(a.z, a.w, N),
                                 uniform64(b.x, b.y, N), uniform64(b.z, b.w, N));
        } else {
            if (PG_CHECK_OUT(e, n_edges))
                Pair2<Id>::store1(out, e, uniform64(a.x, a.y, N), uniform64(a.z, a.w, N));
        }
    }
}

template <typename K>
int grid_for(K kernel, uint64_t work_items, int threads, size_t smem = 0)
{
    const int sms = device_sm_count();   // of the current device
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const uint64_t full = (uint64_t)sms * per_sm;
    const uint64_t need = (work_items + threads - 1) / threads;
    return (int)(need < full ? (need > 0 ? need : 1) : full);
}

}  // namespace

PG_CHECK_UNIT(kron)

cudaError_t launch_kron_stochastic(const KronParams& p, int id64, void* d_out, uint64_t e_begin,
                                   uint64_t n_edges, cudaStream_t s)
{
    if (n_edges == 0) return cudaSuccess;
    const uint64_t pairs = (n_edges + 1) / 2;
    TraceScope trace(p.n0 == 2 ? "kron_descent_n0_2" : "kron_descent", s);
    if (p.n0 == 2) {
        // 32-bit descent state when every id fits (k <= 32)
        const bool full = p.n_zero == 0 && p.n_u == 3;
        if (p.k <= 32 && e_begin + n_edges < ((uint64_t)1 << 32)) {
            // every edge index below 2^32: 32-bit indices and counters
            const uint32_t b = (uint32_t)e_begin, n = (uint32_t)n_edges;
            if (id64) {
                auto k = full ? kron2_kernel32<uint64_t, true> : kron2_kernel32<uint64_t, false>;
                { k<<<grid_for(k, pairs, 256), 256, 0, s>>>(p, (uint64_t*)d_out, b, n); note_launch(); }
            } else {
                auto k = full ? kron2_kernel32<uint32_t, true> : kron2_kernel32<uint32_t, false>;
                { k<<<grid_for(k, pairs, 256), 256, 0, s>>>(p, (uint32_t*)d_out, b, n); note_launch(); }
            }
        } else if (id64 && p.k > 32) {
            auto k = full ? kron2_kernel<uint64_t, uint64_t, true> : kron2_kernel<uint64_t, uint64_t, false>;
            { k<<<grid_for(k, pairs, 256), 256, 0, s>>>(p, (uint64_t*)d_out, e_begin, n_edges); note_launch(); }
        } else if (id64) {
            auto k = full ? kron2_kernel<uint64_t, uint32_t, true> : kron2_kernel<uint64_t, uint32_t, false>;
            { k<<<grid_for(k, pairs, 256), 256, 0, s>>>(p, (uint64_t*)d_out, e_begin, n_edges); note_launch(); }
        } else {
            auto k = full ? kron2_kernel<uint32_t, uint32_t, true> : kron2_kernel<uint32_t, uint32_t, false>;
            { k<<<grid_for(k, pairs, 256), 256, 0, s>>>(p, (uint32_t*)d_out, e_begin, n_edges); note_launch(); }
        }
    } else {
        if (id64) {
            auto k = kron_generic_kernel<uint64_t>;
            { k<<<grid_for(k, pairs, 256), 256, 0, s>>>(p, (uint64_t*)d_out, e_begin, n_edges); note_launch(); }
        } else {
            auto k = kron_generic_kernel<uint32_t>;
            { k<<<grid_for(k, pairs, 256), 256, 0, s>>>(p, (uint32_t*)d_out, e_begin, n_edges); note_launch(); }
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_kron_det(const KronDetParams& p, int id64, void* d_out, uint64_t e_begin,
                            uint64_t n_edges, cudaStream_t s)
{
    if (n_edges == 0) return cudaSuccess;
    const uint64_t pairs = (n_edges + 1) / 2;
    // 32-bit digits when every edge index of the launch and every id is below 2^32
    uint64_t n_vertices = 1;
    for (uint32_t l = 0; l < p.k && n_vertices <= ((uint64_t)1 << 32); ++l) n_vertices *= p.n0;
    const bool narrow = e_begin + n_edges <= ((uint64_t)1 << 32) &&
                        n_vertices <= ((uint64_t)1 << 32);
    const size_t smem = kron_det_smem(p);
    // the opt-in shared-memory size of every variant, set once per device
    static PerDeviceOnce attrs;
    const cudaError_t ae = attrs.run_current([] {
        const int most = (int)(kDetGroupTable * 4 + kMaxDetSeedEdges * 2);
        return first_error({
            cudaFuncSetAttribute(kron_det_kernel<uint64_t, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, most),
            cudaFuncSetAttribute(kron_det_kernel<uint64_t, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, most),
            cudaFuncSetAttribute(kron_det_kernel<uint32_t, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, most),
            cudaFuncSetAttribute(kron_det_kernel<uint32_t, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, most)});
    });
    if (ae != cudaSuccess) return ae;
    TraceScope trace("kron_det", s);
    if (id64) {
        auto k = narrow ? kron_det_kernel<uint64_t, true> : kron_det_kernel<uint64_t, false>;
        { k<<<grid_for(k, pairs, kDetThreads, smem), kDetThreads, smem, s>>>(p, (uint64_t*)d_out, e_begin, n_edges); note_launch(); }
    } else {
        auto k = narrow ? kron_det_kernel<uint32_t, true> : kron_det_kernel<uint32_t, false>;
        { k<<<grid_for(k, pairs, kDetThreads, smem), kDetThreads, smem, s>>>(p, (uint32_t*)d_out, e_begin, n_edges); note_launch(); }
    }
    return cudaGetLastError();
}

cudaError_t launch_random_cells(const Key& key, uint64_t n_vertices, int id64, void* d_out,
                                uint64_t e_begin, uint64_t n_edges, cudaStream_t s)
{
    if (n_edges == 0) return cudaSuccess;
    const uint64_t pairs = (n_edges + 1) / 2;
    TraceScope trace("random_cells", s);
    if (id64) {
        auto k = random_cells_kernel<uint64_t>;
        { k<<<grid_for(k, pairs, 256), 256, 0, s>>>(key, n_vertices, (uint64_t*)d_out, e_begin, n_edges); note_launch(); }
    } else {
        auto k = random_cells_kernel<uint32_t>;
        { k<<<grid_for(k, pairs, 256), 256, 0, s>>>(key, n_vertices, (uint32_t*)d_out, e_begin, n_edges); note_launch(); }
    }
    return cudaGetLastError();
}

}  // namespace pgen

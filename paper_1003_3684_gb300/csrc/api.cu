// C ABI of libpgen (declared in include/pgen.h): argument validation, host
// set-up (thresholds, divisors, geometry) and dispatch to the kernels.
// Every check happens before the first launch, so an invalid call leaves the
// device untouched.
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>
#include <mutex>

#include "../../include/pgen.h"
#include "pg_internal.h"

namespace pgen {

int device_sm_count()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return sms > 0 ? sms : 1;
}

}  // namespace pgen

using namespace pgen;

namespace {

typedef unsigned __int128 u128;

bool aligned(const void* p, size_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

pg_status from_cuda(cudaError_t e) { return e == cudaSuccess ? PG_OK : PG_ECUDA; }

uint64_t seed_edges(uint32_t n0) { return (uint64_t)n0 * (n0 - 1) / 2; }

// Inter-faction coin threshold min(2^32 - 1, round_half_even(f * 2^32)).
uint32_t coin_threshold(double f)
{
    const double t = std::nearbyint(std::ldexp(f, 32));
    if (!(t > 0.0)) return 0;
    if (t >= 4294967295.0) return 0xFFFFFFFFu;
    return (uint32_t)t;
}

struct PbaCheck {
    pg_status st;
    uint64_t n_b, N_e, edges;
};

PbaCheck check_pba(uint64_t n, uint32_t m, uint32_t B, uint32_t n0, uint32_t W, double f,
                   pg_idwidth w)
{
    PbaCheck c{PG_EINVAL, 0, 0, 0};
    if (m < 1 || n0 < 2 || n0 > 65536 || B < 1 || B > 1024 || W < 1 || B % W != 0) return c;
    if (n % B != 0) return c;
    if (!(f >= 0.0 && f <= 1.0)) return c;
    if (w != PG_ID32 && w != PG_ID64) return c;
    const uint64_t n_b = n / B;
    const u128 N_e = (u128)n_b * m;
    const u128 e0 = seed_edges(n0);
    const u128 edges = (u128)B * (e0 + N_e);
    if (edges >> 62) return c;
    const u128 ids = (u128)B * (n0 + (u128)n_b);
    if (w == PG_ID32 && ids > ((u128)1 << 32)) return c;
    if ((u128)n0 + n_b >= ((u128)1 << 32)) return c;       // local ids are 32-bit
    if (N_e >= ((u128)1 << 32)) return c;                  // entries per block are 32-bit
    // phase-2 index arithmetic: (total entries) * n_b must stay below 2^63
    if ((u128)B * N_e * (n_b ? n_b : 1) >= ((u128)1 << 63)) return c;
    c.st = PG_OK;
    c.n_b = n_b;
    c.N_e = (uint64_t)N_e;
    c.edges = (uint64_t)edges;
    return c;
}

PbaGeom make_geom(uint64_t n_b, uint64_t N_e, uint32_t m, uint32_t B, uint32_t n0, uint32_t W,
                  double f, uint64_t seed)
{
    PbaGeom g;
    std::memset(&g, 0, sizeof(g));
    g.n_b = n_b;
    g.N_e = N_e;
    g.e0 = seed_edges(n0);
    g.span = n0 + n_b;
    g.A_stride = (N_e + 7) & ~(uint64_t)7;
    g.m = m;
    g.B = B;
    g.W = W;
    g.n0 = n0;
    g.coin_thr = coin_threshold(f);
    g.coin_on = (B > W && g.coin_thr > 0) ? 1 : 0;
    g.key = make_key(seed);
    g.S = pba_segments(N_e, B, device_sm_count());
    g.seg_len = pba_segment_length(N_e, g.S);
    g.P = pba_prefix_len(N_e);
    g.nb_shift = 0xFFFFFFFFu;
    if (n_b > 0 && (n_b & (n_b - 1)) == 0) {
        g.nb_shift = 0;
        while (((uint64_t)1 << g.nb_shift) < n_b) ++g.nb_shift;
        g.lean_add = (n_b - 1) + (g.e0 << g.nb_shift);
    }
    g.div_m = make_fastdiv(m);
    g.div_m32 = make_fastdiv32(m);
    g.div_nb = make_fastdiv(n_b > 0 ? n_b : 1);
    return g;
}

// Kronecker thresholds T_c, c < n0^2 - 1 (left-to-right double sums).
bool kron_thresholds(const double* P, uint32_t n0, uint64_t* T)
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

// n0^k as a 128-bit value (saturating at 2^127).
u128 ipow(uint64_t b, uint32_t k)
{
    u128 r = 1;
    for (uint32_t i = 0; i < k; ++i) {
        if (r > ((u128)1 << 100)) return (u128)1 << 127;
        r *= b;
    }
    return r;
}

}  // namespace

extern "C" {

const char* pg_status_string(pg_status s)
{
    switch (s) {
    case PG_OK: return "ok";
    case PG_EINVAL: return "invalid argument";
    case PG_ENOSPC: return "output capacity too small";
    case PG_ECUDA: return "CUDA error";
    case PG_ETIMEOUT: return "device wait timed out";
    case PG_ENOMEM: return "workspace too small";
    }
    return "unknown status";
}

int pg_device_sm_count(void) { return device_sm_count(); }

const char* pg_version(void) { return "pgen 0.1 (sm_103a)"; }

void pg_force_wide_path(int on) { set_wide_path_forced(on != 0); }

int pg_test_per_device_once(const int* devs, int n, int threads, int fail_dev, int* calls,
                            int* status)
{
    if (!devs || !calls || !status || n < 0 || threads < 1 || threads > 64) return PG_EINVAL;
    PerDeviceOnce once;
    std::atomic<int> count[kMaxDevices];
    for (int d = 0; d < kMaxDevices; ++d) count[d].store(0);
    // every thread runs the whole sequence on the one shared instance
    auto body = [&](int t) {
        for (int i = 0; i < n; ++i) {
            const int dev = devs[i];
            const cudaError_t e = once.run(dev, [&] {
                count[dev].fetch_add(1);
                return dev == fail_dev ? cudaErrorInvalidValue : cudaSuccess;
            });
            if (t == 0) status[i] = (int)e;
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t) pool.emplace_back(body, t);
    body(0);
    for (auto& th : pool) th.join();
    for (int d = 0; d < kMaxDevices; ++d) calls[d] = count[d].load();
    return PG_OK;
}

uint64_t pg_pba_edge_count(uint64_t n, uint32_t m, uint32_t blocks, uint32_t n0)
{
    const PbaCheck c = check_pba(n, m, blocks, n0, blocks ? blocks : 1, 0.0, PG_ID64);
    return c.st == PG_OK ? c.edges : 0;
}

size_t pg_pba_workspace_size(uint64_t n, uint32_t m, uint32_t blocks)
{
    if (blocks <= 1) return 0;
    const PbaCheck c = check_pba(n, m, blocks, 2, blocks, 0.0, PG_ID64);
    if (c.st != PG_OK) return 0;
    const uint32_t S = pba_segments(c.N_e, blocks, device_sm_count());
    return pba_workspace_layout((c.N_e + 7) & ~(uint64_t)7, blocks, S).total;
}

pg_status gen_pba(uint64_t n, uint32_t m, uint32_t blocks, uint32_t n0, uint32_t faction_width,
                  double inter_frac, uint64_t seed, pg_idwidth w, void* d_edges,
                  uint64_t cap_edges, uint64_t* n_edges_out, void* d_ws, size_t ws_bytes,
                  void* stream)
{
    const PbaCheck c = check_pba(n, m, blocks, n0, faction_width, inter_frac, w);
    if (c.st != PG_OK) return c.st;
    if (n_edges_out) *n_edges_out = c.edges;
    if (cap_edges < c.edges) return PG_ENOSPC;
    if (c.edges > 0 && (!d_edges || !aligned(d_edges, 16))) return PG_EINVAL;
    const PbaGeom g = make_geom(c.n_b, c.N_e, m, blocks, n0, faction_width, inter_frac, seed);
    cudaStream_t s = (cudaStream_t)stream;
    if (blocks == 1) return from_cuda(launch_ba(g, w == PG_ID64, d_edges, s));
    const size_t need = pba_workspace_layout(g.A_stride, blocks, g.S).total;
    if (!d_ws || ws_bytes < need) return PG_ENOMEM;
    if (!aligned(d_ws, 256)) return PG_EINVAL;
    return from_cuda(launch_pba(g, w == PG_ID64, d_edges, d_ws, s));
}

size_t pg_pba_faction_table_size(uint32_t blocks)
{
    if (blocks < 1 || blocks > 1024) return 0;
    return (size_t)blocks * kFacStride * sizeof(uint16_t);
}

pg_status pg_pba_faction_table(uint32_t blocks, const uint32_t* h_offsets,
                               const uint32_t* h_members, void* h_table, size_t table_bytes)
{
    if (blocks < 1 || blocks > 1024 || !h_offsets || !h_members || !h_table) return PG_EINVAL;
    for (uint32_t p = 0; p < blocks; ++p) {
        if (h_offsets[p + 1] <= h_offsets[p] || h_offsets[p + 1] - h_offsets[p] > kFacSlots)
            return PG_EINVAL;
        for (uint32_t t = h_offsets[p]; t < h_offsets[p + 1]; ++t)
            if (h_members[t] >= blocks) return PG_EINVAL;
    }
    if (table_bytes < pg_pba_faction_table_size(blocks)) return PG_ENOSPC;
    uint16_t* tab = (uint16_t*)h_table;
    std::memset(tab, 0, pg_pba_faction_table_size(blocks));
    std::vector<uint8_t> inside(blocks);
    for (uint32_t p = 0; p < blocks; ++p) {
        uint16_t* rec = tab + (size_t)p * kFacStride;
        const uint32_t a = h_offsets[p], s = h_offsets[p + 1] - a;
        std::fill(inside.begin(), inside.end(), 0);
        for (uint32_t t = 0; t < s; ++t) {
            rec[kFacHeader + t] = (uint16_t)h_members[a + t];
            inside[h_members[a + t]] = 1;
        }
        uint32_t n_out = 0;
        for (uint32_t b = 0; b < blocks; ++b)
            if (!inside[b]) rec[kFacHeader + kFacSlots + n_out++] = (uint16_t)b;
        rec[0] = (uint16_t)s;
        rec[1] = (uint16_t)n_out;
    }
    return PG_OK;
}

pg_status gen_pba_factions(uint64_t n, uint32_t m, uint32_t blocks, uint32_t n0,
                           const void* d_faction_table, double inter_frac, uint64_t seed,
                           pg_idwidth w, void* d_edges, uint64_t cap_edges,
                           uint64_t* n_edges_out, void* d_ws, size_t ws_bytes, void* stream)
{
    const PbaCheck c = check_pba(n, m, blocks, n0, 1, inter_frac, w);
    if (c.st != PG_OK) return c.st;
    if (n_edges_out) *n_edges_out = c.edges;
    if (cap_edges < c.edges) return PG_ENOSPC;
    if (c.edges > 0 && (!d_edges || !aligned(d_edges, 16))) return PG_EINVAL;
    if (!d_faction_table || !aligned(d_faction_table, 16)) return PG_EINVAL;
    PbaGeom g = make_geom(c.n_b, c.N_e, m, blocks, n0, 1, inter_frac, seed);
    cudaStream_t s = (cudaStream_t)stream;
    // one block: every list holds only block 0, so phase 1 is trivial
    if (blocks == 1) return from_cuda(launch_ba(g, w == PG_ID64, d_edges, s));
    g.ftab = (const uint16_t*)d_faction_table;
    const size_t need = pba_workspace_layout(g.A_stride, blocks, g.S).total;
    if (!d_ws || ws_bytes < need) return PG_ENOMEM;
    if (!aligned(d_ws, 256)) return PG_EINVAL;
    return from_cuda(launch_pba(g, w == PG_ID64, d_edges, d_ws, s));
}

pg_status pg_pba_prepare(uint64_t n, uint32_t m, uint32_t blocks, uint32_t n0,
                         uint32_t faction_width, const void* d_faction_table, double inter_frac,
                         uint64_t seed, void* d_ws, size_t ws_bytes, void* stream)
{
    const uint32_t W = d_faction_table ? 1 : faction_width;
    const PbaCheck c = check_pba(n, m, blocks, n0, W, inter_frac, PG_ID64);
    if (c.st != PG_OK) return c.st;
    if (blocks == 1) return PG_OK;              // serial BA has no phase 1
    if (d_faction_table && !aligned(d_faction_table, 16)) return PG_EINVAL;
    PbaGeom g = make_geom(c.n_b, c.N_e, m, blocks, n0, W, inter_frac, seed);
    g.ftab = (const uint16_t*)d_faction_table;
    const size_t need = pba_workspace_layout(g.A_stride, blocks, g.S).total;
    if (!d_ws || ws_bytes < need) return PG_ENOMEM;
    if (!aligned(d_ws, 256)) return PG_EINVAL;
    return from_cuda(launch_pba_phase1(g, d_ws, (cudaStream_t)stream));
}

pg_status gen_pba_blocks(uint64_t n, uint32_t m, uint32_t blocks, uint32_t n0, uint64_t seed,
                         pg_idwidth w, uint32_t b_begin, uint32_t b_end, void* d_edges,
                         uint64_t cap_edges, uint64_t* n_edges_out, const void* d_ws,
                         size_t ws_bytes, void* stream)
{
    const PbaCheck c = check_pba(n, m, blocks, n0, 1, 0.0, w);
    if (c.st != PG_OK) return c.st;
    if (b_begin > b_end || b_end > blocks) return PG_EINVAL;
    const uint64_t per = c.edges / blocks;
    const uint64_t count = (uint64_t)(b_end - b_begin) * per;
    if (n_edges_out) *n_edges_out = count;
    if (cap_edges < count) return PG_ENOSPC;
    if (count == 0) return PG_OK;
    if (!d_edges || !aligned(d_edges, 16)) return PG_EINVAL;
    const PbaGeom g = make_geom(c.n_b, c.N_e, m, blocks, n0, 1, 0.0, seed);
    cudaStream_t s = (cudaStream_t)stream;
    if (blocks == 1) return from_cuda(launch_ba(g, w == PG_ID64, d_edges, s));
    const size_t need = pba_workspace_layout(g.A_stride, blocks, g.S).total;
    if (!d_ws || ws_bytes < need) return PG_ENOMEM;
    if (!aligned(d_ws, 256)) return PG_EINVAL;
    return from_cuda(launch_pba_emit(g, w == PG_ID64, d_edges, d_ws, b_begin, b_end, s));
}

}  // extern "C"

namespace pgen {

// Argument checks and launch geometry of gen_pba, for other entry points.
int pba_setup(uint64_t n, uint32_t m, uint32_t blocks, uint32_t n0, uint32_t faction_width,
              double inter_frac, uint64_t seed, int id64, PbaGeom* g, uint64_t* n_edges)
{
    const PbaCheck c = check_pba(n, m, blocks, n0, faction_width, inter_frac,
                                 id64 ? PG_ID64 : PG_ID32);
    if (c.st != PG_OK) return c.st;
    *g = make_geom(c.n_b, c.N_e, m, blocks, n0, faction_width, inter_frac, seed);
    *n_edges = c.edges;
    return PG_OK;
}

}  // namespace pgen

namespace {

// The copy stream and events of gen_pba_to_host on the current device. On a
// failure every handle already created is destroyed again.
cudaError_t make_host_copy(HostCopy* h)
{
    *h = HostCopy{};
    cudaError_t e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
    uint32_t n_done = 0;
    bool copied = false;
    if (e == cudaSuccess)
        for (; n_done < kMaxCopyChunks; ++n_done)
            if ((e = cudaEventCreateWithFlags(&h->done[n_done], cudaEventDisableTiming)) !=
                cudaSuccess)
                break;
    if (e == cudaSuccess)
        copied = (e = cudaEventCreateWithFlags(&h->copied, cudaEventDisableTiming)) == cudaSuccess;
    if (e != cudaSuccess) {
        for (uint32_t i = 0; i < n_done; ++i) cudaEventDestroy(h->done[i]);
        if (copied) cudaEventDestroy(h->copied);
        if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
        *h = HostCopy{};
    }
    return e;
}

}  // namespace

extern "C" {

pg_status gen_pba_to_host(uint64_t n, uint32_t m, uint32_t blocks, uint32_t n0,
                          uint32_t faction_width, double inter_frac, uint64_t seed, pg_idwidth w,
                          void* h_edges, void* d_edges, uint64_t cap_edges, uint64_t* n_edges_out,
                          void* d_ws, size_t ws_bytes, void* stream)
{
    if (!h_edges) return PG_EINVAL;
    const PbaCheck c = check_pba(n, m, blocks, n0, faction_width, inter_frac, w);
    if (c.st != PG_OK) return c.st;
    if (n_edges_out) *n_edges_out = c.edges;
    if (cap_edges < c.edges) return PG_ENOSPC;
    if (c.edges > 0 && (!d_edges || !aligned(d_edges, 16))) return PG_EINVAL;
    const PbaGeom g = make_geom(c.n_b, c.N_e, m, blocks, n0, faction_width, inter_frac, seed);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = c.edges * (w == PG_ID64 ? 16 : 8);
    if (blocks == 1) {
        if (launch_ba(g, w == PG_ID64, d_edges, s) != cudaSuccess) return PG_ECUDA;
        return cudaMemcpyAsync(h_edges, d_edges, bytes, cudaMemcpyDeviceToHost, s) == cudaSuccess
                   ? PG_OK : PG_ECUDA;
    }
    const size_t need = pba_workspace_layout(g.A_stride, blocks, g.S).total;
    if (!d_ws || ws_bytes < need) return PG_ENOMEM;
    if (!aligned(d_ws, 256)) return PG_EINVAL;
    // one copy stream and its events per device, made on first use; a
    // set-up that fails destroys what it made, and its status is kept
    static PerDeviceOnce once;
    static HostCopy per_dev[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PG_ECUDA;
    const cudaError_t made = once.run(dev, [dev] { return make_host_copy(&per_dev[dev]); });
    if (made != cudaSuccess) return PG_ECUDA;
    HostCopy hc = per_dev[dev];
    hc.h_edges = h_edges;
    // about one wave of emit CTAs per chunk
    const uint64_t ctas_per_block = (g.S + 7) / 8;
    const uint64_t wave = (uint64_t)device_sm_count() * 4;
    uint64_t per = (wave + ctas_per_block - 1) / ctas_per_block;
    uint64_t chunks = (blocks + per - 1) / per;
    if (chunks > kMaxCopyChunks) chunks = kMaxCopyChunks;
    if (chunks < 1) chunks = 1;
    hc.chunks = (uint32_t)chunks;
    return from_cuda(launch_pba(g, w == PG_ID64, d_edges, d_ws, s, &hc));
}

uint64_t pg_kron_edge_count(const double* h_initiator, uint32_t n0, uint32_t k, uint64_t n_edges,
                            pg_kron_mode mode)
{
    if (mode == PG_KRON_STOCHASTIC) return n_edges;
    if (!h_initiator || n0 < 1 || n0 > 256 || k < 1) return 0;
    uint64_t e0 = 0;
    for (uint32_t c = 0; c < n0 * n0; ++c) e0 += h_initiator[c] > 0.0;
    const u128 total = ipow(e0, k);
    return (total >> 63) ? 0 : (uint64_t)total;
}

}  // extern "C"

namespace {

// gen_kronecker and gen_kronecker_range: edges [e_begin, e_end) of the graph
// (e_end = ~0: to the last edge) into d_edges[0 ...].
pg_status kron_common(const double* h_initiator, uint32_t n0, uint32_t k, uint64_t n_edges,
                      uint64_t seed, pg_kron_mode mode, pg_idwidth w, uint64_t e_begin,
                      uint64_t e_end, void* d_edges, uint64_t cap_edges, uint64_t* n_edges_out,
                      void* stream)
{
    if (!h_initiator || k < 1 || k > 64 || (w != PG_ID32 && w != PG_ID64)) return PG_EINVAL;
    if (mode != PG_KRON_STOCHASTIC && mode != PG_KRON_DETERMINISTIC) return PG_EINVAL;
    const uint32_t max_n0 = mode == PG_KRON_STOCHASTIC ? 16 : 256;
    if (n0 < 1 || n0 > max_n0) return PG_EINVAL;
    const u128 n_vertices = ipow(n0, k);
    const u128 id_limit = (w == PG_ID32) ? ((u128)1 << 32) : ((u128)1 << 64);
    if (n_vertices > id_limit) return PG_EINVAL;
    const uint32_t cells = n0 * n0;
    for (uint32_t c = 0; c < cells; ++c)
        if (!(h_initiator[c] >= 0.0) || !std::isfinite(h_initiator[c])) return PG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;

    if (mode == PG_KRON_STOCHASTIC) {
        uint64_t T[kMaxKronThr];
        KronParams p;
        std::memset(&p, 0, sizeof(p));
        if (!kron_thresholds(h_initiator, n0, T)) return PG_EINVAL;
        p.n0 = n0;
        p.k = k;
        p.key = make_key(seed);
        for (int t = 0; t < kMaxKronThr; ++t) p.u[t] = 0xFFFFFFFFu;
        uint32_t c = 0;
        while (c + 1 < cells && T[c] == 0) ++c;
        p.n_zero = c;
        for (; c + 1 < cells && T[c] < ((uint64_t)1 << 32); ++c) p.u[p.n_u++] = (uint32_t)(T[c] - 1);
        if (e_end == ~(uint64_t)0) e_end = n_edges;
        if (e_begin > e_end || e_end > n_edges) return PG_EINVAL;
        const uint64_t count = e_end - e_begin;
        if (n_edges_out) *n_edges_out = count;
        if (cap_edges < count) return PG_ENOSPC;
        if (count > 0 && (!d_edges || !aligned(d_edges, 16))) return PG_EINVAL;
        return from_cuda(launch_kron_stochastic(p, w == PG_ID64, d_edges, e_begin, count, s));
    }

    KronDetParams p;
    std::memset(&p, 0, sizeof(p));
    uint32_t e0 = 0;
    for (uint32_t c = 0; c < cells; ++c) {
        if (h_initiator[c] > 0.0) {
            if (e0 >= (uint32_t)kMaxDetSeedEdges) return PG_EINVAL;
            p.ab[e0++] = (uint16_t)((c / n0) | ((c % n0) << 8));
        }
    }
    if (e0 == 0) return PG_EINVAL;
    const u128 total = ipow(e0, k);
    if (total >> 62) return PG_EINVAL;
    p.n0 = n0;
    p.k = k;
    p.e0 = e0;
    p.div_e0 = make_fastdiv(e0);
    p.div_e0_32 = make_fastdiv32(e0);
    // the widest digit group whose table fits and whose row and column parts
    // fit 16 bits each
    uint64_t E = e0, n0g = n0;
    uint32_t g = 1;
    while (g < k && E * e0 <= kDetGroupTable && n0g * n0 <= 65536) {
        ++g;
        E *= e0;
        n0g *= n0;
    }
    p.g = g;
    p.E = (uint32_t)E;
    p.n_groups = k / g;
    p.n_rest = k % g;
    p.n0g = n0g;
    p.div_E = make_fastdiv(E);
    p.div_E32 = make_fastdiv32((uint32_t)E);
    if (e_end == ~(uint64_t)0) e_end = (uint64_t)total;
    if (e_begin > e_end || e_end > (uint64_t)total) return PG_EINVAL;
    const uint64_t count = e_end - e_begin;
    if (n_edges_out) *n_edges_out = count;
    if (cap_edges < count) return PG_ENOSPC;
    if (count > 0 && (!d_edges || !aligned(d_edges, 16))) return PG_EINVAL;
    return from_cuda(launch_kron_det(p, w == PG_ID64, d_edges, e_begin, count, s));
}

}  // namespace

extern "C" {

pg_status gen_kronecker(const double* h_initiator, uint32_t n0, uint32_t k, uint64_t n_edges,
                        uint64_t seed, pg_kron_mode mode, pg_idwidth w, void* d_edges,
                        uint64_t cap_edges, uint64_t* n_edges_out, void* stream)
{
    return kron_common(h_initiator, n0, k, n_edges, seed, mode, w, 0, ~(uint64_t)0, d_edges,
                       cap_edges, n_edges_out, stream);
}

pg_status gen_random_cells(uint64_t n_vertices, uint64_t n_edges, uint64_t seed, pg_idwidth w,
                           void* d_edges, uint64_t cap_edges, void* stream)
{
    if (w != PG_ID32 && w != PG_ID64) return PG_EINVAL;
    if (n_edges > 0 && n_vertices == 0) return PG_EINVAL;
    if (w == PG_ID32 && n_vertices > ((uint64_t)1 << 32)) return PG_EINVAL;
    if (cap_edges < n_edges) return PG_ENOSPC;
    if (n_edges > 0 && (!d_edges || !aligned(d_edges, 16))) return PG_EINVAL;
    return from_cuda(launch_random_cells(make_key(seed), n_vertices, w == PG_ID64, d_edges, 0,
                                         n_edges, (cudaStream_t)stream));
}

pg_status gen_kronecker_range(const double* h_initiator, uint32_t n0, uint32_t k,
                              uint64_t n_edges, uint64_t seed, pg_kron_mode mode, pg_idwidth w,
                              uint64_t e_begin, uint64_t e_end, void* d_edges,
                              uint64_t cap_edges, void* stream)
{
    if (e_end == ~(uint64_t)0) return PG_EINVAL;
    return kron_common(h_initiator, n0, k, n_edges, seed, mode, w, e_begin, e_end, d_edges,
                       cap_edges, nullptr, stream);
}

size_t pg_csr_opts_workspace_size(uint64_t n_edges, uint64_t n_vertices, uint32_t flags)
{
    if (flags == 0) return csr_workspace_bytes(n_edges, n_vertices);
    return csr_opts_workspace_bytes(n_edges, n_vertices, flags);
}

pg_status edges_to_csr_opts(const void* d_edges, uint64_t n_edges, uint64_t n_vertices,
                            pg_idwidth w, uint32_t flags, uint64_t* d_row_ptr, void* d_col,
                            uint64_t cap_col, void* d_ws, size_t ws_bytes, void* stream)
{
    if (flags & ~(uint32_t)(PG_CSR_SYMMETRIZE | PG_CSR_DEDUP | PG_CSR_NO_LOOPS | PG_CSR_ODD))
        return PG_EINVAL;
    if (w != PG_ID32 && w != PG_ID64) return PG_EINVAL;
    if (n_edges > 0 && n_vertices == 0) return PG_EINVAL;
    if (!d_row_ptr || !aligned(d_row_ptr, 8)) return PG_EINVAL;
    if (n_edges >> 62) return PG_EINVAL;
    const uint64_t listed = (flags & PG_CSR_SYMMETRIZE) ? 2 * n_edges : n_edges;
    if (cap_col < listed) return PG_ENOSPC;
    if (n_edges > 0 && (!d_edges || !d_col || !aligned(d_edges, w == PG_ID64 ? 16 : 8)))
        return PG_EINVAL;
    if (w == PG_ID32 && n_vertices > ((uint64_t)1 << 32)) return PG_EINVAL;
    const size_t need = pg_csr_opts_workspace_size(n_edges, n_vertices, flags);
    if (ws_bytes < need || (need > 0 && !d_ws)) return PG_ENOMEM;
    if (d_ws && !aligned(d_ws, 256)) return PG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (flags == 0)
        return from_cuda(launch_csr(d_edges, n_edges, n_vertices, w == PG_ID64, d_row_ptr, d_col,
                                    d_ws, ws_bytes, s));
    return from_cuda(launch_csr_opts(d_edges, n_edges, n_vertices, w == PG_ID64, flags, d_row_ptr,
                                     d_col, d_ws, s));
}

size_t pg_csr_wait_error_offset(uint64_t n_edges, uint64_t n_vertices, pg_idwidth w,
                                uint32_t flags)
{
    if (flags & ~(uint32_t)(PG_CSR_SYMMETRIZE | PG_CSR_DEDUP | PG_CSR_NO_LOOPS | PG_CSR_ODD))
        return SIZE_MAX;
    if (w != PG_ID32 && w != PG_ID64) return SIZE_MAX;
    if (n_edges == 0 || n_vertices < 2 || (n_edges >> 62)) return SIZE_MAX;
    return csr_wait_error_offset(n_edges, n_vertices, flags, w == PG_ID64);
}

pg_status pg_csr_check(const void* d_ws, uint64_t n_edges, uint64_t n_vertices, pg_idwidth w,
                       uint32_t flags, void* stream)
{
    if (flags & ~(uint32_t)(PG_CSR_SYMMETRIZE | PG_CSR_DEDUP | PG_CSR_NO_LOOPS | PG_CSR_ODD))
        return PG_EINVAL;
    if (w != PG_ID32 && w != PG_ID64) return PG_EINVAL;
    const size_t off = pg_csr_wait_error_offset(n_edges, n_vertices, w, flags);
    if (off == SIZE_MAX) return PG_OK;   // no edges to sort: the call had no wait
    if (!d_ws) return PG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t word = 0;
    if (cudaMemcpyAsync(&word, (const unsigned char*)d_ws + off, 4, cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
        return PG_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PG_ECUDA;
    return word ? PG_ETIMEOUT : PG_OK;
}

void pg_csr_test_wait_hook(uint32_t spin_limit, uint32_t withhold_tile)
{
    set_csr_wait_hook(spin_limit, withhold_tile);
}

int pg_checked_build(void) { return kChecked ? 1 : 0; }

#ifdef PGEN_CHECKED
namespace {
using CheckAccess = cudaError_t (*)(CheckRecord*, int, uint32_t, cudaStream_t);
// indexed by CheckUnit
constexpr CheckAccess kCheckUnits[] = {nullptr, check_access_kron, check_access_pba,
                                       check_access_csr, check_access_batch,
                                       check_access_analyze};
constexpr uint32_t kNumCheckUnits = sizeof(kCheckUnits) / sizeof(kCheckUnits[0]);
}  // namespace
#endif

pg_status pg_check_read(int reset, uint32_t* count, uint32_t* unit, uint32_t* line,
                        uint64_t* index, uint64_t* bound, void* stream)
{
    uint64_t total = 0;
    uint32_t first_unit = 0;
    CheckRecord first{0, 0, 0, 0};
#ifdef PGEN_CHECKED
    for (uint32_t u = 1; u < kNumCheckUnits; ++u) {
        CheckRecord r{0, 0, 0, 0};
        if (kCheckUnits[u](&r, reset, 0xFFFFFFFFu, (cudaStream_t)stream) != cudaSuccess)
            return PG_ECUDA;
        if (r.count && !first_unit) {
            first_unit = u;
            first = r;
        }
        total += r.count;
    }
#else
    (void)reset;
    (void)stream;
#endif
    if (count) *count = total > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)total;
    if (unit) *unit = first_unit;
    if (line) *line = first.line;
    if (index) *index = first.index;
    if (bound) *bound = first.bound;
    return PG_OK;
}

pg_status pg_check_test_out_shift(uint32_t shift, void* stream)
{
#ifdef PGEN_CHECKED
    if (shift > 63) return PG_EINVAL;
    for (uint32_t u = 1; u < kNumCheckUnits; ++u)
        if (kCheckUnits[u](nullptr, 0, shift, (cudaStream_t)stream) != cudaSuccess)
            return PG_ECUDA;
    return PG_OK;
#else
    (void)shift;
    (void)stream;
    return PG_EINVAL;
#endif
}

size_t pg_csr_workspace_size(uint64_t n_edges, uint64_t n_vertices)
{
    return csr_workspace_bytes(n_edges, n_vertices);
}

pg_status edges_to_csr(const void* d_edges, uint64_t n_edges, uint64_t n_vertices, pg_idwidth w,
                       uint64_t* d_row_ptr, void* d_col, void* d_ws, size_t ws_bytes,
                       void* stream)
{
    if (w != PG_ID32 && w != PG_ID64) return PG_EINVAL;
    if (n_edges > 0 && n_vertices == 0) return PG_EINVAL;
    if (!d_row_ptr || !aligned(d_row_ptr, 8)) return PG_EINVAL;
    if (n_edges > 0 && (!d_edges || !d_col || !aligned(d_edges, w == PG_ID64 ? 16 : 8)))
        return PG_EINVAL;
    if (w == PG_ID32 && n_vertices > ((uint64_t)1 << 32)) return PG_EINVAL;
    const size_t need = csr_workspace_bytes(n_edges, n_vertices);
    if (ws_bytes < need || (need > 0 && !d_ws)) return PG_ENOMEM;
    if (d_ws && !aligned(d_ws, 256)) return PG_EINVAL;
    return from_cuda(launch_csr(d_edges, n_edges, n_vertices, w == PG_ID64, d_row_ptr, d_col, d_ws,
                                ws_bytes, (cudaStream_t)stream));
}

}  // extern "C"

// Internal launch interface between the C ABI (api.cu) and the kernel
// translation units. Host-only declarations; every launcher enqueues work on
// `stream` and returns the cudaGetLastError() of its launches.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <initializer_list>
#include <mutex>
#include <cuda_runtime.h>

#include "pg_check.cuh"
#include "pg_common.cuh"

namespace pgen {

// Kernels launched by the library in this process (pg_launch_count): every
// launch site calls note_launch() right after its launch.
extern std::atomic<uint64_t> g_launch_count;
inline void note_launch() { g_launch_count.fetch_add(1, std::memory_order_relaxed); }

// Once-per-device set-up (kernel attributes such as the opt-in shared-memory
// size apply to the device that is current when they are set). run() calls
// `setup` the first time it sees a device id, under a mutex, and remembers
// its status: every later call for that device returns the same status
// without calling it again. Ids outside [0, kMaxDevices) fail.
constexpr int kMaxDevices = 64;
class PerDeviceOnce {
public:
    template <class F>
    cudaError_t run(int dev, F&& setup)
    {
        if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
        std::lock_guard<std::mutex> lk(mu_);
        if (!done_[dev]) {
            status_[dev] = setup();
            done_[dev] = true;
        }
        return status_[dev];
    }
    // The same, for the device that is current on this host thread.
    template <class F>
    cudaError_t run_current(F&& setup)
    {
        int dev = 0;
        const cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        return run(dev, setup);
    }

private:
    std::mutex mu_;
    bool done_[kMaxDevices] = {};
    cudaError_t status_[kMaxDevices] = {};
};

// The first failure among several CUDA calls (cudaSuccess when none failed).
inline cudaError_t first_error(std::initializer_list<cudaError_t> errs)
{
    for (cudaError_t e : errs)
        if (e != cudaSuccess) return e;
    return cudaSuccess;
}

constexpr int kMaxKronThr = 255;   // n0 <= 16 -> at most 255 thresholds

// Stochastic Kronecker descent parameters. With thresholds T_c (c < n0^2-1),
// a word w passes T_c when w >= T_c. Thresholds equal to 0 are always passed
// (n_zero of them, at the front); the next n_u are stored as u = T_c - 1 so
// that the test is w > u in 32 bits; thresholds equal to 2^32 are never
// passed and are dropped. u[] is ascending and padded with 0xffffffff.
struct KronParams {
    uint32_t n0, k, n_zero, n_u;
    Key key;
    uint32_t u[kMaxKronThr];
};

// Deterministic Kronecker: seed edges (row-major; a in the low byte, b in
// the high byte, so n0 <= 256) and the divisor for base-e0 digits. The k
// digits of an edge index are taken g at a time from the least significant
// end: n_groups groups of g digits, each resolved by one lookup in a table of
// all E = e0^g digit groups, then n_rest = k - g * n_groups single digits.
constexpr int kMaxDetSeedEdges = 8192;
constexpr uint32_t kDetGroupTable = 16384;   // entries of the digit-group table (64 KB)
struct KronDetParams {
    uint32_t n0, k, e0, pad;
    FastDiv div_e0;
    FastDiv32 div_e0_32;   // for edge indices below 2^32
    uint32_t g, E, n_groups, n_rest;
    uint64_t n0g;          // n0^g: the weight of one digit group in row and column
    FastDiv div_E;
    FastDiv32 div_E32;
    uint16_t ab[kMaxDetSeedEdges];
};

cudaError_t launch_kron_stochastic(const KronParams& p, int id64, void* d_out, uint64_t e_begin,
                                   uint64_t n_edges, cudaStream_t s);
cudaError_t launch_kron_det(const KronDetParams& p, int id64, void* d_out, uint64_t e_begin,
                            uint64_t n_edges, cudaStream_t s);
cudaError_t launch_random_cells(const Key& key, uint64_t n_vertices, int id64, void* d_out,
                                uint64_t e_begin, uint64_t n_edges, cudaStream_t s);

// PBA (two-phase preferential attachment) geometry.
struct PbaGeom {
    uint64_t n_b, N_e, e0, span;   // span = n0 + n_b (ids per block)
    uint64_t A_stride;             // entries between rows of A (N_e rounded up to 8)
    uint32_t m, B, W, n0;
    uint32_t coin_on, coin_thr;    // inter-faction coin: w2 < coin_thr
    Key key;
    uint32_t S;                    // segments per block (one emit warp each)
    uint64_t seg_len;              // entries per segment (a multiple of 16384)
    uint32_t P;                    // phase-1 prefix kept in shared memory
    uint32_t nb_shift;             // log2(n_b) when n_b is a power of two, else 0xffffffff
    uint64_t lean_add;             // (n_b - 1) + e0 * n_b when n_b is a power of two
    FastDiv div_m, div_nb;
    FastDiv32 div_m32;             // j div m for j < 2^32
    const uint16_t* ftab;          // faction table (device), or null: aligned width-W factions
};

// Faction table: one record of kFacStride uint16 per block: [0] list size s
// (1..1024), [1] complement size, [2..7] zero, then the list (1024 slots) and
// the blocks outside it in ascending order (1024 slots).
constexpr uint32_t kFacHeader = 8;
constexpr uint32_t kFacSlots = 1024;
constexpr uint32_t kFacStride = kFacHeader + 2 * kFacSlots;

// Workspace layout for B > 1 (all offsets 256-byte aligned).
struct PbaWorkspace {
    size_t off_A, off_cnt, off_off, off_R, off_magic, off_recip, off_flag, off_stab, total;
};
PbaWorkspace pba_workspace_layout(uint64_t A_stride, uint32_t B, uint32_t S);
uint32_t pba_segments(uint64_t N_e, uint32_t B, int sm_count);
uint32_t pba_prefix_len(uint64_t N_e);
uint64_t pba_segment_length(uint64_t N_e, uint32_t S);

void set_wide_path_forced(bool on);
bool wide_path_forced();
cudaError_t launch_ba(const PbaGeom& g, int id64, void* d_out, cudaStream_t s);
int pba_setup(uint64_t n, uint32_t m, uint32_t blocks, uint32_t n0, uint32_t faction_width,
              double inter_frac, uint64_t seed, int id64, PbaGeom* g, uint64_t* n_edges);
// Optional copy of the edge list to host memory, overlapped with the emit
// kernels: emit runs in `chunks` block ranges and each range is copied on
// copy_stream as soon as it is written; `s` then waits for the last copy.
struct HostCopy {
    void* h_edges;
    uint32_t chunks;                 // at most kMaxCopyChunks
    cudaStream_t copy_stream;
    cudaEvent_t done[32];
    cudaEvent_t copied;
};
constexpr uint32_t kMaxCopyChunks = 32;

cudaError_t launch_pba_phase1(const PbaGeom& g, void* d_ws, cudaStream_t s);
cudaError_t launch_pba_emit(const PbaGeom& g, int id64, void* d_out, const void* d_ws,
                            uint32_t b_begin, uint32_t b_end, cudaStream_t s,
                            const HostCopy* hc = nullptr);
cudaError_t launch_pba(const PbaGeom& g, int id64, void* d_out, void* d_ws, cudaStream_t s,
                       const HostCopy* hc = nullptr);

// CSR assembly.
size_t csr_opts_workspace_bytes(uint64_t n_edges, uint64_t n_vertices, uint32_t flags);
cudaError_t launch_csr_opts(const void* d_edges, uint64_t n_edges, uint64_t n_vertices, int id64,
                            uint32_t flags, uint64_t* d_row_ptr, void* d_col, void* d_ws,
                            cudaStream_t s);
// n_dst (0: n_vertices) bounds the destination ids: the sort orders them on
// the bits of n_dst - 1 only (a CSR whose rows hold local ids of smaller
// graphs, as the batch CSR's union). The workspace and wait-word offset of
// a call depend on it.
size_t csr_workspace_bytes(uint64_t n_edges, uint64_t n_vertices, uint64_t n_dst = 0);
size_t csr_wait_error_offset(uint64_t n_edges, uint64_t n_vertices, uint32_t flags, int id64,
                             uint64_t n_dst = 0);
void set_csr_wait_hook(uint32_t spin_limit, uint32_t withhold_tile);
cudaError_t launch_csr(const void* d_edges, uint64_t n_edges, uint64_t n_vertices, int id64,
                       uint64_t* d_row_ptr, void* d_col, void* d_ws, size_t ws_bytes,
                       cudaStream_t s, uint64_t n_dst = 0);

int device_sm_count();

#ifdef PGEN_CHECKED
// Per-unit bounds-check records of the checked build (pg_check.cuh).
cudaError_t check_access_kron(CheckRecord* out, int reset, uint32_t shift, cudaStream_t s);
cudaError_t check_access_pba(CheckRecord* out, int reset, uint32_t shift, cudaStream_t s);
cudaError_t check_access_csr(CheckRecord* out, int reset, uint32_t shift, cudaStream_t s);
cudaError_t check_access_batch(CheckRecord* out, int reset, uint32_t shift, cudaStream_t s);
cudaError_t check_access_analyze(CheckRecord* out, int reset, uint32_t shift, cudaStream_t s);
#endif

}  // namespace pgen

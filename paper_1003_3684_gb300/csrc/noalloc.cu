// gen_pba_noalloc: the two-phase PBA generator for callers that cannot
// allocate device memory.
//
// gen_pba needs a device workspace (the phase-1 lists A, the count matrix,
// the offsets, per-block divisors) that its caller allocates. Some callers
// cannot: code embedded in a host application whose allocator has reserved
// the whole device and forbids outside cudaMalloc calls, plugins that are
// handed device buffers but no allocation API, and latency-critical paths
// that must not pay for cudaMalloc/cudaFree and the device-wide
// synchronisation they bring. This entry point takes the same arguments as
// gen_pba minus the workspace, and uses a fixed scratch array compiled into
// the library instead.
#include <mutex>

#include "../../include/pgen.h"
#include "pg_internal.h"

namespace pgen {
namespace {

constexpr size_t kScratchBytes = (size_t)32 << 20;   // 32 MiB, see pgen.h

// Device-side scratch for gen_pba_noalloc. Every GPU that loads this part of
// the library holds it until the process exits.
__device__ __align__(256) unsigned char g_pba_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};   // device address of g_pba_scratch, per device

// Device address of the scratch array on the current device. In host code
// the name g_pba_scratch is only a host-side stand-in; the address a kernel
// may use is obtained once per device with cudaGetSymbolAddress.
void* scratch_on_current_device(pg_status* st)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        *st = PG_ECUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_pba_scratch) != cudaSuccess || !p) {
            *st = PG_ECUDA;
            return nullptr;
        }
        g_scratch_ptr[dev] = p;
    }
    *st = PG_OK;
    return g_scratch_ptr[dev];
}

}  // namespace
}  // namespace pgen

using namespace pgen;

extern "C" {

size_t pg_pba_noalloc_scratch_bytes(void) { return kScratchBytes; }

pg_status gen_pba_noalloc(uint64_t n, uint32_t m, uint32_t blocks, uint32_t n0,
                          uint32_t faction_width, double inter_frac, uint64_t seed, pg_idwidth w,
                          void* d_edges, uint64_t cap_edges, uint64_t* n_edges_out, void* stream)
{
    if (w != PG_ID32 && w != PG_ID64) return PG_EINVAL;
    PbaGeom g;
    uint64_t edges = 0;
    const int rc = pba_setup(n, m, blocks, n0, faction_width, inter_frac, seed, w == PG_ID64,
                             &g, &edges);
    if (rc != PG_OK) return (pg_status)rc;
    if (n_edges_out) *n_edges_out = edges;
    if (cap_edges < edges) return PG_ENOSPC;
    if (edges > 0 && (!d_edges || ((uintptr_t)d_edges & 15))) return PG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (blocks == 1) return launch_ba(g, w == PG_ID64, d_edges, s) == cudaSuccess ? PG_OK : PG_ECUDA;
    // the graph must fit the fixed scratch; nothing is launched otherwise
    if (pba_workspace_layout(g.A_stride, g.B, g.S).total > kScratchBytes) return PG_ENOMEM;
    pg_status st;
    void* scratch = scratch_on_current_device(&st);
    if (!scratch) return st;
    // launch_pba clears the counts and the flag it needs on the stream before
    // use, so the array's leftovers from an earlier call do not matter
    return launch_pba(g, w == PG_ID64, d_edges, scratch, s) == cudaSuccess ? PG_OK : PG_ECUDA;
}

}  // extern "C"

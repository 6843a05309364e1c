// Integer throughput probe: Philox4x32-10 calls per second on this device.
//
// The generators are bound by 32-bit integer issue (Philox rounds and index
// arithmetic), not by memory. Their roofline denominator is derived from the
// SM count, 128 int32 lanes per SM and the clock; this kernel measures what
// the same Philox code reaches when nothing else runs, so a kernel's
// fraction can also be read against a measured ceiling.
#include "../../include/pgen.h"
#include "pg_common.cuh"
#include "pg_internal.h"

namespace pgen {
namespace {

constexpr int kProbeThreads = 256;

// Every thread makes `calls` independent Philox calls (four interleaved
// chains) and folds the words into one result, so no call is dead code.
__global__ void __launch_bounds__(kProbeThreads) philox_probe_kernel(uint32_t* __restrict__ out,
                                                                      uint32_t calls, Key key)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
#pragma unroll 4
    for (uint32_t i = 0; i < calls; ++i) {
        const uint4 w = philox(make_uint4(tid, i, 7u, 3u), key);
        acc ^= w.x ^ w.y ^ w.z ^ w.w;
    }
    out[tid] = acc;
}

// Integer pipe rates: 8 dependency chains per thread, each applying one kind
// of operation `iters` times (8 independent operations per step); the
// results are folded into one word so no chain is dead code. op 0: 32x32->64
// multiply (the Philox round's product), 1: 32-bit multiply-add, 2: a
// three-input logic operation (x ^ (y & z): not linear, so no XOR terms can
// cancel across steps), 3: three-input add.
__global__ void __launch_bounds__(kProbeThreads) int_probe_kernel(uint32_t* __restrict__ out,
                                                                  uint32_t iters, int op,
                                                                  uint32_t k0, uint32_t k1)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = tid * 0x9E3779B9u + c;
    uint32_t h[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) h[c] = c;
    if (op == 0) {
        for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const uint64_t p = (uint64_t)a[c] * k0;
                a[c] = (uint32_t)p;
                h[c] += (uint32_t)(p >> 32);
            }
        }
    } else if (op == 1) {
        for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < 8; ++c) a[c] = a[c] * k0 + k1;
        }
    } else if (op == 2) {
        // each chain also reads its neighbour's value of the previous step, so
        // no chain has a closed form the compiler could substitute
        for (uint32_t i = 0; i < iters; ++i) {
            uint32_t b[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) b[c] = a[c] ^ (a[(c + 3) & 7] & a[(c + 5) & 7]);
#pragma unroll
            for (int c = 0; c < 8; ++c) a[c] = b[c];
        }
    } else {
        for (uint32_t i = 0; i < iters; ++i) {
            uint32_t b[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) b[c] = a[c] + a[(c + 1) & 7] + k1;
#pragma unroll
            for (int c = 0; c < 8; ++c) a[c] = b[c];
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) acc ^= a[c] ^ h[c];
    out[tid] = acc;
}

}  // namespace
}  // namespace pgen

extern "C" {

pg_status pg_int_probe(int op, uint32_t iters, uint32_t* d_out, size_t out_words, void* stream)
{
    const size_t threads = pg_philox_probe_threads();
    if (op < 0 || op > 3 || !d_out || out_words < threads || iters == 0) return PG_EINVAL;
    { pgen::int_probe_kernel<<<(unsigned)(threads / pgen::kProbeThreads), pgen::kProbeThreads, 0,
                             (cudaStream_t)stream>>>(d_out, iters, op, 0x9E3779B9u, 0x7F4A7C15u); pgen::note_launch(); }
    return cudaGetLastError() == cudaSuccess ? PG_OK : PG_ECUDA;
}


size_t pg_philox_probe_threads(void)
{
    return (size_t)pgen::device_sm_count() * 8 * pgen::kProbeThreads;
}

pg_status pg_philox_probe(uint32_t calls_per_thread, uint32_t* d_out, size_t out_words,
                          void* stream)
{
    const size_t threads = pg_philox_probe_threads();
    if (!d_out || out_words < threads || calls_per_thread == 0) return PG_EINVAL;
    const pgen::Key key = pgen::make_key(0x9E3779B97F4A7C15ull);
    { pgen::philox_probe_kernel<<<(unsigned)(threads / pgen::kProbeThreads), pgen::kProbeThreads, 0,
                                (cudaStream_t)stream>>>(d_out, calls_per_thread, key); pgen::note_launch(); }
    return cudaGetLastError() == cudaSuccess ? PG_OK : PG_ECUDA;
}

}  // extern "C"

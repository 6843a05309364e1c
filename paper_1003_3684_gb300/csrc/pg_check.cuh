// Bounds checks of the checked build (compiled with -DPGEN_CHECKED into
// libpgen_checked.so; the default library compiles them away).
//
// Every global or shared-memory access whose index comes from data rather
// than from the loop structure -- a random draw, a block id read from the
// phase-1 lists, a vertex id, a position from a scan -- is guarded by
// PG_CHECK(index, bound). In a checked build a failed check skips the access
// (a load yields 0) and records the violation in a per-translation-unit
// device record; nothing traps, so the context stays usable and the host
// reads the record after the launch (pg_check_read in include/pgen.h).
// PG_CHECK_OUT guards the final store of a result element; a test hook can
// shrink only those bounds (bound >> shift), so a test can make real kernels
// skip stores that are in fact in bounds and see them reported.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pgen {

struct CheckRecord {
    uint32_t count;   // failed checks since the last reset
    uint32_t line;    // source line of the first one
    uint64_t index;   // its index and bound
    uint64_t bound;
};

// Translation units with kernels, as reported by pg_check_read.
enum CheckUnit : uint32_t {
    kUnitKron = 1,
    kUnitPba = 2,
    kUnitCsr = 3,
    kUnitBatch = 4,
    kUnitAnalyze = 5,
};

#ifdef PGEN_CHECKED
constexpr bool kChecked = true;

// One record per translation unit (internal linkage: each unit's module has
// its own copy, read through that unit's check_access_* function).
static __device__ CheckRecord g_pg_check;
static __device__ uint32_t g_pg_out_shift;

static __device__ __noinline__ void pg_check_fail(uint64_t i, uint64_t n, uint32_t line)
{
    if (atomicAdd(&g_pg_check.count, 1u) == 0) {
        g_pg_check.line = line;
        g_pg_check.index = i;
        g_pg_check.bound = n;
    }
}

static __device__ __forceinline__ bool pg_check(uint64_t i, uint64_t n, uint32_t line)
{
    if (i < n) return true;
    pg_check_fail(i, n, line);
    return false;
}

static __device__ __forceinline__ bool pg_check_out(uint64_t i, uint64_t n, uint32_t line)
{
    return pg_check(i, n >> *(volatile uint32_t*)&g_pg_out_shift, line);
}

#define PG_CHECK(i, n) ::pgen::pg_check((uint64_t)(i), (uint64_t)(n), __LINE__)
#define PG_CHECK_OUT(i, n) ::pgen::pg_check_out((uint64_t)(i), (uint64_t)(n), __LINE__)

// Host access to this unit's record: copies it to *out (when out is not
// null), then zeroes it when `reset`, and sets the output-bound shift when
// `shift` <= 63; stream-ordered on s, and synchronises s.
#define PG_CHECK_UNIT(name)                                                                     \
    cudaError_t check_access_##name(CheckRecord* out, int reset, uint32_t shift, cudaStream_t s) \
    {                                                                                           \
        const CheckRecord zero{0, 0, 0, 0};                                                     \
        cudaError_t e = cudaSuccess;                                                            \
        if (out)                                                                                \
            e = cudaMemcpyFromSymbolAsync(out, g_pg_check, sizeof(CheckRecord), 0,              \
                                          cudaMemcpyDeviceToHost, s);                           \
        if (e == cudaSuccess && reset)                                                          \
            e = cudaMemcpyToSymbolAsync(g_pg_check, &zero, sizeof(CheckRecord), 0,              \
                                        cudaMemcpyHostToDevice, s);                             \
        if (e == cudaSuccess && shift <= 63)                                                    \
            e = cudaMemcpyToSymbolAsync(g_pg_out_shift, &shift, sizeof(uint32_t), 0,            \
                                        cudaMemcpyHostToDevice, s);                             \
        /* the host copies above must outlive the transfers */                                  \
        const cudaError_t e2 = cudaStreamSynchronize(s);                                        \
        return e != cudaSuccess ? e : e2;                                                       \
    }
#else
constexpr bool kChecked = false;
#define PG_CHECK(i, n) true
#define PG_CHECK_OUT(i, n) true
#define PG_CHECK_UNIT(name)
#endif

}  // namespace pgen

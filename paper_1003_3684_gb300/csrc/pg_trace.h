// Per-launch timing scope (see trace.cu). Construct right before a launch on
// stream s and let it go out of scope right after it.
#pragma once

#include <cuda_runtime.h>

namespace pgen {

class TraceScope {
public:
    TraceScope(const char* name, cudaStream_t s);
    ~TraceScope();
    TraceScope(const TraceScope&) = delete;
    TraceScope& operator=(const TraceScope&) = delete;

private:
    int idx_;
    cudaStream_t s_;
};

}  // namespace pgen

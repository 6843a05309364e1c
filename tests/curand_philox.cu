// Test helper: the first four words of cuRAND's Philox4_32_10 generator
// (device API) for given (seed, subsequence, offset) -- an independent
// implementation to compare the oracle's Philox4x32-10 against.
#include <cstdint>
#include <curand_kernel.h>

__global__ void first_words(unsigned long long seed, const unsigned long long* subseq,
                            const unsigned long long* offset, uint4* out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed, subseq[i], offset[i], &st);
    out[i] = curand4(&st);
}

extern "C" int curand_philox_first(unsigned long long seed, const unsigned long long* h_subseq,
                                   const unsigned long long* h_offset, unsigned int* h_out, int n)
{
    unsigned long long *d_sub = nullptr, *d_off = nullptr;
    uint4* d_out = nullptr;
    if (cudaMalloc(&d_sub, n * 8) || cudaMalloc(&d_off, n * 8) || cudaMalloc(&d_out, n * 16))
        return 1;
    cudaMemcpy(d_sub, h_subseq, n * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(d_off, h_offset, n * 8, cudaMemcpyHostToDevice);
    first_words<<<(n + 127) / 128, 128>>>(seed, d_sub, d_off, d_out, n);
    const int rc = cudaMemcpy(h_out, d_out, n * 16, cudaMemcpyDeviceToHost) != cudaSuccess;
    cudaFree(d_sub);
    cudaFree(d_off);
    cudaFree(d_out);
    return rc;
}

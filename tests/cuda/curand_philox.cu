// Test helper: word 0 of cuRAND's device Philox-4x32-10 (curand_Philox4x32_10
// from the cuRAND device API headers) for counters (c0[i], c1[i], 0, 0) and
// key (k0, k1), so that the library's and the oracle's implementations can be
// compared with NVIDIA's.  Built by tests/test_gpu_philox.py with nvcc.
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_philox4x32_x.h>

__global__ void curand_words(const uint32_t *c0, const uint32_t *c1, uint32_t k0, uint32_t k1, uint32_t n,
                             uint32_t *out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = curand_Philox4x32_10(make_uint4(c0[i], c1[i], 0u, 0u), make_uint2(k0, k1)).x;
}

// Host arrays of n entries; returns 0 or a cudaError_t.
extern "C" int curand_philox_word0(const uint32_t *c0, const uint32_t *c1, uint32_t k0, uint32_t k1, uint32_t n,
                                   uint32_t *out) {
    uint32_t *d = nullptr;
    const size_t bytes = 4ull * n;
    cudaError_t e = cudaMalloc(&d, 3 * bytes);
    if (e != cudaSuccess) return (int)e;
    e = cudaMemcpy(d, c0, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + n, c1, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        curand_words<<<(n + 255u) / 256u, 256>>>(d, d + n, k0, k1, n, d + 2ull * n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, d + 2ull * n, bytes, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return (int)e;
}

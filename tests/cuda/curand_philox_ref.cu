// Test helper (not part of the library): Philox4x32-10 outputs from cuRAND's
// device generator, used to pin the oracle's own Philox implementation.
// curand_init(seed, subsequence, offset) sets key = seed and counter =
// (offset / 4 in words 0-1, subsequence in words 2-3); curand4 returns the
// block of the current counter.
#include <cuda_runtime.h>
#include <curand_kernel.h>
#include <stdint.h>

__global__ void k_ref(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    const unsigned long long seed = (unsigned long long)key[2 * i] | ((unsigned long long)key[2 * i + 1] << 32);
    const unsigned long long sub = (unsigned long long)ctr[4 * i + 2] | ((unsigned long long)ctr[4 * i + 3] << 32);
    const unsigned long long off = ((unsigned long long)ctr[4 * i] | ((unsigned long long)ctr[4 * i + 1] << 32)) * 4ull;
    curand_init(seed, sub, off, &st);
    const uint4 r = curand4(&st);
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

extern "C" int curand_philox_ref(const uint32_t* ctr_h, const uint32_t* key_h, uint32_t* out_h, int n)
{
    uint32_t *c, *k, *o;
    if (cudaMalloc(&c, 16ull * n) || cudaMalloc(&k, 8ull * n) || cudaMalloc(&o, 16ull * n)) return -1;
    cudaMemcpy(c, ctr_h, 16ull * n, cudaMemcpyHostToDevice);
    cudaMemcpy(k, key_h, 8ull * n, cudaMemcpyHostToDevice);
    k_ref<<<(n + 127) / 128, 128>>>(c, k, o, n);
    const cudaError_t e = cudaMemcpy(out_h, o, 16ull * n, cudaMemcpyDeviceToHost);
    cudaFree(c);
    cudaFree(k);
    cudaFree(o);
    return e == cudaSuccess ? 0 : -2;
}

// Every float n: the library's division by 40 (natural cubic spline) against
// CUDA's IEEE division __fdiv_rn(n, 40.0f), compared bit for bit (NaN results
// compare equal as NaN).  Prints the mismatch count; exit status 0 iff none.
#include <cstdio>
#include <cstdint>
#include <cstring>

#include "common.cuh"

__global__ void k_check(unsigned long long *count, uint32_t *first)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < (1ull << 32); i += stride) {
        const uint32_t bits = (uint32_t)i;
        const float n = __uint_as_float(bits);
        const float ref = __fdiv_rn(n, 40.0f);
        const float got = gi::div40_rn(n);
        if (ref != ref && got != got) continue;
        if (__float_as_uint(ref) != __float_as_uint(got)) {
            const unsigned long long c = atomicAdd(count, 1ull);
            if (c < 8) first[c] = bits;
        }
    }
}

int main()
{
    unsigned long long *count = nullptr;
    uint32_t *first = nullptr;
    if (cudaMalloc(&count, sizeof(*count)) != cudaSuccess || cudaMalloc(&first, 8 * sizeof(uint32_t)) != cudaSuccess)
        return 2;
    cudaMemset(count, 0, sizeof(*count));
    cudaMemset(first, 0, 8 * sizeof(uint32_t));
    k_check<<<1024, 256>>>(count, first);
    const cudaError_t e = cudaDeviceSynchronize();
    unsigned long long h = 0;
    uint32_t hf[8] = {0};
    cudaMemcpy(&h, count, sizeof(h), cudaMemcpyDeviceToHost);
    cudaMemcpy(hf, first, sizeof(hf), cudaMemcpyDeviceToHost);
    printf("status=%s mismatches=%llu\n", cudaGetErrorString(e), h);
    for (unsigned long long i = 0; i < h && i < 8; ++i) printf("  0x%08x\n", hf[i]);
    return (e == cudaSuccess && h == 0) ? 0 : 1;
}

// probe.cu -- measured denominator for the shared-memory lookup roofline.
//
// The count kernels are bound by random reads of a Zech table in shared
// memory (Sec. 4 attributes the limits of the method to random table access).
// This probe times the same access pattern alone: every thread performs a
// chain of dependent, uniformly random 16-bit reads from a shared table of
// the given size, with many warps per SM, and reports reads per second.
#include "hwc_internal.cuh"

namespace hwc {
namespace {

__global__ void k_gather(uint32_t entries, uint32_t iters, unsigned long long *sink)
{
    extern __shared__ __align__(16) uint16_t tab[];
    for (uint32_t i = threadIdx.x; i < entries; i += blockDim.x)
        tab[i] = (uint16_t)((i * 2654435761u) >> 7);
    __syncthreads();
    // four independent chains per thread; index = (table value + LCG) mod entries
    uint32_t s0 = threadIdx.x * 747796405u + blockIdx.x * 2891336453u + 1u;
    uint32_t s1 = s0 ^ 0x9E3779B9u, s2 = s0 ^ 0x85EBCA6Bu, s3 = s0 ^ 0xC2B2AE35u;
    uint32_t u0 = s0 % entries, u1 = s1 % entries, u2 = s2 % entries, u3 = s3 % entries;
    uint32_t acc = 0;
    for (uint32_t it = 0; it < iters; ++it) {
        uint32_t z0 = tab[u0], z1 = tab[u1], z2 = tab[u2], z3 = tab[u3];
        s0 = s0 * 1664525u + 1013904223u;
        s1 = s1 * 1664525u + 1013904223u;
        s2 = s2 * 1664525u + 1013904223u;
        s3 = s3 * 1664525u + 1013904223u;
        u0 = __umulhi(s0 ^ z0, entries);
        u1 = __umulhi(s1 ^ z1, entries);
        u2 = __umulhi(s2 ^ z2, entries);
        u3 = __umulhi(s3 ^ z3, entries);
        acc += z0 ^ z1 ^ z2 ^ z3;
    }
    if (acc == 0x7FFFFFFFu) atomicAdd(sink, 1ull);
}

}  // namespace
}  // namespace hwc

using namespace hwc;

extern "C" int hwc_probe_smem_gather(uint32_t entries, uint32_t iters, double *reads_per_s)
{
    if (!reads_per_s || entries < 32 || entries > 100000 || iters == 0)
        return set_error(HWC_ERR_ARG, "bad probe arguments");
    const uint32_t smem = ((entries * 2 + 15) / 16) * 16;
    cudaFuncAttributes fa{};
    HWC_CUDA_TRY(cudaFuncGetAttributes(&fa, (const void *)k_gather));
    HWC_CUDA_TRY(cudaFuncSetAttribute((const void *)k_gather, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)device_smem_optin() - (int)fa.sharedSizeBytes));
    int ctas = 0;
    HWC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, (const void *)k_gather, 256, smem));
    if (ctas <= 0) return set_error(HWC_ERR_TOO_LARGE, "probe table does not fit");
    const int grid = ctas * device_sm_count();
    unsigned long long *sink = nullptr;
    HWC_CUDA_TRY(cudaMalloc(&sink, sizeof(unsigned long long)));
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k_gather<<<grid, 256, smem>>>(entries, iters / 4 + 1, sink);   // warm-up
    cudaEventRecord(a);
    k_gather<<<grid, 256, smem>>>(entries, iters, sink);
    cudaEventRecord(b);
    cudaError_t ce = cudaEventSynchronize(b);
    float ms = 0;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    if (ce != cudaSuccess) return set_error(HWC_ERR_CUDA, "probe: %s", cudaGetErrorString(ce));
    *reads_per_s = (double)grid * 256.0 * 4.0 * iters / (ms * 1e-3);
    return HWC_OK;
}

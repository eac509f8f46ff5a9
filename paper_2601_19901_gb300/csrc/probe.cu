// Roofline probe for the splat's depth test: throughput of 64-bit atomicMin
// on global memory (resolved in L2) at random or warp-coherent addresses, and
// on shared memory. Each thread takes operations k = tid, tid + stride, ... of
// (idx[k], val[k]).
#include "lfdpr_internal.cuh"

namespace lfdpr {
namespace {

// Indices at or beyond n_words are skipped (the probe never writes outside
// the caller's buffer).
__global__ void __launch_bounds__(256) k_probe_global(unsigned long long* words, uint64_t n_words,
                                                       const uint32_t* __restrict__ idx,
                                                       const unsigned long long* __restrict__ val,
                                                       uint64_t n_ops) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_ops;
         k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t i = __ldg(idx + k);
        if (i < n_words) atomicMin(words + i, __ldg(val + k));
    }
}

// Coherent variant: the 32 operations of warp group q = k / 32 hit the 32
// consecutive words from (idx[32 q] & ~31): one warp instruction covers 256
// contiguous bytes. The grid stride is a multiple of 32, so a warp's lanes
// always form one group.
__global__ void __launch_bounds__(256) k_probe_coherent(unsigned long long* words, uint64_t n_words,
                                                         const uint32_t* __restrict__ idx,
                                                         const unsigned long long* __restrict__ val,
                                                         uint64_t n_ops) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_ops;
         k += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = uint64_t(__ldg(idx + (k & ~uint64_t(31))) & ~31u) + (k & 31u);
        if (i < n_words) atomicMin(words + i, __ldg(val + k));
    }
}

// Shared variant: each block keeps a private copy of the first n_words words
// (n_words <= 8192), applies its share of the operations there, and merges the
// copy into global memory with one atomicMin per word.
__global__ void __launch_bounds__(256) k_probe_shared(unsigned long long* words, uint32_t n_words,
                                                       const uint32_t* __restrict__ idx,
                                                       const unsigned long long* __restrict__ val,
                                                       uint64_t n_ops) {
    extern __shared__ unsigned long long s_words[];
    for (uint32_t w = threadIdx.x; w < n_words; w += blockDim.x) s_words[w] = ~0ull;
    __syncthreads();
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_ops;
         k += (uint64_t)gridDim.x * blockDim.x)
        atomicMin(s_words + (__ldg(idx + k) % n_words), __ldg(val + k));
    __syncthreads();
    for (uint32_t w = threadIdx.x; w < n_words; w += blockDim.x)
        if (s_words[w] != ~0ull) atomicMin(words + w, s_words[w]);
}

}  // namespace

cudaError_t launch_probe_atomic(uint64_t* words, uint64_t n_words, const uint32_t* idx, const uint64_t* val,
                                uint64_t n_ops, int mode, int sm_count, cudaStream_t s) {
    auto* w = reinterpret_cast<unsigned long long*>(words);
    auto* v = reinterpret_cast<const unsigned long long*>(val);
    if (mode == 2) {
        k_probe_coherent<<<sm_count * 8, 256, 0, s>>>(w, n_words, idx, v, n_ops);
    } else if (mode == 1) {
        const size_t smem = (size_t)n_words * 8u;
        cudaError_t e = cudaFuncSetAttribute(k_probe_shared, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        k_probe_shared<<<sm_count * 2, 256, smem, s>>>(w, uint32_t(n_words), idx, v, n_ops);
    } else {
        k_probe_global<<<sm_count * 8, 256, 0, s>>>(w, n_words, idx, v, n_ops);
    }
    return cudaGetLastError();
}

}  // namespace lfdpr

// Roofline microbenchmarks for the reach kernel (diagnostics; the paper has no counterpart).
//
// The converged step of the reach kernel is two lane-private shared-memory gathers per text byte:
// the class of the byte, then the next state.  ridfa_bench_smem_gather times exactly that step on
// every SM (a byte stream made in registers, lane-replicated 32 KB class table and transition
// table, the transition dependent on the previous state), so its rate is the ceiling the reach
// kernel can approach on this GPU.  ridfa_bench_hbm_read times a streaming read of a device
// buffer with 16-byte loads.
#include <cuda_runtime.h>

#include <cstdint>

#include "ridfa.h"

namespace {

__device__ __forceinline__ uint32_t lds32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

constexpr int kStates = 64;   // transition table: 64 states x 16 classes, lane-replicated

__global__ void __launch_bounds__(1024, 1) smem_gather_kernel(uint32_t iters, uint32_t seed, uint32_t *sink) {
    extern __shared__ __align__(16) uint32_t sm[];
    uint32_t *cls = sm;                    // 256 bytes x 32 lanes: class offset (class * 16 * 128)
    uint32_t *tab = sm + 256 * 32;         // (64 * 16) entries x 32 lanes: next-state offset
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t i = threadIdx.x; i < 256 * 32; i += blockDim.x) cls[i] = (((i >> 5) * 13u) & 15u) * 128u;
    for (uint32_t i = threadIdx.x; i < kStates * 16 * 32; i += blockDim.x)
        tab[i] = ((((i >> 5) * 37u + 11u) % kStates) * 16u) * 128u;
    __syncthreads();
    const uint32_t bc = static_cast<uint32_t>(__cvta_generic_to_shared(cls)) + lane * 4;
    const uint32_t bt = static_cast<uint32_t>(__cvta_generic_to_shared(tab)) + lane * 4;
    uint32_t s = ((threadIdx.x * 7u) % kStates) * 16u * 128u;
    uint32_t x = threadIdx.x * 2654435761u + seed;
    for (uint32_t it = 0; it < iters; ++it) {
        x = x * 1664525u + 1013904223u;
        const uint32_t c = lds32(bc + (x >> 24) * 128u);   // offsets stay inside both tables
        s = lds32(bt + s + c);
    }
    if (s == 0xFFFFFFFFu) *sink = s;
}

__global__ void hbm_read_kernel(const uint4 *p, size_t n16, uint32_t *sink) {
    uint32_t acc = 0;
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n16;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const uint4 v = __ldg(p + i);
        acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
    if (acc == 0x9E3779B9u) *sink = acc;
}

int fail(cudaError_t e) {
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? RIDFA_E_NOMEM : RIDFA_E_CUDA;
}

}  // namespace

extern "C" int ridfa_bench_smem_gather(uint32_t iters, double *bytes_per_s, double *ms_out) {
    if (!bytes_per_s || iters == 0) return RIDFA_E_ARG;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(e);
    const size_t smem = (256 * 32 + kStates * 16 * 32) * sizeof(uint32_t);
    e = cudaFuncSetAttribute(smem_gather_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return fail(e);
    uint32_t *sink = nullptr;
    e = cudaMalloc(&sink, 4);
    if (e != cudaSuccess) return fail(e);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float ms = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // first launch warms up
        cudaEventRecord(a);
        smem_gather_kernel<<<sms, 1024, smem>>>(iters, 17u + rep, sink);
        cudaEventRecord(b);
        e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    if (e != cudaSuccess) return fail(e);
    // one step = one text byte's two gathers
    *bytes_per_s = static_cast<double>(sms) * 1024.0 * iters / (ms * 1e-3);
    if (ms_out) *ms_out = ms;
    return RIDFA_OK;
}

extern "C" int ridfa_bench_hbm_read(const uint8_t *d_buf, size_t bytes, double *bytes_per_s, double *ms_out) {
    if (!d_buf || !bytes_per_s || bytes < 16 || (reinterpret_cast<uintptr_t>(d_buf) & 15)) return RIDFA_E_ARG;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(e);
    uint32_t *sink = nullptr;
    e = cudaMalloc(&sink, 4);
    if (e != cudaSuccess) return fail(e);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float ms = 0.f;
    const size_t n16 = bytes / 16;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        cudaEventRecord(a);
        hbm_read_kernel<<<sms * 8, 512>>>(reinterpret_cast<const uint4 *>(d_buf), n16, sink);
        cudaEventRecord(b);
        e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    if (e != cudaSuccess) return fail(e);
    *bytes_per_s = static_cast<double>(n16) * 16.0 / (ms * 1e-3);
    if (ms_out) *ms_out = ms;
    return RIDFA_OK;
}

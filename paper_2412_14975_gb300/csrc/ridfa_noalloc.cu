// ridfa_recognize_noalloc: the RID path on memory that already exists, for callers that must not
// allocate device memory while they serve requests.
//
// cudaMalloc can stall every stream of the device, and it can fail outright when another
// framework's caching allocator already holds the memory.  A service with a strict latency
// budget, or a plug-in whose host application owns every device allocation, therefore cannot let
// a recognize call allocate.  This entry point keeps the program's tables and all of the kernels'
// scratch in one fixed array of device memory declared below, so a call only copies the tables
// in, clears two counters and launches the usual reach and join kernels.
#include <cuda_runtime.h>

#include <mutex>

#include "ridfa_internal.h"

namespace {

// Tables + scratch of ridfa_recognize_noalloc.  Every GPU that loads the library keeps this
// array until the process exits.
constexpr size_t kNoallocBytes = RIDFA_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_ptr[kMaxDevices] = {};   // device address of g_noalloc_scratch, per device

inline size_t al256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Once per device, with that device current: the array's device address.  In host code the
// array's name is only a stand-in, so the address has to come from cudaGetSymbolAddress.
int scratch_address(int dev, uint8_t **out) {
    if (dev < 0 || dev >= kMaxDevices) return RIDFA_E_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || ptr == nullptr) {
            (void)cudaGetLastError();
            return RIDFA_E_CUDA;
        }
        g_scratch_ptr[dev] = ptr;
    }
    *out = static_cast<uint8_t *>(g_scratch_ptr[dev]);
    return RIDFA_OK;
}

}  // namespace

extern "C" int ridfa_recognize_noalloc(const ridfa_program *prog, const uint8_t *d_text, size_t len,
                                       uint32_t n_chunks, uint8_t *d_accept, uint16_t *d_chunk_maps,
                                       void *stream) {
    if (!prog || !d_accept) return RIDFA_E_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const ridfa::HostAutomaton &H = prog->rid;
    if (len == 0) {
        if (n_chunks != 0) return RIDFA_E_CHUNKS;
        const int acc = H.final_flag.empty() ? 0 : H.final_flag[H.slot_state[H.q0_slot]];
        cudaError_t e = cudaMemsetAsync(d_accept, acc, 1, st);
        return e == cudaSuccess ? RIDFA_OK : RIDFA_E_CUDA;
    }
    if (!d_text || !d_chunk_maps) return RIDFA_E_ARG;
    if (n_chunks == 0 || n_chunks > len) return RIDFA_E_CHUNKS;
    if (H.k > RIDFA_MAX_SLOTS) return RIDFA_E_UNSUPPORTED;

    // layout inside the fixed array; everything is sized before anything is copied
    const size_t bt = H.trans.size() * 2, bf = H.final_bits.size() * 4, bi = H.ifmask.size() * 4,
                 bs = H.slot_state.size() * 2;
    size_t off = 0;
    const size_t counters_off = off;  off += 256;                // ticket, status
    const size_t partials_off = off;  off += al256(ridfa::kMaxJoinBlocks * ridfa::kPartialWords * 4);
    const size_t trans_off = off;     off += al256(bt);
    const size_t cls_off = off;       off += 256;
    const size_t fin_off = off;       off += al256(bf);
    const size_t ifm_off = off;       off += al256(bi);
    const size_t slot_off = off;      off += al256(bs);
    const size_t dinfo_off = off;     off += al256(static_cast<size_t>(n_chunks) * 4);
    if (off > kNoallocBytes) return RIDFA_E_TOO_LARGE;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return RIDFA_E_CUDA;
    uint8_t *base = nullptr;
    int err = scratch_address(dev, &base);
    if (err != RIDFA_OK) return err;

    // the array keeps the previous call's contents: the tables are copied in every time, and the
    // join's ticket and status word must start at zero
    e = cudaMemcpyAsync(base + trans_off, H.trans.data(), bt, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + cls_off, H.classmap.data(), 256, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && bf) e = cudaMemcpyAsync(base + fin_off, H.final_bits.data(), bf, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && bi) e = cudaMemcpyAsync(base + ifm_off, H.ifmask.data(), bi, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && bs) e = cudaMemcpyAsync(base + slot_off, H.slot_state.data(), bs, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + counters_off, 0, 256, st);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return RIDFA_E_CUDA;
    }
    ridfa::PreparedBuffers B{};
    B.trans = reinterpret_cast<const uint16_t *>(base + trans_off);
    B.classmap = base + cls_off;
    B.final_bits = reinterpret_cast<const uint32_t *>(base + fin_off);
    B.ifmask = reinterpret_cast<const uint32_t *>(base + ifm_off);
    B.slot_state = reinterpret_cast<const uint16_t *>(base + slot_off);
    B.maps = d_chunk_maps;
    B.dinfo = reinterpret_cast<uint32_t *>(base + dinfo_off);
    B.partials = reinterpret_cast<uint32_t *>(base + partials_off);
    B.ticket = reinterpret_cast<uint32_t *>(base + counters_off);
    B.status = reinterpret_cast<uint32_t *>(base + counters_off + 128);
    B.accept = d_accept;
    return ridfa::launch_with_buffers(H, B, d_text, len, n_chunks, stream);
}

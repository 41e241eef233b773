// The NFA variant of the classic speculative algorithm (Sec. 2; the NFA columns of Table 3), as a
// comparator for the RID.  Chunk automaton A_i = the position NFA with every state initial (chunk
// 1: only q0); each start state's set of active NFA states is simulated on its own over the chunk,
// rho(q, y_i) = the set reached (Follow of the active set, intersected with the positions that read
// the byte's class), with no merging of runs: the mapping lambda_i relates q to every state of
// rho(q, y_i).  The join composes the chunk relations (PLAS_i = lambda_i(PLAS_{i-1}), Sec. 2) as
// a tree of relation compositions, and the text is accepted iff the composed relation takes q0 to
// a set that meets F.
//
// Kernels:
//   rid_nfa_reach_kernel<NW>: one warp per chunk, lane l holding start states l, 32 + l, ... as
//     bitsets of NW 32-bit words; per byte every live set is advanced by OR-ing the follow rows of
//     its members (shared memory) and masking with the byte's class row.  Writes lambda_i rows.
//   rid_nfa_compose_kernel<NW>: one warp composes G consecutive relations (lane = row q): row(q)
//     <- union of the next relation's rows over the members of row(q).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "ridfa_internal.h"

namespace ridfa {
namespace {

constexpr int kNfaCompose = 64;   // relations composed by one warp per level

__device__ __forceinline__ uint64_t dev_chunk_begin(uint64_t i, uint64_t len, uint64_t c) {
    return i * (len / c) + (i * (len % c)) / c;
}

struct NfaArgs {
    const uint8_t *classmap;
    const uint32_t *follow;    // [n][NW]
    const uint32_t *cls;       // [C][NW]
    const uint8_t *text;
    uint64_t len;
    uint32_t c, n, C;
    uint32_t *rel;             // [c][n][NW]
};

template <int NW>
__global__ void __launch_bounds__(256) rid_nfa_reach_kernel(NfaArgs a) {
    extern __shared__ __align__(16) uint32_t sm[];
    uint32_t *s_follow = sm;                               // [n][NW]
    uint32_t *s_cls = sm + a.n * NW;                       // [C][NW]
    uint8_t *s_map = reinterpret_cast<uint8_t *>(s_cls + a.C * NW);
    for (uint32_t i = threadIdx.x; i < a.n * NW; i += blockDim.x) s_follow[i] = a.follow[i];
    for (uint32_t i = threadIdx.x; i < a.C * NW; i += blockDim.x) s_cls[i] = a.cls[i];
    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) s_map[i] = a.classmap[i];
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t ch = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; ch < a.c; ch += warps) {
        const uint64_t beg = dev_chunk_begin(ch, a.len, a.c), end = dev_chunk_begin(ch + 1, a.len, a.c);
        // lane l, register r: start state q = 32 r + l (chunk 1: q0 only)
        uint32_t S[NW][NW];
#pragma unroll
        for (int r = 0; r < NW; ++r)
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const uint32_t q = 32 * r + lane;
                const bool start = q < a.n && (ch > 0 || q == 0);
                S[r][w] = (start && w == r) ? (1u << lane) : 0u;
            }
        for (uint64_t pos = beg; pos < end; ++pos) {
            uint32_t any = 0;
#pragma unroll
            for (int r = 0; r < NW; ++r)
#pragma unroll
                for (int w = 0; w < NW; ++w) any |= S[r][w];
            if (!__any_sync(0xFFFFFFFFu, any != 0)) break;          // every run died
            const uint32_t *cm = s_cls + s_map[a.text[pos]] * NW;
#pragma unroll
            for (int r = 0; r < NW; ++r) {
                uint32_t F[NW];
#pragma unroll
                for (int v = 0; v < NW; ++v) F[v] = 0;
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    uint32_t m = S[r][w];
                    while (m) {
                        const uint32_t q = 32 * w + (__ffs(m) - 1);
                        m &= m - 1;
#pragma unroll
                        for (int v = 0; v < NW; ++v) F[v] |= s_follow[q * NW + v];
                    }
                }
#pragma unroll
                for (int v = 0; v < NW; ++v) S[r][v] = F[v] & cm[v];
            }
        }
#pragma unroll
        for (int r = 0; r < NW; ++r) {
            const uint32_t q = 32 * r + lane;
            if (q < a.n) {
                uint32_t *row = a.rel + (ch * a.n + q) * NW;
#pragma unroll
                for (int w = 0; w < NW; ++w) row[w] = S[r][w];
            }
        }
    }
}

// out[g] = in[g*G] o in[g*G + 1] o ... (relations of n rows of NW words); one warp per g, lane l
// holding rows l, 32 + l, ...
template <int NW>
__global__ void __launch_bounds__(256) rid_nfa_compose_kernel(const uint32_t *in, uint64_t m, uint32_t n,
                                                              uint32_t *out) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t g = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t first = g * kNfaCompose;
    if (first >= m) return;
    const uint64_t last = min(m, first + kNfaCompose);
    const size_t rel_words = static_cast<size_t>(n) * NW;
    uint32_t R[NW][NW];
#pragma unroll
    for (int r = 0; r < NW; ++r) {
        const uint32_t q = 32 * r + lane;
#pragma unroll
        for (int w = 0; w < NW; ++w) R[r][w] = q < n ? in[first * rel_words + q * NW + w] : 0u;
    }
    for (uint64_t j = first + 1; j < last; ++j) {
        const uint32_t *B = in + j * rel_words;
#pragma unroll
        for (int r = 0; r < NW; ++r) {
            uint32_t T[NW];
#pragma unroll
            for (int v = 0; v < NW; ++v) T[v] = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                uint32_t mm = R[r][w];
                while (mm) {
                    const uint32_t p = 32 * w + (__ffs(mm) - 1);
                    mm &= mm - 1;
#pragma unroll
                    for (int v = 0; v < NW; ++v) T[v] |= B[p * NW + v];
                }
            }
#pragma unroll
            for (int v = 0; v < NW; ++v) R[r][v] = T[v];
        }
    }
#pragma unroll
    for (int r = 0; r < NW; ++r) {
        const uint32_t q = 32 * r + lane;
        if (q < n)
#pragma unroll
            for (int w = 0; w < NW; ++w) out[g * rel_words + q * NW + w] = R[r][w];
    }
}

// accept = row q0 of the single composed relation meets F
__global__ void rid_nfa_accept_kernel(const uint32_t *rel, const uint32_t *finals, uint32_t nw, uint8_t *accept) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint32_t hit = 0;
    for (uint32_t w = 0; w < nw; ++w) hit |= rel[w] & finals[w];
    *accept = hit ? 1 : 0;
}

template <int NW>
cudaError_t nfa_launch(const NfaArgs &a, int sms, uint32_t *lvl0, uint32_t *lvl1, const uint32_t *finals,
                       uint8_t *d_accept, cudaStream_t st) {
    const size_t smem = (static_cast<size_t>(a.n) + a.C) * NW * 4 + 256;
    const uint64_t warps_needed = a.c;
    const int grid = static_cast<int>(std::min<uint64_t>((warps_needed + 7) / 8, static_cast<uint64_t>(sms) * 8));
    rid_nfa_reach_kernel<NW><<<grid, 256, smem, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // compose levels until one relation is left; ping-pong between the two level buffers (the
    // caller's lambda rows are read, never overwritten)
    const uint32_t *in = a.rel;
    uint64_t m = a.c;
    uint32_t *bufs[2] = {lvl0, lvl1};
    int b = 0;
    while (m > 1) {
        const uint64_t groups = (m + kNfaCompose - 1) / kNfaCompose;
        rid_nfa_compose_kernel<NW><<<static_cast<unsigned>((groups + 7) / 8), 256, 0, st>>>(in, m, a.n, bufs[b]);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        in = bufs[b];
        b ^= 1;
        m = groups;
    }
    rid_nfa_accept_kernel<<<1, 32, 0, st>>>(in, finals, NW, d_accept);
    return cudaGetLastError();
}

DeviceNfa *nfa_device(const ridfa_program *P, int dev, int *err) {
    for (auto &d : P->dev_nfa)
        if (d.device == dev) return &d;
    const HostNfa &H = P->nfa;
    const size_t bf = H.follow.size() * 4, bc = H.cls.size() * 4, bfin = H.finals.size() * 4;
    const size_t total = 256 + bf + bc + bfin;
    DeviceNfa D;
    D.device = dev;
    cudaError_t e = cudaMalloc(&D.base, total);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&D.h_accept_pinned), 16, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        if (D.base) cudaFree(D.base);
        *err = cuda_fail(e);
        return nullptr;
    }
    std::vector<uint8_t> img(total);
    std::memcpy(img.data(), H.classmap.data(), 256);
    std::memcpy(img.data() + 256, H.follow.data(), bf);
    std::memcpy(img.data() + 256 + bf, H.cls.data(), bc);
    std::memcpy(img.data() + 256 + bf + bc, H.finals.data(), bfin);
    e = cudaMemcpy(D.base, img.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(D.base);
        cudaFreeHost(D.h_accept_pinned);
        *err = cuda_fail(e);
        return nullptr;
    }
    uint8_t *b = static_cast<uint8_t *>(D.base);
    D.classmap = b;
    D.follow = reinterpret_cast<const uint32_t *>(b + 256);
    D.cls = reinterpret_cast<const uint32_t *>(b + 256 + bf);
    D.finals = reinterpret_cast<const uint32_t *>(b + 256 + bf + bc);
    P->dev_nfa.push_back(D);
    return &P->dev_nfa.back();
}

}  // namespace

void release_nfa(const ridfa_program *P) {
    for (auto &d : P->dev_nfa) {
        cudaSetDevice(d.device);
        if (d.base) cudaFree(d.base);
        if (d.scratch) cudaFree(d.scratch);
        if (d.h_accept_pinned) cudaFreeHost(d.h_accept_pinned);
    }
    (void)cudaGetLastError();
}

}  // namespace ridfa

extern "C" int ridfa_recognize_nfa(const ridfa_program *prog, const uint8_t *d_text, size_t len, uint32_t n_chunks,
                                   uint8_t *h_accept, uint32_t *d_sets, void *stream) {
    using namespace ridfa;
    if (!prog || !h_accept) return RIDFA_E_ARG;
    const HostNfa &H = prog->nfa;
    if (H.n == 0) return RIDFA_E_UNSUPPORTED;
    if (len == 0) {
        if (n_chunks != 0) return RIDFA_E_CHUNKS;
        *h_accept = (H.finals[0] & 1u) ? 1 : 0;           // q0 in F: the empty word is in L
        return RIDFA_OK;
    }
    if (!d_text) return RIDFA_E_ARG;
    if (n_chunks == 0 || n_chunks > len) return RIDFA_E_CHUNKS;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lock(prog->mu);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    int err = RIDFA_OK;
    DeviceNfa *D = nfa_device(prog, dev, &err);
    if (!D) return err;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t rel_bytes = static_cast<size_t>(H.n) * H.nw * 4;
    const uint64_t c = n_chunks;
    const uint64_t g1 = (c + kNfaCompose - 1) / kNfaCompose;
    auto al = [](size_t x) { return (x + 255) & ~static_cast<size_t>(255); };
    const size_t own = d_sets ? 0 : al(c * rel_bytes);
    const size_t need = own + 2 * al(g1 * rel_bytes) + 256;
    if (D->scratch_bytes < need) {
        if (D->scratch) cudaFree(D->scratch);
        D->scratch = nullptr;
        D->scratch_bytes = 0;
        e = cudaMalloc(&D->scratch, need);
        if (e != cudaSuccess) {
            D->scratch = nullptr;
            return cuda_fail(e);
        }
        D->scratch_bytes = need;
    }
    uint8_t *base = static_cast<uint8_t *>(D->scratch);
    uint32_t *rel = d_sets ? d_sets : reinterpret_cast<uint32_t *>(base);
    uint32_t *lvl0 = reinterpret_cast<uint32_t *>(base + own);
    uint32_t *lvl1 = reinterpret_cast<uint32_t *>(base + own + al(g1 * rel_bytes));
    uint8_t *d_acc = base + own + 2 * al(g1 * rel_bytes);
    NfaArgs a{D->classmap, D->follow, D->cls, d_text, len, n_chunks, H.n, H.n_classes, rel};
    {
        NvtxRange range("ridfa nfa variant");
        switch (H.nw) {
            case 1: e = nfa_launch<1>(a, sms, lvl0, lvl1, D->finals, d_acc, st); break;
            case 2: e = nfa_launch<2>(a, sms, lvl0, lvl1, D->finals, d_acc, st); break;
            case 3: e = nfa_launch<3>(a, sms, lvl0, lvl1, D->finals, d_acc, st); break;
            default: e = nfa_launch<4>(a, sms, lvl0, lvl1, D->finals, d_acc, st); break;
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(D->h_accept_pinned, d_acc, 1, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    *h_accept = D->h_accept_pinned[0];
    return RIDFA_OK;
}

// Per-chunk join states: the full scan of the join (Sec. 3.2) instead of its reduction.
//
// For every chunk i the entry set E_i = if_min(PLAS_{i-1}) ∩ PIS_i (E_1 = {q0's slot} ∩ PIS_1),
// i.e. the interface slots through which chunk i is entered on the way to PLAS_i = λ_i(E_i), and
// the first chunk whose PLAS_i is empty (the text is rejected there).  The recurrence
// PLAS_i = PLAS_{i-1} · M_i runs over the distinct end states D_i of each chunk (M_i as in the
// join kernel), in three launches:
//   1. one thread per segment of kScanSeg boundaries: the product of the segment's M_i;
//   2. one block: the product of each thread's run of segments, then the incoming PLAS vector of
//      every segment (vector × matrix, sequential over 256 thread totals, then per segment);
//   3. one thread per segment: walk its boundaries from the incoming vector, writing E_i.
// When some chunk has more than 32 distinct end states, one block propagates the k-bit sets
// chunk by chunk instead (exact, sequential in c).
#include <cuda_runtime.h>

#include <cstdint>

#include "ridfa_internal.h"
#include "ridfa_kernels.cuh"

namespace ridfa {
namespace {

constexpr uint32_t kScanSeg = 64;          // boundaries per thread of launches 1 and 3
constexpr uint32_t kScanThreads = 256;
constexpr uint32_t kScanWords = 1 + kMaxD; // a product: nrows (0xFFFFFFFF = identity) + rows

struct ScanArgs {
    Automaton A;
    const uint16_t *maps;      // [c][k]
    uint32_t c, nseg;
    uint32_t *prods;           // [nseg][kScanWords]
    uint32_t *vin;             // [nseg]: PLAS before the segment's first boundary, over its D
    uint32_t *entry;           // [c][kw], or null
    unsigned long long *reject;
    uint32_t *status;
};

// Distinct defined values of a row, ascending (0xFFFFFFFF when more than kMaxD).
__device__ uint32_t row_distinct(const uint16_t *row, uint32_t k, uint16_t *D) {
    uint32_t cnt = 0;
    for (uint32_t a = 0; a < k; ++a) {
        const uint16_t v = row[a];
        if (v == kUndef) continue;
        uint32_t j = 0;
        while (j < cnt && D[j] < v) ++j;
        if (j < cnt && D[j] == v) continue;
        if (cnt == kMaxD) return 0xFFFFFFFFu;
        for (uint32_t t = cnt; t > j; --t) D[t] = D[t - 1];
        D[j] = v;
        ++cnt;
    }
    return cnt;
}

__device__ __forceinline__ uint32_t row_index(const uint16_t *D, uint32_t m, uint16_t v) {
    for (uint32_t j = 0; j < m; ++j)
        if (D[j] == v) return j;
    return 0xFFFFFFFFu;
}

// Entry slots of a chunk from the previous chunk's PLAS (bits v over Dp): if_min(PLAS) ∩ PIS.
// Writes them to out (kw words) when non-null and returns the next PLAS as bits over Dc.
__device__ uint32_t step_plas(const Automaton &A, const uint16_t *row, const uint16_t *Dp, uint32_t v,
                              const uint16_t *Dc, uint32_t mc, uint32_t *out, bool *bad) {
    uint32_t next = 0;
    for (uint32_t w = 0; w < A.kw; ++w) {
        uint32_t e = 0;
        for (uint32_t bits = v; bits; bits &= bits - 1)
            e |= A.ifmask[static_cast<uint64_t>(Dp[__ffs(bits) - 1]) * A.kw + w];
        uint32_t live = 0;
        for (uint32_t bits = e; bits; bits &= bits - 1) {
            const uint32_t a = w * 32 + __ffs(bits) - 1;
            const uint16_t s = row[a];
            if (s == kUndef) continue;
            live |= 1u << (a & 31);
            const uint32_t y = row_index(Dc, mc, s);
            if (y == 0xFFFFFFFFu) *bad = true;
            else next |= 1u << y;
        }
        if (out) out[w] = live;
    }
    return next;
}

__device__ uint32_t vec_times(uint32_t v, const uint32_t *prod) {   // v · P (P may be identity)
    if (prod[0] == 0xFFFFFFFFu) return v;
    uint32_t out = 0;
    for (uint32_t bits = v; bits; bits &= bits - 1) out |= prod[1 + __ffs(bits) - 1];
    return out;
}

__device__ void prod_compose(uint32_t *a, const uint32_t *b) {       // a <- a · b
    if (b[0] == 0xFFFFFFFFu) return;
    if (a[0] == 0xFFFFFFFFu) {
        for (uint32_t r = 0; r < kScanWords; ++r) a[r] = b[r];
        return;
    }
    for (uint32_t x = 0; x < a[0]; ++x) a[1 + x] = vec_times(a[1 + x], b);
}

// Launch 1: the product of each segment's transfer matrices.
__global__ void __launch_bounds__(kScanThreads) rid_scan_products(ScanArgs p) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.nseg) return;
    const Automaton &A = p.A;
    const uint64_t b0 = 1 + static_cast<uint64_t>(t) * kScanSeg;
    const uint64_t b1 = b0 + kScanSeg < p.c ? b0 + kScanSeg : p.c;
    uint16_t Dp[kMaxD], Dc[kMaxD];
    uint32_t *P = p.prods + static_cast<uint64_t>(t) * kScanWords;
    uint32_t mp = row_distinct(p.maps + (b0 - 1) * A.k, A.k, Dp);
    if (mp == 0xFFFFFFFFu) {
        atomicOr(p.status, kStatusWide);
        return;
    }
    // rows stay over the segment's first D; the columns move on to each next D
    uint32_t rows[kMaxD];
    for (uint32_t x = 0; x < mp; ++x) rows[x] = 1u << x;
    uint32_t mcur = mp;
    bool bad = false;
    for (uint64_t i = b0; i < b1; ++i) {
        const uint16_t *row = p.maps + i * A.k;
        const uint32_t mc = row_distinct(row, A.k, Dc);
        if (mc == 0xFFFFFFFFu) {
            atomicOr(p.status, kStatusWide);
            return;
        }
        uint32_t M[kMaxD];                       // row z of M_i: D_{i-1}[z] -> bits over D_i
        for (uint32_t z = 0; z < mcur; ++z) M[z] = step_plas(A, row, Dp, 1u << z, Dc, mc, nullptr, &bad);
        for (uint32_t x = 0; x < mp; ++x) {
            uint32_t out = 0;
            for (uint32_t bits = rows[x]; bits; bits &= bits - 1) out |= M[__ffs(bits) - 1];
            rows[x] = out;
        }
        for (uint32_t j = 0; j < mc; ++j) Dp[j] = Dc[j];
        mcur = mc;
    }
    if (bad) atomicOr(p.status, kStatusBad);
    P[0] = mp;
    for (uint32_t x = 0; x < kMaxD; ++x) P[1 + x] = x < mp ? rows[x] : 0;
}

// Launch 2 (one block): incoming PLAS vector of every segment, and chunk 0's entry set.
__global__ void __launch_bounds__(kScanThreads) rid_scan_prefix(ScanArgs p) {
    __shared__ uint32_t s_tot[kScanThreads][kScanWords];
    __shared__ uint32_t s_in[kScanThreads];
    const Automaton &A = p.A;
    const uint32_t tid = threadIdx.x;
    const uint32_t per = (p.nseg + kScanThreads - 1) / kScanThreads;
    const uint32_t s0 = tid * per, s1 = min(p.nseg, s0 + per);
    s_tot[tid][0] = 0xFFFFFFFFu;
    for (uint32_t sg = s0; sg < s1; ++sg) prod_compose(s_tot[tid], p.prods + static_cast<uint64_t>(sg) * kScanWords);
    __syncthreads();
    if (tid == 0) {
        // PLAS_1 = {λ_1(q0)} over D_1 (chunk 0 here); E_1 = {q0's slot} if that move is defined
        uint16_t D0[kMaxD];
        const uint32_t m0 = row_distinct(p.maps, A.k, D0);
        const uint16_t v0 = p.maps[A.q0_slot];
        uint32_t v = 0;
        if (v0 != kUndef && m0 != 0xFFFFFFFFu) {
            const uint32_t x = row_index(D0, m0, v0);
            if (x != 0xFFFFFFFFu) v = 1u << x;
        }
        if (p.entry)
            for (uint32_t w = 0; w < A.kw; ++w)
                p.entry[w] = (v0 != kUndef && (A.q0_slot >> 5) == w) ? (1u << (A.q0_slot & 31)) : 0u;
        if (v0 == kUndef) atomicMin(p.reject, 0ull);
        for (uint32_t t = 0; t < kScanThreads; ++t) {
            s_in[t] = v;
            v = vec_times(v, s_tot[t]);
        }
    }
    __syncthreads();
    uint32_t v = s_in[tid];
    for (uint32_t sg = s0; sg < s1; ++sg) {
        p.vin[sg] = v;
        v = vec_times(v, p.prods + static_cast<uint64_t>(sg) * kScanWords);
    }
}

// Launch 3: walk each segment's boundaries from its incoming vector.
__global__ void __launch_bounds__(kScanThreads) rid_scan_walk(ScanArgs p) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.nseg) return;
    const Automaton &A = p.A;
    const uint64_t b0 = 1 + static_cast<uint64_t>(t) * kScanSeg;
    const uint64_t b1 = b0 + kScanSeg < p.c ? b0 + kScanSeg : p.c;
    uint16_t Dp[kMaxD], Dc[kMaxD];
    row_distinct(p.maps + (b0 - 1) * A.k, A.k, Dp);
    uint32_t v = p.vin[t];
    bool bad = false;
    for (uint64_t i = b0; i < b1; ++i) {
        const uint16_t *row = p.maps + i * A.k;
        const uint32_t mc = row_distinct(row, A.k, Dc);
        const uint32_t nv = step_plas(A, row, Dp, v, Dc, mc, p.entry ? p.entry + i * A.kw : nullptr, &bad);
        if (nv == 0 && v != 0) atomicMin(p.reject, static_cast<unsigned long long>(i));
        v = nv;
        for (uint32_t j = 0; j < mc; ++j) Dp[j] = Dc[j];
    }
    if (bad) atomicOr(p.status, kStatusBad);
}

// Some chunk has more than kMaxD end states: one block propagates the k-bit slot sets.
__global__ void __launch_bounds__(kScanThreads) rid_scan_wide(ScanArgs p) {
    __shared__ uint32_t s_vec[RIDFA_MAX_SLOTS / 32], s_nvec[RIDFA_MAX_SLOTS / 32];
    __shared__ uint32_t s_any;
    const Automaton &A = p.A;
    const uint32_t tid = threadIdx.x;
    for (uint32_t w = tid; w < A.kw; w += blockDim.x) s_vec[w] = (A.q0_slot >> 5) == w ? 1u << (A.q0_slot & 31) : 0u;
    __syncthreads();
    for (uint64_t i = 0; i < p.c; ++i) {
        const uint16_t *row = p.maps + i * A.k;
        for (uint32_t w = tid; w < A.kw; w += blockDim.x) s_nvec[w] = 0;
        if (tid == 0) s_any = 0;
        __syncthreads();
        // entry set E_i = s_vec ∩ PIS_i; next slots = if_min(λ_i(E_i))
        for (uint32_t a = tid; a < A.k; a += blockDim.x) {
            const bool in = (s_vec[a >> 5] >> (a & 31)) & 1;
            if (!in || row[a] == kUndef) continue;
            s_any = 1;
            for (uint32_t w = 0; w < A.kw; ++w) {
                const uint32_t m = A.ifmask[static_cast<uint64_t>(row[a]) * A.kw + w];
                if (m) atomicOr(&s_nvec[w], m);
            }
        }
        __syncthreads();
        if (p.entry)
            for (uint32_t w = tid; w < A.kw; w += blockDim.x) {
                uint32_t live = 0;
                for (uint32_t b = 0; b < 32; ++b) {
                    const uint32_t a = w * 32 + b;
                    if (a < A.k && ((s_vec[w] >> b) & 1) && row[a] != kUndef) live |= 1u << b;
                }
                p.entry[i * A.kw + w] = live;
            }
        if (tid == 0 && !s_any) atomicMin(p.reject, static_cast<unsigned long long>(i));
        __syncthreads();
        for (uint32_t w = tid; w < A.kw; w += blockDim.x) s_vec[w] = s_nvec[w];
        __syncthreads();
    }
}

}  // namespace
}  // namespace ridfa

extern "C" int ridfa_join_scan(const ridfa_program *prog, const uint16_t *d_maps, uint32_t n_chunks,
                               uint32_t *d_entry, int64_t *h_reject, void *stream) {
    using namespace ridfa;
    if (!prog || !d_maps || !h_reject || n_chunks == 0) return RIDFA_E_ARG;
    const HostAutomaton &H = prog->rid;
    if (H.k > RIDFA_MAX_SLOTS) return RIDFA_E_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    const DeviceAutomaton *D = nullptr;
    {
        std::lock_guard<std::mutex> lock(prog->mu);
        int err = RIDFA_OK;
        D = device_copy(prog, false, dev, &err);
        if (!D) return err;
    }
    const uint32_t c = n_chunks;
    const uint32_t nseg = c > 1 ? (c - 1 + kScanSeg - 1) / kScanSeg : 0;
    const size_t bytes = 256 + static_cast<size_t>(nseg) * (kScanWords + 1) * 4;
    uint8_t *scratch = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void **>(&scratch), bytes, st);
    if (e != cudaSuccess) return cuda_fail(e);
    unsigned long long *reject = reinterpret_cast<unsigned long long *>(scratch);
    uint32_t *status = reinterpret_cast<uint32_t *>(scratch + 8);
    uint32_t *prods = reinterpret_cast<uint32_t *>(scratch + 256);
    uint32_t *vin = prods + static_cast<size_t>(nseg) * kScanWords;
    ScanArgs a{Automaton{D->trans, D->classmap, D->final_bits, D->ifmask, D->slot_state, H.n_states, H.n_classes,
                         H.k, H.kw, H.q0_slot},
               d_maps, c, nseg, prods, vin, d_entry, reject, status};
    uint64_t h[2] = {~0ull, 0};
    e = cudaMemsetAsync(scratch, 0xFF, 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, 4, st);
    if (e == cudaSuccess && nseg) {
        rid_scan_products<<<(nseg + kScanThreads - 1) / kScanThreads, kScanThreads, 0, st>>>(a);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h[1], status, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    int err = RIDFA_OK;
    if (e == cudaSuccess && (h[1] & kStatusBad)) err = RIDFA_E_STATE;
    if (e == cudaSuccess && err == RIDFA_OK) {
        if (h[1] & kStatusWide) {
            rid_scan_wide<<<1, kScanThreads, 0, st>>>(a);
        } else {
            rid_scan_prefix<<<1, kScanThreads, 0, st>>>(a);
            if (nseg) rid_scan_walk<<<(nseg + kScanThreads - 1) / kScanThreads, kScanThreads, 0, st>>>(a);
        }
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h[0], reject, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h[1], status, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && (h[1] & kStatusBad)) err = RIDFA_E_STATE;
    }
    cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return cuda_fail(e);
    if (err != RIDFA_OK) return err;
    *h_reject = h[0] == ~0ull ? -1 : static_cast<int64_t>(h[0]);
    return RIDFA_OK;
}

// Device side of the RID recognizer for sm_103a: table upload, scratch, the reach kernel, the
// join kernel and the recognize entry points of the C ABI.
//
// Reach phase (Sec. 3.2): chunk i = text[b_i, b_{i+1}), b_i = floor(i*len/c).  For every
// interface slot a the chunk automaton runs from the slot's start state; lambda_i(a) is the
// state reached at the chunk end, or undefined (0xFFFF) once a move is undefined.
// Kernel layout: a warp owns 32 consecutive chunks.
//   * Speculative phase, one chunk at a time: the warp's lanes hold the chunk's runs (slot
//     a = r*32 + lane in register r), all reading the same byte.  Every `probe` bytes the warp
//     checks whether all live runs are in one state (redux min == max); runs that merged
//     collapse into one (convergence), dead runs are dropped.
//   * Converged phase: each lane takes its own chunk and finishes the surviving run alone (or,
//     when the live runs sit in at most 8 distinct states, each of them as a run of its own, or
//     all of them together on the set path), reading the text staged in shared memory or with
//     16-byte vector loads; the chunk map row is the surviving state for the slots alive at
//     convergence and undefined for the others.
//   A chunk whose runs never merge finishes in the speculative phase.
// Few chunks: each chunk is cut into pieces run from every state (or, for large automata, from
// each piece's look-back start set) and the piece functions are composed into the chunk's row.
// Join phase (Sec. 3.2 / 3.4): let D_i be the distinct defined values of lambda_i (m_i <= 32).
// Between chunks i-1 and i the transfer is the m_{i-1} x m_i Boolean matrix
//   M_i[x][y] = exists a in if_min({D_{i-1}[x]}) with lambda_i(a) = D_i[y],
// PLAS_c = lambda_1(q0) M_2 ... M_c, and the text is accepted iff PLAS_c meets F^RID.  The
// matrices are multiplied in a chain: sequentially inside a thread, by a tree inside a block,
// and over blocks by the last block to finish (an atomic ticket).  If some chunk has more than
// 32 distinct end states, block 0 instead propagates if(PLAS_i) as a k-bit set chunk by chunk.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "ridfa_internal.h"
#include "ridfa_reach.cuh"

namespace ridfa {
// --------------------------------------------------------------------------- host side
int cuda_fail(cudaError_t e) {
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? RIDFA_E_NOMEM : RIDFA_E_CUDA;
}

int upload(const HostAutomaton &H, DeviceAutomaton &D, int dev) {
    D.device = dev;
    const size_t bt = H.trans.size() * 2, bf = H.final_bits.size() * 4, bi = H.ifmask.size() * 4,
                 bs = H.slot_state.size() * 2, ba = static_cast<size_t>(H.n_states) * 2;
    auto al = [](size_t x) { return (x + 255) & ~static_cast<size_t>(255); };
    const size_t total = al(bt) + al(256) + al(bf) + al(bi) + al(bs) + al(ba);
    uint8_t *base = nullptr;
    cudaError_t e = cudaMalloc(&base, total);
    if (e != cudaSuccess) return cuda_fail(e);
    size_t off = 0;
    D.trans = reinterpret_cast<uint16_t *>(base + off); off += al(bt);
    D.classmap = base + off; off += al(256);
    D.final_bits = reinterpret_cast<uint32_t *>(base + off); off += al(bf);
    D.ifmask = reinterpret_cast<uint32_t *>(base + off); off += al(bi);
    D.slot_state = reinterpret_cast<uint16_t *>(base + off); off += al(bs);
    D.all_states = reinterpret_cast<uint16_t *>(base + off); off += al(ba);
    D.bytes = total;
    std::vector<uint16_t> iota(H.n_states);
    for (uint32_t i = 0; i < H.n_states; ++i) iota[i] = static_cast<uint16_t>(i);
    e = cudaMemcpy(D.trans, H.trans.data(), bt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(D.classmap, H.classmap.data(), 256, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && bf) e = cudaMemcpy(D.final_bits, H.final_bits.data(), bf, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && bi) e = cudaMemcpy(D.ifmask, H.ifmask.data(), bi, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && bs) e = cudaMemcpy(D.slot_state, H.slot_state.data(), bs, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && ba) e = cudaMemcpy(D.all_states, iota.data(), ba, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(base);
        D = DeviceAutomaton{};
        return cuda_fail(e);
    }
    return RIDFA_OK;
}

const DeviceAutomaton *device_copy(const ridfa_program *P, bool dfa, int dev, int *err) {
    auto &vec = dfa ? P->dev_dfa : P->dev_rid;
    for (auto &d : vec)
        if (d.device == dev) return &d;
    DeviceAutomaton D;
    *err = upload(dfa ? P->dfa : P->rid, D, dev);
    if (*err != RIDFA_OK) return nullptr;
    vec.push_back(D);
    return &vec.back();
}

cudaError_t ensure_smem_cap(const void *kern, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> caps;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    size_t &cap = caps[{kern, dev}];
    if (bytes <= cap) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
    if (e == cudaSuccess) cap = bytes;
    return e;
}

int smem_optin_limit() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}


namespace {

// ------------------------------------------------------------------------------- join
struct JoinArgs {
    Automaton A;
    uint32_t c;
    const uint16_t *maps;
    const uint32_t *dinfo;
    uint32_t *status;
    uint32_t *partials;       // [gridDim.x][2 + kMaxD]
    uint32_t *ticket;
    uint8_t *accept;
    uint32_t per_thread;      // boundaries per thread
    ridfa_shard_summary *summary;   // non-null: write the shard's relation instead of accept
};

// Distinct defined values of lambda_i, ascending (at most kMaxD; caller checked m <= kMaxD).
__device__ uint32_t distinct_of(const JoinArgs &p, uint32_t i, uint16_t *D) {
    const uint32_t info = p.dinfo[i];
    const uint32_t m = info >> 16;
    if (m <= 1) {
        D[0] = static_cast<uint16_t>(info & 0xFFFF);
        return m;
    }
    const uint16_t *row = p.maps + static_cast<uint64_t>(i) * p.A.k;
    uint32_t cnt = 0;
    for (uint32_t a = 0; a < p.A.k; ++a) {
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

__device__ __forceinline__ uint32_t index_of(const uint16_t *D, uint32_t m, uint16_t v) {
    for (uint32_t j = 0; j < m; ++j)
        if (D[j] == v) return j;
    return 0xFFFFFFFFu;
}

// Row x of M_i: bits y with lambda_i(a) = D_i[y] for some slot a in if_min({D_{i-1}[x]}).
__device__ uint32_t transfer_row(const JoinArgs &p, uint32_t i, uint16_t d_prev, const uint16_t *D,
                                 uint32_t m, bool *bad) {
    const uint32_t *mask = p.A.ifmask + static_cast<uint64_t>(d_prev) * p.A.kw;
    const uint16_t *row = p.maps + static_cast<uint64_t>(i) * p.A.k;
    uint32_t out = 0;
    for (uint32_t w = 0; w < p.A.kw; ++w) {
        uint32_t bits = mask[w];
        while (bits) {
            const uint32_t a = w * 32 + __ffs(bits) - 1;
            bits &= bits - 1;
            const uint16_t v = row[a];
            if (v == kUndef) continue;
            const uint32_t y = index_of(D, m, v);
            if (y == 0xFFFFFFFFu) *bad = true;
            else out |= 1u << y;
        }
    }
    return out;
}

// Product of a thread's run of boundaries: rows over D_{s-1}, columns over D_{e-1}.
struct Prod {
    uint32_t nrows;           // 0xFFFFFFFF = identity (no boundary)
    uint32_t rows[kMaxD];
};

__device__ void compose(Prod &a, const Prod &b) {   // a <- a x b
    if (b.nrows == 0xFFFFFFFFu) return;
    if (a.nrows == 0xFFFFFFFFu) {
        a = b;
        return;
    }
    for (uint32_t x = 0; x < a.nrows; ++x) {
        uint32_t bits = a.rows[x], out = 0;
        while (bits) {
            const uint32_t z = __ffs(bits) - 1;
            bits &= bits - 1;
            out |= b.rows[z];
        }
        a.rows[x] = out;
    }
}

__device__ bool is_final(const Automaton &A, uint32_t s) {
    return s < A.n && ((A.final_bits[s >> 5] >> (s & 31)) & 1);
}

// Shard summary when some chunk has more than kMaxD distinct end states (block 0 alone):
// for every distinct state x the shard's first chunk ends in, propagate if_min({x}) chunk by
// chunk and record the end states reached, as bits over the last chunk's distinct end states.
__device__ void summary_wide(const JoinArgs &p, uint32_t *s_vec, uint32_t *s_nvec) {
    const Automaton &A = p.A;
    const uint32_t tid = threadIdx.x;
    ridfa_shard_summary *S = p.summary;
    __shared__ uint16_t s_out[RIDFA_MAX_SLOTS];
    __shared__ uint32_t s_nout, s_bits[RIDFA_MAX_SLOTS / 32];
    const uint16_t *row0 = p.maps;
    const uint16_t *last = p.maps + static_cast<uint64_t>(p.c - 1) * A.k;
    if (tid == 0) {
        // distinct defined end states of the last chunk, ascending
        uint32_t n = 0;
        for (uint32_t a = 0; a < A.k; ++a) {
            const uint16_t v = last[a];
            if (v == kUndef) continue;
            uint32_t j = 0;
            while (j < n && s_out[j] < v) ++j;
            if (j < n && s_out[j] == v) continue;
            for (uint32_t t = n; t > j; --t) s_out[t] = s_out[t - 1];
            s_out[j] = v;
            ++n;
        }
        s_nout = n;
        S->k = A.k;
        S->n_out = n;
    }
    __syncthreads();
    for (uint32_t a = tid; a < RIDFA_MAX_SLOTS; a += blockDim.x) {
        S->out_state[a] = a < s_nout ? s_out[a] : kUndef;
        S->entry[a] = a < A.k ? row0[a] : kUndef;
        for (uint32_t w = 0; w < RIDFA_MAX_SLOTS / 32; ++w) S->reach[a][w] = 0;
    }
    __syncthreads();
    for (uint32_t a0 = 0; a0 < A.k; ++a0) {
        const uint16_t x = row0[a0];
        if (x == kUndef) continue;
        bool seen = false;                    // handled with an earlier slot of the same state
        for (uint32_t b = 0; b < a0 && !seen; ++b) seen = row0[b] == x;
        if (seen) continue;
        if (tid < RIDFA_MAX_SLOTS / 32) s_bits[tid] = 0;
        __syncthreads();
        if (p.c == 1) {
            if (tid == 0)
                for (uint32_t y = 0; y < s_nout; ++y)
                    if (s_out[y] == x) s_bits[y >> 5] |= 1u << (y & 31);
        } else {
            for (uint32_t w = tid; w < A.kw; w += blockDim.x) s_vec[w] = A.ifmask[static_cast<uint64_t>(x) * A.kw + w];
            __syncthreads();
            for (uint32_t i = 1; i + 1 < p.c; ++i) {
                for (uint32_t w = tid; w < A.kw; w += blockDim.x) s_nvec[w] = 0;
                __syncthreads();
                const uint16_t *row = p.maps + static_cast<uint64_t>(i) * A.k;
                for (uint32_t a = tid; a < A.k; a += blockDim.x) {
                    if (!((s_vec[a >> 5] >> (a & 31)) & 1)) continue;
                    const uint16_t v = row[a];
                    if (v == kUndef) continue;
                    for (uint32_t w = 0; w < A.kw; ++w) {
                        const uint32_t m = A.ifmask[static_cast<uint64_t>(v) * A.kw + w];
                        if (m) atomicOr(&s_nvec[w], m);
                    }
                }
                __syncthreads();
                for (uint32_t w = tid; w < A.kw; w += blockDim.x) s_vec[w] = s_nvec[w];
                __syncthreads();
            }
            for (uint32_t a = tid; a < A.k; a += blockDim.x) {
                if (!((s_vec[a >> 5] >> (a & 31)) & 1) || last[a] == kUndef) continue;
                for (uint32_t y = 0; y < s_nout; ++y)
                    if (s_out[y] == last[a]) atomicOr(&s_bits[y >> 5], 1u << (y & 31));
            }
        }
        __syncthreads();
        for (uint32_t a = tid; a < A.k; a += blockDim.x)
            if (row0[a] == x)
                for (uint32_t w = 0; w < RIDFA_MAX_SLOTS / 32; ++w) S->reach[a][w] = s_bits[w];
        __syncthreads();
    }
}

// Shard summary from the chain product (thread 0 of the last block): tot maps the first chunk's
// distinct end states D_1 to the last chunk's D_c.
__device__ void summary_matrix(const JoinArgs &p, const Prod &tot) {
    const Automaton &A = p.A;
    ridfa_shard_summary *S = p.summary;
    uint16_t D0[kMaxD], Dl[kMaxD];
    const uint32_t m0 = distinct_of(p, 0, D0);
    const uint32_t ml = distinct_of(p, p.c - 1, Dl);
    if (m0 == 0xFFFFFFFFu || ml == 0xFFFFFFFFu || (p.c > 1 && tot.nrows == 0xFFFFFFFFu)) {
        atomicOr(p.status, kStatusBad);
        return;
    }
    S->k = A.k;
    S->n_out = ml;
    for (uint32_t y = 0; y < RIDFA_MAX_SLOTS; ++y) S->out_state[y] = y < ml ? Dl[y] : kUndef;
    for (uint32_t a = 0; a < RIDFA_MAX_SLOTS; ++a) {
        const uint16_t x = a < A.k ? p.maps[a] : kUndef;
        S->entry[a] = x;
        uint32_t bits = 0;
        if (x != kUndef) {
            const uint32_t xi = index_of(D0, m0, x);
            if (xi == 0xFFFFFFFFu) atomicOr(p.status, kStatusBad);
            else bits = p.c == 1 ? (1u << xi) : tot.rows[xi];
        }
        S->reach[a][0] = bits;
        for (uint32_t w = 1; w < RIDFA_MAX_SLOTS / 32; ++w) S->reach[a][w] = 0;
    }
}

__global__ void __launch_bounds__(kJoinThreads) rid_join_kernel(JoinArgs p) {
    __shared__ Prod s_prod[kJoinThreads];
    __shared__ bool s_last;
    __shared__ uint32_t s_vec[RIDFA_MAX_SLOTS / 32], s_nvec[RIDFA_MAX_SLOTS / 32];
    const uint32_t tid = threadIdx.x;
    const Automaton &A = p.A;
    const uint32_t status0 = *reinterpret_cast<volatile uint32_t *>(p.status);

    if (status0 & kStatusWide) {
        // some chunk has more than kMaxD distinct end states: block 0 propagates if(PLAS_i)
        if (blockIdx.x != 0) return;
        if (p.summary) {
            summary_wide(p, s_vec, s_nvec);
            return;
        }
        const uint16_t *row0 = p.maps;
        const uint16_t v0 = row0[A.q0_slot];
        if (p.c == 1 || v0 == kUndef) {
            if (tid == 0) *p.accept = (v0 != kUndef && is_final(A, v0)) ? 1 : 0;
            return;
        }
        for (uint32_t w = tid; w < A.kw; w += blockDim.x)
            s_vec[w] = A.ifmask[static_cast<uint64_t>(v0) * A.kw + w];
        __syncthreads();
        for (uint32_t i = 1; i + 1 < p.c; ++i) {
            for (uint32_t w = tid; w < A.kw; w += blockDim.x) s_nvec[w] = 0;
            __syncthreads();
            const uint16_t *row = p.maps + static_cast<uint64_t>(i) * A.k;
            for (uint32_t a = tid; a < A.k; a += blockDim.x) {
                if (!((s_vec[a >> 5] >> (a & 31)) & 1)) continue;
                const uint16_t v = row[a];
                if (v == kUndef) continue;
                for (uint32_t w = 0; w < A.kw; ++w) {
                    const uint32_t m = A.ifmask[static_cast<uint64_t>(v) * A.kw + w];
                    if (m) atomicOr(&s_nvec[w], m);
                }
            }
            __syncthreads();
            for (uint32_t w = tid; w < A.kw; w += blockDim.x) s_vec[w] = s_nvec[w];
            __syncthreads();
        }
        __shared__ uint32_t s_acc;
        if (tid == 0) s_acc = 0;
        __syncthreads();
        const uint16_t *last = p.maps + static_cast<uint64_t>(p.c - 1) * A.k;
        for (uint32_t a = tid; a < A.k; a += blockDim.x)
            if (((s_vec[a >> 5] >> (a & 31)) & 1) && last[a] != kUndef && is_final(A, last[a]))
                s_acc = 1;
        __syncthreads();
        if (tid == 0) *p.accept = s_acc ? 1 : 0;
        return;
    }

    // ---- chain product of the transfer matrices M_1 .. M_{c-1} (0-based boundaries)
    const uint64_t nbound = p.c > 0 ? p.c - 1 : 0;
    const uint64_t b0 = 1 + (static_cast<uint64_t>(blockIdx.x) * blockDim.x + tid) * p.per_thread;
    const uint64_t b1 = min(b0 + p.per_thread, nbound + 1);
    Prod P;
    P.nrows = 0xFFFFFFFFu;
    bool bad = false;
    if (b0 < b1) {
        uint16_t Dp[kMaxD], Dc[kMaxD];
        uint32_t mp = distinct_of(p, static_cast<uint32_t>(b0 - 1), Dp);
        P.nrows = mp;
        for (uint32_t x = 0; x < mp; ++x) P.rows[x] = 1u << x;
        for (uint64_t i = b0; i < b1; ++i) {
            const uint32_t mc = distinct_of(p, static_cast<uint32_t>(i), Dc);
            uint32_t M[kMaxD];
            for (uint32_t z = 0; z < mp; ++z) M[z] = transfer_row(p, static_cast<uint32_t>(i), Dp[z], Dc, mc, &bad);
            for (uint32_t x = 0; x < P.nrows; ++x) {
                uint32_t bits = P.rows[x], out = 0;
                while (bits) {
                    const uint32_t z = __ffs(bits) - 1;
                    bits &= bits - 1;
                    out |= M[z];
                }
                P.rows[x] = out;
            }
            for (uint32_t j = 0; j < mc; ++j) Dp[j] = Dc[j];
            mp = mc;
        }
    }
    if (bad) atomicOr(p.status, kStatusBad);
    s_prod[tid] = P;
    __syncthreads();
    for (uint32_t stride = 1; stride < blockDim.x; stride *= 2) {
        if ((tid % (2 * stride)) == 0 && tid + stride < blockDim.x) compose(s_prod[tid], s_prod[tid + stride]);
        __syncthreads();
    }
    uint32_t *mine = p.partials + static_cast<uint64_t>(blockIdx.x) * (1 + kMaxD);
    if (tid == 0) {
        mine[0] = s_prod[0].nrows;
        for (uint32_t x = 0; x < kMaxD; ++x) mine[1 + x] = s_prod[0].rows[x];
        __threadfence();
        const uint32_t t = atomicAdd(p.ticket, 1);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // ---- last block: compose the block products in order (256 at a time, tree in shared
    // memory), then the head lambda_1(q0) and the acceptance test on D_c
    Prod tot;
    tot.nrows = 0xFFFFFFFFu;
    for (uint32_t base = 0; base < gridDim.x; base += blockDim.x) {
        Prod x;
        x.nrows = 0xFFFFFFFFu;
        if (base + tid < gridDim.x) {
            const volatile uint32_t *q = p.partials + static_cast<uint64_t>(base + tid) * (1 + kMaxD);
            x.nrows = q[0];
            if (x.nrows != 0xFFFFFFFFu)
                for (uint32_t r = 0; r < x.nrows; ++r) x.rows[r] = q[1 + r];
        }
        __syncthreads();
        s_prod[tid] = x;
        __syncthreads();
        for (uint32_t stride = 1; stride < blockDim.x; stride *= 2) {
            if ((tid % (2 * stride)) == 0 && tid + stride < blockDim.x) compose(s_prod[tid], s_prod[tid + stride]);
            __syncthreads();
        }
        if (tid == 0) compose(tot, s_prod[0]);
        __syncthreads();
    }
    if (tid != 0) return;
    *p.ticket = 0;   // ready for the next launch on this scratch
    if (p.summary) {
        summary_matrix(p, tot);
        return;
    }
    const uint16_t v0 = p.maps[A.q0_slot];
    uint8_t acc = 0;
    if (v0 != kUndef) {
        if (p.c == 1) {
            acc = is_final(A, v0) ? 1 : 0;
        } else {
            uint16_t D0[kMaxD], Dl[kMaxD];
            const uint32_t m0 = distinct_of(p, 0, D0);
            const uint32_t x0 = index_of(D0, m0, v0);
            const uint32_t ml = distinct_of(p, p.c - 1, Dl);
            if (x0 == 0xFFFFFFFFu || tot.nrows == 0xFFFFFFFFu || ml == 0xFFFFFFFFu) {
                atomicOr(p.status, kStatusBad);
            } else {
                const uint32_t bits = tot.rows[x0];
                for (uint32_t y = 0; y < ml; ++y)
                    if (((bits >> y) & 1) && is_final(A, Dl[y])) acc = 1;
            }
        }
    }
    *p.accept = acc;
}

// ------------------------------------------------------------ intra-chunk speculation (pieces)
// One warp per piece, the whole piece in lockstep: lanes hold the runs from every state (state
// a = 32*r + lane in register r), every lane reads the same 16 bytes (one transaction), the
// class lookup is the lane's own replica, and registers whose runs all died are skipped.  The
// piece's row (f_j(x) for every state x, kUndef when the run dies) is written at the end.
template <int R, class LUT>
__global__ void __launch_bounds__(256) rid_piece_kernel(ReachArgs p, int table_in_smem) {
    extern __shared__ __align__(128) uint8_t smem[];
    const Automaton &A = p.A;
    LUT T;
    T.setup(A, smem, static_cast<uint32_t>(table_in_smem));
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t dead = T.enc(A.n);
    const uint64_t warp0 = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t j = warp0; j < p.c; j += n_warps) {
        uint32_t s[R];
        uint32_t live = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t a = r * 32 + lane;
            s[r] = a < A.k ? T.enc(__ldg(A.slot_state + a)) : dead;
            if (r * 32 < static_cast<int>(A.k)) live |= 1u << r;
        }
        uint64_t pos = chunk_begin(j, p.len, p.c);
        const uint64_t end = chunk_begin(j + 1, p.len, p.c);
        auto step = [&](uint32_t b) {
            const uint32_t c = T.cls_of(b);
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (live & (1u << r)) s[r] = T.next(s[r], c);
        };
        while (pos < end && (reinterpret_cast<uintptr_t>(p.text + pos) & 15)) step(__ldg(p.text + pos++));
        while (pos + 16 <= end && live) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p.text + pos));
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const uint32_t c = T.cls_at(w[q >> 2], q & 3);
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (live & (1u << r)) s[r] = T.next(s[r], c);
            }
            pos += 16;
            uint32_t nl = 0;
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (__any_sync(kFull, s[r] != dead)) nl |= 1u << r;
            live &= nl;
        }
        while (pos < end && live) step(__ldg(p.text + pos++));
        uint16_t *row = p.maps + j * p.stride;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t a = r * 32 + lane;
            if (a < A.k) row[a] = s[r] == dead ? kUndef : static_cast<uint16_t>(T.id(s[r]));
        }
    }
}

template <int R, class LUT>
cudaError_t piece_one(const ReachArgs &a, int grid, size_t smem, int tis, cudaStream_t st) {
    auto kern = rid_piece_kernel<R, LUT>;
    cudaError_t e = ensure_smem_cap(reinterpret_cast<const void *>(kern), smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 256, smem, st>>>(a, tis);
    return cudaGetLastError();
}

template <class LUT>
cudaError_t piece_r(int R, const ReachArgs &a, int grid, size_t smem, int tis, cudaStream_t st) {
    switch (R) {
        case 1: return piece_one<1, LUT>(a, grid, smem, tis, st);
        case 2: return piece_one<2, LUT>(a, grid, smem, tis, st);
        case 4: return piece_one<4, LUT>(a, grid, smem, tis, st);
        default: return piece_one<8, LUT>(a, grid, smem, tis, st);
    }
}

// Look-back start sets for pieces (automata too large to run every piece from every state):
// inside chunk i, the run's state at piece j's first byte b is delta(y, text[w, b)) for the state
// y it had at w, for any w from the chunk start b_i to b, so it lies in delta(P, text[w, b)), the
// states that survive the window from every state.  One warp per piece: for windows of 16, 64,
// 256, ... bytes back (never before b_i) every state is run over the window, 32 at a time, and the
// distinct live end states are gathered; once at most 32 remain they are the piece's start set.
// The first piece of a chunk starts from the interface slots (k <= 32).  A piece whose set never
// falls to 32 has its whole function written here instead: every state run over the piece.
struct LookbackArgs {
    Automaton A;              // A.slot_state[0..k): the interface slots' start states
    const uint8_t *text;
    uint64_t len;
    uint64_t pieces;          // c * spc
    uint32_t spc;             // pieces per chunk
    uint16_t *slots;          // [pieces][32] start states, 0xFFFF = none
    uint16_t *F;              // [pieces][A.n] piece functions, pre-filled with 0xFFFF
    uint32_t cap;             // largest start set kept (1..32)
};

constexpr int kLbRegs = 4;         // states per lane and pass of the look-back kernel

// Every state x in [s0, s0 + 32*kLbRegs) run over text[w, e) (the warp in lockstep, all lanes on
// the same byte); the live end states, in the policy's encoding, in s[].  With a two-byte table a
// lane's states take each pair of bytes in one lookup through the pair's column.
template <class LUT>
__device__ __forceinline__ void run_all_states(const LUT &T, const Automaton &A, const uint8_t *text, uint64_t w,
                                               uint64_t e, uint32_t s0, uint32_t lane, uint32_t dead,
                                               uint32_t (&s)[kLbRegs]) {
#pragma unroll
    for (int r = 0; r < kLbRegs; ++r) {
        const uint32_t x = s0 + r * 32 + lane;
        s[r] = x < A.n ? T.enc(x) : dead;
    }
    for (uint64_t q = w; q < e;) {
        const uint64_t stop = min(e, q + 8);
        if constexpr (has_pairs<LUT>::value) {
            for (; q + 1 < stop; q += 2) {
                const uint32_t pc = T.pair_col(T.cls_of(__ldg(text + q)), T.cls_of(__ldg(text + q + 1)));
#pragma unroll
                for (int r = 0; r < kLbRegs; ++r) s[r] = T.next_pc(s[r], pc);
            }
        }
        for (; q < stop; ++q) {
            const uint32_t c = T.cls_of(__ldg(text + q));
#pragma unroll
            for (int r = 0; r < kLbRegs; ++r) s[r] = T.next(s[r], c);
        }
        bool any = false;
#pragma unroll
        for (int r = 0; r < kLbRegs; ++r) any |= s[r] != dead;
        if (!__any_sync(kFull, any)) break;
    }
}

template <class LUT>
__global__ void __launch_bounds__(512, 2) rid_lookback_kernel(LookbackArgs p, int table_in_smem) {
    extern __shared__ __align__(128) uint8_t smem[];
    const Automaton &A = p.A;
    LUT T;
    T.setup(A, smem, static_cast<uint32_t>(table_in_smem));
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t dead = T.enc(A.n);
    const uint64_t nw = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t j = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; j < p.pieces; j += nw) {
        uint16_t *out = p.slots + j * 32;
        const uint64_t t = j % p.spc;
        if (t == 0) {
            out[lane] = lane < A.k ? A.slot_state[lane] : kUndef;
            continue;
        }
        const uint64_t b = chunk_begin(j, p.len, p.pieces);
        const uint64_t cb = chunk_begin(j - t, p.len, p.pieces);
        uint32_t mine = kUndef;             // lane g: the g-th surviving state
        bool found = false;
        for (uint64_t L = 16;; L *= 4) {
            const uint64_t w = b - cb <= L ? cb : b - L;
            uint32_t cnt = 0;
            mine = kUndef;
            bool over = false;
            for (uint32_t s0 = 0; s0 < A.n && !over; s0 += 32 * kLbRegs) {
                uint32_t s[kLbRegs];
                run_all_states(T, A, p.text, w, b, s0, lane, dead, s);
#pragma unroll
                for (int r = 0; r < kLbRegs; ++r) {
                    uint32_t v = s[r] != dead ? T.id(s[r]) : kUndef;
                    for (uint32_t g = 0; g < cnt; ++g)          // already gathered
                        if (__shfl_sync(kFull, mine, g) == v) v = kUndef;
                    while (!over) {                             // new ones, ascending
                        const uint32_t lo = __reduce_min_sync(kFull, v);
                        if (lo == kUndef) break;
                        if (cnt == p.cap) {
                            over = true;
                            break;
                        }
                        if (lane == cnt) mine = lo;
                        ++cnt;
                        if (v == lo) v = kUndef;
                    }
                }
            }
            if (!over) {
                found = true;
                break;
            }
            if (w == cb) break;
        }
        out[lane] = static_cast<uint16_t>(found ? mine : kUndef);
        if (!found) {
            // no small start set: the piece's whole function, every state over the piece
            const uint64_t e = chunk_begin(j + 1, p.len, p.pieces);
            for (uint32_t s0 = 0; s0 < A.n; s0 += 32 * kLbRegs) {
                uint32_t s[kLbRegs];
                run_all_states(T, A, p.text, b, e, s0, lane, dead, s);
#pragma unroll
                for (int r = 0; r < kLbRegs; ++r) {
                    const uint32_t x = s0 + r * 32 + lane;
                    if (x < A.n) p.F[j * A.n + x] = s[r] != dead ? static_cast<uint16_t>(T.id(s[r])) : kUndef;
                }
            }
        }
    }
}

// Piece rows of the per-piece start sets (slot g of piece j started from slots[j][g]) scattered
// into the piece functions: F_j(slots[j][g]) = row_j[g].  One thread per (piece, slot).
__global__ void rid_scatter_kernel(const uint16_t *slots, const uint16_t *rows, uint64_t pieces, uint32_t P,
                                   uint16_t *F) {
    const uint64_t t = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= pieces * 32) return;
    const uint32_t x = slots[t];
    if (x < P) F[(t >> 5) * P + x] = rows[t];
}

// A chunk cut into pieces y_i = p_1 ... p_s: each piece is run from every state x of the automaton
// (the reach kernel with every state as a slot), giving f_j(x) = δ(x, p_j) or ⊥, and
// δ(x, y_i) = f_s(...f_1(x)) because the automaton is deterministic; the chunk's map row is that
// composition applied to the interface slots' start states.  Exact, whatever the convergence.
constexpr uint32_t kComposeGroup = 32;     // functions composed per thread and level
constexpr uint32_t kMaxPieceGroups = 4;    // pieces for automata of up to 4 x 256 states
constexpr uint64_t kManyPieceLen = 1024;   // shortest piece of the many-pieces path (bytes)
constexpr uint64_t kMaxPieceBytes = 1ull << 30;   // scratch of the piece functions, at most

// One level: function g of chunk i = the composition, in order, of input functions
// [g*G, (g+1)*G) of that chunk.  One thread per (chunk, group, start state).
__global__ void rid_compose_kernel(const uint16_t *in, uint32_t in_per_chunk, uint16_t *out, uint32_t out_per_chunk,
                                   uint32_t c, uint32_t P) {
    const uint64_t t = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= static_cast<uint64_t>(c) * out_per_chunk * P) return;
    const uint32_t x = static_cast<uint32_t>(t % P);
    const uint64_t cg = t / P;
    const uint64_t g = cg % out_per_chunk, i = cg / out_per_chunk;
    const uint64_t f0 = i * in_per_chunk + g * kComposeGroup;
    const uint64_t f1 = min(f0 + kComposeGroup, (i + 1) * in_per_chunk);
    uint32_t y = x;
    for (uint64_t f = f0; f < f1 && y != kUndef; ++f) y = in[f * P + y];
    out[cg * P + x] = static_cast<uint16_t>(y);
}

// Chunk map rows from the composed functions F_i: λ_i(a) = F_i(start state of slot a), and each
// row's D_i summary (number of distinct defined end states and the smallest).  One warp per chunk.
__global__ void rid_apply_kernel(const uint16_t *F, uint32_t P, const uint16_t *slot_state, uint32_t k, uint32_t c,
                                 uint16_t *maps, uint32_t *dinfo, uint32_t *status, const uint32_t *piece_status) {
    const uint64_t i = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = threadIdx.x & 31;
    if (i == 0 && lane == 0) {
        // failures of the pieces' reach carry over; their "wide" bit does not (pieces are not joined)
        const uint32_t ps = *piece_status & (kStatusBad | kStatusTimeout);
        if (ps) atomicOr(status, ps);
    }
    if (i >= c) return;                       // whole warps leave together
    constexpr int kMaxR = RIDFA_MAX_SLOTS / 32;
    uint32_t v[kMaxR];
#pragma unroll
    for (int r = 0; r < kMaxR; ++r) {
        const uint32_t a = r * 32 + lane;
        v[r] = a < k ? F[i * P + slot_state[a]] : kUndef;
        if (a < k) maps[i * k + a] = static_cast<uint16_t>(v[r]);
    }
    uint32_t cnt = 0, first = kUndef, cur = 0;
    for (;;) {
        uint32_t m = 0xFFFFFFFFu;
#pragma unroll
        for (int r = 0; r < kMaxR; ++r)
            if (v[r] != kUndef && (cnt == 0 || v[r] > cur)) m = min(m, v[r]);
        m = __reduce_min_sync(kFull, m);
        if (m == 0xFFFFFFFFu) break;
        if (cnt == 0) first = m;
        cur = m;
        if (++cnt > kMaxD) break;
    }
    if (lane == 0) {
        if (cnt > kMaxD) {
            dinfo[i] = (0xFFu << 16) | first;
            atomicOr(status, kStatusWide);
        } else {
            dinfo[i] = cnt ? ((cnt << 16) | first) : static_cast<uint32_t>(kUndef);
        }
    }
}

struct Layout {   // scratch layout for one call
    size_t maps_off, dinfo_off, partials_off, ticket_off, status_off, accept_off, runs_off, finals_off,
        summary_off, pmaps_off, pdinfo_off, comp_off, lbslots_off, lbrows_off, total;
};

Layout layout_for(uint64_t c, uint32_t k, bool need_maps, uint32_t join_blocks, uint64_t grid_warps,
                  uint64_t pieces = 0, uint32_t P = 0, uint64_t comp_funcs = 0, bool lookback = false) {
    auto al = [](size_t x) { return (x + 255) & ~static_cast<size_t>(255); };
    Layout L{};
    size_t off = 0;
    L.ticket_off = off; off += 256;
    L.status_off = off; off += 256;
    L.accept_off = off; off += 256;
    L.partials_off = off; off += al(static_cast<size_t>(join_blocks) * (1 + kMaxD) * 4);
    L.dinfo_off = off; off += al(c * 4);
    L.runs_off = off; off += al(grid_warps * kRunsPerWarp * sizeof(RunEntry));
    L.finals_off = off; off += al(grid_warps * kFinalsPerWarp * 4);
    L.summary_off = off; off += al(sizeof(ridfa_shard_summary));
    L.pmaps_off = off; off += al(pieces * P * 2);
    L.pdinfo_off = off; off += al(pieces * 4);
    L.comp_off = off; off += 2 * al(comp_funcs * P * 2);      // two buffers of composed functions
    L.lbslots_off = off; off += lookback ? al(pieces * 32 * 2) : 0;   // look-back start sets
    L.lbrows_off = off; off += lookback ? al(pieces * 32 * 2) : 0;    // their rows
    L.maps_off = off; off += need_maps ? al(c * k * 2) : 0;
    L.total = off;
    return L;
}

DeviceScratch *scratch_for(const ridfa_program *P, int dev, size_t bytes, int *err) {
    DeviceScratch *S = nullptr;
    for (auto &s : P->scratch)
        if (s.device == dev) S = &s;
    if (!S) {
        P->scratch.push_back(DeviceScratch{});
        S = &P->scratch.back();
        S->device = dev;
        cudaError_t e = cudaMallocHost(&S->h_accept_pinned, 64);
        if (e != cudaSuccess) { *err = cuda_fail(e); return nullptr; }
        S->h_status_pinned = reinterpret_cast<uint32_t *>(S->h_accept_pinned + 16);
    }
    if (S->bytes < bytes) {
        if (S->base) {
            cudaDeviceSynchronize();
            cudaFree(S->base);
            S->base = nullptr;
            S->bytes = 0;
        }
        size_t want = std::max(bytes, static_cast<size_t>(1) << 20);
        cudaError_t e = cudaMalloc(&S->base, want);
        if (e != cudaSuccess) { *err = cuda_fail(e); return nullptr; }
        e = cudaMemset(S->base, 0, 1024);   // ticket and status start at zero
        if (e != cudaSuccess) { *err = cuda_fail(e); return nullptr; }
        S->bytes = want;
    }
    return S;
}

cudaError_t reach_dispatch(const ReachArgs &a, const ReachPlan &pl, cudaStream_t st, int *per_sm) {
    switch (pl.path) {
        case kPathCoop: return reach_path_coop(a, pl, st, per_sm);
        case kPathCoop2: return reach_path_coop2(a, pl, st, per_sm);
        case kPathCoopSet: return reach_path_set(a, pl, st, per_sm);
        default: return reach_path_global(a, pl, st, per_sm);
    }
}

// Launch the piece kernel with the table layout a reach plan chose (table only, no staging).
cudaError_t piece_dispatch(const ReachArgs &a, const ReachPlan &pl, int sms, cudaStream_t st) {
    const size_t smem = pl.path == kPathGlobal ? pl.smem : pl.staging_offset;
    const uint64_t blocks = (static_cast<uint64_t>(a.c) + 7) / 8;
    const int grid = static_cast<int>(std::min<uint64_t>(blocks, static_cast<uint64_t>(sms) * 8));
    switch (pl.mode) {
        case kModeRep16: return piece_r<LutRep<true>>(pl.R, a, grid, smem, pl.tis, st);
        case kModeRep32: return piece_r<LutRep<false>>(pl.R, a, grid, smem, pl.tis, st);
        case kModePart16: return piece_r<LutPart>(pl.R, a, grid, smem, pl.tis, st);
        case kModeRep16x4: return piece_r<LutRep16x4>(pl.R, a, grid, smem, pl.tis, st);
        case kModeRep16x4C: return piece_r<LutRep16x4C>(pl.R, a, grid, smem, pl.tis, st);
        case kModePair: return piece_r<LutPair>(pl.R, a, grid, smem, pl.tis, st);
        case kModePairC: return piece_r<LutPairC>(pl.R, a, grid, smem, pl.tis, st);
        case kModePairF: return piece_r<LutPairF>(pl.R, a, grid, smem, pl.tis, st);
        case kModePairH: return piece_r<LutPairH>(pl.R, a, grid, smem, pl.tis, st);
        case kModePlain: return piece_r<LutPlain>(pl.R, a, grid, smem, pl.tis, st);
        default: return piece_r<LutFlat>(pl.R, a, grid, smem, pl.tis, st);
    }
}

// Launch the look-back kernel: its work is latency-bound lockstep runs, so it takes a compact
// table (small, leaving room for many warps) whatever layout the reach launch uses: the two-byte
// one where it fits (each lane steps 4 states over every byte pair through one column; the
// regexp family k = 9 at 4,096 chunks 522 -> 616 GB/s, k = 7 1,228 -> 1,245), else the one-byte
// one.  Two blocks of 512 threads an SM (64 registers: at 70 the two-byte kernel ran one block an
// SM and lost its gain).
template <class LUT>
cudaError_t lookback_one(const LookbackArgs &a, int sms, size_t smem, int tis, cudaStream_t st) {
    auto kern = rid_lookback_kernel<LUT>;
    cudaError_t e = ensure_smem_cap(reinterpret_cast<const void *>(kern), smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 512, smem);
    if (e != cudaSuccess) return e;
    const uint64_t blocks = (a.pieces + 15) / 16;
    const int grid = static_cast<int>(std::min<uint64_t>(blocks, static_cast<uint64_t>(sms) * std::max(per_sm, 1)));
    kern<<<grid, 512, smem, st>>>(a, tis);
    return cudaGetLastError();
}

cudaError_t lookback_dispatch(const LookbackArgs &a, int sms, cudaStream_t st) {
    const size_t limit = static_cast<size_t>(smem_optin_limit()) - 1024;
    if (LutPairC::fits(a.A) && LutPairC::smem_bytes(a.A) <= limit / 2)
        return lookback_one<LutPairC>(a, sms, LutPairC::smem_bytes(a.A), 0, st);
    if (LutPlain::fits(a.A) && LutPlain::smem_bytes(a.A) <= limit)
        return lookback_one<LutPlain>(a, sms, LutPlain::smem_bytes(a.A), 0, st);
    const size_t flat = LutFlat::smem_bytes(a.A);
    return flat <= limit ? lookback_one<LutFlat>(a, sms, flat, 1, st) : lookback_one<LutFlat>(a, sms, 256, 0, st);
}

// Choose the layout of a reach launch.  Defaults: the smallest lane-replicated table that fits
// (16-bit, then 32-bit offsets), else the compact table; text staged warp-cooperatively in
// shared memory when the text is 16-byte aligned and the staging buffers fit next to the table;
// one block per SM with as many warps as fit; a grid of one wave.
int plan_reach(const Automaton &A, const ridfa_tuning *tuning, const uint8_t *text,
               const ReachArgs &ra, int sms, ReachPlan *out, bool allow_pair = true) {
    ReachPlan pl;
    pl.R = A.k <= 32 ? 1 : A.k <= 64 ? 2 : A.k <= 128 ? 4 : 8;
    const size_t limit = static_cast<size_t>(smem_optin_limit()) - 1024;
    uint32_t mode = tuning ? tuning->table_mode : 0;
    const size_t rep16 = LutRep<true>::smem_bytes(A), rep32 = LutRep<false>::smem_bytes(A),
                 part16 = LutPart::smem_bytes(A);
    // (the half-replicated layout does not replace the compact one: on the codon RE it measured
    // slower -- its gathers conflict less, but its larger footprint leaves fewer warps and the
    // time goes to run imbalance, not conflicts)
    const size_t plain = LutPlain::smem_bytes(A), flat = LutFlat::smem_bytes(A), rep16x4 = LutRep16x4::smem_bytes(A),
                 rep16x4c = LutRep16x4C::smem_bytes(A), pair = LutPair::smem_bytes(A),
                 pairc = LutPairC::smem_bytes(A);
    const bool ok16 = LutRep<true>::fits16(A) && rep16 <= limit, ok32 = rep32 <= limit,
               okp = LutPart::fits(A) && part16 <= limit, okplain = LutPlain::fits(A) && plain <= limit,
               ok16x4 = LutRep16x4::fits(A) && rep16x4 <= limit,
               ok16x4c = LutRep16x4C::fits(A) && rep16x4c + 4 * static_cast<size_t>(kWarpCoopBytes) <= limit,
               okpair = LutPair::fits(A) && pair + 4 * static_cast<size_t>(kWarpCoopBytes) <= limit,
               okpairc = LutPairC::fits(A) && pairc + 4 * static_cast<size_t>(kWarpCoopBytes) <= limit;
    // two-byte tables in lane copies (byte and half-word offsets): the most copies (16, 8, 4 or 2)
    // whose entries fit 16 bits and that leave room beside the table for the warps the launch
    // wants, one per task up to the block cap (a table that leaves fewer starts a second round of
    // tasks: the any-field record lines with half-word offsets at 4 copies, 28 warps for 32 tasks
    // per SM, ran at 1,647 against 2,782 GB/s at 2 copies); on request, room for 4 warps is enough
    const uint64_t coop_tasks = (static_cast<uint64_t>(ra.c) + 31) / 32;
    const size_t w_want = std::min<uint64_t>(pl.R <= 4 ? 32 : 16,
                                             std::max<uint64_t>(4, (coop_tasks + sms - 1) / sms));
    auto copies = [&](auto fits_f, auto bytes_f, size_t warps) -> uint32_t {
        for (uint32_t f = 16; f >= 2; f /= 2) {
            if (!fits_f(f)) continue;
            const size_t t = (bytes_f(f) + 127) & ~static_cast<size_t>(127);
            if (t + warps * kWarpCoopBytes <= limit) return f;
        }
        return 0;
    };
    auto f_fits = [&](uint32_t f) { return LutPairF::fits(A, f); };
    auto f_bytes = [&](uint32_t f) { return LutPairF::smem_bytes(A, f); };
    auto h_fits = [&](uint32_t f) { return LutPairH::fits(A, f); };
    auto h_bytes = [&](uint32_t f) { return LutPairH::smem_bytes(A, f); };
    const uint32_t want_mode = tuning ? tuning->table_mode : 0;
    uint32_t pair_f = copies(f_fits, f_bytes, w_want), pair_h = copies(h_fits, h_bytes, w_want);
    if (want_mode == kModePairF && !pair_f) pair_f = copies(f_fits, f_bytes, 4);
    if (want_mode == kModePairH && !pair_h) pair_h = copies(h_fits, h_bytes, 4);
    const size_t pairf = pair_f ? LutPairF::smem_bytes(A, pair_f) : 0;
    const size_t pairh = pair_h ? LutPairH::smem_bytes(A, pair_h) : 0;
    // replicated layouts that leave room for at least 16 warps' staging come first; a 32-bit table
    // that leaves fewer is taken only when no scaled 16-bit one fits (measured: a 6-warp 32-bit
    // table ran at a third of the speed of a 26-warp scaled one)
    const size_t room16w = 16 * static_cast<size_t>(kWarpCoopBytes);
    const bool roomy32 = ok32 && rep32 + room16w <= limit, roomy16x4 = ok16x4 && rep16x4 + room16w <= limit;
    if (mode == 0) {
        mode = ok16 ? kModeRep16 : roomy32 ? kModeRep32 : roomy16x4 ? kModeRep16x4 : ok32 ? kModeRep32 : kModePlain;
        // a large conflict-free table gives way to the half-replicated one (at most two wavefronts
        // a gather) when that leaves at least a quarter more warps: measured on the any-field
        // record lines (Rep16x4, 23 warps: 2,330 GB/s; half-replicated, 31 warps: 2,548) and the
        // regexp family (Rep32, 21 warps: 1,740; half-replicated: 2,080)
        if ((mode == kModeRep32 || mode == kModeRep16x4) && okp) {
            const size_t wmax = pl.R <= 4 ? 32 : 16;    // the block's warp cap
            auto warps_beside = [&](size_t table) {
                const size_t off = (table + 127) & ~static_cast<size_t>(127);
                return std::min<size_t>(wmax, off < limit ? (limit - off) / kWarpCoopBytes : 0);
            };
            const size_t w_cf = warps_beside(mode == kModeRep32 ? rep32 : rep16x4);
            const size_t w_part = warps_beside(part16);
            if (4 * w_part >= 5 * w_cf) mode = kModePart16;
        }
        // small automata take two bytes per transition lookup when the pair table leaves room for
        // a full block's staging (regexp family k = 3..5: 2,716 -> 3,088 GB/s; the C1 RE on 1 GiB:
        // 2,507 -> 2,911); not for the lockstep pieces, whose kernel steps one byte at a time
        // (C1 on 1 MiB: 20.6 -> 17.6 GB/s with pairs)
        const uint32_t tp = tuning ? tuning->text_path : 0;
        if (allow_pair && okpair && (tp == 0 || tp == 1 || tp == 3) &&
            pair + 32 * static_cast<size_t>(kWarpCoopBytes) <= limit)
            mode = kModePair;
        // automata left with the compact table (runs that stay apart, several to a lane on the
        // set path) take its two-byte form where it fits beside a full set-path block: a lane's
        // runs then share each pair's column and pay half the transition lookups (the codon RE
        // on 1 GiB, 65,536 chunks: 1,057 -> 1,256 GB/s; on the regexp family, whose replicated
        // tables keep one run a lane, the two-byte compact table measured 16 % slower)
        // (automata whose runs merge on random text -- the compile-time hint -- take the two-byte
        // table in lane copies below instead, one run per lane: the regexp family k = 9, 2,067
        // against 1,839 GB/s)
        const bool copies_ok = pair_f || pair_h;
        if (allow_pair && mode == kModePlain && A.merges && copies_ok && (tp == 0 || tp == 1 || tp == 3))
            mode = kModePart16;               // (replaced by a table in lane copies just below)
        else if (allow_pair && mode == kModePlain && okplain && okpairc && (tp == 0 || tp == 1 || tp == 5) &&
                 pairc + 16 * static_cast<size_t>(kWarpCoopBytes) <= limit)
            mode = kModePairC;
        // the half-replicated one-byte table gives way to the two-byte table in lane copies (a pair
        // gather of at most 32/F wavefronts pays for two bytes where a half-replicated lookup costs
        // up to 2 for one): byte offsets at 16 copies, else half-word offsets at 16 copies (one
        // shift-add more a step; regexp family k = 7: 2,658 GB/s against 2,413 with byte offsets
        // at 8 copies and 2,289 with Part16), else byte offsets at the most copies that fit (the
        // any-field record lines, 2 copies: 2,876 against 2,782); not where the fully replicated
        // pair table fits (regexp k = 5: 16 copies ran 10 % slower than 32)
        if (allow_pair && mode == kModePart16 && (tp == 0 || tp == 1 || tp == 3)) {
            if (pair_f == 16 || (pair_f && pair_f >= pair_h)) mode = kModePairF;
            else if (pair_h) mode = kModePairH;
        }
    }
    if (mode == kModeRep16x4 && !ok16x4) return RIDFA_E_ARG;
    if (mode == kModeRep16x4C && !ok16x4c) return RIDFA_E_ARG;
    if (mode == kModePair && !okpair) return RIDFA_E_ARG;
    if (mode == kModePairC && !okpairc) return RIDFA_E_ARG;
    if (mode == kModePairF && !pair_f) return RIDFA_E_ARG;
    if (mode == kModePairH && !pair_h) return RIDFA_E_ARG;
    if (mode == kModePlain && !okplain) mode = kModeFlat;    // the compact table, through generic loads
    if ((mode == kModeRep16 && !ok16) || (mode == kModeRep32 && !ok32) || (mode == kModePart16 && !okp))
        return RIDFA_E_ARG;
    if (mode < kModePlain || mode > kModePairH) return RIDFA_E_ARG;
    pl.mode = mode;
    pl.tis = mode == kModePairF ? static_cast<int>(pair_f) : mode == kModePairH ? static_cast<int>(pair_h)
             : (mode == kModeFlat && flat <= limit) ? 1 : 0;
    const size_t table_smem = mode == kModeRep16 ? rep16 : mode == kModeRep32 ? rep32 : mode == kModePart16 ? part16
                              : mode == kModeRep16x4 ? rep16x4 : mode == kModeRep16x4C ? rep16x4c
                              : mode == kModePair ? pair : mode == kModePairC ? pairc : mode == kModePairF ? pairf
                              : mode == kModePairH ? pairh
                              : mode == kModePlain ? plain : (pl.tis ? flat : 256);
    const int cap = pl.R <= 4 ? 1024 : 512;
    const uint32_t text_path = tuning ? tuning->text_path : 0;
    if (text_path > 5) return RIDFA_E_ARG;
    pl.staging_offset = static_cast<uint32_t>((table_smem + 127) & ~static_cast<size_t>(127));
    const size_t room = limit > pl.staging_offset ? limit - pl.staging_offset : 0;
    const bool aligned = (reinterpret_cast<uintptr_t>(text) & 15) == 0;
    int block = (tuning && tuning->block_threads) ? static_cast<int>(tuning->block_threads) : 0;
    auto fits = [&](uint32_t per_warp) {
        const int w = static_cast<int>(std::min<size_t>(cap / 32, room / per_warp));
        return (block == 0 ? w >= 4 : block / 32 <= w) ? w : 0;
    };
    const int cap2 = pl.R <= 4 ? 768 : 512;
    auto fits2 = [&](uint32_t per_warp) {
        const int w = static_cast<int>(std::min<size_t>(cap2 / 32, room / per_warp));
        return (block == 0 ? w >= 4 : block / 32 <= w) ? w : 0;
    };
    const int w_coop = fits(kWarpCoopBytes), w_coop2 = fits2(kWarpCoop2Bytes);
    const int w_set = std::min(w_coop, 512 / 32);
    // auto: one chain per lane with cooperative staging (16-byte-aligned text, buffers fit),
    // else plain global loads.  (Two chains per lane measured slower on GB300; so did per-lane
    // bulk copies, a path since retired so that no kernel can leave with a copy in flight.)
    // Automata whose table is too large to replicate are the ones whose runs stay apart: there a
    // lane finishes all of its chunk's runs together (measured on the codon RE: 1.21x; on
    // replicated-table workloads the 512-thread cap of that variant cost 8-13%).
    // (the one-byte compact table of an automaton whose runs merge -- too large for any two-byte
    // form, e.g. the regexp family at k = 11 -- keeps one run per lane)
    const bool many_runs = (mode == kModePlain && !A.merges) || mode == kModeFlat || mode == kModeRep16x4C ||
                           mode == kModePairC;
    if (text_path == 0)
        pl.path = !aligned ? kPathGlobal
                  : !w_coop ? kPathGlobal
                  : many_runs && w_set >= 4 && block <= 512 ? kPathCoopSet : kPathCoop;
    else if (text_path == 1) pl.path = kPathGlobal;
    else if (text_path == 2) return RIDFA_E_ARG;   // retired: per-lane bulk copies
    else if (text_path == 3) pl.path = kPathCoop;
    else if (text_path == 4) pl.path = kPathCoop2;
    else pl.path = kPathCoopSet;
    if (pl.path == kPathCoop && !(aligned && w_coop)) return RIDFA_E_ARG;
    if (pl.path == kPathCoop2 && !(aligned && w_coop2)) return RIDFA_E_ARG;
    if (pl.path == kPathCoopSet && !(aligned && w_set)) return RIDFA_E_ARG;
    // the compact class table is built for the set path (and plain global loads), two-byte steps
    // for the single-run cooperative path (and plain global loads)
    if (mode == kModeRep16x4C && pl.path != kPathCoopSet && pl.path != kPathGlobal) return RIDFA_E_ARG;
    if (mode == kModePair && pl.path != kPathCoop && pl.path != kPathGlobal) return RIDFA_E_ARG;
    if (mode == kModePairC && pl.path != kPathCoopSet && pl.path != kPathGlobal) return RIDFA_E_ARG;
    if ((mode == kModePairF || mode == kModePairH) && pl.path != kPathCoop && pl.path != kPathGlobal) return RIDFA_E_ARG;
    const int warps_fit = pl.path == kPathCoop      ? w_coop
                          : pl.path == kPathCoopSet ? w_set
                          : pl.path == kPathCoop2 ? w_coop2
                                                  : cap / 32;
    const uint64_t tasks = (static_cast<uint64_t>(ra.c) + (pl.path == kPathCoop2 ? 63 : 31)) /
                           (pl.path == kPathCoop2 ? 64 : 32);
    if (block == 0) {
        block = pl.path == kPathGlobal ? (mode == kModeFlat && !pl.tis ? 256 : cap) : warps_fit * 32;
        // fewer tasks than SMs x warps: spread them over every SM instead of filling some SMs'
        // blocks and leaving the rest idle (at least 4 warps a block: each block loads the tables)
        if (pl.path != kPathGlobal) {
            const uint64_t per_sm_warps = std::max<uint64_t>(4, (tasks + sms - 1) / sms);
            if (per_sm_warps < static_cast<uint64_t>(block / 32)) block = static_cast<int>(per_sm_warps) * 32;
        }
    }
    const int bcap = pl.path == kPathCoop2 ? cap2 : pl.path == kPathCoopSet ? 512 : cap;
    if (block < 32 || block > bcap || block % 32) return RIDFA_E_ARG;
    pl.block = block;
    pl.smem = pl.path == kPathCoop || pl.path == kPathCoopSet
                  ? pl.staging_offset + static_cast<size_t>(block / 32) * kWarpCoopBytes
              : pl.path == kPathCoop2 ? pl.staging_offset + static_cast<size_t>(block / 32) * kWarpCoop2Bytes
                                      : table_smem;
    if (tuning && tuning->grid_blocks) {
        pl.grid = static_cast<int>(tuning->grid_blocks);
    } else {
        int per_sm = 0;
        cudaError_t e = reach_dispatch(ra, pl, nullptr, &per_sm);
        if (e != cudaSuccess) return cuda_fail(e);
        if (per_sm < 1) return RIDFA_E_UNSUPPORTED;
        const uint64_t wpb = block / 32;
        const uint64_t need = (tasks + wpb - 1) / wpb;
        pl.grid = static_cast<int>(std::min<uint64_t>(need, static_cast<uint64_t>(sms) * per_sm));
    }
    *out = pl;
    return RIDFA_OK;
}

int recognize_impl(const ridfa_program *P, bool use_dfa, const uint8_t *d_text, size_t len,
                   uint32_t n_chunks, const ridfa_tuning *tuning, uint8_t *d_accept_user,
                   uint8_t *h_accept, uint16_t *d_maps_user, cudaStream_t st,
                   ridfa_shard_summary *h_summary = nullptr) {
    if (!P) return RIDFA_E_ARG;
    if (use_dfa && !P->has_dfa) return RIDFA_E_NO_DFA;
    const HostAutomaton &H = use_dfa ? P->dfa : P->rid;
    if (len == 0) {
        if (n_chunks != 0) return RIDFA_E_CHUNKS;
        // empty text: accept iff the start state is final (no device work needed for the answer)
        const uint8_t acc = H.final_flag.empty() ? 0 : H.final_flag[H.slot_state[H.q0_slot]];
        if (h_accept) *h_accept = acc;
        if (d_accept_user) {
            cudaError_t e = cudaMemcpyAsync(d_accept_user, &acc, 1, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e);
            e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(e);
        }
        return RIDFA_OK;
    }
    if (!d_text) return RIDFA_E_ARG;
    if (n_chunks == 0 || n_chunks > len) return RIDFA_E_CHUNKS;
    if (H.k > RIDFA_MAX_SLOTS) return RIDFA_E_UNSUPPORTED;

    std::lock_guard<std::mutex> lock(P->mu);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    int err = RIDFA_OK;
    const DeviceAutomaton *D = device_copy(P, use_dfa, dev, &err);
    if (!D) return err;

    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t c = n_chunks;
    const uint64_t nbound = c - 1;
    const uint64_t per_block_max = 1024;
    uint32_t per_thread = static_cast<uint32_t>(std::max<uint64_t>(
        1, (nbound + static_cast<uint64_t>(kJoinThreads) * per_block_max - 1) /
               (static_cast<uint64_t>(kJoinThreads) * per_block_max)));
    uint32_t join_blocks = static_cast<uint32_t>(std::max<uint64_t>(
        1, (nbound + static_cast<uint64_t>(kJoinThreads) * per_thread - 1) /
               (static_cast<uint64_t>(kJoinThreads) * per_thread)));
    Automaton A{D->trans, D->classmap, D->final_bits, D->ifmask, D->slot_state,
                H.n_states, H.n_classes, H.k, H.kw, H.q0_slot, H.merges};
    // intra-chunk speculation: too few chunks to fill the GPU, each long enough to cut into pieces.
    // Pieces run from every state; automata of more than 256 states run theirs in groups of at
    // most 256 states (one reach launch per group into one row of all states).
    const uint32_t piece_req = tuning ? tuning->piece_len : 0;
    if (piece_req > 1 && piece_req < 64) return RIDFA_E_ARG;
    const uint32_t NS = H.n_states;
    // automata of more than 256 states whose interface fits one register start each piece from its
    // look-back start set instead (one launch, no repeated runs)
    const uint32_t text_path = tuning ? tuning->text_path : 0;
    const bool lb_able = NS > RIDFA_MAX_SLOTS && H.k <= 32 && text_path != 2 && text_path != 4;
    const uint32_t lb_cap = tuning && tuning->lookback_cap ? tuning->lookback_cap : 32;
    if (lb_cap > 32) return RIDFA_E_ARG;
    const uint32_t groups = lb_able ? 1 : (NS + RIDFA_MAX_SLOTS - 1) / RIDFA_MAX_SLOTS;
    uint64_t spc = 1;                                  // pieces per chunk
    if (piece_req != 1 && NS >= 1 && groups <= kMaxPieceGroups) {
        const uint64_t warps = static_cast<uint64_t>(sms) * 32, lanes = warps * 32;
        const uint64_t rall = NS <= 32 ? 1 : NS <= 64 ? 2 : NS <= 128 ? 4 : 8;
        // a short text: a lockstep piece costs a warp (1 + ceil(P/32)) lookups per byte where a
        // chunk costs a lane 2, worth it only while the chunks leave most resident warps idle
        if (NS <= RIDFA_MAX_SLOTS && c * (1 + rall) * 4 <= warps) {
            const uint64_t plen = piece_req >= 64 ? piece_req : 256;
            spc = std::min<uint64_t>(2 * lanes / c, len / (c * plen));
        }
        // a long text in chunks that fill at most half of the lanes (a quarter with look-back start
        // sets, whose look-back costs extra; a quarter per state group when the states run in
        // groups, whose launches repeat the merged runs): pieces through the reach kernel, at most
        // one per lane, at least kManyPieceLen bytes each
        const uint64_t fill = lb_able ? 4 : groups == 1 ? 2 : 4 * groups;
        if (spc < 2 && c * fill <= lanes) {
            const uint64_t plen = piece_req >= 64 ? piece_req : kManyPieceLen;
            // automata whose runs stay apart (the compile-time hint) run on the set path, at most
            // 16 warps a block and one block an SM: one piece per lane of that one round (the
            // codon RE at 4,096 chunks: 155,648 pieces 535 GB/s, 77,824 pieces 776)
            const uint64_t plimit = lb_able && !H.merges ? static_cast<uint64_t>(sms) * 16 * 32 : lanes;
            spc = std::min<uint64_t>(plimit / c, len / (c * plen));
        }
        // the piece functions take pieces * P * 2 bytes of scratch: at most kMaxPieceBytes
        spc = std::min<uint64_t>(spc, kMaxPieceBytes / (c * NS * 2));
        if (spc < 2) spc = 1;
    }
    // many pieces (a long text in few chunks): the reach kernel runs them, one lane per piece
    // once its runs merge; few pieces: one lockstep warp per piece
    const bool lockstep = spc > 1 && NS <= RIDFA_MAX_SLOTS && c * spc <= static_cast<uint64_t>(sms) * 32 * 8;
    const uint64_t pieces = c * spc;
    const bool lookback = spc > 1 && lb_able;
    const uint32_t n_launch = spc > 1 ? groups : 1;
    // plan the reach launches first: the run-list scratch is sized by their grids
    ReachArgs ras[kMaxPieceGroups];
    ReachPlan plans[kMaxPieceGroups];
    uint64_t grid_warps = 0;
    for (uint32_t g = 0; g < n_launch; ++g) {
        // look-back pieces: 32 start slots per piece, rows of 32 scattered afterwards
        const uint32_t kg = lookback ? 32 : spc > 1 ? std::min<uint32_t>(RIDFA_MAX_SLOTS, NS - g * RIDFA_MAX_SLOTS) : H.k;
        const Automaton Ag = spc > 1 ? Automaton{D->trans, D->classmap, D->final_bits, D->ifmask,
                                                 lookback ? D->slot_state : D->all_states + g * RIDFA_MAX_SLOTS,
                                                 H.n_states, H.n_classes, kg, (kg + 31) / 32, 0}
                                     : A;
        ras[g] = ReachArgs{Ag, d_text, len, static_cast<uint32_t>(pieces), nullptr, nullptr, nullptr, 8,
                           nullptr, nullptr, lookback ? 32u : spc > 1 ? NS : H.k, nullptr};
        if (tuning && tuning->probe_interval) ras[g].probe = tuning->probe_interval;
        err = plan_reach(ras[g].A, tuning, d_text, ras[g], sms, &plans[g], !lockstep);
        if (err != RIDFA_OK) return err;
        plans[g].pslot = lookback;
        // warps past the last 32-chunk task never write their run list (the lockstep kernel has none)
        if (!lockstep)
            grid_warps = std::max<uint64_t>(grid_warps, std::min<uint64_t>(static_cast<uint64_t>(plans[g].grid) *
                                                                               (plans[g].block / 32),
                                                                           (pieces + 31) / 32));
    }
    const uint64_t comp_funcs = spc > 1 ? c * ((spc + kComposeGroup - 1) / kComposeGroup) : 0;
    const Layout L = layout_for(c, H.k, d_maps_user == nullptr, join_blocks, grid_warps, spc > 1 ? pieces : 0,
                                spc > 1 ? NS : 0, comp_funcs, lookback);
    DeviceScratch *S = scratch_for(P, dev, L.total, &err);
    if (!S) return err;
    {
        const ReachPlan &p0 = plans[0];
        const bool copies = p0.mode == kModePairF || p0.mode == kModePairH;
        S->last_plan = ridfa_plan_report{p0.mode,
                                         p0.path == kPathCoop ? 3u : p0.path == kPathCoop2 ? 4u : p0.path == kPathCoopSet ? 5u : 1u,
                                         copies ? static_cast<uint32_t>(p0.tis) : 0u, static_cast<uint32_t>(p0.block),
                                         static_cast<uint32_t>(p0.grid), (spc > 1 || lockstep) ? 1u : 0u};
        S->planned = true;
    }
    uint8_t *base = static_cast<uint8_t *>(S->base);
    uint32_t *ticket = reinterpret_cast<uint32_t *>(base + L.ticket_off);
    uint32_t *status = reinterpret_cast<uint32_t *>(base + L.status_off);
    uint8_t *accept = d_accept_user ? d_accept_user : base + L.accept_off;
    uint16_t *maps = d_maps_user ? d_maps_user : reinterpret_cast<uint16_t *>(base + L.maps_off);
    uint32_t *dinfo = reinterpret_cast<uint32_t *>(base + L.dinfo_off);
    uint32_t *partials = reinterpret_cast<uint32_t *>(base + L.partials_off);
    uint32_t *piece_status = status + 1;
    uint16_t *pmaps = reinterpret_cast<uint16_t *>(base + L.pmaps_off);
    for (uint32_t g = 0; g < n_launch; ++g) {
        ReachArgs &ra = ras[g];
        ra.maps = lookback ? reinterpret_cast<uint16_t *>(base + L.lbrows_off)
                  : spc > 1 ? pmaps + g * RIDFA_MAX_SLOTS : maps;
        if (lookback) ra.piece_slots = reinterpret_cast<const uint16_t *>(base + L.lbslots_off);
        ra.dinfo = spc > 1 ? reinterpret_cast<uint32_t *>(base + L.pdinfo_off) : dinfo;
        ra.status = spc > 1 ? piece_status : status;
        ra.runs = reinterpret_cast<RunEntry *>(base + L.runs_off);
        ra.finals = reinterpret_cast<uint32_t *>(base + L.finals_off);
    }
    e = cudaMemsetAsync(status, 0, 8, st);
    if (e != cudaSuccess) return cuda_fail(e);

    const bool prof = tuning && tuning->profile;
    if (prof) {
        for (auto &ev : S->ev)
            if (!ev) {
                cudaEvent_t x;
                e = cudaEventCreate(&x);
                if (e != cudaSuccess) return cuda_fail(e);
                ev = x;
            }
        cudaEventRecord(static_cast<cudaEvent_t>(S->ev[0]), st);
    }
    if (lookback) {
        // piece functions start undefined; the look-back kernel writes each piece's start set (or
        // the whole function of a piece without a small one)
        e = cudaMemsetAsync(pmaps, 0xFF, pieces * NS * 2, st);
        if (e != cudaSuccess) return cuda_fail(e);
        LookbackArgs la{ras[0].A, d_text, len, pieces, static_cast<uint32_t>(spc),
                        reinterpret_cast<uint16_t *>(base + L.lbslots_off), pmaps, lb_cap};
        la.A.k = H.k;
        e = lookback_dispatch(la, sms, st);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    // (the groups' launches share the run lists: they run one after another on the stream)
    NvtxRange reach_range("ridfa reach");
    for (uint32_t g = 0; g < n_launch; ++g) {
        e = lockstep ? piece_dispatch(ras[g], plans[g], sms, st) : reach_dispatch(ras[g], plans[g], st, nullptr);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    if (lookback) {
        rid_scatter_kernel<<<static_cast<unsigned>((pieces * 32 + 255) / 256), 256, 0, st>>>(
            reinterpret_cast<const uint16_t *>(base + L.lbslots_off),
            reinterpret_cast<const uint16_t *>(base + L.lbrows_off), pieces, NS, pmaps);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e);
    }
    if (spc > 1) {
        // compose each chunk's piece functions, kComposeGroup per thread and level, then apply
        // them to the interface slots' start states
        const uint16_t *in = pmaps;
        uint64_t in_per = spc;
        uint16_t *bufs[2] = {reinterpret_cast<uint16_t *>(base + L.comp_off),
                             reinterpret_cast<uint16_t *>(base + L.comp_off + ((comp_funcs * NS * 2 + 255) & ~255ull))};
        int b = 0;
        while (in_per > 1) {
            const uint64_t out_per = (in_per + kComposeGroup - 1) / kComposeGroup;
            const uint64_t threads = c * out_per * NS;
            rid_compose_kernel<<<static_cast<unsigned>((threads + 255) / 256), 256, 0, st>>>(
                in, static_cast<uint32_t>(in_per), bufs[b], static_cast<uint32_t>(out_per), static_cast<uint32_t>(c), NS);
            in = bufs[b];
            b ^= 1;
            in_per = out_per;
        }
        rid_apply_kernel<<<static_cast<unsigned>((c * 32 + 255) / 256), 256, 0, st>>>(
            in, NS, D->slot_state, H.k, static_cast<uint32_t>(c), maps, dinfo, status, piece_status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e);
    }
    if (prof) cudaEventRecord(static_cast<cudaEvent_t>(S->ev[1]), st);

    // ---- join
    NvtxRange join_range("ridfa join");
    ridfa_shard_summary *d_summary =
        h_summary ? reinterpret_cast<ridfa_shard_summary *>(base + L.summary_off) : nullptr;
    JoinArgs ja{A, n_chunks, maps, dinfo, status, partials, ticket, accept, per_thread, d_summary};
    rid_join_kernel<<<join_blocks, kJoinThreads, 0, st>>>(ja);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    if (h_summary) {
        e = cudaMemcpyAsync(h_summary, d_summary, sizeof(ridfa_shard_summary), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(S->h_status_pinned, status, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e);
        if (*S->h_status_pinned & kStatusTimeout) return RIDFA_E_TIMEOUT;
        if (*S->h_status_pinned & kStatusBad) return RIDFA_E_STATE;
        return RIDFA_OK;
    }
    if (prof) {
        cudaEventRecord(static_cast<cudaEvent_t>(S->ev[2]), st);
        S->profiled = true;
    }

    if (h_accept) {
        e = cudaMemcpyAsync(S->h_accept_pinned, accept, 1, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(S->h_status_pinned, status, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e);
        *h_accept = *S->h_accept_pinned;
        if (*S->h_status_pinned & kStatusTimeout) return RIDFA_E_TIMEOUT;
        if (*S->h_status_pinned & kStatusBad) return RIDFA_E_STATE;
    }
    return RIDFA_OK;
}

}  // namespace

void release_device(const ridfa_program *P) {
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    auto free_on = [&](int dev, void *ptr) {
        if (!ptr) return;
        cudaSetDevice(dev);
        cudaFree(ptr);
    };
    release_nfa(P);
    for (auto &d : P->dev_rid) free_on(d.device, d.trans);
    for (auto &d : P->dev_dfa) free_on(d.device, d.trans);
    for (auto &s : P->scratch) {
        free_on(s.device, s.base);
        if (s.h_accept_pinned) cudaFreeHost(s.h_accept_pinned);
        for (void *ev : s.ev)
            if (ev) cudaEventDestroy(static_cast<cudaEvent_t>(ev));
    }
    cudaSetDevice(cur);
    (void)cudaGetLastError();
}

int launch_with_buffers(const HostAutomaton &H, const PreparedBuffers &B, const uint8_t *d_text,
                        uint64_t len, uint32_t n_chunks, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t c = n_chunks;
    const uint64_t nbound = c - 1;
    const uint64_t per_thread = std::max<uint64_t>(
        1, (nbound + static_cast<uint64_t>(kJoinThreads) * kMaxJoinBlocks - 1) /
               (static_cast<uint64_t>(kJoinThreads) * kMaxJoinBlocks));
    const uint32_t join_blocks = static_cast<uint32_t>(std::max<uint64_t>(
        1, (nbound + kJoinThreads * per_thread - 1) / (kJoinThreads * per_thread)));
    Automaton A{B.trans, B.classmap, B.final_bits, B.ifmask, B.slot_state,
                H.n_states, H.n_classes, H.k, H.kw, H.q0_slot, H.merges};
    ReachArgs ra{A, d_text, len, n_chunks, B.maps, B.dinfo, B.status, 8, nullptr, nullptr, H.k};
    ReachPlan plan;
    int err = plan_reach(A, nullptr, d_text, ra, sms, &plan);
    if (err != RIDFA_OK) return err;
    e = reach_dispatch(ra, plan, st, nullptr);
    if (e != cudaSuccess) return cuda_fail(e);
    JoinArgs ja{A, n_chunks, B.maps, B.dinfo, B.status, B.partials, B.ticket, B.accept,
                static_cast<uint32_t>(per_thread)};
    rid_join_kernel<<<join_blocks, kJoinThreads, 0, st>>>(ja);
    e = cudaGetLastError();
    return e == cudaSuccess ? RIDFA_OK : cuda_fail(e);
}

}  // namespace ridfa

namespace ridfa {
namespace {
// The library's bounded mbarrier wait, exercised alone: one warp waits on a fresh mbarrier for
// its first phase, at most `limit` polls.  With `arrive` lane 0 completes the phase first; without
// it nothing ever arrives and the wait must run out.  *status gets kStatusTimeout when it did.
__global__ void rid_wait_check_kernel(uint32_t limit, int arrive, uint32_t *status) {
    __shared__ __align__(8) uint64_t bar_word;
    const uint32_t bar = smem_addr(&bar_word);
    if (threadIdx.x == 0) mbar_init(bar, 1);
    fence_mbar_init();
    __syncwarp();
    if (arrive && threadIdx.x == 0) mbar_arrive(bar);
    __syncwarp();
    const bool ok = mbar_wait_warp(bar, 0, limit);
    if (threadIdx.x == 0) *status = ok ? 0u : kStatusTimeout;
}
}  // namespace
}  // namespace ridfa

extern "C" int ridfa_check_bounded_wait(uint32_t limit, int arrive, void *stream) {
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t *d_status = nullptr;
    cudaError_t e = cudaMalloc(&d_status, sizeof(uint32_t));
    if (e != cudaSuccess) return ridfa::cuda_fail(e);
    uint32_t h_status = 0;
    e = cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess) {
        ridfa::rid_wait_check_kernel<<<1, 32, 0, st>>>(limit, arrive, d_status);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_status);
    if (e != cudaSuccess) return ridfa::cuda_fail(e);
    return (h_status & ridfa::kStatusTimeout) ? RIDFA_E_TIMEOUT : RIDFA_OK;
}

extern "C" int ridfa_recognize(const ridfa_program *prog, const uint8_t *d_text, size_t len,
                               uint32_t n_chunks, const ridfa_tuning *tuning, uint8_t *h_accept,
                               uint16_t *d_chunk_maps, void *stream) {
    if (!h_accept) return RIDFA_E_ARG;
    return ridfa::recognize_impl(prog, false, d_text, len, n_chunks, tuning, nullptr, h_accept,
                                 d_chunk_maps, static_cast<cudaStream_t>(stream));
}

extern "C" int ridfa_recognize_host(const ridfa_program *prog, const uint8_t *h_text, size_t len,
                                    uint32_t n_chunks, const ridfa_tuning *tuning, uint8_t *d_staging,
                                    uint8_t *h_accept, void *stream) {
    if (!prog || !h_accept || (len && (!h_text || !d_staging))) return RIDFA_E_ARG;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (len) {
        const cudaError_t e = cudaMemcpyAsync(d_staging, h_text, len, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return ridfa::cuda_fail(e);
    }
    return ridfa::recognize_impl(prog, false, d_staging, len, n_chunks, tuning, nullptr, h_accept, nullptr, st);
}

extern "C" int ridfa_recognize_async(const ridfa_program *prog, const uint8_t *d_text, size_t len,
                                     uint32_t n_chunks, const ridfa_tuning *tuning, uint8_t *d_accept,
                                     uint16_t *d_chunk_maps, void *stream) {
    if (!d_accept) return RIDFA_E_ARG;
    return ridfa::recognize_impl(prog, false, d_text, len, n_chunks, tuning, d_accept, nullptr,
                                 d_chunk_maps, static_cast<cudaStream_t>(stream));
}

extern "C" int ridfa_recognize_dfa(const ridfa_program *prog, const uint8_t *d_text, size_t len,
                                   uint32_t n_chunks, const ridfa_tuning *tuning, uint8_t *h_accept,
                                   uint16_t *d_chunk_maps, void *stream) {
    if (!h_accept) return RIDFA_E_ARG;
    return ridfa::recognize_impl(prog, true, d_text, len, n_chunks, tuning, nullptr, h_accept,
                                 d_chunk_maps, static_cast<cudaStream_t>(stream));
}

extern "C" int ridfa_recognize_dfa_async(const ridfa_program *prog, const uint8_t *d_text,
                                         size_t len, uint32_t n_chunks, const ridfa_tuning *tuning,
                                         uint8_t *d_accept, uint16_t *d_chunk_maps, void *stream) {
    if (!d_accept) return RIDFA_E_ARG;
    return ridfa::recognize_impl(prog, true, d_text, len, n_chunks, tuning, d_accept, nullptr,
                                 d_chunk_maps, static_cast<cudaStream_t>(stream));
}

extern "C" int ridfa_recognize_shard(const ridfa_program *prog, const uint8_t *d_text, size_t len,
                                     uint32_t n_chunks, const ridfa_tuning *tuning, ridfa_shard_summary *h_out,
                                     void *stream) {
    if (!h_out || len == 0) return RIDFA_E_ARG;
    return ridfa::recognize_impl(prog, false, d_text, len, n_chunks, tuning, nullptr, nullptr, nullptr,
                                 static_cast<cudaStream_t>(stream), h_out);
}

extern "C" int ridfa_last_status(const ridfa_program *prog, void *stream) {
    if (!prog) return RIDFA_E_ARG;
    std::lock_guard<std::mutex> lock(prog->mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ridfa::cuda_fail(cudaGetLastError());
    for (auto &s : prog->scratch) {
        if (s.device != dev || !s.base) continue;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        uint32_t *status = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(s.base) + 256);
        cudaError_t e = cudaMemcpyAsync(s.h_status_pinned, status, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return ridfa::cuda_fail(e);
        if (*s.h_status_pinned & 4u) return RIDFA_E_TIMEOUT;
        return (*s.h_status_pinned & 2u) ? RIDFA_E_STATE : RIDFA_OK;
    }
    return RIDFA_OK;
}

extern "C" int ridfa_last_plan(const ridfa_program *prog, ridfa_plan_report *out) {
    if (!prog || !out) return RIDFA_E_ARG;
    std::lock_guard<std::mutex> lock(prog->mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ridfa::cuda_fail(cudaGetLastError());
    for (auto &s : prog->scratch)
        if (s.device == dev && s.planned) {
            *out = s.last_plan;
            return RIDFA_OK;
        }
    return RIDFA_E_ARG;
}

extern "C" int ridfa_last_timings(const ridfa_program *prog, float *reach_ms, float *join_ms) {
    if (!prog) return RIDFA_E_ARG;
    std::lock_guard<std::mutex> lock(prog->mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ridfa::cuda_fail(cudaGetLastError());
    for (auto &s : prog->scratch) {
        if (s.device != dev || !s.profiled) continue;
        cudaError_t e = cudaEventSynchronize(static_cast<cudaEvent_t>(s.ev[2]));
        float a = 0.f, b = 0.f;
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&a, static_cast<cudaEvent_t>(s.ev[0]), static_cast<cudaEvent_t>(s.ev[1]));
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&b, static_cast<cudaEvent_t>(s.ev[1]), static_cast<cudaEvent_t>(s.ev[2]));
        if (e != cudaSuccess) return ridfa::cuda_fail(e);
        if (reach_ms) *reach_ms = a;
        if (join_ms) *join_ms = b;
        return RIDFA_OK;
    }
    return RIDFA_E_ARG;
}

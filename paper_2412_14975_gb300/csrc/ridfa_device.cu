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
//   * Converged phase: each lane takes its own chunk and finishes the single surviving run
//     alone, with 16-byte vector loads of the text; the chunk map row is the surviving state
//     for the slots alive at convergence and undefined for the others.
//   A chunk whose runs never merge finishes in the speculative phase.
// Join phase (Sec. 3.2 / 3.4): let D_i be the distinct defined values of lambda_i (m_i <= 32).
// Between chunks i-1 and i the transfer is the m_{i-1} x m_i Boolean matrix
//   M_i[x][y] = exists a in if_min({D_{i-1}[x]}) with lambda_i(a) = D_i[y],
// PLAS_c = lambda_1(q0) M_2 ... M_c, and the text is accepted iff PLAS_c meets F^RID.  The
// matrices are multiplied in a chain: sequentially inside a thread, by a tree inside a block,
// and over blocks by the last block to finish (an atomic ticket).  If some chunk has more than
// 32 distinct end states, block 0 instead propagates if(PLAS_i) as a k-bit set chunk by chunk.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "ridfa_internal.h"

namespace ridfa {
namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint16_t kUndef = 0xFFFF;
constexpr uint32_t kStatusWide = 1u;      // some chunk has > 32 distinct end states
constexpr uint32_t kStatusBad = 2u;       // a device consistency check failed
constexpr int kMaxD = 32;                 // distinct end states handled by the matrix join
constexpr int kJoinThreads = 256;

struct Automaton {            // device view of one automaton
    const uint16_t *trans;    // [(n+1) * C]
    const uint8_t *classmap;  // [256]
    const uint32_t *final_bits;
    const uint32_t *ifmask;   // [(n+1) * kw]
    const uint16_t *slot_state;
    uint32_t n, C, k, kw, q0_slot;
};

__host__ __device__ inline uint64_t chunk_begin(uint64_t i, uint64_t len, uint64_t c) {
    // floor(i * len / c) without 128-bit products: i*(len/c) + (i*(len%c))/c
    return i * (len / c) + (i * (len % c)) / c;
}

// ------------------------------------------------------------------------------ reach
struct ReachArgs {
    Automaton A;
    const uint8_t *text;
    uint64_t len;
    uint32_t c;
    uint16_t *maps;           // [c][k]
    uint32_t *dinfo;          // [c]: (m << 16) | min defined end state (0xFFFF if none)
    uint32_t *status;
    uint32_t probe;
    int table_in_smem;
};

template <bool SMEM>
struct Tab {
    const uint16_t *t;
    const uint8_t *cls;
    uint32_t C;
    __device__ __forceinline__ uint32_t cls_of(uint32_t b) const { return cls[b]; }
    __device__ __forceinline__ uint32_t next(uint32_t s, uint32_t c) const { return t[s * C + c]; }
};

template <int R, bool SMEM>
__global__ void __launch_bounds__(256) rid_reach_kernel(ReachArgs p) {
    extern __shared__ __align__(16) uint8_t smem[];
    const Automaton &A = p.A;
    uint8_t *s_cls = smem;
    uint16_t *s_t = reinterpret_cast<uint16_t *>(smem + 256);
    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) s_cls[i] = A.classmap[i];
    const uint32_t tab_n = (A.n + 1) * A.C;
    if (SMEM)
        for (uint32_t i = threadIdx.x; i < tab_n; i += blockDim.x) s_t[i] = A.trans[i];
    __syncthreads();
    Tab<SMEM> T{SMEM ? s_t : A.trans, s_cls, A.C};

    const uint32_t lane = threadIdx.x & 31;
    const uint32_t dead = A.n;
    const uint64_t n_tasks = (static_cast<uint64_t>(p.c) + 31) / 32;
    const uint64_t warp0 = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;

    // slot start states of this lane (slot a = r*32 + lane)
    uint32_t start_state[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        uint32_t a = r * 32 + lane;
        start_state[r] = a < A.k ? A.slot_state[a] : dead;
    }

    for (uint64_t task = warp0; task < n_tasks; task += n_warps) {
        const uint64_t chunk0 = task * 32;
        // what this lane must still do for chunk chunk0 + lane
        uint64_t my_pos = 0;
        uint32_t my_state = dead;
        uint32_t my_alive[R];
        bool my_pending = false;
#pragma unroll
        for (int r = 0; r < R; ++r) my_alive[r] = 0;

        // ---------------- speculative phase, one chunk at a time, lanes = runs
        for (uint32_t j = 0; j < 32; ++j) {
            const uint64_t ch = chunk0 + j;
            if (ch >= p.c) break;
            const uint64_t beg = chunk_begin(ch, p.len, p.c);
            const uint64_t end = chunk_begin(ch + 1, p.len, p.c);
            uint32_t s[R];
#pragma unroll
            for (int r = 0; r < R; ++r) s[r] = start_state[r];
            uint64_t pos = beg;
            bool converged = false;
            uint32_t conv_state = dead;
            while (pos < end) {
                const uint64_t stop = min(end, pos + p.probe);
                for (; pos < stop; ++pos) {
                    const uint32_t c = T.cls_of(__ldg(p.text + pos));
#pragma unroll
                    for (int r = 0; r < R; ++r) s[r] = T.next(s[r], c);
                }
                // convergence check: all live runs in one state?
                uint32_t lo = 0xFFFFFFFFu, hi = 0;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (s[r] != dead) {
                        lo = min(lo, s[r]);
                        hi = max(hi, s[r]);
                    }
                lo = __reduce_min_sync(kFull, lo);
                hi = __reduce_max_sync(kFull, hi);
                if (lo == 0xFFFFFFFFu || lo == hi) {
                    converged = true;
                    conv_state = (lo == 0xFFFFFFFFu) ? dead : lo;
                    break;
                }
            }
            uint16_t *row = p.maps + ch * A.k;
            if (converged && pos < end && conv_state != dead) {
                // hand the single surviving run to lane j
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    uint32_t b = __ballot_sync(kFull, s[r] != dead);
                    if (lane == j) my_alive[r] = b;
                }
                if (lane == j) {
                    my_pos = pos;
                    my_state = conv_state;
                    my_pending = true;
                }
            } else {
                // finished in the speculative phase: write the row (coalesced) and D_i's size
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    uint32_t a = r * 32 + lane;
                    if (a < A.k) row[a] = s[r] == dead ? kUndef : static_cast<uint16_t>(s[r]);
                }
                uint32_t cnt = 0, first = kUndef, cur = 0;
                bool more = true;
                while (more) {
                    uint32_t v = 0xFFFFFFFFu;
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        if (s[r] != dead && (cnt == 0 || s[r] > cur)) v = min(v, s[r]);
                    v = __reduce_min_sync(kFull, v);
                    if (v == 0xFFFFFFFFu) {
                        more = false;
                    } else {
                        if (cnt == 0) first = v;
                        cur = v;
                        if (++cnt > kMaxD) more = false;
                    }
                }
                if (lane == 0) {
                    if (cnt > kMaxD) {
                        p.dinfo[ch] = (0xFFu << 16) | first;
                        atomicOr(p.status, kStatusWide);
                    } else {
                        p.dinfo[ch] = (cnt << 16) | first;
                    }
                }
            }
        }

        // ---------------- converged phase: each lane finishes its own chunk's single run
        if (my_pending) {
            const uint64_t ch = chunk0 + lane;
            const uint64_t end = chunk_begin(ch + 1, p.len, p.c);
            uint64_t pos = my_pos;
            uint32_t s = my_state;
            const uint8_t *t = p.text;
            while (pos < end && (reinterpret_cast<uintptr_t>(t + pos) & 15)) {
                s = T.next(s, T.cls_of(__ldg(t + pos)));
                ++pos;
            }
            while (pos + 16 <= end && s != dead) {
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(t + pos));
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
#pragma unroll
                    for (int bb = 0; bb < 4; ++bb) s = T.next(s, T.cls_of((w[q] >> (8 * bb)) & 0xFF));
                }
                pos += 16;
            }
            while (pos < end && s != dead) {
                s = T.next(s, T.cls_of(__ldg(t + pos)));
                ++pos;
            }
            uint16_t *row = p.maps + ch * A.k;
            const uint16_t val = s == dead ? kUndef : static_cast<uint16_t>(s);
            bool any = false;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint32_t m = my_alive[r];
                any |= m != 0;
                for (uint32_t l = 0; l < 32; ++l) {
                    const uint32_t a = r * 32 + l;
                    if (a < A.k) row[a] = ((m >> l) & 1) ? val : kUndef;
                }
            }
            const bool live = any && s != dead;
            p.dinfo[ch] = live ? ((1u << 16) | s) : static_cast<uint32_t>(kUndef);
        }
    }
}

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
    if (!s_last || tid != 0) return;
    __threadfence();
    // ---- last block: compose the block products in order, then head and acceptance
    Prod tot;
    tot.nrows = 0xFFFFFFFFu;
    for (uint32_t b = 0; b < gridDim.x; ++b) {
        const volatile uint32_t *q = p.partials + static_cast<uint64_t>(b) * (1 + kMaxD);
        Prod x;
        x.nrows = q[0];
        for (uint32_t r = 0; r < kMaxD; ++r) x.rows[r] = q[1 + r];
        compose(tot, x);
    }
    *p.ticket = 0;   // ready for the next launch on this scratch
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

// --------------------------------------------------------------------------- host side
inline int cuda_fail(cudaError_t e) {
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? RIDFA_E_NOMEM : RIDFA_E_CUDA;
}

int upload(const HostAutomaton &H, DeviceAutomaton &D, int dev) {
    D.device = dev;
    const size_t bt = H.trans.size() * 2, bf = H.final_bits.size() * 4, bi = H.ifmask.size() * 4,
                 bs = H.slot_state.size() * 2;
    auto al = [](size_t x) { return (x + 255) & ~static_cast<size_t>(255); };
    const size_t total = al(bt) + al(256) + al(bf) + al(bi) + al(bs);
    uint8_t *base = nullptr;
    cudaError_t e = cudaMalloc(&base, total);
    if (e != cudaSuccess) return cuda_fail(e);
    size_t off = 0;
    D.trans = reinterpret_cast<uint16_t *>(base + off); off += al(bt);
    D.classmap = base + off; off += al(256);
    D.final_bits = reinterpret_cast<uint32_t *>(base + off); off += al(bf);
    D.ifmask = reinterpret_cast<uint32_t *>(base + off); off += al(bi);
    D.slot_state = reinterpret_cast<uint16_t *>(base + off); off += al(bs);
    D.bytes = total;
    e = cudaMemcpy(D.trans, H.trans.data(), bt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(D.classmap, H.classmap.data(), 256, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && bf) e = cudaMemcpy(D.final_bits, H.final_bits.data(), bf, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && bi) e = cudaMemcpy(D.ifmask, H.ifmask.data(), bi, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && bs) e = cudaMemcpy(D.slot_state, H.slot_state.data(), bs, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(base);
        D = DeviceAutomaton{};
        return cuda_fail(e);
    }
    return RIDFA_OK;
}

struct Layout {   // scratch layout for one call
    size_t maps_off, dinfo_off, partials_off, ticket_off, status_off, accept_off, total;
};

Layout layout_for(uint64_t c, uint32_t k, bool need_maps, uint32_t join_blocks) {
    auto al = [](size_t x) { return (x + 255) & ~static_cast<size_t>(255); };
    Layout L{};
    size_t off = 0;
    L.ticket_off = off; off += 256;
    L.status_off = off; off += 256;
    L.accept_off = off; off += 256;
    L.partials_off = off; off += al(static_cast<size_t>(join_blocks) * (1 + kMaxD) * 4);
    L.dinfo_off = off; off += al(c * 4);
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

int smem_optin_limit() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

template <int R, bool SMEM>
cudaError_t launch_reach_t(const ReachArgs &a, int grid, int block, size_t smem, cudaStream_t st) {
    auto kern = rid_reach_kernel<R, SMEM>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

template <bool SMEM>
cudaError_t launch_reach_r(int R, const ReachArgs &a, int grid, int block, size_t smem, cudaStream_t st) {
    switch (R) {
        case 1: return launch_reach_t<1, SMEM>(a, grid, block, smem, st);
        case 2: return launch_reach_t<2, SMEM>(a, grid, block, smem, st);
        case 4: return launch_reach_t<4, SMEM>(a, grid, block, smem, st);
        default: return launch_reach_t<8, SMEM>(a, grid, block, smem, st);
    }
}

int recognize_impl(const ridfa_program *P, bool use_dfa, const uint8_t *d_text, size_t len,
                   uint32_t n_chunks, const ridfa_tuning *tuning, uint8_t *d_accept_user,
                   uint8_t *h_accept, uint16_t *d_maps_user, cudaStream_t st) {
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
    uint32_t per_thread = static_cast<uint32_t>(std::max<uint64_t>(1, (nbound + static_cast<uint64_t>(kJoinThreads) * sms * 2 - 1) /
                                                                         (static_cast<uint64_t>(kJoinThreads) * sms * 2)));
    uint32_t join_blocks = static_cast<uint32_t>(std::max<uint64_t>(1, (nbound + static_cast<uint64_t>(kJoinThreads) * per_thread - 1) /
                                                                           (static_cast<uint64_t>(kJoinThreads) * per_thread)));
    const Layout L = layout_for(c, H.k, d_maps_user == nullptr, join_blocks);
    DeviceScratch *S = scratch_for(P, dev, L.total, &err);
    if (!S) return err;
    uint8_t *base = static_cast<uint8_t *>(S->base);
    uint32_t *ticket = reinterpret_cast<uint32_t *>(base + L.ticket_off);
    uint32_t *status = reinterpret_cast<uint32_t *>(base + L.status_off);
    uint8_t *accept = d_accept_user ? d_accept_user : base + L.accept_off;
    uint16_t *maps = d_maps_user ? d_maps_user : reinterpret_cast<uint16_t *>(base + L.maps_off);
    uint32_t *dinfo = reinterpret_cast<uint32_t *>(base + L.dinfo_off);
    uint32_t *partials = reinterpret_cast<uint32_t *>(base + L.partials_off);

    Automaton A{D->trans, D->classmap, D->final_bits, D->ifmask, D->slot_state,
                H.n_states, H.n_classes, H.k, H.kw, H.q0_slot};
    e = cudaMemsetAsync(status, 0, 4, st);
    if (e != cudaSuccess) return cuda_fail(e);

    // ---- reach
    ReachArgs ra{A, d_text, len, n_chunks, maps, dinfo, status, 8, 0};
    if (tuning && tuning->probe_interval) ra.probe = tuning->probe_interval;
    const int R = H.k <= 32 ? 1 : H.k <= 64 ? 2 : H.k <= 128 ? 4 : 8;
    const size_t tab_bytes = static_cast<size_t>(H.n_states + 1) * H.n_classes * 2;
    const size_t smem_full = 256 + tab_bytes;
    const bool in_smem = smem_full <= static_cast<size_t>(smem_optin_limit()) - 1024;
    const int block = (tuning && tuning->block_threads) ? static_cast<int>(tuning->block_threads) : 256;
    if (block < 32 || block > 256 || block % 32) return RIDFA_E_ARG;
    const uint64_t tasks = (c + 31) / 32;
    int grid;
    if (tuning && tuning->grid_blocks) {
        grid = static_cast<int>(tuning->grid_blocks);
    } else {
        int per_sm = 0;
        if (in_smem) {
            switch (R) {
                case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rid_reach_kernel<1, true>, block, smem_full); break;
                case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rid_reach_kernel<2, true>, block, smem_full); break;
                case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rid_reach_kernel<4, true>, block, smem_full); break;
                default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rid_reach_kernel<8, true>, block, smem_full); break;
            }
        }
        per_sm = std::max(per_sm, 1);
        const uint64_t warps_per_block = block / 32;
        const uint64_t need = (tasks + warps_per_block - 1) / warps_per_block;
        grid = static_cast<int>(std::min<uint64_t>(need, static_cast<uint64_t>(sms) * per_sm));
    }
    ra.table_in_smem = in_smem ? 1 : 0;
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
    e = in_smem ? launch_reach_r<true>(R, ra, grid, block, smem_full, st)
                : launch_reach_r<false>(R, ra, grid, block, 256, st);
    if (e != cudaSuccess) return cuda_fail(e);
    if (prof) cudaEventRecord(static_cast<cudaEvent_t>(S->ev[1]), st);

    // ---- join
    JoinArgs ja{A, n_chunks, maps, dinfo, status, partials, ticket, accept, per_thread};
    rid_join_kernel<<<join_blocks, kJoinThreads, 0, st>>>(ja);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
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

}  // namespace ridfa

extern "C" int ridfa_recognize(const ridfa_program *prog, const uint8_t *d_text, size_t len,
                               uint32_t n_chunks, const ridfa_tuning *tuning, uint8_t *h_accept,
                               uint16_t *d_chunk_maps, void *stream) {
    if (!h_accept) return RIDFA_E_ARG;
    return ridfa::recognize_impl(prog, false, d_text, len, n_chunks, tuning, nullptr, h_accept,
                                 d_chunk_maps, static_cast<cudaStream_t>(stream));
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
        return (*s.h_status_pinned & 2u) ? RIDFA_E_STATE : RIDFA_OK;
    }
    return RIDFA_OK;
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

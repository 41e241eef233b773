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
static_assert(kPartialWords == 1 + kMaxD, "join partial layout");

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
};

__device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ uint32_t lds_u16(uint32_t addr) {
    uint16_t v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ void sts_u32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(v));
}
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Table lookup policies.  A run's state is kept in the policy's own encoding (`enc`); `id`
// recovers the automaton state number.
//
// Plain: compact uint16 table [(n+1) * C] and uint8 class map, in shared memory (or global
// memory when it does not fit).  Lanes gathering different entries may hit the same bank.
struct LutPlain {
    const uint16_t *t;
    const uint8_t *cls;
    uint32_t C;
    static size_t smem_bytes(const Automaton &A) { return 256 + static_cast<size_t>(A.n + 1) * A.C * 2; }
    __device__ void setup(const Automaton &A, uint8_t *smem, bool table_in_smem) {
        uint8_t *s_cls = smem;
        uint16_t *s_t = reinterpret_cast<uint16_t *>(smem + 256);
        for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) s_cls[i] = A.classmap[i];
        if (table_in_smem)
            for (uint32_t i = threadIdx.x; i < (A.n + 1) * A.C; i += blockDim.x) s_t[i] = A.trans[i];
        t = table_in_smem ? s_t : A.trans;
        cls = s_cls;
        C = A.C;
    }
    __device__ __forceinline__ uint32_t enc(uint32_t id) const { return id; }
    __device__ __forceinline__ uint32_t id(uint32_t s) const { return s; }
    __device__ __forceinline__ uint32_t cls_of(uint32_t b) const { return cls[b]; }
    __device__ __forceinline__ uint32_t next(uint32_t s, uint32_t c) const { return t[s * C + c]; }
};

// Lane-replicated tables: every entry is stored 32 times, lane l's copy in bank l, so a warp's
// 32 gathers are always one shared-memory wavefront whatever states and bytes the lanes hold.
// Entries hold byte offsets, so a step is one add and one load:
//   class table, 32-bit words: word (b * 32 + l) = class offset of byte b;
//   Rep16 transition table, 16-bit halves: entry (s, c) at byte
//       (s * Cp/2 + c/2) * 128 + l * 4 + (c & 1) * 2,   value = state offset s' * Cp * 64;
//   Rep32 transition table, 32-bit words: entry (s, c) at word (s * C + c) * 32 + l,
//       value = s' * C * 128.
template <bool W16>
struct LutRep {
    uint32_t lc, lt;          // shared addresses of this lane's class / transition copies
    uint32_t row;             // state offset stride
    __host__ __device__ static uint32_t cpad(const Automaton &A) { return W16 ? (A.C + 1) & ~1u : A.C; }
    static size_t smem_bytes(const Automaton &A) {
        return 256 * 128 + static_cast<size_t>(A.n + 1) * cpad(A) * (W16 ? 64 : 128);
    }
    static bool fits16(const Automaton &A) {
        return static_cast<uint64_t>(A.n) * cpad(A) * 64 + 128 * ((cpad(A) - 1) / 2) + 2 <= 0xFFFF;
    }
    __device__ __forceinline__ uint32_t cls_off(uint32_t c) const {
        return W16 ? (c >> 1) * 128 + (c & 1) * 2 : c * 128;
    }
    __device__ void setup(const Automaton &A, uint8_t *smem, bool) {
        const uint32_t Cp = cpad(A);
        row = W16 ? Cp * 64 : Cp * 128;
        const uint32_t base_c = smem_addr(smem);
        const uint32_t base_t = base_c + 256 * 128;
        for (uint32_t i = threadIdx.x; i < 256 * 32; i += blockDim.x)
            sts_u32(base_c + i * 4, cls_off(A.classmap[i >> 5]));
        const uint32_t words = W16 ? (A.n + 1) * Cp / 2 : (A.n + 1) * Cp;
        for (uint32_t i = threadIdx.x; i < words * 32; i += blockDim.x) {
            const uint32_t w = i >> 5;
            uint32_t v;
            if (W16) {
                const uint32_t s = (2 * w) / Cp, c0 = (2 * w) % Cp;
                const uint32_t n0 = A.trans[s * A.C + c0];
                const uint32_t n1 = (c0 + 1 < A.C) ? A.trans[s * A.C + c0 + 1] : A.n;
                v = (n0 * row) | ((n1 * row) << 16);
            } else {
                v = A.trans[w] * row;
            }
            sts_u32(base_t + i * 4, v);
        }
        const uint32_t lane = threadIdx.x & 31;
        lc = base_c + lane * 4;
        lt = base_t + lane * 4;
    }
    __device__ __forceinline__ uint32_t enc(uint32_t id) const { return id * row; }
    __device__ __forceinline__ uint32_t id(uint32_t s) const { return s / row; }
    __device__ __forceinline__ uint32_t cls_of(uint32_t b) const { return lds_u32(lc + b * 128); }
    __device__ __forceinline__ uint32_t next(uint32_t s, uint32_t c) const {
        return W16 ? lds_u16(lt + s + c) : lds_u32(lt + s + c);
    }
};

// Chunk-map row of one chunk written by one lane: entries of alive slots get `val`.
template <int R>
__device__ __forceinline__ void write_row(uint16_t *row, uint32_t k, const uint32_t (&alive)[R],
                                          uint16_t val) {
    if ((k & 1) == 0) {
        uint32_t *row32 = reinterpret_cast<uint32_t *>(row);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t m = alive[r];
            for (uint32_t l = 0; l < 32; l += 2) {
                const uint32_t a = r * 32 + l;
                if (a >= k) break;
                const uint32_t lo = ((m >> l) & 1) ? val : kUndef;
                const uint32_t hi = ((m >> (l + 1)) & 1) ? val : kUndef;
                row32[a >> 1] = lo | (hi << 16);
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t m = alive[r];
            for (uint32_t l = 0; l < 32; ++l) {
                const uint32_t a = r * 32 + l;
                if (a >= k) break;
                row[a] = ((m >> l) & 1) ? val : kUndef;
            }
        }
    }
}

template <int R, class LUT, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1) rid_reach_kernel(ReachArgs p, int table_in_smem) {
    extern __shared__ __align__(16) uint8_t smem[];
    const Automaton &A = p.A;
    LUT T;
    T.setup(A, smem, table_in_smem != 0);
    __syncthreads();

    const uint32_t lane = threadIdx.x & 31;
    const uint32_t dead = T.enc(A.n);
    const uint64_t n_tasks = (static_cast<uint64_t>(p.c) + 31) / 32;
    const uint64_t warp0 = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;

    // slot start states of this lane (slot a = r*32 + lane)
    uint32_t start_state[R];
    uint32_t start_live = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t a = r * 32 + lane;
        start_state[r] = a < A.k ? T.enc(A.slot_state[a]) : dead;
        if (r * 32 < static_cast<int>(A.k)) start_live |= 1u << r;
    }

    for (uint64_t task = warp0; task < n_tasks; task += n_warps) {
        const uint64_t chunk0 = task * 32;
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
            uint32_t live_regs = start_live;       // registers holding at least one live run
            uint64_t pos = beg;
            bool converged = false;
            uint32_t conv_state = dead;
            while (pos < end) {
                const uint64_t stop = min(end, pos + p.probe);
                for (; pos < stop; ++pos) {
                    const uint32_t c = T.cls_of(__ldg(p.text + pos));
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        if (live_regs & (1u << r)) s[r] = T.next(s[r], c);
                }
                // convergence: are all live runs in one state?  (dead runs are dropped)
                uint32_t lo = 0xFFFFFFFFu, hi = 0;
                live_regs = 0;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (__any_sync(kFull, s[r] != dead)) live_regs |= 1u << r;
                    if (s[r] != dead) {
                        lo = min(lo, s[r]);
                        hi = max(hi, s[r]);
                    }
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
                    const uint32_t b = __ballot_sync(kFull, s[r] != dead);
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
                    const uint32_t a = r * 32 + lane;
                    if (a < A.k) row[a] = s[r] == dead ? kUndef : static_cast<uint16_t>(T.id(s[r]));
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
                        if (cnt == 0) first = T.id(v);
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
                uint32_t cl[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) cl[q] = T.cls_of((w[q >> 2] >> (8 * (q & 3))) & 0xFF);
#pragma unroll
                for (int q = 0; q < 16; ++q) s = T.next(s, cl[q]);
                pos += 16;
            }
            while (pos < end && s != dead) {
                s = T.next(s, T.cls_of(__ldg(t + pos)));
                ++pos;
            }
            bool any = false;
#pragma unroll
            for (int r = 0; r < R; ++r) any |= my_alive[r] != 0;
            const uint32_t sid = T.id(s);
            const uint16_t val = s == dead ? kUndef : static_cast<uint16_t>(sid);
            write_row<R>(p.maps + ch * A.k, A.k, my_alive, val);
            const bool live = any && s != dead;
            p.dinfo[ch] = live ? ((1u << 16) | sid) : static_cast<uint32_t>(kUndef);
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

enum Mode : uint32_t { kModePlain = 1, kModeRep16 = 2, kModeRep32 = 3 };

template <int R>
constexpr int block_cap() { return R <= 4 ? 1024 : 512; }

// Launch (or, with per_sm != nullptr, size) one instantiation of the reach kernel.
template <int R, class LUT>
cudaError_t reach_one(const ReachArgs &a, int table_in_smem, int grid, int block, size_t smem,
                      cudaStream_t st, int *per_sm) {
    auto kern = rid_reach_kernel<R, LUT, block_cap<R>()>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    if (per_sm) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, block, smem);
    kern<<<grid, block, smem, st>>>(a, table_in_smem);
    return cudaGetLastError();
}

template <class LUT>
cudaError_t reach_r(int R, const ReachArgs &a, int tis, int grid, int block, size_t smem,
                    cudaStream_t st, int *per_sm) {
    switch (R) {
        case 1: return reach_one<1, LUT>(a, tis, grid, block, smem, st, per_sm);
        case 2: return reach_one<2, LUT>(a, tis, grid, block, smem, st, per_sm);
        case 4: return reach_one<4, LUT>(a, tis, grid, block, smem, st, per_sm);
        default: return reach_one<8, LUT>(a, tis, grid, block, smem, st, per_sm);
    }
}

cudaError_t reach_dispatch(uint32_t mode, int R, const ReachArgs &a, int tis, int grid, int block,
                           size_t smem, cudaStream_t st, int *per_sm) {
    switch (mode) {
        case kModeRep16: return reach_r<LutRep<true>>(R, a, tis, grid, block, smem, st, per_sm);
        case kModeRep32: return reach_r<LutRep<false>>(R, a, tis, grid, block, smem, st, per_sm);
        default: return reach_r<LutPlain>(R, a, tis, grid, block, smem, st, per_sm);
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
    const uint64_t per_block_max = 1024;
    uint32_t per_thread = static_cast<uint32_t>(std::max<uint64_t>(
        1, (nbound + static_cast<uint64_t>(kJoinThreads) * per_block_max - 1) /
               (static_cast<uint64_t>(kJoinThreads) * per_block_max)));
    uint32_t join_blocks = static_cast<uint32_t>(std::max<uint64_t>(
        1, (nbound + static_cast<uint64_t>(kJoinThreads) * per_thread - 1) /
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
    ReachArgs ra{A, d_text, len, n_chunks, maps, dinfo, status, 8};
    if (tuning && tuning->probe_interval) ra.probe = tuning->probe_interval;
    const int R = H.k <= 32 ? 1 : H.k <= 64 ? 2 : H.k <= 128 ? 4 : 8;
    const size_t limit = static_cast<size_t>(smem_optin_limit()) - 1024;
    // table layout: lane-replicated 16-bit offsets, else 32-bit offsets, else the compact table
    uint32_t mode = tuning ? tuning->table_mode : 0;
    const size_t rep16 = LutRep<true>::smem_bytes(A), rep32 = LutRep<false>::smem_bytes(A);
    if (mode == 0)
        mode = (LutRep<true>::fits16(A) && rep16 <= limit) ? kModeRep16
               : (rep32 <= limit) ? kModeRep32 : kModePlain;
    if (mode == kModeRep16 && !(LutRep<true>::fits16(A) && rep16 <= limit)) return RIDFA_E_ARG;
    if (mode == kModeRep32 && rep32 > limit) return RIDFA_E_ARG;
    if (mode < kModePlain || mode > kModeRep32) return RIDFA_E_ARG;
    const size_t plain_bytes = LutPlain::smem_bytes(A);
    const int tis = (mode == kModePlain && plain_bytes <= limit) ? 1 : 0;
    const size_t smem = mode == kModeRep16 ? rep16 : mode == kModeRep32 ? rep32 : (tis ? plain_bytes : 256);
    const int cap = R <= 4 ? 1024 : 512;
    int block = (tuning && tuning->block_threads) ? static_cast<int>(tuning->block_threads)
                                                  : (mode == kModePlain ? 256 : cap);
    if (block < 32 || block > cap || block % 32) return RIDFA_E_ARG;
    const uint64_t tasks = (c + 31) / 32;
    int grid;
    if (tuning && tuning->grid_blocks) {
        grid = static_cast<int>(tuning->grid_blocks);
    } else {
        int per_sm = 0;
        e = reach_dispatch(mode, R, ra, tis, 0, block, smem, st, &per_sm);
        if (e != cudaSuccess) return cuda_fail(e);
        if (per_sm < 1) return RIDFA_E_UNSUPPORTED;
        const uint64_t warps_per_block = block / 32;
        const uint64_t need = (tasks + warps_per_block - 1) / warps_per_block;
        grid = static_cast<int>(std::min<uint64_t>(need, static_cast<uint64_t>(sms) * per_sm));
    }
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
    e = reach_dispatch(mode, R, ra, tis, grid, block, smem, st, nullptr);
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
                H.n_states, H.n_classes, H.k, H.kw, H.q0_slot};
    ReachArgs ra{A, d_text, len, n_chunks, B.maps, B.dinfo, B.status, 8};
    const int R = H.k <= 32 ? 1 : H.k <= 64 ? 2 : H.k <= 128 ? 4 : 8;
    const size_t limit = static_cast<size_t>(smem_optin_limit()) - 1024;
    const size_t rep16 = LutRep<true>::smem_bytes(A), rep32 = LutRep<false>::smem_bytes(A);
    const uint32_t mode = (LutRep<true>::fits16(A) && rep16 <= limit) ? kModeRep16
                          : (rep32 <= limit) ? kModeRep32 : kModePlain;
    const size_t plain_bytes = LutPlain::smem_bytes(A);
    const int tis = (mode == kModePlain && plain_bytes <= limit) ? 1 : 0;
    const size_t smem = mode == kModeRep16 ? rep16 : mode == kModeRep32 ? rep32 : (tis ? plain_bytes : 256);
    const int block = mode == kModePlain ? 256 : (R <= 4 ? 1024 : 512);
    int per_sm = 0;
    e = reach_dispatch(mode, R, ra, tis, 0, block, smem, st, &per_sm);
    if (e != cudaSuccess) return cuda_fail(e);
    if (per_sm < 1) return RIDFA_E_UNSUPPORTED;
    const uint64_t tasks = (c + 31) / 32;
    const uint64_t need = (tasks + block / 32 - 1) / (block / 32);
    const int grid = static_cast<int>(std::min<uint64_t>(need, static_cast<uint64_t>(sms) * per_sm));
    e = reach_dispatch(mode, R, ra, tis, grid, block, smem, st, nullptr);
    if (e != cudaSuccess) return cuda_fail(e);
    JoinArgs ja{A, n_chunks, B.maps, B.dinfo, B.status, B.partials, B.ticket, B.accept,
                static_cast<uint32_t>(per_thread)};
    rid_join_kernel<<<join_blocks, kJoinThreads, 0, st>>>(ja);
    e = cudaGetLastError();
    return e == cudaSuccess ? RIDFA_OK : cuda_fail(e);
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

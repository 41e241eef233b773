// Batched recognition: many texts against many programs in one CUDA graph.
//
// The paper recognises one text at a time (Sec. 3.2).  A batch runs the same reach and join,
// exactly, for every (text, program) item, with all items' chunks in one persistent reach launch
// per table layout and one join launch, captured once into a CUDA graph and replayed by
// ridfa_batch_run:
//   * reach: CTAs take tasks (up to 32 chunks per warp of one program) from an atomic ticket;
//     tasks are ordered by program, so a CTA reloads its shared-memory tables only when the
//     program changes.  Each warp runs the speculative phase of its chunks (lanes = runs) and
//     then finishes the converged runs one per lane, with the text staged by cp.async exactly as
//     the single-text kernel does.  Chunk i of an item covers text[floor(i*len/c), ...).
//   * join: one block per segment of up to 256 chunk boundaries of one text; each thread forms
//     one transfer matrix M_i (as in the single-text join), the block multiplies them, and the
//     last segment of a text (per-text atomic ticket) multiplies the segment products in order and
//     evaluates lambda_1(q0) and the acceptance test.  A text with more than 32 distinct end
//     states in some chunk is finished by that last block propagating if_min(PLAS_i) chunk by chunk.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "ridfa_batch_plan.h"
#include "ridfa_internal.h"
#include "ridfa_kernels.cuh"

namespace ridfa {
namespace {

struct TextDesc {             // one item
    const uint8_t *text;
    uint64_t len;
    uint64_t chunk_base;      // first chunk of this text in its program's chunk numbering
    uint32_t c;               // chunks (0 for an empty text)
    uint32_t item;            // index into d_accept
};

struct ProgDesc {
    Automaton A;
    const TextDesc *texts;    // this program's texts, chunk_base ascending
    uint16_t *maps;           // [n_chunks][k]
    uint32_t *dinfo;          // [n_chunks]
    uint32_t n_texts;
    uint32_t tis;             // compact table in shared memory (Plain layout)
    uint32_t text0;           // global index of texts[0]
    uint32_t pad;
};

struct TaskDesc {
    uint64_t chunk0;
    uint32_t prog;
    uint32_t count;
};

struct SegDesc {
    uint64_t b0;              // first boundary (chunk index >= 1) of the segment
    uint32_t prog, text;      // text: global text index
    uint32_t count, seg, nseg, part0;
};

struct BatchReachArgs {
    const ProgDesc *progs;
    const TaskDesc *tasks;
    uint32_t n_tasks;
    uint32_t probe;
    uint32_t *counter;
    uint32_t *status;
    RunEntry *runs;           // [grid warps][kRunsPerWarp]
    uint32_t *finals;         // [grid warps][kFinalsPerWarp]
};

struct BatchJoinArgs {
    const ProgDesc *progs;
    const TextDesc *texts;    // all texts, grouped by program
    const SegDesc *segs;
    uint32_t *partials;       // [segments][kPartialWords]
    uint32_t *tickets;        // [texts]
    uint32_t *flags;          // [texts]
    uint8_t *accept;
    uint32_t *status;
};

constexpr int kBatchJoinThreads = 256;

// Text of program-local chunk ch, starting the search at *t (chunks of a slice ascend).
__device__ __forceinline__ const TextDesc *text_of(const ProgDesc &P, uint64_t ch, uint32_t *t) {
    uint32_t i = *t;
    while (i + 1 < P.n_texts && P.texts[i + 1].chunk_base <= ch) ++i;
    *t = i;
    return &P.texts[i];
}

__device__ __forceinline__ uint32_t first_text(const ProgDesc &P, uint64_t ch) {
    uint32_t lo = 0, hi = P.n_texts - 1;          // last text with chunk_base <= ch
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) / 2;
        if (P.texts[mid].chunk_base <= ch) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// How a batch reach launch's converged runs read the text: plain 16-byte global loads, warp-
// cooperative staging, or staging with each lane finishing all the runs its chunk handed off.
constexpr int kTpGlobal = 0, kTpCoop = 1, kTpSet = 2;

template <int R, class LUT, int BLOCK, int TP>
__global__ void __launch_bounds__(BLOCK, 1) rid_reach_batch_kernel(BatchReachArgs b, uint32_t staging_offset) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ uint32_t s_task;
    LUT T;
    int cur = -1;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t stg_base = smem_addr(smem) + staging_offset + warp * kWarpCoopBytes;
    const uint64_t gwarp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    RunEntry *const wruns = b.runs + gwarp * kRunsPerWarp;
    uint32_t *const wfin = b.finals + gwarp * kFinalsPerWarp;
    uint32_t *const wball = wfin + kRunsPerWarp;
    for (;;) {
        if (threadIdx.x == 0) s_task = atomicAdd(b.counter, 1u);
        __syncthreads();
        const uint32_t t = s_task;
        if (t >= b.n_tasks) break;
        const TaskDesc task = b.tasks[t];
        const ProgDesc &P = b.progs[task.prog];
        const Automaton &A = P.A;
        if (static_cast<int>(task.prog) != cur) {
            T.setup(A, smem, P.tis);
            __syncthreads();
            cur = static_cast<int>(task.prog);
        }
        const uint64_t c0 = task.chunk0 + 32ull * warp;
        const uint64_t cend = task.chunk0 + task.count;
        if (c0 < cend) {
            const uint32_t nch = static_cast<uint32_t>(min(static_cast<uint64_t>(32), cend - c0));
            // slot start states of this lane (slot a = r*32 + lane)
            const uint32_t dead = T.enc(A.n);
            uint32_t start_state[R];
            uint32_t start_live = 0;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint32_t a = r * 32 + lane;
                start_state[r] = a < A.k ? T.enc(__ldg(A.slot_state + a)) : dead;
                if (r * 32 < static_cast<int>(A.k)) start_live |= 1u << r;
            }
            // ---- speculative phase, chunk by chunk; up to kMaxRun runs handed off per chunk
            uint32_t my_hand = 0;     // owner lane j of a handed-off chunk: (m << 16) | first run
            uint32_t my_ti = 0;       // owner lane j: text index of chunk j
            uint32_t nruns = 0, handed = 0;
            uint32_t amask[R];
#pragma unroll
            for (int r = 0; r < R; ++r) amask[r] = 0;
            uint32_t ti = first_text(P, c0);
            for (uint32_t j = 0; j < nch; ++j) {
                const uint64_t ch = c0 + j;
                const TextDesc *td = text_of(P, ch, &ti);
                if (lane == j) my_ti = ti;
                const uint64_t i = ch - td->chunk_base;
                const uint64_t beg = chunk_begin(i, td->len, td->c), end = chunk_begin(i + 1, td->len, td->c);
                uint64_t hp = 0;
                uint32_t d, al[R];
                const int m = speculate<R, LUT, TP == kTpSet ? kMultiMinSet : kMultiMin>(
                    T, A, td->text, beg, end, b.probe, lane, start_state, start_live, dead, P.maps + ch * A.k,
                    P.dinfo + ch, b.status, true, false, &hp, &d, al);
                if (m >= 1) {
                    handed |= 1u << j;
#pragma unroll
                    for (int r = 0; r < R; ++r) amask[r] |= ((al[r] >> lane) & 1u) << j;
                    if (lane < static_cast<uint32_t>(m))
                        wruns[nruns + lane] = RunEntry{hp, d, static_cast<uint16_t>(j), static_cast<uint16_t>(lane)};
                    if (lane == j) my_hand = (static_cast<uint32_t>(m) << 16) | nruns;
                    nruns += static_cast<uint32_t>(m);
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) wball[r * 32 + lane] = amask[r];
            __syncwarp();
            // ---- converged phase: each lane finishes one run (rounds of 32 runs); on the set
            // path, when some chunk handed off several runs, each lane finishes its chunk's runs
            // together
            uint32_t fin_reg = dead;
            const bool set_path = TP == kTpSet && nruns != static_cast<uint32_t>(__popc(handed));
            if (set_path) {
                const uint32_t m = my_hand >> 16, run0 = my_hand & 0xFFFF;
                uint32_t stv[kMaxRun];
                uint64_t pos = 0, end = 0, lim = 0;
                const uint8_t *tx = nullptr;
#pragma unroll
                for (int g = 0; g < kMaxRun; ++g) stv[g] = dead;
                if (m) {
#pragma unroll
                    for (int g = 0; g < kMaxRun; ++g)
                        if (g < static_cast<int>(m)) stv[g] = wruns[run0 + g].state;
                    pos = wruns[run0].pos;
                    const TextDesc &td = P.texts[my_ti];
                    end = chunk_begin(c0 + lane - td.chunk_base + 1, td.len, td.c);
                    lim = td.len & ~static_cast<uint64_t>(15);
                    tx = td.text;
                }
                uint32_t rep = 0xFFFFFFFFu;            // group g -> its slot (4 bits; 0xF dead)
#pragma unroll
                for (int g = 0; g < kMaxRun; ++g)
                    if (g < static_cast<int>(m)) rep = (rep & ~(0xFu << (4 * g))) | (static_cast<uint32_t>(g) << (4 * g));
                coop_converge_set(T, stg_base, lane, m != 0, tx, lim, min(end, lim), pos, stv, rep, dead);
                if (m) finish_set_runs(T, tx, pos, end, stv, rep, m, wfin + run0, dead);
            }
            for (uint32_t rb = 0; rb < (set_path ? 0u : nruns); rb += 32) {
                const uint32_t idx = rb + lane;
                const bool pending = idx < nruns;
                uint64_t pos = 0, end = 0, lim = 0;
                uint32_t s = dead, jj = 0;
                if (pending) {
                    const RunEntry e = wruns[idx];
                    pos = e.pos;
                    s = e.state;
                    jj = e.chunk;
                }
                const uint32_t tix = __shfl_sync(kFull, my_ti, jj);
                const uint8_t *tx = nullptr;
                if (pending) {
                    const TextDesc &td = P.texts[tix];
                    end = chunk_begin(c0 + jj - td.chunk_base + 1, td.len, td.c);
                    lim = td.len & ~static_cast<uint64_t>(15);
                    tx = td.text;
                }
                if (TP != kTpGlobal && __any_sync(kFull, pending))
                    coop_converge<LUT, false>(T, stg_base, lane, pending, tx, lim, min(end, lim), pos, s, dead);
                if (pending) {
                    tail_converge<LUT, TP == kTpGlobal>(T, tx, pos, end, s, dead);
                    if (nruns > 32) wfin[idx] = s;
                    else fin_reg = s;
                }
            }
            __syncwarp();
            // ---- rows of the handed-off chunks, one chunk at a time by the warp
#pragma unroll
            for (int r = 0; r < R; ++r) amask[r] = wball[r * 32 + lane];
            for (uint32_t hm = handed; hm; hm &= hm - 1) {
                const uint32_t j = __ffs(hm) - 1;
                const uint32_t hand = __shfl_sync(kFull, my_hand, j);
                const uint32_t m = hand >> 16, run0 = hand & 0xFFFF;
                const uint32_t src = run0 + min(lane, m - 1);
                uint32_t fin = __shfl_sync(kFull, fin_reg, src & 31);
                if (nruns > 32 || set_path) fin = wfin[src];
                uint32_t am = 0;
#pragma unroll
                for (int r = 0; r < R; ++r) am |= ((amask[r] >> j) & 1u) << r;
                finish_handed_row<R, LUT>(T, P.maps + (c0 + j) * A.k, A.k, m, m >= 2, lane, am, fin, dead,
                                          P.dinfo + c0 + j);
            }
        }
        __syncthreads();   // every warp is done with this task before the tables may change
    }
}

// ---------------------------------------------------------------------------- batch join
struct BProd {
    uint32_t nrows;           // 0xFFFFFFFF = identity
    uint32_t rows[kMaxD];
};

__device__ void bcompose(BProd &a, const BProd &b) {
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

// Distinct defined values of row i (ascending, at most kMaxD; 0xFFFFFFFF when wider).
__device__ uint32_t bdistinct(const Automaton &A, const uint16_t *maps_t, const uint32_t *dinfo_t, uint64_t i,
                              uint16_t *D) {
    const uint32_t info = dinfo_t[i];
    const uint32_t m = info >> 16;
    if (m <= 1) {
        D[0] = static_cast<uint16_t>(info & 0xFFFF);
        return m;
    }
    if (m > kMaxD) return 0xFFFFFFFFu;
    const uint16_t *row = maps_t + i * A.k;
    uint32_t cnt = 0;
    for (uint32_t a = 0; a < A.k; ++a) {
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

__device__ __forceinline__ uint32_t bindex(const uint16_t *D, uint32_t m, uint16_t v) {
    for (uint32_t j = 0; j < m; ++j)
        if (D[j] == v) return j;
    return 0xFFFFFFFFu;
}

__global__ void __launch_bounds__(kBatchJoinThreads) rid_join_batch_kernel(BatchJoinArgs J) {
    __shared__ BProd s_prod[kBatchJoinThreads];
    __shared__ bool s_last, s_wide;
    __shared__ uint32_t s_vec[RIDFA_MAX_SLOTS / 32], s_nvec[RIDFA_MAX_SLOTS / 32];
    __shared__ uint32_t s_acc;
    __shared__ int s_wideflag, s_badflag;
    if (threadIdx.x == 0) {
        s_wideflag = 0;
        s_badflag = 0;
    }
    __syncthreads();
    const SegDesc seg = J.segs[blockIdx.x];
    const ProgDesc &P = J.progs[seg.prog];
    const Automaton &A = P.A;
    const TextDesc &td = J.texts[seg.text];
    const uint16_t *maps_t = P.maps + td.chunk_base * A.k;
    const uint32_t *dinfo_t = P.dinfo + td.chunk_base;
    const uint32_t tid = threadIdx.x;

    BProd Pr;
    Pr.nrows = 0xFFFFFFFFu;
    bool wide = false, bad = false;
    if (tid < seg.count) {
        const uint64_t i = seg.b0 + tid;            // boundary between chunks i-1 and i
        uint16_t Dp[kMaxD], Dc[kMaxD];
        const uint32_t mp = bdistinct(A, maps_t, dinfo_t, i - 1, Dp);
        const uint32_t mc = bdistinct(A, maps_t, dinfo_t, i, Dc);
        if (mp == 0xFFFFFFFFu || mc == 0xFFFFFFFFu) {
            wide = true;
        } else {
            Pr.nrows = mp;
            const uint16_t *row = maps_t + i * A.k;
            for (uint32_t x = 0; x < mp; ++x) {
                const uint32_t *mask = A.ifmask + static_cast<uint64_t>(Dp[x]) * A.kw;
                uint32_t out = 0;
                for (uint32_t w = 0; w < A.kw; ++w) {
                    uint32_t bits = mask[w];
                    while (bits) {
                        const uint32_t a = w * 32 + __ffs(bits) - 1;
                        bits &= bits - 1;
                        const uint16_t v = row[a];
                        if (v == kUndef) continue;
                        const uint32_t y = bindex(Dc, mc, v);
                        if (y == 0xFFFFFFFFu) bad = true;
                        else out |= 1u << y;
                    }
                }
                Pr.rows[x] = out;
            }
        }
    }
    if (bad) s_badflag = 1;
    if (wide) s_wideflag = 1;
    s_prod[tid] = Pr;
    __syncthreads();
    for (uint32_t stride = 1; stride < blockDim.x; stride *= 2) {
        if ((tid % (2 * stride)) == 0 && tid + stride < blockDim.x) bcompose(s_prod[tid], s_prod[tid + stride]);
        __syncthreads();
    }
    uint32_t *mine = J.partials + static_cast<uint64_t>(seg.part0 + seg.seg) * kPartialWords;
    if (tid == 0) {
        if (s_badflag) atomicOr(J.status, kStatusBad);
        if (s_wideflag) atomicOr(&J.flags[seg.text], 1u);
        mine[0] = s_prod[0].nrows;
        if (s_prod[0].nrows != 0xFFFFFFFFu)
            for (uint32_t x = 0; x < s_prod[0].nrows; ++x) mine[1 + x] = s_prod[0].rows[x];
        __threadfence();
        const uint32_t t = atomicAdd(&J.tickets[seg.text], 1u);
        s_last = (t == seg.nseg - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (tid == 0) s_wide = (*reinterpret_cast<volatile uint32_t *>(&J.flags[seg.text]) & 1u) != 0;
    __syncthreads();
    const uint64_t c = td.c;
    if (c == 0) {   // empty text: is the empty word in L?
        if (tid == 0) J.accept[td.item] = is_final_state(A, A.slot_state[A.q0_slot]) ? 1 : 0;
    } else if (s_wide) {
        // sequential propagation of if_min(PLAS_i) over this text's chunks
        const uint16_t v0 = maps_t[A.q0_slot];
        if (c == 1 || v0 == kUndef) {
            if (tid == 0) J.accept[td.item] = (v0 != kUndef && is_final_state(A, v0)) ? 1 : 0;
        } else {
            for (uint32_t w = tid; w < A.kw; w += blockDim.x) s_vec[w] = A.ifmask[static_cast<uint64_t>(v0) * A.kw + w];
            __syncthreads();
            for (uint64_t i = 1; i + 1 < c; ++i) {
                for (uint32_t w = tid; w < A.kw; w += blockDim.x) s_nvec[w] = 0;
                __syncthreads();
                const uint16_t *row = maps_t + i * A.k;
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
            if (tid == 0) s_acc = 0;
            __syncthreads();
            const uint16_t *last = maps_t + (c - 1) * A.k;
            for (uint32_t a = tid; a < A.k; a += blockDim.x)
                if (((s_vec[a >> 5] >> (a & 31)) & 1) && last[a] != kUndef && is_final_state(A, last[a])) s_acc = 1;
            __syncthreads();
            if (tid == 0) J.accept[td.item] = s_acc ? 1 : 0;
        }
    } else if (tid == 0) {
        BProd tot;
        tot.nrows = 0xFFFFFFFFu;
        for (uint32_t sgi = 0; sgi < seg.nseg; ++sgi) {
            const volatile uint32_t *q = J.partials + static_cast<uint64_t>(seg.part0 + sgi) * kPartialWords;
            BProd x;
            x.nrows = q[0];
            if (x.nrows != 0xFFFFFFFFu)
                for (uint32_t r = 0; r < x.nrows; ++r) x.rows[r] = q[1 + r];
            bcompose(tot, x);
        }
        const uint16_t v0 = maps_t[A.q0_slot];
        uint8_t acc = 0;
        if (v0 != kUndef) {
            if (c == 1) {
                acc = is_final_state(A, v0) ? 1 : 0;
            } else {
                uint16_t D0[kMaxD], Dl[kMaxD];
                const uint32_t m0 = bdistinct(A, maps_t, dinfo_t, 0, D0);
                const uint32_t x0 = bindex(D0, m0, v0);
                const uint32_t ml = bdistinct(A, maps_t, dinfo_t, c - 1, Dl);
                if (x0 == 0xFFFFFFFFu || tot.nrows == 0xFFFFFFFFu || ml == 0xFFFFFFFFu) {
                    atomicOr(J.status, kStatusBad);
                } else {
                    const uint32_t bits = tot.rows[x0];
                    for (uint32_t y = 0; y < ml; ++y)
                        if (((bits >> y) & 1) && is_final_state(A, Dl[y])) acc = 1;
                }
            }
        }
        J.accept[td.item] = acc;
    }
    if (tid == 0) {   // ready for the next replay
        J.tickets[seg.text] = 0;
        J.flags[seg.text] = 0;
    }
}

// ---------------------------------------------------------------------------- host side
enum BMode : uint32_t { kBPlain = 1, kBRep16 = 2, kBRep32 = 3, kBFlat = 4, kBRep16x4 = 5 };

struct LaunchGroup {          // one persistent reach launch
    uint32_t mode = kBPlain;
    int R = 1;
    int tp = kTpGlobal;            // how converged runs read the text
    std::vector<uint32_t> progs;   // batch program indices in this launch
    uint32_t task0 = 0, n_tasks = 0;
    size_t table_smem = 0;
    uint64_t run0 = 0;             // first warp of this launch's run lists (groups may run at once)
    int block = 0, grid = 0;
    uint32_t stg = 0;              // staging offset in dynamic shared memory
    size_t smem = 0;               // dynamic shared memory
};

template <int R, class LUT, int TP>
cudaError_t batch_reach_one(const BatchReachArgs &a, int grid, int block, size_t smem, uint32_t stg,
                            cudaStream_t st, int *per_sm) {
    auto kern = rid_reach_batch_kernel<R, LUT, (R <= 4 && TP != kTpSet ? 1024 : 512), TP>;
    cudaError_t e = ensure_smem_cap(reinterpret_cast<const void *>(kern), smem);
    if (e != cudaSuccess) return e;
    if (per_sm) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, block, smem);
    kern<<<grid, block, smem, st>>>(a, stg);
    return cudaGetLastError();
}

template <class LUT, int TP>
cudaError_t batch_reach_r(int R, const BatchReachArgs &a, int grid, int block, size_t smem, uint32_t stg,
                          cudaStream_t st, int *per_sm) {
    switch (R) {
        case 1: return batch_reach_one<1, LUT, TP>(a, grid, block, smem, stg, st, per_sm);
        case 2: return batch_reach_one<2, LUT, TP>(a, grid, block, smem, stg, st, per_sm);
        case 4: return batch_reach_one<4, LUT, TP>(a, grid, block, smem, stg, st, per_sm);
        default: return batch_reach_one<8, LUT, TP>(a, grid, block, smem, stg, st, per_sm);
    }
}

cudaError_t batch_reach(const LaunchGroup &g, const BatchReachArgs &a, cudaStream_t st, int *per_sm) {
#define RIDFA_BATCH_MODES(TPV)                                                                                  \
    switch (g.mode) {                                                                                           \
        case kBRep16: return batch_reach_r<LutRep<true>, TPV>(g.R, a, g.grid, g.block, g.smem, g.stg, st, per_sm);  \
        case kBRep32: return batch_reach_r<LutRep<false>, TPV>(g.R, a, g.grid, g.block, g.smem, g.stg, st, per_sm); \
        case kBPlain: return batch_reach_r<LutPlain, TPV>(g.R, a, g.grid, g.block, g.smem, g.stg, st, per_sm);      \
        case kBRep16x4: return batch_reach_r<LutRep16x4, TPV>(g.R, a, g.grid, g.block, g.smem, g.stg, st, per_sm);  \
        default: return batch_reach_r<LutFlat, TPV>(g.R, a, g.grid, g.block, g.smem, g.stg, st, per_sm);           \
    }
    if (g.tp == kTpSet) { RIDFA_BATCH_MODES(kTpSet) }
    if (g.tp == kTpCoop) { RIDFA_BATCH_MODES(kTpCoop) }
    RIDFA_BATCH_MODES(kTpGlobal)
#undef RIDFA_BATCH_MODES
}

// Resident blocks per SM of a launch group's kernel, cached: setting the shared-memory attribute
// and querying occupancy once per (device, layout, R, path, block, shared memory).
int blocks_per_sm(int device, const LaunchGroup &g, int *per_sm) {
    static std::mutex mu;
    static std::map<std::tuple<int, uint32_t, int, int, int, size_t>, int> cache;
    const auto key = std::make_tuple(device, g.mode, g.R, g.tp, g.block, g.smem);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *per_sm = it->second;
        return RIDFA_OK;
    }
    BatchReachArgs a{};
    cudaError_t e = batch_reach(g, a, nullptr, per_sm);
    if (e != cudaSuccess) return cuda_fail(e);
    cache[key] = *per_sm;
    return RIDFA_OK;
}

inline size_t al256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// What the batch autotuner found for a batch: chunk length and launch shape.
struct BatchTune {
    uint32_t chunk_len = 0;
    BatchShape shape;
    bool operator==(const BatchTune &o) const {
        return chunk_len == o.chunk_len && shape.warps_cap == o.shape.warps_cap && shape.set_mode == o.shape.set_mode;
    }
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, BatchTune> g_tune_cache;   // (log2 |P|, log2 k, log2 C) -> tune

int log2i(uint32_t v) {
    int r = 0;
    while ((1u << (r + 1)) <= v && r < 30) ++r;
    return r;
}

}  // namespace

struct BatchPlan {
    std::vector<const ridfa_program *> progs;
    std::vector<const DeviceAutomaton *> dev;
    std::vector<uint32_t> tis, n_texts_of, text0;
    std::vector<uint64_t> maps_off, dinfo_off;   // within the maps / summaries regions
    std::vector<TextDesc> texts;                 // grouped by program
    std::vector<TaskDesc> tasks;
    std::vector<SegDesc> segs;
    std::vector<LaunchGroup> groups;
    uint32_t n_items = 0;
    uint64_t total_bytes = 0, total_chunks = 0;
    // block layout; everything before o_part is the host image
    size_t o_counters = 0, o_progs = 0, o_texts = 0, o_tasks = 0, o_segs = 0, o_tick = 0, o_flags = 0;
    size_t o_part = 0, o_runs = 0, o_finals = 0, o_maps = 0, o_dinfo = 0, total = 0;
};

BatchPlan *plan_new() { return new (std::nothrow) BatchPlan(); }
void plan_delete(BatchPlan *pl) { delete pl; }
size_t plan_device_bytes(const BatchPlan *pl) { return pl->total; }
size_t plan_image_bytes(const BatchPlan *pl) { return pl->o_part; }
size_t plan_status_offset(const BatchPlan *pl) { return pl->o_counters + 32 * 4; }

PlanStats plan_stats(const BatchPlan *pl) {
    PlanStats s{};
    s.total_bytes = pl->total_bytes;
    s.total_chunks = pl->total_chunks;
    s.n_programs = static_cast<uint32_t>(pl->progs.size());
    s.n_launches = static_cast<uint32_t>(pl->groups.size()) + (pl->segs.empty() ? 0 : 1);
    s.n_tasks = static_cast<uint32_t>(pl->tasks.size());
    s.n_segments = static_cast<uint32_t>(pl->segs.size());
    return s;
}

int plan_build(BatchPlan *pl, const ridfa_program *const *progs, uint32_t np, const ridfa_batch_item *items,
               uint32_t ni, uint32_t L, int device, const BatchShape &shape) {
    if (!pl || !progs || !np || (ni && !items) || L == 0) return RIDFA_E_ARG;
    for (uint32_t p = 0; p < np; ++p)
        if (!progs[p] || progs[p]->rid.k > RIDFA_MAX_SLOTS) return progs[p] ? RIDFA_E_UNSUPPORTED : RIDFA_E_ARG;
    for (uint32_t i = 0; i < ni; ++i) {
        const ridfa_batch_item &it = items[i];
        if (it.prog >= np || (it.len && !it.d_text)) return RIDFA_E_ARG;
        if (it.n_chunks > it.len || (it.len == 0 && it.n_chunks)) return RIDFA_E_CHUNKS;
    }
    BatchPlan &P = *pl;
    P.progs.assign(progs, progs + np);
    P.n_items = ni;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const size_t limit = static_cast<size_t>(smem_optin_limit()) - 1024 - 64;
    // per-program device tables and layout
    P.dev.assign(np, nullptr);
    std::vector<uint32_t> mode(np, kBPlain);
    P.tis.assign(np, 0);
    std::vector<size_t> tbytes(np, 0);
    for (uint32_t p = 0; p < np; ++p) {
        const ridfa_program *R = progs[p];
        std::lock_guard<std::mutex> lock(R->mu);
        int err = RIDFA_OK;
        P.dev[p] = device_copy(R, false, device, &err);
        if (!P.dev[p]) return err;
        const HostAutomaton &H = R->rid;
        Automaton A{nullptr, nullptr, nullptr, nullptr, nullptr, H.n_states, H.n_classes, H.k, H.kw, H.q0_slot};
        const size_t r16 = LutRep<true>::smem_bytes(A), r32 = LutRep<false>::smem_bytes(A),
                     pln = LutPlain::smem_bytes(A), flt = LutFlat::smem_bytes(A);
        if (LutRep<true>::fits16(A) && r16 + 8 * kWarpCoopBytes <= limit) { mode[p] = kBRep16; tbytes[p] = r16; }
        else if (r32 + 8 * kWarpCoopBytes <= limit) { mode[p] = kBRep32; tbytes[p] = r32; }
        // (the scaled 16-bit table only when 16 warps' staging still fits beside it: its launch
        // group takes the warp count of its largest table)
        else if (LutRep16x4::fits(A) && LutRep16x4::smem_bytes(A) + 16 * kWarpCoopBytes <= limit) {
            mode[p] = kBRep16x4;
            tbytes[p] = LutRep16x4::smem_bytes(A);
        }
        else if (LutPlain::fits(A) && pln + 8 * kWarpCoopBytes <= limit) { mode[p] = kBPlain; tbytes[p] = pln; }
        else if (flt + 8 * kWarpCoopBytes <= limit) { mode[p] = kBFlat; P.tis[p] = 1; tbytes[p] = flt; }
        else { mode[p] = kBFlat; P.tis[p] = 0; tbytes[p] = 256; }
    }
    // texts grouped by program; chunk counts
    std::vector<std::vector<uint32_t>> by_prog(np);
    for (uint32_t i = 0; i < ni; ++i) by_prog[items[i].prog].push_back(i);
    P.texts.clear();
    std::vector<uint64_t> prog_chunks(np, 0);
    P.text0.assign(np, 0);
    P.n_texts_of.assign(np, 0);
    bool aligned_all = true;
    P.total_bytes = 0;
    for (uint32_t p = 0; p < np; ++p) {
        P.text0[p] = static_cast<uint32_t>(P.texts.size());
        P.n_texts_of[p] = static_cast<uint32_t>(by_prog[p].size());
        for (uint32_t i : by_prog[p]) {
            const ridfa_batch_item &it = items[i];
            TextDesc td{it.d_text, it.len, prog_chunks[p], 0, i};
            if (it.len == 0) td.c = 0;
            else if (it.n_chunks) td.c = it.n_chunks;
            else td.c = static_cast<uint32_t>(std::max<uint64_t>(1, std::min<uint64_t>(it.len, (it.len + L - 1) / L)));
            if (it.len && (reinterpret_cast<uintptr_t>(it.d_text) & 15)) aligned_all = false;
            prog_chunks[p] += td.c;
            P.total_bytes += it.len;
            P.texts.push_back(td);
        }
    }
    P.total_chunks = 0;
    for (uint32_t p = 0; p < np; ++p) P.total_chunks += prog_chunks[p];
    // launch groups by layout; tasks ordered by group then program
    P.groups.clear();
    P.tasks.clear();
    uint64_t run_warps = 0;
    for (uint32_t m = kBPlain; m <= kBRep16x4; ++m) {
        LaunchGroup g;
        g.mode = m;
        // staged text when every text is 16-byte aligned; tables too large to replicate (their
        // runs stay apart) finish a chunk's runs together, at up to 512 threads
        g.tp = !aligned_all ? kTpGlobal : (m == kBPlain || m == kBFlat) && shape.set_mode != 2 ? kTpSet : kTpCoop;
        for (uint32_t p = 0; p < np; ++p)
            if (mode[p] == m && prog_chunks[p]) {
                g.progs.push_back(p);
                const uint32_t k = progs[p]->rid.k;
                g.R = std::max(g.R, k <= 32 ? 1 : k <= 64 ? 2 : k <= 128 ? 4 : 8);
                g.table_smem = std::max(g.table_smem, tbytes[p]);
            }
        if (g.progs.empty()) continue;
        g.task0 = static_cast<uint32_t>(P.tasks.size());
        const int cap = g.R <= 4 && g.tp != kTpSet ? 1024 : 512;
        g.stg = static_cast<uint32_t>((g.table_smem + 127) & ~static_cast<size_t>(127));
        int warps = g.tp != kTpGlobal ? static_cast<int>(std::min<size_t>(cap / 32, (limit - g.stg) / kWarpCoopBytes)) : cap / 32;
        if (shape.warps_cap) warps = std::min<int>(warps, static_cast<int>(shape.warps_cap));
        warps = std::max(warps, 1);
        g.block = warps * 32;
        g.smem = g.tp != kTpGlobal ? g.stg + static_cast<size_t>(warps) * kWarpCoopBytes : g.table_smem;
        const uint64_t per_task = 32ull * warps;
        for (uint32_t p : g.progs)
            for (uint64_t c0 = 0; c0 < prog_chunks[p]; c0 += per_task)
                P.tasks.push_back(TaskDesc{c0, p, static_cast<uint32_t>(std::min<uint64_t>(per_task, prog_chunks[p] - c0))});
        g.n_tasks = static_cast<uint32_t>(P.tasks.size()) - g.task0;
        // persistent: as many blocks as fit on every SM, no more than there are tasks
        int per_sm = 0;
        const int err = blocks_per_sm(device, g, &per_sm);
        if (err != RIDFA_OK) return err;
        if (per_sm < 1) return RIDFA_E_UNSUPPORTED;
        g.grid = static_cast<int>(std::min<uint64_t>(g.n_tasks, static_cast<uint64_t>(sms) * per_sm));
        g.run0 = run_warps;
        run_warps += static_cast<uint64_t>(g.grid) * warps;
        P.groups.push_back(g);
    }
    // join segments
    P.segs.clear();
    for (uint32_t p = 0; p < np; ++p)
        for (uint32_t t = P.text0[p]; t < P.text0[p] + P.n_texts_of[p]; ++t) {
            const TextDesc &td = P.texts[t];
            const uint64_t nb = td.c > 1 ? td.c - 1 : 0;
            const uint32_t nseg = nb ? static_cast<uint32_t>((nb + kBatchJoinThreads - 1) / kBatchJoinThreads) : 1;
            const uint32_t part0 = static_cast<uint32_t>(P.segs.size());
            for (uint32_t sgi = 0; sgi < nseg; ++sgi) {
                const uint64_t b0 = 1 + static_cast<uint64_t>(sgi) * kBatchJoinThreads;
                const uint32_t cnt = nb ? static_cast<uint32_t>(std::min<uint64_t>(kBatchJoinThreads, nb + 1 - b0)) : 0;
                P.segs.push_back(SegDesc{b0, p, t, cnt, sgi, nseg, part0});
            }
        }
    // block layout: the host image first, then device-only scratch
    uint64_t maps_bytes = 0, dinfo_bytes = 0;
    P.maps_off.assign(np, 0);
    P.dinfo_off.assign(np, 0);
    for (uint32_t p = 0; p < np; ++p) {
        P.maps_off[p] = maps_bytes;
        P.dinfo_off[p] = dinfo_bytes;
        maps_bytes += al256(prog_chunks[p] * progs[p]->rid.k * 2);
        dinfo_bytes += al256(prog_chunks[p] * 4);
    }
    size_t off = 0;
    P.o_counters = off; off += 256;
    P.o_progs = off;    off += al256(np * sizeof(ProgDesc));
    P.o_texts = off;    off += al256(P.texts.size() * sizeof(TextDesc));
    P.o_tasks = off;    off += al256(P.tasks.size() * sizeof(TaskDesc));
    P.o_segs = off;     off += al256(P.segs.size() * sizeof(SegDesc));
    P.o_tick = off;     off += al256(P.texts.size() * 4);
    P.o_flags = off;    off += al256(P.texts.size() * 4);
    P.o_part = off;     off += al256(P.segs.size() * kPartialWords * 4);
    P.o_runs = off;     off += al256(run_warps * kRunsPerWarp * sizeof(RunEntry));
    P.o_finals = off;   off += al256(run_warps * kFinalsPerWarp * 4);
    P.o_maps = off;     off += maps_bytes;
    P.o_dinfo = off;    off += dinfo_bytes;
    P.total = off;
    return RIDFA_OK;
}

void plan_image(const BatchPlan *pl, uint8_t *base, uint8_t *img) {
    const BatchPlan &P = *pl;
    std::memset(img, 0, P.o_part);
    const uint32_t np = static_cast<uint32_t>(P.progs.size());
    ProgDesc *pd = reinterpret_cast<ProgDesc *>(img + P.o_progs);
    for (uint32_t p = 0; p < np; ++p) {
        const HostAutomaton &H = P.progs[p]->rid;
        const DeviceAutomaton *D = P.dev[p];
        pd[p].A = Automaton{D->trans, D->classmap, D->final_bits, D->ifmask, D->slot_state,
                            H.n_states, H.n_classes, H.k, H.kw, H.q0_slot};
        pd[p].texts = reinterpret_cast<const TextDesc *>(base + P.o_texts) + P.text0[p];
        pd[p].maps = reinterpret_cast<uint16_t *>(base + P.o_maps + P.maps_off[p]);
        pd[p].dinfo = reinterpret_cast<uint32_t *>(base + P.o_dinfo + P.dinfo_off[p]);
        pd[p].n_texts = P.n_texts_of[p];
        pd[p].tis = P.tis[p];
        pd[p].text0 = P.text0[p];
        pd[p].pad = 0;
    }
    if (!P.texts.empty()) std::memcpy(img + P.o_texts, P.texts.data(), P.texts.size() * sizeof(TextDesc));
    if (!P.tasks.empty()) std::memcpy(img + P.o_tasks, P.tasks.data(), P.tasks.size() * sizeof(TaskDesc));
    if (!P.segs.empty()) std::memcpy(img + P.o_segs, P.segs.data(), P.segs.size() * sizeof(SegDesc));
}

int make_fork(LaunchFork *f) {
    f->ok = false;
    for (int i = 0; i < kMaxLaunchGroups - 1; ++i) {
        cudaError_t e = cudaStreamCreateWithFlags(&f->aux[i], cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    for (int i = 0; i < kMaxLaunchGroups; ++i) {
        cudaError_t e = cudaEventCreateWithFlags(&f->ev[i], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    f->ok = true;
    return RIDFA_OK;
}

void free_fork(LaunchFork *f) {
    for (auto &s : f->aux)
        if (s) cudaStreamDestroy(s);
    for (auto &e : f->ev)
        if (e) cudaEventDestroy(e);
    *f = LaunchFork{};
}

int plan_enqueue(const BatchPlan *pl, uint8_t *base, uint8_t *d_accept, cudaStream_t st, bool zero_counters,
                 const LaunchFork *fork) {
    const BatchPlan &P = *pl;
    uint32_t *counters = reinterpret_cast<uint32_t *>(base + P.o_counters);
    uint32_t *status = counters + 32;
    if (zero_counters) {
        cudaError_t e = cudaMemsetAsync(counters, 0, 256, st);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    const ProgDesc *progs = reinterpret_cast<const ProgDesc *>(base + P.o_progs);
    const TaskDesc *tasks = reinterpret_cast<const TaskDesc *>(base + P.o_tasks);
    RunEntry *runs = reinterpret_cast<RunEntry *>(base + P.o_runs);
    uint32_t *finals = reinterpret_cast<uint32_t *>(base + P.o_finals);
    const bool concurrent = fork && fork->ok && P.groups.size() > 1 && P.groups.size() <= kMaxLaunchGroups;
    if (concurrent) {
        cudaError_t e = cudaEventRecord(fork->ev[0], st);
        for (size_t gi = 1; gi < P.groups.size() && e == cudaSuccess; ++gi) e = cudaStreamWaitEvent(fork->aux[gi - 1], fork->ev[0], 0);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    for (size_t gi = 0; gi < P.groups.size(); ++gi) {
        const LaunchGroup &g = P.groups[gi];
        if (g.n_tasks == 0) continue;
        BatchReachArgs a{progs, tasks + g.task0, g.n_tasks, 8, counters + gi, status, runs + g.run0 * kRunsPerWarp,
                         finals + g.run0 * kFinalsPerWarp};
        cudaError_t e = batch_reach(g, a, (concurrent && gi > 0) ? fork->aux[gi - 1] : st, nullptr);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    if (concurrent) {
        for (size_t gi = 1; gi < P.groups.size(); ++gi) {
            cudaError_t e = cudaEventRecord(fork->ev[gi], fork->aux[gi - 1]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, fork->ev[gi], 0);
            if (e != cudaSuccess) return cuda_fail(e);
        }
    }
    if (!P.segs.empty()) {
        BatchJoinArgs J{progs, reinterpret_cast<const TextDesc *>(base + P.o_texts),
                        reinterpret_cast<const SegDesc *>(base + P.o_segs),
                        reinterpret_cast<uint32_t *>(base + P.o_part), reinterpret_cast<uint32_t *>(base + P.o_tick),
                        reinterpret_cast<uint32_t *>(base + P.o_flags), d_accept, status};
        rid_join_batch_kernel<<<static_cast<unsigned>(P.segs.size()), kBatchJoinThreads, 0, st>>>(J);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return RIDFA_OK;
}

}  // namespace ridfa

struct ridfa_batch {
    int device = -1;
    std::vector<const ridfa_program *> progs;
    std::vector<ridfa_batch_item> items;
    uint8_t *d_accept = nullptr;
    uint32_t chunk_len = 0;
    ridfa::BatchShape shape;
    bool use_graph = true;
    ridfa::BatchPlan *plan = nullptr;
    void *dmem = nullptr;
    size_t dbytes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ridfa::LaunchFork fork;
};

namespace ridfa {
namespace {

void batch_release(ridfa_batch *B) {
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    B->exec = nullptr;
    B->graph = nullptr;
    if (B->dmem) cudaFree(B->dmem);
    B->dmem = nullptr;
    B->dbytes = 0;
}

// Plan and allocate the batch for chunk length L, write its image and capture the graph.
int batch_build(ridfa_batch *B, uint32_t L) {
    batch_release(B);
    if (!B->plan) B->plan = plan_new();
    if (!B->plan) return RIDFA_E_NOMEM;
    int err = plan_build(B->plan, B->progs.data(), static_cast<uint32_t>(B->progs.size()), B->items.data(),
                         static_cast<uint32_t>(B->items.size()), L, B->device, B->shape);
    if (err != RIDFA_OK) return err;
    const size_t total = plan_device_bytes(B->plan);
    cudaError_t e = cudaMalloc(&B->dmem, total);
    if (e != cudaSuccess) {
        B->dmem = nullptr;
        return cuda_fail(e);
    }
    B->dbytes = total;
    uint8_t *base = static_cast<uint8_t *>(B->dmem);
    std::vector<uint8_t> img(plan_image_bytes(B->plan));
    plan_image(B->plan, base, img.data());
    e = cudaMemcpy(base, img.data(), img.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e);
    if (B->use_graph) {
        cudaStream_t cs;
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e);
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        err = e == cudaSuccess ? plan_enqueue(B->plan, base, B->d_accept, cs, true, &B->fork) : cuda_fail(e);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        if (err != RIDFA_OK) {
            if (g) cudaGraphDestroy(g);
            return err;
        }
        if (e2 != cudaSuccess) return cuda_fail(e2);
        B->graph = g;
        e = cudaGraphInstantiate(&B->exec, g, 0);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return RIDFA_OK;
}

int batch_run(ridfa_batch *B, cudaStream_t st) {
    if (B->exec) {
        cudaError_t e = cudaGraphLaunch(B->exec, st);
        return e == cudaSuccess ? RIDFA_OK : cuda_fail(e);
    }
    return plan_enqueue(B->plan, static_cast<uint8_t *>(B->dmem), B->d_accept, st, true, &B->fork);
}

// Chunk length and launch shape for the batch.  Every program is keyed by (log2 |P|, log2 k,
// log2 C); when all keys are in the cache and agree, that tune is used.  Otherwise the batch itself
// is timed (one warm-up and 3 replays per candidate, CUDA events), one knob after another: the
// chunk length (4-32 KiB), then the warps per block of the reach groups (as many as fit, 16, 8),
// then -- when some table is too large to replicate -- whether a lane finishes all of its chunk's
// runs together or one run per lane.  The winner is recorded under every key.  Knobs the caller
// fixed (opts->block_warps, opts->set_mode) are not searched.
int batch_autotune(ridfa_batch *B, bool fixed_warps, bool fixed_set, BatchTune *out) {
    std::vector<std::tuple<int, int, int>> keys;
    bool large_table = false;
    for (const ridfa_program *P : B->progs) {
        keys.emplace_back(log2i(P->rid.n_states), log2i(P->rid.k), log2i(P->rid.n_classes));
        const HostAutomaton &H = P->rid;
        Automaton A{nullptr, nullptr, nullptr, nullptr, nullptr, H.n_states, H.n_classes, H.k, H.kw, H.q0_slot};
        if (!LutRep<true>::fits16(A) && !LutRep16x4::fits(A)) large_table = true;
    }
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        BatchTune v;
        bool all = true, first = true;
        for (auto &k : keys) {
            auto it = g_tune_cache.find(k);
            if (it == g_tune_cache.end() || (!first && !(it->second == v))) {
                all = false;
                break;
            }
            v = it->second;
            first = false;
        }
        if (all && v.chunk_len) {
            if (fixed_warps) v.shape.warps_cap = B->shape.warps_cap;
            if (fixed_set) v.shape.set_mode = B->shape.set_mode;
            *out = v;
            return RIDFA_OK;
        }
    }
    cudaStream_t st;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    int err = RIDFA_OK;
    BatchTune best;
    best.chunk_len = 8192;
    best.shape = B->shape;
    float best_ms = 1e30f;
    auto trial = [&](const BatchTune &t) {
        B->shape = t.shape;
        err = batch_build(B, t.chunk_len);
        if (err != RIDFA_OK) return;
        batch_run(B, st);                       // warm-up
        cudaEventRecord(a, st);
        for (int r = 0; r < 3; ++r) batch_run(B, st);
        cudaEventRecord(b, st);
        e = cudaEventSynchronize(b);
        if (e != cudaSuccess) {
            err = cuda_fail(e);
            return;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best_ms) {
            best_ms = ms;
            best = t;
        }
    };
    for (uint32_t L : {4096u, 8192u, 16384u, 32768u}) {
        if (err != RIDFA_OK) break;
        BatchTune t = best;
        t.chunk_len = L;
        trial(t);
    }
    if (!fixed_warps)
        for (uint32_t w : {16u, 8u}) {
            if (err != RIDFA_OK) break;
            BatchTune t = best;
            t.shape.warps_cap = w;
            trial(t);
        }
    if (!fixed_set && large_table && err == RIDFA_OK) {
        BatchTune t = best;
        t.shape.set_mode = best.shape.set_mode == 2 ? 1 : 2;
        trial(t);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamDestroy(st);
    if (err != RIDFA_OK) return err;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (auto &k : keys) g_tune_cache[k] = best;
    }
    *out = best;
    return RIDFA_OK;
}

}  // namespace
}  // namespace ridfa

extern "C" int ridfa_batch_create(const ridfa_program *const *progs, uint32_t n_progs,
                                  const ridfa_batch_item *items, uint32_t n_items, uint8_t *d_accept,
                                  const ridfa_batch_opts *opts, ridfa_batch **out) {
    if (!progs || !n_progs || !items || !n_items || !d_accept || !out) return RIDFA_E_ARG;
    for (uint32_t p = 0; p < n_progs; ++p) {
        if (!progs[p]) return RIDFA_E_ARG;
        if (progs[p]->rid.k > RIDFA_MAX_SLOTS) return RIDFA_E_UNSUPPORTED;
    }
    for (uint32_t i = 0; i < n_items; ++i) {
        const ridfa_batch_item &it = items[i];
        if (it.prog >= n_progs || (it.len && !it.d_text)) return RIDFA_E_ARG;
        if (it.n_chunks > it.len || (it.len == 0 && it.n_chunks)) return RIDFA_E_CHUNKS;
    }
    ridfa::NvtxRange range("ridfa batch create");
    ridfa_batch *B = new (std::nothrow) ridfa_batch();
    if (!B) return RIDFA_E_NOMEM;
    if (cudaGetDevice(&B->device) != cudaSuccess) {
        delete B;
        return ridfa::cuda_fail(cudaGetLastError());
    }
    B->progs.assign(progs, progs + n_progs);
    B->items.assign(items, items + n_items);
    B->d_accept = d_accept;
    B->use_graph = !(opts && opts->no_graph);
    uint32_t L = opts ? opts->chunk_len : 0;
    B->shape.warps_cap = opts ? opts->block_warps : 0;
    B->shape.set_mode = opts ? opts->set_mode : 0;
    if (B->shape.warps_cap > 32 || B->shape.set_mode > 2) {
        delete B;
        return RIDFA_E_ARG;
    }
    int err = ridfa::make_fork(&B->fork);
    if (err == RIDFA_OK && L == 0) {
        ridfa::BatchTune t;
        err = ridfa::batch_autotune(B, B->shape.warps_cap != 0, B->shape.set_mode != 0, &t);
        if (err == RIDFA_OK) {
            L = t.chunk_len;
            B->shape = t.shape;
        }
    }
    if (err == RIDFA_OK) err = ridfa::batch_build(B, L);
    if (err != RIDFA_OK) {
        ridfa::batch_release(B);
        ridfa::plan_delete(B->plan);
        ridfa::free_fork(&B->fork);
        delete B;
        return err;
    }
    B->chunk_len = L;
    *out = B;
    return RIDFA_OK;
}

extern "C" int ridfa_batch_run(ridfa_batch *b, void *stream) {
    if (!b) return RIDFA_E_ARG;
    ridfa::NvtxRange range("ridfa batch run");
    return ridfa::batch_run(b, static_cast<cudaStream_t>(stream));
}

extern "C" int ridfa_batch_get_stats(const ridfa_batch *b, ridfa_batch_stats *out) {
    if (!b || !out) return RIDFA_E_ARG;
    std::memset(out, 0, sizeof(*out));
    const ridfa::PlanStats s = ridfa::plan_stats(b->plan);
    out->total_bytes = s.total_bytes;
    out->total_chunks = s.total_chunks;
    out->n_programs = s.n_programs;
    out->n_launches = s.n_launches;
    out->n_tasks = s.n_tasks;
    out->n_segments = s.n_segments;
    out->chunk_len = b->chunk_len;
    out->block_warps = b->shape.warps_cap;
    out->set_mode = b->shape.set_mode;
    out->graph = b->exec ? 1 : 0;
    out->device_bytes = b->dbytes;
    return RIDFA_OK;
}

extern "C" void ridfa_batch_free(ridfa_batch *b) {
    if (!b) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    ridfa::batch_release(b);
    ridfa::plan_delete(b->plan);
    ridfa::free_fork(&b->fork);
    cudaSetDevice(cur);
    (void)cudaGetLastError();
    delete b;
}

extern "C" int ridfa_recognize_batch(const ridfa_program *const *progs, uint32_t n_progs,
                                     const ridfa_batch_item *items, uint32_t n_items, uint8_t *d_accept,
                                     void *stream) {
    ridfa_batch_opts o{8192, 1, 0, 0};   // one run: no graph
    ridfa_batch *b = nullptr;
    int err = ridfa_batch_create(progs, n_progs, items, n_items, d_accept, &o, &b);
    if (err != RIDFA_OK) return err;
    err = ridfa_batch_run(b, stream);
    if (err == RIDFA_OK && cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess)
        err = ridfa::cuda_fail(cudaGetLastError());
    ridfa_batch_free(b);
    return err;
}

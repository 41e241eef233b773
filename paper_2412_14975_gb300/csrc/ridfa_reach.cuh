// The reach kernel (Sec. 3.2 reach phase; one chunk's speculative runs per warp, then one
// converged run -- or one chunk's set of runs -- per lane) and the launch of one instantiation
// per (interface registers R, table layout, text path).  Each text path's instantiations are
// compiled in a translation unit of their own (ridfa_reach_<path>.cu) so that the library builds
// in parallel; ridfa_device.cu plans the launches and calls reach_path_<path>.
#pragma once

#include "ridfa_kernels.cuh"

namespace ridfa {

// table layouts (ridfa_tuning::table_mode)
enum Mode : uint32_t { kModePlain = 1, kModeRep16 = 2, kModeRep32 = 3, kModePart16 = 4, kModeFlat = 5,
                       kModeRep16x4 = 6, kModeRep16x4C = 7, kModePair = 8, kModePairC = 9,
                       kModePairF = 10, kModePairH = 11 };

// How one reach launch is laid out: table layout, text path, block/grid, shared memory.
struct ReachPlan {
    uint32_t mode = kModePlain;
    int R = 1;
    int tis = 0;                 // layout parameter: Flat, table in shared memory (1) or not (0);
                                 // PairF / PairH, the number of lane copies
    int path = kPathGlobal;      // how the converged phase reads the text
    int block = 256;
    int grid = 1;
    size_t smem = 0;
    uint32_t staging_offset = 0;
    bool pslot = false;          // per-chunk start states (ReachArgs::piece_slots; R = 1 only)
};


cudaError_t ensure_smem_cap(const void *kern, size_t bytes);   // ridfa_device.cu

// One launch (or, with per_sm != nullptr, the blocks per SM it would get) of the reach kernel for
// the plan's layout and R, one function per text path.
cudaError_t reach_path_global(const ReachArgs &a, const ReachPlan &pl, cudaStream_t st, int *per_sm);
cudaError_t reach_path_coop(const ReachArgs &a, const ReachPlan &pl, cudaStream_t st, int *per_sm);
cudaError_t reach_path_coop2(const ReachArgs &a, const ReachPlan &pl, cudaStream_t st, int *per_sm);
cudaError_t reach_path_set(const ReachArgs &a, const ReachPlan &pl, cudaStream_t st, int *per_sm);

namespace {

template <int R, class LUT, int BLOCK, int PATH, bool PSLOT = false>
__global__ void __launch_bounds__(BLOCK, 1) rid_reach_kernel(ReachArgs p, int table_in_smem,
                                                            uint32_t staging_offset) {
    extern __shared__ __align__(128) uint8_t smem[];
    const Automaton &A = p.A;
    LUT T;
    T.setup(A, smem, static_cast<uint32_t>(table_in_smem));
    // per-warp staging buffers of the cooperative text paths
    const uint32_t warp_in_block = threadIdx.x >> 5;
    const uint32_t stg_base = smem_addr(smem) + staging_offset + warp_in_block * kWarpCoopBytes;
    __syncthreads();

    const uint32_t lane = threadIdx.x & 31;
    const uint32_t dead = T.enc(A.n);
    const uint64_t n_tasks = (static_cast<uint64_t>(p.c) + 31) / 32;
    const uint64_t warp0 = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
    RunEntry *wruns = p.runs ? p.runs + warp0 * kRunsPerWarp : nullptr;
    uint32_t *wfin = p.finals ? p.finals + warp0 * kFinalsPerWarp : nullptr;   // null with wruns
    uint32_t *wball = wfin ? wfin + kRunsPerWarp : nullptr;

    // slot start states of this lane (slot a = r*32 + lane)
    static_assert(!PSLOT || R == 1, "per-chunk start states take one register");
    uint32_t start_state[R];
    uint32_t start_live = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t a = r * 32 + lane;
        start_state[r] = (!PSLOT && a < A.k) ? T.enc(A.slot_state[a]) : dead;
        if (!PSLOT && r * 32 < static_cast<int>(A.k)) start_live |= 1u << r;
    }

    for (uint64_t task = warp0; task < n_tasks; task += n_warps) {
        const uint64_t chunk0 = task * 32;
        // the speculative phase reads the first bytes of the task's chunks one chunk after the
        // other: lane j asks for chunk j's first line now, so the 32 reads overlap (record lines
        // +1.6 %).  A prefetch needs only an address near the chunk start, so it is taken in
        // double precision rather than by the exact 64-bit division of chunk_begin.
        if (chunk0 + lane < p.c) {
            const double at = static_cast<double>(chunk0 + lane) * (static_cast<double>(p.len) / p.c);
            const uint64_t first = min(static_cast<uint64_t>(at), p.len - 1);
            asm volatile("prefetch.global.L1 [%0];" ::"l"(p.text + first));
        }
        // ---------------- speculative phase, one chunk at a time, lanes = runs
        // A chunk whose live runs reduce to m <= kMaxRun distinct states hands them off as m
        // runs; without a run list (no scratch) only m = 1, kept by lane j.
        uint32_t my_hand = 0;         // owner lane j of a handed-off chunk: (m << 16) | first run
        uint32_t nruns = 0, handed = 0;
        uint32_t amask[R];            // bit j: this lane's slot of register r alive at chunk j's hand-off
#pragma unroll
        for (int r = 0; r < R; ++r) amask[r] = 0;
        uint64_t one_pos = 0;
        uint32_t one_state = dead;
        for (uint32_t j = 0; j < 32; ++j) {
            const uint64_t ch = chunk0 + j;
            if (ch >= p.c) break;
            const uint64_t beg = chunk_begin(ch, p.len, p.c);
            const uint64_t end = chunk_begin(ch + 1, p.len, p.c);
            if constexpr (PSLOT) {
                // this chunk's own start states (one register: at most 32)
                const uint32_t v = p.piece_slots[ch * 32 + lane];
                start_state[0] = v < A.n ? T.enc(v) : dead;
                start_live = __any_sync(kFull, start_state[0] != dead) ? 1u : 0u;
            }
            uint32_t d, alive[R];
            uint64_t hp = 0;
            const int m = speculate<R, LUT, PATH == kPathCoopSet ? kMultiMinSet : kMultiMin>(
                T, A, p.text, beg, end, p.probe, lane, start_state, start_live, dead, p.maps + ch * p.stride,
                p.dinfo + ch, p.status, wruns != nullptr, wruns == nullptr, &hp, &d, alive);
            if (m >= 1) {
                handed |= 1u << j;
#pragma unroll
                for (int r = 0; r < R; ++r) amask[r] |= ((alive[r] >> lane) & 1u) << j;
                if (wruns) {
                    if (lane < static_cast<uint32_t>(m))
                        wruns[nruns + lane] = RunEntry{hp, d, static_cast<uint16_t>(j), static_cast<uint16_t>(lane)};
                    if (lane == j) {
                        my_hand = (static_cast<uint32_t>(m) << 16) | nruns;
                    }
                    nruns += static_cast<uint32_t>(m);
                } else if (lane == j) {
                    my_hand = (1u << 16) | j;
                    one_pos = hp;
                    one_state = d;
                }
            }
        }
        // the alive bits wait in the finals area while the runs go on (registers are scarce
        // there); without it the rows carry tags instead
        if (wball) {
#pragma unroll
            for (int r = 0; r < R; ++r) wball[r * 32 + lane] = amask[r];
        }
        __syncwarp();

        // ---------------- converged phase: each lane finishes one run (rounds of 32 runs); when
        // some chunk handed off several runs (staged path), each lane finishes its chunk's runs
        // together instead
        const uint32_t total_runs = wruns ? nruns : 32;
        uint32_t fin_reg = dead;      // final state of run `lane` when there are at most 32 runs
        const bool set_path = PATH == kPathCoopSet && wruns && nruns != static_cast<uint32_t>(__popc(handed));
        if (set_path) {
            const uint32_t m = my_hand >> 16, run0 = my_hand & 0xFFFF;
            uint32_t st[kMaxRun];
            uint64_t pos = 0, end = 0;
#pragma unroll
            for (int g = 0; g < kMaxRun; ++g) st[g] = dead;
            if (m) {
#pragma unroll
                for (int g = 0; g < kMaxRun; ++g)
                    if (g < static_cast<int>(m)) st[g] = wruns[run0 + g].state;
                pos = wruns[run0].pos;
                end = chunk_begin(chunk0 + lane + 1, p.len, p.c);
            }
            const uint64_t lim = p.len & ~static_cast<uint64_t>(15);
            uint32_t rep = 0xFFFFFFFFu;                // group g -> its slot (4 bits; 0xF dead)
#pragma unroll
            for (int g = 0; g < kMaxRun; ++g)
                if (g < static_cast<int>(m)) rep = (rep & ~(0xFu << (4 * g))) | (static_cast<uint32_t>(g) << (4 * g));
            coop_converge_set(T, stg_base, lane, m != 0, p.text, lim, min(end, lim), pos, st, rep, dead);
            if (m) finish_set_runs(T, p.text, pos, end, st, rep, m, wfin + run0, dead);
        }
        for (uint32_t rb = 0; rb < (set_path ? 0u : total_runs); rb += 32) {
            bool my_pending;
            uint64_t pos = 0, end = 0;
            uint32_t s = dead, jj = lane;
            const uint32_t idx = rb + lane;
            if (wruns) {
                my_pending = idx < nruns;
                if (my_pending) {
                    const RunEntry e = wruns[idx];
                    pos = e.pos;
                    s = e.state;
                    jj = e.chunk;
                }
            } else {
                my_pending = my_hand != 0;
                pos = one_pos;
                s = one_state;
            }
            if (my_pending) end = chunk_begin(chunk0 + jj + 1, p.len, p.c);
            if ((PATH == kPathCoop || PATH == kPathCoopSet) && __any_sync(kFull, my_pending)) {
                const uint64_t lim = p.len & ~static_cast<uint64_t>(15);
                coop_converge<LUT, true>(T, stg_base, lane, my_pending, p.text, lim, min(end, lim), pos, s, dead);
            }
            if (my_pending) {
                tail_converge<LUT, PATH == kPathGlobal>(T, p.text, pos, end, s, dead);
                if (total_runs > 32) wfin[idx] = s;
                else fin_reg = s;
            }
        }
        __syncwarp();
        // ---------------- rows of the handed-off chunks, one chunk at a time by the warp
        if (wball) {
#pragma unroll
            for (int r = 0; r < R; ++r) amask[r] = wball[r * 32 + lane];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) amask[r] = 0xFFFFFFFFu;    // tags decide
        }
        for (uint32_t hm = handed; hm; hm &= hm - 1) {
            const uint32_t j = __ffs(hm) - 1;
            const uint32_t hand = __shfl_sync(kFull, my_hand, j);
            const uint32_t m = hand >> 16, run0 = hand & 0xFFFF;
            const uint32_t src = run0 + min(lane, m - 1);     // lane g < m: run of group g
            uint32_t fin = __shfl_sync(kFull, fin_reg, src & 31);
            if (total_runs > 32 || set_path) fin = wfin[src];
            uint32_t am = 0;
#pragma unroll
            for (int r = 0; r < R; ++r) am |= ((amask[r] >> j) & 1u) << r;
            finish_handed_row<R, LUT>(T, p.maps + (chunk0 + j) * p.stride, A.k, m, m >= 2 || !wball, lane, am, fin,
                                      dead, p.dinfo + chunk0 + j);
        }
    }
}

// ------------------------------------------------------------------ reach, two chains per lane
// Speculative phase of one chunk by the whole warp (lanes = runs).  Returns true when the live
// runs merged into one state before the chunk end; then *out_pos / *out_state hold where and
// what, and alive[] the ballots of the slots still alive (the same in every lane).  Otherwise the
// chunk finished here: its map row and D_i summary are written and false is returned.
template <int R, class LUT>
__device__ __forceinline__ bool speculate_chunk(const ReachArgs &p, const LUT &T, uint64_t ch,
                                                uint32_t lane, const uint32_t (&start_state)[R],
                                                uint32_t start_live, uint32_t dead, uint64_t *out_pos,
                                                uint32_t *out_state, uint32_t (&alive)[R]) {
    return speculate_range<R, LUT>(T, p.A, p.text, chunk_begin(ch, p.len, p.c), chunk_begin(ch + 1, p.len, p.c),
                                   p.probe, lane, start_state, start_live, dead, p.maps + ch * p.stride,
                                   p.dinfo + ch, p.status, out_pos, out_state, alive);
}

// The same for two independent chains, interleaved so their lookups overlap.
template <class LUT>
__device__ __forceinline__ void run_granule2(const LUT &T, uint32_t &s0, uint32_t a0, uint32_t &s1,
                                             uint32_t a1) {
    const uint4 x = lds_v4(a0), y = lds_v4(a1);
    const uint32_t w0[4] = {x.x, x.y, x.z, x.w}, w1[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t c0[8], c1[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int b = h * 8 + q;
            c0[q] = T.cls_at(w0[b >> 2], b & 3);
            c1[q] = T.cls_at(w1[b >> 2], b & 3);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            s0 = T.next(s0, c0[q]);
            s1 = T.next(s1, c1[q]);
        }
    }
}

// Cooperative text path with two chunks per lane.  A warp owns 64 consecutive chunks: lane l
// finishes chunks l and 32 + l after the speculative phase, interleaving the two runs.  Each
// round the warp loads one 32-byte window of each of its 64 chunks with coalesced 16-byte loads
// (16 chunks' windows per instruction, two lanes per window), one round ahead, into a shared
// buffer whose windows sit 48 bytes apart (3 granules, odd: conflict-free 16-byte reads).
constexpr uint32_t kC2Win = 32;
constexpr uint32_t kC2Stride = 48;
constexpr uint32_t kWarpCoop2Bytes = 64 * kC2Stride;

template <int R, class LUT, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1) rid_reach2_kernel(ReachArgs p, int table_in_smem,
                                                             uint32_t staging_offset) {
    extern __shared__ __align__(128) uint8_t smem[];
    const Automaton &A = p.A;
    LUT T;
    T.setup(A, smem, static_cast<uint32_t>(table_in_smem));
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t stg = smem_addr(smem) + staging_offset + (threadIdx.x >> 5) * kWarpCoop2Bytes;
    const uint32_t dead = T.enc(A.n);
    const uint64_t n_tasks = (static_cast<uint64_t>(p.c) + 63) / 64;
    const uint64_t warp0 = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
    const uint64_t lim = p.len & ~static_cast<uint64_t>(15);

    uint32_t start_state[R];
    uint32_t start_live = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t a = r * 32 + lane;
        start_state[r] = a < A.k ? T.enc(A.slot_state[a]) : dead;
        if (r * 32 < static_cast<int>(A.k)) start_live |= 1u << r;
    }

    for (uint64_t task = warp0; task < n_tasks; task += n_warps) {
        const uint64_t chunk0 = task * 64;
        uint64_t pos[2] = {0, 0}, end[2] = {0, 0};
        uint32_t s[2] = {dead, dead};
        uint32_t alive[2][R];
        bool pend[2] = {false, false};
#pragma unroll
        for (int nb = 0; nb < 2; ++nb) {
#pragma unroll
            for (int r = 0; r < R; ++r) alive[nb][r] = 0;
            for (uint32_t j = 0; j < 32; ++j) {
                const uint64_t ch = chunk0 + nb * 32 + j;
                if (ch >= p.c) break;
                uint64_t cp;
                uint32_t cs;
                uint32_t al[R];
                if (speculate_chunk<R, LUT>(p, T, ch, lane, start_state, start_live, dead, &cp, &cs, al)) {
                    if (lane == j) {
                        pos[nb] = cp;
                        s[nb] = cs;
                        pend[nb] = true;
#pragma unroll
                        for (int r = 0; r < R; ++r) alive[nb][r] = al[r];
                    }
                }
            }
        }
        // ---------------- converged phase: two chains per lane over shared windows
        uint64_t wb[2];
        uint32_t nwin[2];
#pragma unroll
        for (int nb = 0; nb < 2; ++nb) {
            if (pend[nb]) end[nb] = chunk_begin(chunk0 + nb * 32 + lane + 1, p.len, p.c);
            const uint64_t stop = min(end[nb], lim);
            wb[nb] = pos[nb] & ~static_cast<uint64_t>(15);
            nwin[nb] = (pend[nb] && wb[nb] < stop)
                           ? static_cast<uint32_t>((stop - wb[nb] + kC2Win - 1) / kC2Win) : 0;
        }
        const uint32_t max_win = __reduce_max_sync(kFull, max(nwin[0], nwin[1]));
        if (max_win) {
            const uint32_t g = lane & 1;
            uint4 v[4];
            // instruction u loads window j = 16u + (lane >> 1) (chunk chunk0 + j), granule g
            auto fetch = [&](uint32_t r) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int src = (16 * u + (lane >> 1)) & 31;
                    const int nb = u >> 1;
                    const uint64_t a = __shfl_sync(kFull, wb[nb], src) + static_cast<uint64_t>(kC2Win) * r + 16 * g;
                    const uint32_t nw = __shfl_sync(kFull, nwin[nb], src);
                    v[u] = (r < nw && a + 16 <= lim) ? __ldg(reinterpret_cast<const uint4 *>(p.text + a))
                                                     : make_uint4(0, 0, 0, 0);
                }
            };
            auto stash = [&]() {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t j = 16 * u + (lane >> 1);
                    const uint32_t addr = stg + j * kC2Stride + 16 * g;
                    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};"
                                 ::"r"(addr), "r"(v[u].x), "r"(v[u].y), "r"(v[u].z), "r"(v[u].w) : "memory");
                }
            };
            fetch(0);
            stash();
            __syncwarp();
            const uint32_t sb0 = stg + lane * kC2Stride, sb1 = stg + (32 + lane) * kC2Stride;
            for (uint32_t r = 0; r < max_win; ++r) {
                if (r + 1 < max_win) fetch(r + 1);
                bool full[2], have[2];
                uint64_t lo[2], hi[2], ws[2];
#pragma unroll
                for (int nb = 0; nb < 2; ++nb) {
                    ws[nb] = wb[nb] + static_cast<uint64_t>(kC2Win) * r;
                    have[nb] = r < nwin[nb] && s[nb] != dead;
                    const uint64_t stop = min(end[nb], lim);
                    lo[nb] = max(pos[nb], ws[nb]);
                    hi[nb] = min(stop, ws[nb] + kC2Win);
                    full[nb] = have[nb] && lo[nb] == ws[nb] && hi[nb] == ws[nb] + kC2Win;
                }
                if (full[0] && full[1]) {
                    run_granule2(T, s[0], sb0, s[1], sb1);
                    run_granule2(T, s[0], sb0 + 16, s[1], sb1 + 16);
                } else {
#pragma unroll
                    for (int nb = 0; nb < 2; ++nb) {
                        if (!have[nb]) continue;
                        const uint32_t sb = nb ? sb1 : sb0;
                        if (full[nb]) {
                            s[nb] = run_granule(T, s[nb], sb);
                            s[nb] = run_granule(T, s[nb], sb + 16);
                        } else {
                            for (uint64_t q = lo[nb]; q < hi[nb]; ++q)
                                s[nb] = T.next(s[nb], T.cls_of(lds_u8(sb + static_cast<uint32_t>(q - ws[nb]))));
                        }
                    }
                }
#pragma unroll
                for (int nb = 0; nb < 2; ++nb)
                    if (have[nb]) pos[nb] = hi[nb];
                __syncwarp();
                if (r + 1 < max_win) {
                    stash();
                    __syncwarp();
                }
            }
        }
        // tails past the last 16-byte boundary of the text, then rows and summaries
#pragma unroll
        for (int nb = 0; nb < 2; ++nb) {
            if (!pend[nb]) continue;
            while (pos[nb] < end[nb] && s[nb] != dead) {
                s[nb] = T.next(s[nb], T.cls_of(__ldg(p.text + pos[nb])));
                ++pos[nb];
            }
            const uint64_t ch = chunk0 + nb * 32 + lane;
            bool any = false;
#pragma unroll
            for (int r = 0; r < R; ++r) any |= alive[nb][r] != 0;
            const uint32_t sid = T.id(s[nb]);
            const uint16_t val = s[nb] == dead ? kUndef : static_cast<uint16_t>(sid);
            write_row<R>(p.maps + ch * p.stride, A.k, alive[nb], val);
            p.dinfo[ch] = (any && s[nb] != dead) ? ((1u << 16) | sid) : static_cast<uint32_t>(kUndef);
        }
    }
}

template <int R, int PATH = kPathCoop>
constexpr int block_cap() { return R <= 4 && PATH != kPathCoopSet ? 1024 : 512; }

// Launch (or, with per_sm != nullptr, size) one instantiation of the reach kernel.
template <int R>
constexpr int block_cap2() { return R <= 4 ? 768 : 512; }

template <int R, class LUT, int PATH>
cudaError_t reach_one(const ReachArgs &a, const ReachPlan &pl, cudaStream_t st, int *per_sm) {
    using KernT = void (*)(ReachArgs, int, uint32_t);
    KernT kern;
    if constexpr (PATH == kPathCoop2) kern = rid_reach2_kernel<R, LUT, block_cap2<R>()>;
    else kern = rid_reach_kernel<R, LUT, block_cap<R, PATH>(), PATH>;
    if (pl.pslot) {
        if constexpr (R == 1 && (PATH == kPathGlobal || PATH == kPathCoop || PATH == kPathCoopSet))
            kern = rid_reach_kernel<1, LUT, block_cap<1, PATH>(), PATH, true>;
        else
            return cudaErrorInvalidValue;
    }
    cudaError_t e = ensure_smem_cap(reinterpret_cast<const void *>(kern), pl.smem);
    if (e != cudaSuccess) return e;
    if (per_sm) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, pl.block, pl.smem);
    kern<<<pl.grid, pl.block, pl.smem, st>>>(a, pl.tis, pl.staging_offset);
    return cudaGetLastError();
}

template <class LUT, int PATH>
cudaError_t reach_r(const ReachArgs &a, const ReachPlan &pl, cudaStream_t st, int *per_sm) {
    switch (pl.R) {
        case 1: return reach_one<1, LUT, PATH>(a, pl, st, per_sm);
        case 2: return reach_one<2, LUT, PATH>(a, pl, st, per_sm);
        case 4: return reach_one<4, LUT, PATH>(a, pl, st, per_sm);
        default: return reach_one<8, LUT, PATH>(a, pl, st, per_sm);
    }
}

template <int PATH>
cudaError_t reach_m(const ReachArgs &a, const ReachPlan &pl, cudaStream_t st, int *per_sm) {
    switch (pl.mode) {
        case kModeRep16: return reach_r<LutRep<true>, PATH>(a, pl, st, per_sm);
        case kModeRep32: return reach_r<LutRep<false>, PATH>(a, pl, st, per_sm);
        case kModePart16: return reach_r<LutPart, PATH>(a, pl, st, per_sm);
        case kModeRep16x4: return reach_r<LutRep16x4, PATH>(a, pl, st, per_sm);
        case kModeRep16x4C:
            // (the compact class table serves the set path and plain global loads only)
            if constexpr (PATH == kPathCoopSet || PATH == kPathGlobal) return reach_r<LutRep16x4C, PATH>(a, pl, st, per_sm);
            else return cudaErrorInvalidValue;
        case kModePair:
            // (two-byte steps serve the single-run cooperative path and plain global loads)
            if constexpr (PATH == kPathCoop || PATH == kPathGlobal) return reach_r<LutPair, PATH>(a, pl, st, per_sm);
            else return cudaErrorInvalidValue;
        case kModePairF:
            if constexpr (PATH == kPathCoop || PATH == kPathGlobal) return reach_r<LutPairF, PATH>(a, pl, st, per_sm);
            else return cudaErrorInvalidValue;
        case kModePairH:
            if constexpr (PATH == kPathCoop || PATH == kPathGlobal) return reach_r<LutPairH, PATH>(a, pl, st, per_sm);
            else return cudaErrorInvalidValue;
        case kModePairC:
            // (the compact two-byte table serves the set path and plain global loads)
            if constexpr (PATH == kPathCoopSet || PATH == kPathGlobal) return reach_r<LutPairC, PATH>(a, pl, st, per_sm);
            else return cudaErrorInvalidValue;
        case kModePlain: return reach_r<LutPlain, PATH>(a, pl, st, per_sm);
        default: return reach_r<LutFlat, PATH>(a, pl, st, per_sm);
    }
}

}  // namespace
}  // namespace ridfa

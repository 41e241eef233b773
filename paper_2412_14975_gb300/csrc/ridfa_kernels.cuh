// Device building blocks shared by the single-text kernels (ridfa_device.cu) and the batched
// kernels (ridfa_batch.cu): constants, the device view of an automaton, shared-memory and
// asynchronous-copy helpers, the table lookup policies, and the speculative phase of one chunk.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "ridfa_internal.h"

namespace ridfa {

// (the plain structs below have one definition for every translation unit: the reach launches
// of each text path are compiled in a unit of their own)
struct Automaton {            // device view of one automaton
    const uint16_t *trans;    // [(n+1) * C]
    const uint8_t *classmap;  // [256]
    const uint32_t *final_bits;
    const uint32_t *ifmask;   // [(n+1) * kw]
    const uint16_t *slot_state;
    uint32_t n, C, k, kw, q0_slot;
    uint32_t merges;          // host planning hint (HostAutomaton::merges); unused on the device
};

// A run handed from the speculative phase to one lane: chunk j of the warp's task, resume
// position, state (policy encoding), and the group of slots that share it.
struct RunEntry {
    uint64_t pos;
    uint32_t state;
    uint16_t chunk;
    uint16_t group;
};

struct ReachArgs {
    Automaton A;
    const uint8_t *text;
    uint64_t len;
    uint32_t c;
    uint16_t *maps;           // [c][k]
    uint32_t *dinfo;          // [c]: (m << 16) | min defined end state (0xFFFF if none)
    uint32_t *status;
    uint32_t probe;
    RunEntry *runs;           // [grid warps][32 * 8], or null: only single-run hand-offs
    uint32_t *finals;         // [grid warps][kFinalsPerWarp]
    uint32_t stride;          // entries between consecutive rows of maps (A.k, or wider when the
                              // slots are one group of a larger row)
    const uint16_t *piece_slots;   // [c][32] per-chunk start states (0xFFFF: none), or null: the
                                   // slots' start states A.slot_state for every chunk
};

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint16_t kUndef = 0xFFFF;
constexpr uint32_t kStatusWide = 1u;      // some chunk has > 32 distinct end states
constexpr uint32_t kStatusBad = 2u;       // a device consistency check failed
constexpr int kMaxD = 32;                 // distinct end states handled by the matrix join
constexpr int kJoinThreads = 256;
static_assert(kPartialWords == 1 + kMaxD, "join partial layout");


__host__ __device__ inline uint64_t chunk_begin(uint64_t i, uint64_t len, uint64_t c) {
    // floor(i * len / c) without 128-bit products: i*(len/c) + (i*(len%c))/c
    return i * (len / c) + (i * (len % c)) / c;
}

// ------------------------------------------------------------------------------ reach
constexpr int kMaxRun = 8;              // distinct live states one chunk may hand off
// speculated bytes before a multi-run hand-off is tried: on the set path a lane carries all of a
// chunk's runs in one pass, so handing off early is cheap there (the codon RE: 16 bytes 7.7 %
// faster than 64); where each run takes a lane of its own, a late hand-off lets more runs merge
// first (the any-field record lines lost a third at 16)
constexpr uint32_t kMultiMin = 64;
constexpr uint32_t kMultiMinSet = 16;
constexpr uint32_t kRunsPerWarp = 32 * kMaxRun;
// per-warp words of the finals area: the final state of each run, then the alive bits of the
// task's hand-offs (word 32*r + lane: bit j = slot 32*r + lane alive at chunk j's hand-off)
constexpr uint32_t kFinalsPerWarp = kRunsPerWarp + 32 * 8;
static_assert(kMaxRun <= 8, "group tags keep the group in the low 3 bits");


__device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ uint32_t lds_u16(uint32_t addr) {
    uint32_t v;                       // zero-extended into a 32-bit register: no conversion
    asm volatile("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ void sts_u32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(v));
}
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

constexpr uint32_t kStatusTimeout = 4u;   // a bounded device wait gave up
// text paths of the converged phase
constexpr int kPathGlobal = 0;   // each lane: 16-byte global loads of its own chunk
// (1 was per-lane 1-D bulk copies into a shared-memory ring: retired)
constexpr int kPathCoop = 2;     // the warp: coalesced loads of 8 chunks' windows per instruction
constexpr int kPathCoop2 = 3;    // the same with two chunks per lane, interleaved
constexpr int kPathCoopSet = 4;  // kPathCoop, and a lane finishes all runs its chunk handed off together
// cooperative path: one 64-byte window per chunk of the warp; granule g of chunk j's window sits
// at 16-byte unit 4j + (g ^ ((j >> 1) & 3)), so both the stores (lanes write 4 granules of 2
// chunks per 8-lane phase) and the owners' 16-byte reads (8 chunks, one granule each) are
// conflict-free
constexpr uint32_t kCoopWin = 64;
constexpr uint32_t kCoopBufBytes = 32 * kCoopWin;          // one round: a window per chunk
constexpr uint32_t kWarpCoopBytes = 2 * kCoopBufBytes;     // double-buffered

__device__ __forceinline__ void cp_async_16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ uint32_t coop_unit(uint32_t j, uint32_t g) { return 4 * j + (g ^ ((j >> 1) & 3)); }
constexpr uint32_t kSpinLimit = 1u << 24;

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P1;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, P1;\n\t}"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}
// Wait, the whole warp together, for the phase of parity `parity` of the mbarrier at `bar`: at
// most `limit` polls.  False when the limit ran out (the caller reports a timeout and leaves).
__device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity, uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it)
        if (__all_sync(0xFFFFFFFFu, mbar_try_wait(bar, parity))) return true;
    return false;
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ uint4 lds_v4(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr));
    return v;
}
__device__ __forceinline__ uint32_t lds_u8(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}
// Byte q (0..3) of w in the low 8 bits.  Shift and mask run on the integer pipes; a byte permute
// (PRMT) measured slower here, as it competes with the table lookups for the shared-memory pipe.
__device__ __forceinline__ uint32_t byte_of(uint32_t w, int q) { return (w >> (8 * q)) & 0xFF; }

// Table lookup policies.  A run's state is kept in the policy's own encoding (`enc`); `id`
// recovers the automaton state number.
//
// Plain: the compact transition table in shared memory, entries premultiplied 16-bit byte
// offsets (entry (s, c) at byte 2(s*C + c) holds 2*C*s'), so a step is one 3-input add and one
// ld.shared.u16; the class table is the lane-replicated one of LutRep (conflict-free), holding 2c.
// Lanes gathering different transition entries may share a bank.  Needs 2*C*(P+1) <= 64 KiB.
struct LutPlain {
    uint32_t lc, bt;          // this lane's class copy; the transition table
    uint32_t row;             // 2*C: bytes per state row
    static size_t smem_bytes(const Automaton &A) { return 256 * 128 + static_cast<size_t>(A.n + 1) * A.C * 2; }
    static bool fits(const Automaton &A) { return static_cast<uint64_t>(A.n + 1) * A.C * 2 <= 0xFFFF; }
    __device__ void setup(const Automaton &A, uint8_t *smem, uint32_t) {
        row = 2 * A.C;
        const uint32_t base_c = smem_addr(smem);
        bt = base_c + 256 * 128;
        for (uint32_t i = threadIdx.x; i < 256 * 32; i += blockDim.x) sts_u32(base_c + i * 4, 2u * A.classmap[i >> 5]);
        const uint32_t n = (A.n + 1) * A.C;
        for (uint32_t i = threadIdx.x; i < (n + 1) / 2; i += blockDim.x) {
            const uint32_t v0 = A.trans[2 * i] * row;
            const uint32_t v1 = 2 * i + 1 < n ? A.trans[2 * i + 1] * row : 0u;
            sts_u32(bt + i * 4, v0 | (v1 << 16));
        }
        lc = base_c + (threadIdx.x & 31) * 4;
    }
    __device__ __forceinline__ uint32_t enc(uint32_t id) const { return id * row; }
    __device__ __forceinline__ uint32_t id(uint32_t s) const { return s / row; }
    __device__ __forceinline__ uint32_t cls_of(uint32_t b) const { return lds_u32(lc + b * 128); }
    __device__ __forceinline__ uint32_t cls_at(uint32_t w, int q) const { return lds_u32(lc + (byte_of(w, q) << 7)); }
    __device__ __forceinline__ uint32_t next(uint32_t s, uint32_t c) const { return lds_u16(bt + s + c); }
};

// Flat: the uint16 table [(n+1) * C] and uint8 class map through generic pointers, in shared
// memory when the table fits there, else in global memory -- for automata too large for Plain.
struct LutFlat {
    const uint16_t *t;
    const uint8_t *cls;
    uint32_t C;
    static size_t smem_bytes(const Automaton &A) { return 256 + static_cast<size_t>(A.n + 1) * A.C * 2; }
    __device__ void setup(const Automaton &A, uint8_t *smem, uint32_t aux) {
        const bool table_in_smem = aux != 0;
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
    __device__ __forceinline__ uint32_t cls_at(uint32_t w, int q) const { return cls[byte_of(w, q)]; }
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
    __device__ void setup(const Automaton &A, uint8_t *smem, uint32_t) {
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
    // class of byte q of w
    __device__ __forceinline__ uint32_t cls_at(uint32_t w, int q) const { return lds_u32(lc + (byte_of(w, q) << 7)); }
    __device__ __forceinline__ uint32_t next(uint32_t s, uint32_t c) const {
        return W16 ? lds_u16(lt + s + c) : lds_u32(lt + s + c);
    }
};

// Rep16 with states in 4-byte units: the same lane-replicated table of 16-bit entries, holding
// s' * Cp * 16 (the row offset over 4), so automata up to P * Cp <= 4095 fit the entries where
// byte offsets would overflow them; a step is a shift-add of the state, an add of the class offset
// and one ld.shared.u16.
// CC (compact classes): the class table is one copy of 256 16-bit class offsets (512 bytes)
// instead of 32 lane copies (32 KB).  Byte b's entry sits in bank (b >> 1) & 31, so lanes reading
// bytes of one 64-byte stretch (A, C, G, T; ASCII digits) never conflict and others at most
// rarely; the 32 KB it saves go to staging, i.e. to more warps beside a large replicated table.
template <bool CC>
struct LutRep16x4T {
    uint32_t lc, lt;          // shared addresses of this lane's class copy (CC: the one copy) /
                              // transition copy
    uint32_t row4;            // 4-byte units per state row: Cp * 16
    __host__ __device__ static uint32_t cpad(const Automaton &A) { return (A.C + 1) & ~1u; }
    __host__ __device__ static constexpr size_t class_bytes() { return CC ? 512 : 256 * 128; }
    static size_t smem_bytes(const Automaton &A) { return class_bytes() + static_cast<size_t>(A.n + 1) * cpad(A) * 64; }
    static bool fits(const Automaton &A) { return static_cast<uint64_t>(A.n) * cpad(A) * 16 <= 0xFFFF; }
    __device__ __forceinline__ static uint32_t cls_off(uint32_t c) { return (c >> 1) * 128 + (c & 1) * 2; }
    __device__ void setup(const Automaton &A, uint8_t *smem, uint32_t) {
        const uint32_t Cp = cpad(A);
        row4 = Cp * 16;
        const uint32_t base_c = smem_addr(smem);
        const uint32_t base_t = base_c + static_cast<uint32_t>(class_bytes());
        if (CC) {
            for (uint32_t i = threadIdx.x; i < 128; i += blockDim.x)
                sts_u32(base_c + i * 4, cls_off(A.classmap[2 * i]) | (cls_off(A.classmap[2 * i + 1]) << 16));
        } else {
            for (uint32_t i = threadIdx.x; i < 256 * 32; i += blockDim.x)
                sts_u32(base_c + i * 4, cls_off(A.classmap[i >> 5]));
        }
        const uint32_t words = (A.n + 1) * Cp / 2;
        for (uint32_t i = threadIdx.x; i < words * 32; i += blockDim.x) {
            const uint32_t w = i >> 5;
            const uint32_t s = (2 * w) / Cp, c0 = (2 * w) % Cp;
            const uint32_t n0 = A.trans[s * A.C + c0];
            const uint32_t n1 = (c0 + 1 < A.C) ? A.trans[s * A.C + c0 + 1] : A.n;
            sts_u32(base_t + i * 4, (n0 * row4) | ((n1 * row4) << 16));
        }
        const uint32_t lane = threadIdx.x & 31;
        lc = CC ? base_c : base_c + lane * 4;
        lt = base_t + lane * 4;
    }
    __device__ __forceinline__ uint32_t enc(uint32_t id) const { return id * row4; }
    __device__ __forceinline__ uint32_t id(uint32_t s) const { return s / row4; }
    __device__ __forceinline__ uint32_t cls_of(uint32_t b) const {
        return CC ? lds_u16(lc + b * 2) : lds_u32(lc + b * 128);
    }
    __device__ __forceinline__ uint32_t cls_at(uint32_t w, int q) const {
        return CC ? lds_u16(lc + (byte_of(w, q) << 1)) : lds_u32(lc + (byte_of(w, q) << 7));
    }
    __device__ __forceinline__ uint32_t next(uint32_t s, uint32_t c) const { return lds_u16(lt + (s << 2) + c); }
};
using LutRep16x4 = LutRep16x4T<false>;
using LutRep16x4C = LutRep16x4T<true>;

// Two-byte transitions (the super-transition tables among the compatible optimisations of the
// paper's conclusion, Sec. 5): the converged runs take the text two bytes per lookup.  Beside the
// lane-replicated class table (word b*32 + l = class(b) * 128) sits one lane-replicated table of
// 16-bit entries with a column for every pair of classes (c1, c2), entry delta(delta(s, c1), c2),
// and one for every single class c, entry delta(s, c): NP = C*C + C columns.  States are paired so
// that a pair column's offset is the sum of the two class words:
//   entry (s, p) at byte ((s >> 1) * NP + p) * 128 + l * 4 + (s & 1) * 2,
//   enc(s) = (s >> 1) * NP * 128 + (s & 1) * 2,
// so a pair step is s' = T[s + cw1 * C + cw2] (one IMAD, one add, one ld.shared.u16) and a single
// step s' = T[s + C*C*128 + cw] (one add, one load).  A 16-byte granule then costs 16 class lookups
// and 8 transition lookups instead of 16 + 16.  Fits small automata only: (P/2 + 1) * NP <= 511.
struct LutPair {
    static constexpr bool kPairs = true;
    uint32_t lc, lt, lt1;     // this lane's class copy; its transition copy (pairs, singles)
    uint32_t C, NP;
    static uint32_t np_of(const Automaton &A) { return A.C * A.C + A.C; }
    static size_t smem_bytes(const Automaton &A) {
        return 256 * 128 + static_cast<size_t>((A.n + 2) / 2) * np_of(A) * 128;
    }
    static bool fits(const Automaton &A) {
        return (static_cast<uint64_t>(A.n / 2) + 1) * np_of(A) * 128 <= 0xFFFF;
    }
    __device__ __forceinline__ uint32_t enc(uint32_t id) const { return (id >> 1) * NP * 128 + (id & 1) * 2; }
    __device__ __forceinline__ uint32_t id(uint32_t e) const { return ((e >> 7) / NP) * 2 + ((e >> 1) & 1); }
    __device__ void setup(const Automaton &A, uint8_t *smem, uint32_t) {
        C = A.C;
        NP = C * C + C;
        const uint32_t base_c = smem_addr(smem);
        const uint32_t base_t = base_c + 256 * 128;
        for (uint32_t i = threadIdx.x; i < 256 * 32; i += blockDim.x) sts_u32(base_c + i * 4, A.classmap[i >> 5] * 128u);
        const uint32_t n = A.n;               // the dead state: row n maps to itself
        auto step = [&](uint32_t st, uint32_t c) { return st >= n ? n : static_cast<uint32_t>(A.trans[st * C + c]); };
        auto value = [&](uint32_t st, uint32_t col) {
            if (st > n) st = n;
            const uint32_t t = col < C * C ? step(step(st, col / C), col % C) : step(st, col - C * C);
            return enc(t);
        };
        const uint32_t words = ((n + 2) / 2) * NP;
        for (uint32_t i = threadIdx.x; i < words * 32; i += blockDim.x) {
            const uint32_t w = i >> 5;
            const uint32_t sp = w / NP, col = w % NP;
            sts_u32(base_t + i * 4, value(2 * sp, col) | (value(2 * sp + 1, col) << 16));
        }
        const uint32_t lane = threadIdx.x & 31;
        lc = base_c + lane * 4;
        lt = base_t + lane * 4;
        lt1 = lt + C * C * 128;
    }
    __device__ __forceinline__ uint32_t cls_of(uint32_t b) const { return lds_u32(lc + b * 128); }
    __device__ __forceinline__ uint32_t cls_at(uint32_t w, int q) const { return lds_u32(lc + (byte_of(w, q) << 7)); }
    __device__ __forceinline__ uint32_t next(uint32_t s, uint32_t c) const { return lds_u16(lt1 + s + c); }
    // the pair column of classes (c1, c2), shared by every run stepping the same two bytes
    __device__ __forceinline__ uint32_t pair_col(uint32_t c1, uint32_t c2) const { return c1 * C + c2; }
    __device__ __forceinline__ uint32_t next_pc(uint32_t s, uint32_t pc) const { return lds_u16(lt + s + pc); }
    __device__ __forceinline__ uint32_t next2(uint32_t s, uint32_t c1, uint32_t c2) const {
        return next_pc(s, pair_col(c1, c2));
    }
};

// Two-byte transitions in one compact table, for automata whose runs stay apart (the set path,
// where a lane steps all of its chunk's runs over the same bytes): row s holds NP = C*C + C 16-bit
// entries, the C*C pair columns (c1, c2) -> delta(delta(s, c1), c2) and then the C single columns,
// padded to NPr entries (NPr = 2 mod 4: an odd number of words, so that consecutive rows start in
// different banks and the rows of one column cover all 32), each entry the premultiplied row offset
// 2*NPr*s' of its target, so
//   pair step   s' = T[s + 2*(c1*C + c2)]   (the column shared by all of a lane's runs),
//   single step s' = T[s + 2*C*C + 2*c].
// The class table is lane-replicated (word b*32 + l = 2*class(b), conflict-free).  A lane with m
// runs then pays 1 class lookup per byte and m/2 transition lookups instead of m; the gathers
// into the table can share banks, as in Plain.  Needs 2*NPr*(P+1) <= 64 KiB.
struct LutPairC {
    static constexpr bool kPairs = true;
    uint32_t lc, bt, bt1;     // this lane's class copy; the table (pairs, singles)
    uint32_t C, row;          // row: 2*NPr bytes per state
    __host__ __device__ static uint32_t np_of(const Automaton &A) {
        const uint32_t np = A.C * A.C + A.C;
        return np + (6 - np % 4) % 4;          // NPr: the next count = 2 mod 4
    }
    static size_t smem_bytes(const Automaton &A) {
        return 256 * 128 + static_cast<size_t>(A.n + 1) * np_of(A) * 2;
    }
    static bool fits(const Automaton &A) { return static_cast<uint64_t>(A.n + 1) * np_of(A) * 2 <= 0xFFFF; }
    __device__ void setup(const Automaton &A, uint8_t *smem, uint32_t) {
        C = A.C;
        const uint32_t NP = np_of(A);
        row = 2 * NP;
        const uint32_t base_c = smem_addr(smem);
        bt = base_c + 256 * 128;
        bt1 = bt + 2 * C * C;
        for (uint32_t i = threadIdx.x; i < 256 * 32; i += blockDim.x) sts_u32(base_c + i * 4, 2u * A.classmap[i >> 5]);
        const uint32_t n = A.n;               // the dead state: row n maps to itself
        auto value = [&](uint32_t e) -> uint32_t {
            const uint32_t st = e / NP, col = e % NP;
            if (col >= C * C + C) return 0u;  // padding, never read
            const uint32_t t = col < C * C ? A.trans[A.trans[st * C + col / C] * C + col % C]
                                           : A.trans[st * C + col - C * C];
            return t * row;
        };
        const uint32_t cnt = (n + 1) * NP;
        for (uint32_t i = threadIdx.x; i < (cnt + 1) / 2; i += blockDim.x) {
            const uint32_t v0 = value(2 * i);
            const uint32_t v1 = 2 * i + 1 < cnt ? value(2 * i + 1) : 0u;
            sts_u32(bt + i * 4, v0 | (v1 << 16));
        }
        lc = base_c + (threadIdx.x & 31) * 4;
    }
    __device__ __forceinline__ uint32_t enc(uint32_t id) const { return id * row; }
    __device__ __forceinline__ uint32_t id(uint32_t s) const { return s / row; }
    __device__ __forceinline__ uint32_t cls_of(uint32_t b) const { return lds_u32(lc + b * 128); }
    __device__ __forceinline__ uint32_t cls_at(uint32_t w, int q) const { return lds_u32(lc + (byte_of(w, q) << 7)); }
    __device__ __forceinline__ uint32_t next(uint32_t s, uint32_t c) const { return lds_u16(bt1 + s + c); }
    __device__ __forceinline__ uint32_t pair_col(uint32_t c1, uint32_t c2) const { return c1 * C + c2; }
    __device__ __forceinline__ uint32_t next_pc(uint32_t s, uint32_t pc) const { return lds_u16(bt + s + pc); }
    __device__ __forceinline__ uint32_t next2(uint32_t s, uint32_t c1, uint32_t c2) const {
        return next_pc(s, pair_col(c1, c2));
    }
};

// Two-byte transitions in F lane copies (F = 2, 4, 8 or 16, chosen at launch and passed to setup),
// for automata whose fully replicated pair table (LutPair, F = 32) does not fit: lane l reads copy
// l & (F - 1), and word (s >> 1, p) of LutPair's layout (two states per word, 16-bit halves) is
// stored F times side by side:
//   entry (s, p) at byte (((s >> 1) * NPw + p) * F + (l & (F - 1))) * 4 + (s & 1) * 2,
// NPw = (C*C + C) | 1 columns per state pair (odd, so that the rows of one column fall in every
// bank and not in one: with an even row stride all lanes of a copy reading one column would meet
// in the same bank or two).  Lanes of different copies never share a bank, so a pair gather costs
// at most 32/F wavefronts (2 at F = 16; about 3 on average at F = 8 for random rows), and it pays
// for two bytes, where the half-replicated one-byte table (LutPart) costs up to 2 for one.
// Two forms:
//   HW = false: entries are byte offsets enc(s) = (s >> 1) * NPw * 4F + (s & 1) * 2 beside the
//     lane-replicated class table (word b*32 + l = class(b) * 4F): a pair step is one IMAD for the
//     column and s' = T[s + cw1*C + cw2], one add and one load.  Needs (P/2 + 1) * NPw * 4F <= 64 KiB.
//   HW = true: entries are half-word offsets enc(s) = (s >> 1) * NPw * 2F + (s & 1), so twice the
//     copies fit 16 bits, beside one 256-byte table of 8-bit class offsets class(b) * 2F (bytes
//     below 128 read distinct banks, so ASCII text never conflicts there); a step is
//     s' = T[2 * (s + column)], one shift-add more.  Needs (P/2 + 1) * NPw * 2F <= 64 Ki and
//     (C - 1) * 2F <= 255.
template <bool HW>
struct LutPairFT {
    static constexpr bool kPairs = true;
    uint32_t lc, lt, lt1;     // this lane's class table; its transition copy (pairs, singles)
    uint32_t C, NPw, FU;      // FU: offset units per word row (4F bytes, or 2F half-words)
    __host__ __device__ static uint32_t npw_of(uint32_t C) { return (C * C + C) | 1u; }
    __host__ __device__ static constexpr size_t class_bytes() { return HW ? 256 : 256 * 128; }
    static size_t smem_bytes(const Automaton &A, uint32_t F) {
        return class_bytes() + static_cast<size_t>((A.n + 2) / 2) * npw_of(A.C) * 4 * F;
    }
    static bool fits(const Automaton &A, uint32_t F) {
        const uint64_t fu = HW ? 2 * F : 4 * F;
        return (static_cast<uint64_t>(A.n / 2) + 1) * npw_of(A.C) * fu <= 0xFFFF &&
               (!HW || (A.C - 1) * fu <= 255);
    }
    __device__ __forceinline__ uint32_t enc(uint32_t id) const {
        return (id >> 1) * NPw * FU + (id & 1) * (HW ? 1 : 2);
    }
    __device__ __forceinline__ uint32_t id(uint32_t e) const {
        return ((e / FU) / NPw) * 2 + (HW ? (e & 1) : ((e >> 1) & 1));
    }
    // aux = F, the number of lane copies
    __device__ void setup(const Automaton &A, uint8_t *smem, uint32_t aux) {
        const uint32_t F = aux;
        C = A.C;
        const uint32_t NP = C * C + C;
        NPw = npw_of(C);
        FU = HW ? 2 * F : 4 * F;
        const uint32_t base_c = smem_addr(smem);
        const uint32_t base_t = base_c + static_cast<uint32_t>(class_bytes());
        if (HW) {
            for (uint32_t i = threadIdx.x; i < 64; i += blockDim.x) {
                uint32_t v = 0;
                for (uint32_t q = 0; q < 4; ++q) v |= (A.classmap[4 * i + q] * FU) << (8 * q);
                sts_u32(base_c + i * 4, v);
            }
        } else {
            for (uint32_t i = threadIdx.x; i < 256 * 32; i += blockDim.x) sts_u32(base_c + i * 4, A.classmap[i >> 5] * FU);
        }
        const uint32_t n = A.n;               // the dead state: row n maps to itself
        auto step = [&](uint32_t st, uint32_t c) { return st >= n ? n : static_cast<uint32_t>(A.trans[st * C + c]); };
        auto value = [&](uint32_t st, uint32_t col) {
            if (st > n) st = n;
            if (col >= NP) return 0u;         // padding column, never read
            const uint32_t t = col < C * C ? step(step(st, col / C), col % C) : step(st, col - C * C);
            return enc(t);
        };
        const uint32_t words = ((n + 2) / 2) * NPw;
        for (uint32_t i = threadIdx.x; i < words * F; i += blockDim.x) {
            const uint32_t w = i / F;
            const uint32_t sp = w / NPw, col = w % NPw;
            sts_u32(base_t + i * 4, value(2 * sp, col) | (value(2 * sp + 1, col) << 16));
        }
        const uint32_t lane = threadIdx.x & 31;
        lc = HW ? base_c : base_c + lane * 4;
        lt = base_t + (lane & (F - 1)) * 4;
        lt1 = lt + C * C * FU * (HW ? 2 : 1);
    }
    __device__ __forceinline__ uint32_t cls_of(uint32_t b) const {
        return HW ? lds_u8(lc + b) : lds_u32(lc + b * 128);
    }
    __device__ __forceinline__ uint32_t cls_at(uint32_t w, int q) const {
        return HW ? lds_u8(lc + byte_of(w, q)) : lds_u32(lc + (byte_of(w, q) << 7));
    }
    __device__ __forceinline__ uint32_t next(uint32_t s, uint32_t c) const {
        return HW ? lds_u16(lt1 + ((s + c) << 1)) : lds_u16(lt1 + s + c);
    }
    __device__ __forceinline__ uint32_t pair_col(uint32_t c1, uint32_t c2) const { return c1 * C + c2; }
    __device__ __forceinline__ uint32_t next_pc(uint32_t s, uint32_t pc) const {
        return HW ? lds_u16(lt + ((s + pc) << 1)) : lds_u16(lt + s + pc);
    }
    __device__ __forceinline__ uint32_t next2(uint32_t s, uint32_t c1, uint32_t c2) const {
        return next_pc(s, pair_col(c1, c2));
    }
};
using LutPairF = LutPairFT<false>;
using LutPairH = LutPairFT<true>;

template <class LUT, class = void>
struct has_pairs { static constexpr bool value = false; };
template <class LUT>
struct has_pairs<LUT, decltype(void(LUT::kPairs))> { static constexpr bool value = LUT::kPairs; };

// Half-replicated tables, for transition tables too large to replicate 32 times: the class table
// as in LutRep (32 copies, conflict-free), the transition table in F = 16 copies, lane l reading
// copy l & 15.  Entry (s, c) sits at byte ((s * Cp/2 + c/2) * 16 + (l & 15)) * 4 + (c & 1) * 2, so
// lanes of different copies never share a bank and the two lanes of one copy share one only when
// their rows differ with the same parity: at most 2 wavefronts per gather.  States are kept in
// 2-byte units (s * Cp * 16), so a step is one add of a doubled state and the class offset.
struct LutPart {
    static constexpr uint32_t F = 16;
    uint32_t lc, lt;          // shared addresses of this lane's class copy / transition copy
    uint32_t unit;            // 2-byte units per state row: Cp * F
    __host__ __device__ static uint32_t cpad(const Automaton &A) { return (A.C + 1) & ~1u; }
    static size_t smem_bytes(const Automaton &A) {
        return 256 * 128 + static_cast<size_t>(A.n + 1) * (cpad(A) / 2) * (4 * F);
    }
    static bool fits(const Automaton &A) { return static_cast<uint64_t>(A.n) * cpad(A) * F <= 0xFFFF; }
    __device__ __forceinline__ static uint32_t cls_off(uint32_t c) { return (c >> 1) * (4 * F) + (c & 1) * 2; }
    __device__ void setup(const Automaton &A, uint8_t *smem, uint32_t) {
        const uint32_t Cp = cpad(A);
        unit = Cp * F;
        const uint32_t base_c = smem_addr(smem);
        const uint32_t base_t = base_c + 256 * 128;
        for (uint32_t i = threadIdx.x; i < 256 * 32; i += blockDim.x)
            sts_u32(base_c + i * 4, cls_off(A.classmap[i >> 5]));
        const uint32_t words = (A.n + 1) * (Cp / 2) * F;
        for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) {
            const uint32_t rowp = i / F;                       // s * Cp/2 + c/2
            const uint32_t s = rowp / (Cp / 2), c0 = 2 * (rowp % (Cp / 2));
            const uint32_t n0 = A.trans[s * A.C + c0];
            const uint32_t n1 = (c0 + 1 < A.C) ? A.trans[s * A.C + c0 + 1] : A.n;
            sts_u32(base_t + i * 4, (n0 * unit) | ((n1 * unit) << 16));
        }
        const uint32_t lane = threadIdx.x & 31;
        lc = base_c + lane * 4;
        lt = base_t + (lane & (F - 1)) * 4;
    }
    __device__ __forceinline__ uint32_t enc(uint32_t id) const { return id * unit; }
    __device__ __forceinline__ uint32_t id(uint32_t s) const { return s / unit; }
    __device__ __forceinline__ uint32_t cls_of(uint32_t b) const { return lds_u32(lc + b * 128); }
    __device__ __forceinline__ uint32_t cls_at(uint32_t w, int q) const { return lds_u32(lc + (byte_of(w, q) << 7)); }
    __device__ __forceinline__ uint32_t next(uint32_t s, uint32_t c) const { return lds_u16(lt + 2 * s + c); }
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


// Speculative phase of one chunk text[beg, end) by the whole warp (lanes = runs; slot
// a = 32*r + lane in register r).  Every `probe` bytes the warp drops registers whose runs are all
// dead and checks whether the live runs sit in one state (redux.sync min == max).  With `multi`
// set, once MULTI_MIN bytes have been speculated it also hands off as soon as the live runs sit in
// at most kMaxRun distinct states, each as a run of its own.
//
// Return m >= 1 (handed off before `end`): *out_pos is the resume position, lane g < m holds the
// g-th distinct live state (ascending) in *my_d (for m = 1 every lane holds it), alive[] holds
// the ballots of the slots still alive (the same in every lane), and for m >= 2 (or any m when
// `tag_all`) the chunk's map row holds a group tag per alive slot (0x8000 | g) and 0xFFFF for a
// dead one, to be replaced once the runs end.
// Return 0: the chunk finished here; its map row (`row`, k entries) and its D_i summary
// (`*dinfo_slot`) are written.
template <int R, class LUT, uint32_t MULTI_MIN = kMultiMin>
__device__ __forceinline__ int speculate(const LUT &T, const Automaton &A, const uint8_t *text,
                                         uint64_t beg, uint64_t end, uint32_t probe, uint32_t lane,
                                         const uint32_t (&start_state)[R], uint32_t start_live,
                                         uint32_t dead, uint16_t *row, uint32_t *dinfo_slot,
                                         uint32_t *status, bool multi, bool tag_all, uint64_t *out_pos,
                                         uint32_t *my_d, uint32_t (&alive)[R]) {
    uint32_t s[R];
#pragma unroll
    for (int r = 0; r < R; ++r) s[r] = start_state[r];
    uint32_t live_regs = start_live;
    uint64_t pos = beg;
    int m = 0;
    uint32_t d = dead;
    while (pos < end) {
        const uint64_t stop = min(end, pos + probe);
        for (; pos < stop; ++pos) {
            const uint32_t c = T.cls_of(__ldg(text + pos));
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (live_regs & (1u << r)) s[r] = T.next(s[r], c);
        }
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
        if (lo == 0xFFFFFFFFu) break;                     // every run died: finish here
        if (lo == hi) {
            if (pos < end) {
                m = 1;
                d = lo;
            }
            break;
        }
        if (multi && pos < end && pos - beg >= MULTI_MIN) {
            // the distinct live states in ascending order, lane g taking the g-th, while there
            // are at most kMaxRun of them
            uint32_t cnt = 0, cur = 0, mine = dead;
            for (;;) {
                uint32_t v = 0xFFFFFFFFu;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (s[r] != dead && (cnt == 0 || s[r] > cur)) v = min(v, s[r]);
                v = __reduce_min_sync(kFull, v);
                if (v == 0xFFFFFFFFu) break;
                if (cnt == static_cast<uint32_t>(kMaxRun)) {
                    cnt = kMaxRun + 1;
                    break;
                }
                if (lane == cnt) mine = v;
                cur = v;
                ++cnt;
            }
            if (cnt <= static_cast<uint32_t>(kMaxRun)) {
                m = static_cast<int>(cnt);
                d = mine;
                break;
            }
        }
    }
    if (m >= 1) {
#pragma unroll
        for (int r = 0; r < R; ++r) alive[r] = __ballot_sync(kFull, s[r] != dead);
        if (m >= 2 || tag_all) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                uint32_t tag = kUndef;
                for (int g = 0; g < m; ++g) {
                    const uint32_t dg = __shfl_sync(kFull, d, g);     // every lane takes part
                    if (s[r] != dead && dg == s[r]) tag = 0x8000u | g;
                }
                const uint32_t a = r * 32 + lane;
                if (a < A.k) row[a] = static_cast<uint16_t>(tag);
            }
        }
        *out_pos = pos;
        *my_d = d;
        return m;
    }
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
            *dinfo_slot = (0xFFu << 16) | first;
            atomicOr(status, kStatusWide);
        } else {
            *dinfo_slot = (cnt << 16) | first;
        }
    }
    return 0;
}

// The single-run form: true when the live runs merged into one state before `end`
// (*out_state), false when the chunk finished in the speculative phase.
template <int R, class LUT>
__device__ __forceinline__ bool speculate_range(const LUT &T, const Automaton &A, const uint8_t *text,
                                                uint64_t beg, uint64_t end, uint32_t probe,
                                                uint32_t lane, const uint32_t (&start_state)[R],
                                                uint32_t start_live, uint32_t dead, uint16_t *row,
                                                uint32_t *dinfo_slot, uint32_t *status,
                                                uint64_t *out_pos, uint32_t *out_state,
                                                uint32_t (&alive)[R]) {
    return speculate<R, LUT>(T, A, text, beg, end, probe, lane, start_state, start_live, dead, row,
                             dinfo_slot, status, false, false, out_pos, out_state, alive) == 1;
}

// Map row and D_i summary of a handed-off chunk, by the whole warp, once its runs have ended.
// `am` is this lane's alive bit of each of its slots (bit r: slot 32*r + lane); lane g < m holds
// the final state of group g in `fin`.  Untagged rows (m = 1 without tag_all) are written from
// the alive bits alone; tagged rows are read back and their group tags replaced.
template <int R, class LUT>
__device__ __forceinline__ void finish_handed_row(const LUT &T, uint16_t *row, uint32_t k, uint32_t m,
                                                  bool tagged, uint32_t lane, uint32_t am, uint32_t fin,
                                                  uint32_t dead, uint32_t *dinfo_slot) {
    const uint32_t fid = (lane < m && fin != dead) ? T.id(fin) : kUndef;
    if (!tagged) {
        const uint32_t v = __shfl_sync(kFull, fid, 0);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t a = r * 32 + lane;
            if (a < k) row[a] = static_cast<uint16_t>(((am >> r) & 1) ? v : kUndef);
        }
        if (lane == 0) *dinfo_slot = v == kUndef ? static_cast<uint32_t>(kUndef) : ((1u << 16) | v);
        return;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t a = r * 32 + lane;
        const uint32_t t = (a < k && ((am >> r) & 1)) ? row[a] : kUndef;
        const bool live = t != kUndef;
        const uint32_t v = __shfl_sync(kFull, fid, live ? (t & 7) : 0);
        if (a < k) row[a] = static_cast<uint16_t>(live ? v : kUndef);
    }
    // every group owns at least one slot: D_i is the set of defined group finals
    bool dup = false;
    for (uint32_t h = 0; h < m; ++h) {
        const uint32_t fh = __shfl_sync(kFull, fid, h);
        if (h < lane && fh == fid) dup = true;
    }
    const bool uniq = lane < m && fid != kUndef && !dup;
    const uint32_t cnt = __popc(__ballot_sync(kFull, uniq));
    const uint32_t first = __reduce_min_sync(kFull, uniq ? fid : static_cast<uint32_t>(kUndef));
    if (lane == 0) *dinfo_slot = cnt ? ((cnt << 16) | first) : static_cast<uint32_t>(kUndef);
}

// 16 transitions of one run over one 16-byte granule held in shared memory.
template <class LUT>
__device__ __forceinline__ uint32_t run_granule(const LUT &T, uint32_t s, uint32_t addr) {
    const uint4 x = lds_v4(addr);
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
    uint32_t cl[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) cl[q] = T.cls_at(w[q >> 2], q & 3);
    if constexpr (has_pairs<LUT>::value) {
#pragma unroll
        for (int q = 0; q < 16; q += 2) s = T.next2(s, cl[q], cl[q + 1]);
    } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) s = T.next(s, cl[q]);
    }
    return s;
}

// Converged phase of up to 32 runs, one per lane, with the text staged by the warp.  Lane l's
// run (if `pending`) advances from `pos` to `stop` over its own text `base`; `lim` is that
// text's length rounded down to 16 (the same for every lane when ONE_TEXT), and stop <= lim:
// what lies past `lim` is left to the caller's plain loads.  The windows [wb + 64r, +64) of
// each run (wb = the 16-byte boundary at or below `pos`) are copied with cp.async (L2 to shared
// memory, no register or L1 round trip): lane l copies granule (l & 3) of the windows of runs
// (l >> 2) + 8u, u = 0..3, so one instruction moves 8 runs' windows; one round ahead,
// double-buffered, in the XOR-swizzled layout of coop_unit.
template <class LUT, bool ONE_TEXT>
__device__ __forceinline__ void coop_converge(const LUT &T, uint32_t stg_base, uint32_t lane, bool pending,
                                              const uint8_t *base, uint64_t lim, uint64_t stop,
                                              uint64_t &pos, uint32_t &s, uint32_t dead) {
    const uint64_t wb = pos & ~static_cast<uint64_t>(15);
    const uint32_t nwin = (pending && wb < stop)
                              ? static_cast<uint32_t>((stop - wb + kCoopWin - 1) / kCoopWin) : 0;
    const uint64_t waddr = reinterpret_cast<uint64_t>(base) + wb;
    const uint64_t wlim = reinterpret_cast<uint64_t>(base) + lim;
    const uint32_t g = lane & 3;
    const uint32_t max_win = __reduce_max_sync(kFull, nwin);
    auto issue = [&](uint32_t r) {
        const uint32_t buf = stg_base + (r & 1) * kCoopBufBytes;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = u * 8 + (lane >> 2);        // run whose granule g this lane copies
            const uint64_t a = __shfl_sync(kFull, waddr, j) + static_cast<uint64_t>(kCoopWin) * r + 16 * g;
            const uint32_t nw = __shfl_sync(kFull, nwin, j);
            const uint64_t la = ONE_TEXT ? wlim : __shfl_sync(kFull, wlim, j);
            if (r < nw && a + 16 <= la) cp_async_16(buf + 16 * coop_unit(j, g), reinterpret_cast<const void *>(a));
        }
        cp_async_commit();
    };
    issue(0);
    const uint32_t sw = (lane >> 1) & 3;
    for (uint32_t r = 0; r < max_win; ++r) {
        if (r + 1 < max_win) issue(r + 1);
        else cp_async_commit();               // keep one group per round
        cp_async_wait1();                     // this lane's copies of round r have landed
        __syncwarp();                         // ... and every other lane's
        const uint64_t ws = wb + static_cast<uint64_t>(kCoopWin) * r;
        if (r < nwin && s != dead) {
            const uint32_t sb = stg_base + (r & 1) * kCoopBufBytes + 64 * lane;
            const uint64_t lo = max(pos, ws), hi = min(stop, ws + kCoopWin);
            if (lo == ws && hi == ws + kCoopWin) {
#pragma unroll
                for (uint32_t q16 = 0; q16 < kCoopWin / 16; ++q16) s = run_granule(T, s, sb + 16 * (q16 ^ sw));
            } else {
                for (uint64_t q = lo; q < hi; ++q) {
                    const uint32_t o = static_cast<uint32_t>(q - ws);
                    s = T.next(s, T.cls_of(lds_u8(sb + 16 * ((o >> 4) ^ sw) + (o & 15))));
                }
            }
            pos = hi;
        }
        __syncwarp();                         // buffer (r & 1) is refilled next round
    }
    cp_async_wait0();
    __syncwarp();
}

// Runs of one lane on the set path: slots s[0..kMaxRun) hold states (dead where unused), and
// `rep` maps each handed-off group g (4 bits at 4g) to the slot its run lives in, or 0xF once it
// died.  compact_runs drops dead runs and runs in the same state as an earlier slot (they would
// repeat its lookups from here on: the merging of Sec. 5's convergence, now inside the lane) and
// packs the survivors into slots 0..cnt-1 in their order; it returns cnt.  Register arrays are
// only indexed by compile-time constants (select networks), so nothing spills to local memory.
__device__ __forceinline__ uint32_t compact_runs(uint32_t (&s)[kMaxRun], uint32_t &rep, uint32_t dead) {
    uint32_t nidx = 0;        // 4 bits per old slot: its new slot, 0xF when dropped as dead
    uint32_t cnt = 0;
#pragma unroll
    for (int j = 0; j < kMaxRun; ++j) {
        uint32_t idx = 0xF;
        if (s[j] != dead) {
#pragma unroll
            for (int i = 0; i < j; ++i)
                if (idx == 0xF && s[i] == s[j]) idx = (nidx >> (4 * i)) & 0xF;
            if (idx == 0xF) idx = cnt++;
        }
        nidx |= idx << (4 * j);
    }
    uint32_t t[kMaxRun];
#pragma unroll
    for (int k = 0; k < kMaxRun; ++k) t[k] = dead;
#pragma unroll
    for (int j = 0; j < kMaxRun; ++j) {
        const uint32_t idx = (nidx >> (4 * j)) & 0xF;
#pragma unroll
        for (int k = 0; k < kMaxRun; ++k)
            if (idx == static_cast<uint32_t>(k)) t[k] = s[j];     // a merged slot rewrites its leader's value
    }
#pragma unroll
    for (int k = 0; k < kMaxRun; ++k) s[k] = t[k];
    uint32_t nrep = 0;
#pragma unroll
    for (int g = 0; g < kMaxRun; ++g) {
        const uint32_t r = (rep >> (4 * g)) & 0xF;
        nrep |= (r == 0xF ? 0xFu : (nidx >> (4 * r)) & 0xF) << (4 * g);
    }
    rep = nrep;
    return cnt;
}

// One staged 64-byte window for the first M run slots of a lane (M is the same in the whole warp:
// the largest live count; a lane's unused slots hold the dead state, which maps to itself).
template <class LUT, int M>
__device__ __forceinline__ void set_window(const LUT &T, uint32_t sb, uint32_t sw, uint32_t o0, uint32_t o1,
                                           uint32_t (&s)[kMaxRun]) {
    if (o0 == 0 && o1 == kCoopWin) {
        // (one granule of code per M, not four: the eight specialisations share the instruction
        // cache, and the unrolled form measured slower for it)
#pragma unroll 1
        for (uint32_t q16 = 0; q16 < kCoopWin / 16; ++q16) {
            const uint4 x = lds_v4(sb + 16 * (q16 ^ sw));
            const uint32_t w[4] = {x.x, x.y, x.z, x.w};
            uint32_t cl[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) cl[q] = T.cls_at(w[q >> 2], q & 3);
            if constexpr (has_pairs<LUT>::value) {
#pragma unroll
                for (int q = 0; q < 16; q += 2) {
                    const uint32_t pc = T.pair_col(cl[q], cl[q + 1]);
#pragma unroll
                    for (int g = 0; g < M; ++g) s[g] = T.next_pc(s[g], pc);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 16; ++q)
#pragma unroll
                    for (int g = 0; g < M; ++g) s[g] = T.next(s[g], cl[q]);
            }
        }
    } else {
        for (uint32_t o = o0; o < o1; ++o) {
            const uint32_t c = T.cls_of(lds_u8(sb + 16 * ((o >> 4) ^ sw) + (o & 15)));
#pragma unroll
            for (int g = 0; g < M; ++g) s[g] = T.next(s[g], c);
        }
    }
}

// coop_converge for a lane that carries all the runs of one chunk together (up to kMaxRun states
// handed off at one position): the text is staged once per chunk and each byte's class is looked
// up once for all of them, so m runs cost 1 + m lookups per byte instead of 2m.  Every four
// windows the lane's runs are compacted (dead runs dropped, runs that met merged) and the warp's
// loop is respecialised to the largest live count M, so a byte costs 1 + M lookups and no
// instruction is issued for a run that is gone.
template <class LUT>
__device__ __forceinline__ void coop_converge_set(const LUT &T, uint32_t stg_base, uint32_t lane, bool pending,
                                                  const uint8_t *base, uint64_t lim, uint64_t stop, uint64_t &pos,
                                                  uint32_t (&s)[kMaxRun], uint32_t &rep, uint32_t dead) {
    const uint64_t wb = pos & ~static_cast<uint64_t>(15);
    const uint32_t nwin = (pending && wb < stop)
                              ? static_cast<uint32_t>((stop - wb + kCoopWin - 1) / kCoopWin) : 0;
    const uint64_t waddr = reinterpret_cast<uint64_t>(base) + wb;
    const uint64_t wlim = reinterpret_cast<uint64_t>(base) + lim;
    const uint32_t g = lane & 3;
    const uint32_t max_win = __reduce_max_sync(kFull, nwin);
    uint32_t cnt = pending ? compact_runs(s, rep, dead) : 0;
    uint32_t M = __reduce_max_sync(kFull, cnt);
    auto issue = [&](uint32_t r) {
        const uint32_t buf = stg_base + (r & 1) * kCoopBufBytes;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = u * 8 + (lane >> 2);
            const uint64_t a = __shfl_sync(kFull, waddr, j) + static_cast<uint64_t>(kCoopWin) * r + 16 * g;
            const uint32_t nw = __shfl_sync(kFull, nwin, j);
            const uint64_t la = __shfl_sync(kFull, wlim, j);
            if (r < nw && a + 16 <= la) cp_async_16(buf + 16 * coop_unit(j, g), reinterpret_cast<const void *>(a));
        }
        cp_async_commit();
    };
    issue(0);
    const uint32_t sw = (lane >> 1) & 3;
    for (uint32_t r = 0; r < max_win; ++r) {
        if (r + 1 < max_win) issue(r + 1);
        else cp_async_commit();
        cp_async_wait1();
        __syncwarp();
        const uint64_t ws = wb + static_cast<uint64_t>(kCoopWin) * r;
        if (r < nwin && cnt) {
            const uint32_t sb = stg_base + (r & 1) * kCoopBufBytes + 64 * lane;
            const uint64_t lo = max(pos, ws), hi = min(stop, ws + kCoopWin);
            const uint32_t o0 = static_cast<uint32_t>(lo - ws), o1 = static_cast<uint32_t>(hi - ws);
            switch (M) {
                case 1: set_window<LUT, 1>(T, sb, sw, o0, o1, s); break;
                case 2: set_window<LUT, 2>(T, sb, sw, o0, o1, s); break;
                case 3: set_window<LUT, 3>(T, sb, sw, o0, o1, s); break;
                case 4: set_window<LUT, 4>(T, sb, sw, o0, o1, s); break;
                case 5: set_window<LUT, 5>(T, sb, sw, o0, o1, s); break;
                case 6: set_window<LUT, 6>(T, sb, sw, o0, o1, s); break;
                case 7: set_window<LUT, 7>(T, sb, sw, o0, o1, s); break;
                default: set_window<LUT, 8>(T, sb, sw, o0, o1, s); break;
            }
            pos = hi;
        }
        __syncwarp();
        if ((r & 3) == 3) {
            if (cnt) cnt = compact_runs(s, rep, dead);
            M = __reduce_max_sync(kFull, cnt);
        }
    }
    cp_async_wait0();
    __syncwarp();
}

// The rest of one run, text[pos, end), with plain global loads (16-byte vector loads once
// aligned when VEC).
template <class LUT, bool VEC>
__device__ __forceinline__ void tail_converge(const LUT &T, const uint8_t *t, uint64_t &pos, uint64_t end,
                                              uint32_t &s, uint32_t dead) {
    if (VEC) {
        while (pos < end && (reinterpret_cast<uintptr_t>(t + pos) & 15)) {
            s = T.next(s, T.cls_of(__ldg(t + pos)));
            ++pos;
        }
        while (pos + 16 <= end && s != dead) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(t + pos));
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
            uint32_t cl[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) cl[q] = T.cls_at(w[q >> 2], q & 3);
#pragma unroll
            for (int q = 0; q < 16; ++q) s = T.next(s, cl[q]);
            pos += 16;
        }
    }
    while (pos < end && s != dead) {
        s = T.next(s, T.cls_of(__ldg(t + pos)));
        ++pos;
    }
}

// After coop_converge_set: the runs' rest past the staged part (plain loads), then the final state
// of each handed-off group g < m into fin[g] (the dead state when its run died).
template <class LUT>
__device__ __forceinline__ void finish_set_runs(const LUT &T, const uint8_t *text, uint64_t pos, uint64_t end,
                                                uint32_t (&s)[kMaxRun], uint32_t rep, uint32_t m, uint32_t *fin,
                                                uint32_t dead) {
#pragma unroll
    for (int k = 0; k < kMaxRun; ++k) {
        uint64_t pk = pos;
        tail_converge<LUT, false>(T, text, pk, end, s[k], dead);
    }
#pragma unroll
    for (int gg = 0; gg < kMaxRun; ++gg) {
        if (gg >= static_cast<int>(m)) continue;
        const uint32_t r = (rep >> (4 * gg)) & 0xF;
        uint32_t v = dead;
#pragma unroll
        for (int k = 0; k < kMaxRun; ++k)
            if (r == static_cast<uint32_t>(k)) v = s[k];
        fin[gg] = v;
    }
}

__device__ __forceinline__ bool is_final_state(const Automaton &A, uint32_t s) {
    return s < A.n && ((A.final_bits[s >> 5] >> (s & 31)) & 1);
}

}  // namespace
}  // namespace ridfa

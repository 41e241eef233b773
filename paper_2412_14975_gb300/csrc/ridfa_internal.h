// Internal structures shared by the host compiler (ridfa_compile.cpp) and the device code
// (ridfa_device.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cstddef>
#include <cuda_runtime_api.h>
#include <nvtx3/nvToolsExt.h>
#include <mutex>
#include <string>
#include <vector>

#include "ridfa.h"

namespace ridfa {

// A named NVTX range over a host scope (compile, reach launches, join launch, batch and server
// launches), for timeline tools such as Nsight Systems; free when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// One speculative automaton as the device sees it: the RI-DFA B with its interface
// (Sec. 3.1-3.4) or the minimal DFA with every state initial (Sec. 2).
struct HostAutomaton {
    uint32_t n_states = 0;            // |P| (or |Q|); the dead state has id n_states
    uint32_t n_classes = 0;           // byte classes C
    uint32_t k = 0;                   // interface slots
    uint32_t kw = 0;                  // 32-bit words per interface-set row: ceil(k / 32)
    uint32_t q0_slot = 0;             // slot whose start state is {q0} (or the DFA start)
    std::vector<uint16_t> trans;      // [(n_states + 1) * n_classes], dead row / moves = n_states
    std::vector<uint8_t> classmap;    // [256]
    std::vector<uint8_t> final_flag;  // [n_states]
    std::vector<uint32_t> final_bits; // [ceil((n_states + 1) / 32)]
    std::vector<uint32_t> ifmask;     // [(n_states + 1) * kw]: slots of if_min({p}); dead row = 0
    std::vector<uint16_t> slot_state; // [k]: start state of each slot
    uint32_t merges = 0;              // 1: runs from every slot merge on random text (merge_hint)
};

// Device copy of one automaton (one per device it was uploaded to).
struct DeviceAutomaton {
    int device = -1;
    uint16_t *trans = nullptr;
    uint8_t *classmap = nullptr;
    uint32_t *final_bits = nullptr;
    uint32_t *ifmask = nullptr;
    uint16_t *slot_state = nullptr;
    uint16_t *all_states = nullptr;   // [n_states]: state s (every state as a start, for pieces)
    size_t bytes = 0;
};

// The position NFA over byte classes, for the NFA variant of the classic algorithm (the
// comparator of Sec. 2 / Table 3): follow rows, class rows (positions reading the class) and the
// final set as bitsets of nw 32-bit words (bit q of word q / 32 = NFA state q; 0 = q0).  Kept
// only when n <= 128 (nw <= 4); n = 0 otherwise.
struct HostNfa {
    uint32_t n = 0, nw = 0, n_classes = 0;
    std::vector<uint8_t> classmap;    // [256]
    std::vector<uint32_t> follow;     // [n][nw]
    std::vector<uint32_t> cls;        // [n_classes][nw]
    std::vector<uint32_t> finals;     // [nw]
};

// Device copy of a HostNfa (one per device it was uploaded to): one allocation.
struct DeviceNfa {
    int device = -1;
    void *base = nullptr;
    const uint8_t *classmap = nullptr;
    const uint32_t *follow = nullptr, *cls = nullptr, *finals = nullptr;
    void *scratch = nullptr;          // the call's relations (grown on demand)
    size_t scratch_bytes = 0;
    uint8_t *h_accept_pinned = nullptr;
};

// Per-device scratch of a program: chunk maps when the caller passes none, per-chunk summaries,
// the join's partial products, a block ticket, the status word and the accept byte.
struct DeviceScratch {
    int device = -1;
    void *base = nullptr;
    size_t bytes = 0;
    uint8_t *h_accept_pinned = nullptr;
    uint32_t *h_status_pinned = nullptr;
    void *ev[3] = {nullptr, nullptr, nullptr};   // cudaEvent_t: before reach, before join, after
    bool profiled = false;
    ridfa_plan_report last_plan{};               // the reach plan of the last call on this device
    bool planned = false;
};

}  // namespace ridfa

struct ridfa_program {
    std::string re;
    uint32_t n_nfa = 0;
    std::vector<std::vector<uint32_t>> state_sets;   // NFA states of each RI-DFA state
    std::vector<uint32_t> slots;                      // representative NFA state per slot
    std::vector<uint32_t> delegate_slot;              // NFA state -> slot of its representative
    ridfa::HostAutomaton rid;
    ridfa::HostAutomaton dfa;
    bool has_dfa = false;
    ridfa::HostNfa nfa;                               // the NFA variant's tables (n <= 128)
    // device side (filled lazily by the device code)
    mutable std::mutex mu;
    mutable std::vector<ridfa::DeviceAutomaton> dev_rid, dev_dfa;
    mutable std::vector<ridfa::DeviceScratch> scratch;
    mutable std::vector<ridfa::DeviceNfa> dev_nfa;
};

namespace ridfa {
void release_device(const ridfa_program *prog);   // defined in the device code
void release_nfa(const ridfa_program *prog);      // ridfa_nfa.cu

// Device buffers supplied by the caller of launch_with_buffers: the automaton's tables and every
// piece of scratch the reach and join kernels use.  Nothing is allocated by the launch.
struct PreparedBuffers {
    const uint16_t *trans;
    const uint8_t *classmap;
    const uint32_t *final_bits;
    const uint32_t *ifmask;
    const uint16_t *slot_state;
    uint16_t *maps;        // [c][k]
    uint32_t *dinfo;       // [c]
    uint32_t *partials;    // [kMaxJoinBlocks][33]
    uint32_t *ticket;      // zero before the launch
    uint32_t *status;      // zero before the launch
    uint8_t *accept;
};
// Host helpers of the device code (ridfa_device.cu), shared with the batched path.
int cuda_fail(cudaError_t e);
int upload(const HostAutomaton &H, DeviceAutomaton &D, int dev);
const DeviceAutomaton *device_copy(const ridfa_program *P, bool dfa, int dev, int *err);
int smem_optin_limit();
// Raise a kernel's dynamic shared-memory cap on the current device to at least `bytes`.  The cap
// is never lowered, so a launch sized by another thread (or an earlier plan) stays valid.
cudaError_t ensure_smem_cap(const void *kern, size_t bytes);

constexpr uint32_t kMaxJoinBlocks = 1024;
constexpr uint32_t kPartialWords = 33;

// Enqueue the reach and join kernels of the RID path (automatic tuning) on `stream`, on buffers
// that are already resident.  Returns a RIDFA_* status; performs no allocation.
int launch_with_buffers(const HostAutomaton &H, const PreparedBuffers &B, const uint8_t *d_text,
                        uint64_t len, uint32_t n_chunks, void *stream);
}

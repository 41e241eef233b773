// Host composition of shard summaries (the join of Sec. 3.2 applied to whole shards).
//
// A shard summary maps each entry slot a to the set of states the shard can end in when entered
// through a.  The join is a composition of union-distributive relations, so consecutive shards
// compose as the chunks inside them do: the first shard is entered through {q0}'s slot only, the
// next one through the slots of if_min of the states the previous one ended in, and the text is
// accepted iff the last set meets F^RID.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "ridfa.h"
#include "ridfa_internal.h"

extern "C" int ridfa_join_shards(const ridfa_program *prog, const ridfa_shard_summary *shards, uint32_t n,
                                 uint8_t *h_accept) {
    if (!prog || !shards || n == 0 || !h_accept) return RIDFA_E_ARG;
    const ridfa::HostAutomaton &H = prog->rid;
    for (uint32_t j = 0; j < n; ++j)
        if (shards[j].k != H.k || shards[j].n_out > RIDFA_MAX_SLOTS) return RIDFA_E_ARG;
    const uint32_t kw = H.kw;
    std::vector<uint32_t> slots(kw, 0);
    std::vector<uint16_t> plas;            // states the previous shard can end in
    auto end_states = [&](const ridfa_shard_summary &S, const std::vector<uint32_t> &in) {
        std::vector<uint32_t> bits(RIDFA_MAX_SLOTS / 32, 0);
        for (uint32_t a = 0; a < H.k; ++a)
            if ((in[a >> 5] >> (a & 31)) & 1)
                for (uint32_t w = 0; w < RIDFA_MAX_SLOTS / 32; ++w) bits[w] |= S.reach[a][w];
        std::vector<uint16_t> out;
        for (uint32_t y = 0; y < S.n_out; ++y)
            if ((bits[y >> 5] >> (y & 31)) & 1) out.push_back(S.out_state[y]);
        return out;
    };
    slots[H.q0_slot >> 5] |= 1u << (H.q0_slot & 31);
    plas = end_states(shards[0], slots);
    for (uint32_t j = 1; j < n && !plas.empty(); ++j) {
        std::fill(slots.begin(), slots.end(), 0u);
        for (uint16_t x : plas) {
            if (x >= H.n_states) return RIDFA_E_ARG;
            for (uint32_t w = 0; w < kw; ++w) slots[w] |= H.ifmask[static_cast<uint64_t>(x) * kw + w];
        }
        plas = end_states(shards[j], slots);
    }
    uint8_t acc = 0;
    for (uint16_t x : plas)
        if (x < H.n_states && H.final_flag[x]) acc = 1;
    *h_accept = acc;
    return RIDFA_OK;
}

// The recognition on the host's cores: the CPU context of the device numbers, in the setting the
// paper measures its method in (Sec. 4: one text, its chunks on the cores of one machine).
//   n_chunks = 1: the serial recognizer, the table loop from {q0} (Sec. 2's serial run; on the
//                 minimal DFA the classic serial DFA).
//   n_chunks > 1: the chunked speculative recognition (Sec. 3.2): chunk 1 from {q0}'s slot, every
//                 other chunk from every interface slot, runs that meet in one state at one
//                 position merged (Sec. 5's convergence), the chunk maps lambda_i, then the join
//                 PLAS_i = lambda_i(if_min(PLAS_{i-1})) and acceptance PLAS_c n F != {}.  On the
//                 minimal DFA with every state a slot it is the all-states DFA variant (Sec. 2).
// The chunks are split over host threads; the join runs on the calling thread.  ridfa_recognize
// never calls this: it is a separate entry point for comparisons, not a fallback.
#include <algorithm>
#include <cstdint>
#include <new>
#include <thread>
#include <vector>

#include "ridfa.h"
#include "ridfa_internal.h"

namespace ridfa {
namespace {

uint64_t chunk_start(uint64_t i, uint64_t len, uint64_t c) { return i * (len / c) + (i * (len % c)) / c; }

// One run from state s over text[b, e): its end state, or the dead state once it dies.
inline uint32_t walk(const HostAutomaton &H, uint32_t s, const uint8_t *text, uint64_t b, uint64_t e) {
    const uint16_t *T = H.trans.data();
    const uint8_t *cm = H.classmap.data();
    const uint32_t C = H.n_classes, dead = H.n_states;
    for (uint64_t p = b; p < e; ++p) {
        s = T[static_cast<size_t>(s) * C + cm[text[p]]];
        if (s == dead) break;
    }
    return s;
}

// Chunk maps of chunks [c_lo, c_hi) (chunk 0 from q0's slot only) into rows[i * k + a].  The
// distinct live states of a chunk are stepped once per byte; `idx` maps each slot to the entry
// it shares, and is rewritten only at a step where runs merged or died (otherwise the entries
// keep their order).
void reach_range(const HostAutomaton &H, const uint8_t *text, uint64_t len, uint64_t c, uint64_t c_lo,
                 uint64_t c_hi, uint16_t *rows) {
    const uint32_t k = H.k, C = H.n_classes, dead = H.n_states;
    const uint16_t *T = H.trans.data();
    const uint8_t *cm = H.classmap.data();
    std::vector<uint32_t> stamp(dead + 1, 0), where(dead + 1, 0);
    uint32_t gen = 0;
    std::vector<uint32_t> st, st2, remap, idx(k);
    for (uint64_t i = c_lo; i < c_hi; ++i) {
        const uint64_t b = chunk_start(i, len, c), e = chunk_start(i + 1, len, c);
        uint16_t *row = rows + i * k;
        if (i == 0) {
            std::fill(row, row + k, static_cast<uint16_t>(dead));
            row[H.q0_slot] = static_cast<uint16_t>(walk(H, H.slot_state[H.q0_slot], text, b, e));
            continue;
        }
        st.assign(H.slot_state.begin(), H.slot_state.end());     // distinct start states
        for (uint32_t a = 0; a < k; ++a) idx[a] = a;
        uint64_t p = b;
        while (p < e && st.size() > 1) {
            const uint32_t cls = cm[text[p++]];
            if (++gen == 0) {
                std::fill(stamp.begin(), stamp.end(), 0u);
                gen = 1;
            }
            st2.clear();
            remap.assign(st.size(), UINT32_MAX);
            bool same = true;
            for (size_t j = 0; j < st.size(); ++j) {
                const uint32_t s2 = T[static_cast<size_t>(st[j]) * C + cls];
                if (s2 == dead) {
                    same = false;
                    continue;
                }
                if (stamp[s2] != gen) {
                    stamp[s2] = gen;
                    where[s2] = static_cast<uint32_t>(st2.size());
                    st2.push_back(s2);
                }
                remap[j] = where[s2];
                if (remap[j] != j) same = false;
            }
            if (!same)
                for (uint32_t a = 0; a < k; ++a)
                    if (idx[a] != UINT32_MAX) idx[a] = remap[idx[a]];
            st.swap(st2);
        }
        if (st.size() == 1) st[0] = walk(H, st[0], text, p, e);
        for (uint32_t a = 0; a < k; ++a)
            row[a] = static_cast<uint16_t>(idx[a] == UINT32_MAX || st.empty() ? dead : st[idx[a]]);
    }
}

}  // namespace
}  // namespace ridfa

extern "C" int ridfa_cpu_recognize(const ridfa_program *prog, int which, const uint8_t *h_text, size_t len,
                                   uint32_t n_chunks, uint32_t n_threads, uint8_t *h_accept) {
    if (!prog || !h_accept || (len && !h_text) || which < 0 || which > 1) return RIDFA_E_ARG;
    if (which == 1 && !prog->has_dfa) return RIDFA_E_NO_DFA;
    const ridfa::HostAutomaton &H = which ? prog->dfa : prog->rid;
    const uint32_t dead = H.n_states;
    if (len == 0) {
        if (n_chunks != 0) return RIDFA_E_CHUNKS;
        *h_accept = H.final_flag[H.slot_state[H.q0_slot]];
        return RIDFA_OK;
    }
    if (n_chunks == 0 || n_chunks > len) return RIDFA_E_CHUNKS;
    if (n_chunks == 1) {
        const uint32_t s = ridfa::walk(H, H.slot_state[H.q0_slot], h_text, 0, len);
        *h_accept = s != dead && H.final_flag[s];
        return RIDFA_OK;
    }
    const uint64_t c = n_chunks, k = H.k;
    std::vector<uint16_t> rows;
    try {
        rows.resize(c * k);
    } catch (const std::bad_alloc &) {
        return RIDFA_E_NOMEM;
    }
    uint32_t T = n_threads ? n_threads : std::max(1u, std::thread::hardware_concurrency());
    T = static_cast<uint32_t>(std::min<uint64_t>(T, c));
    std::vector<std::thread> th;
    try {
        for (uint32_t t = 1; t < T; ++t)
            th.emplace_back(ridfa::reach_range, std::cref(H), h_text, static_cast<uint64_t>(len), c, c * t / T,
                            c * (t + 1) / T, rows.data());
    } catch (...) {
        for (auto &x : th) x.join();
        return RIDFA_E_NOMEM;
    }
    ridfa::reach_range(H, h_text, len, c, 0, c / T, rows.data());
    for (auto &x : th) x.join();
    // join: PLAS_1 = {lambda_1(q0)}; PLAS_i = lambda_i(if_min(PLAS_{i-1})) without the dead state
    std::vector<uint32_t> plas, next, stamp(dead + 1, 0), in(H.kw);
    uint32_t gen = 1;
    if (rows[H.q0_slot] != dead) plas.push_back(rows[H.q0_slot]);
    for (uint64_t i = 1; i < c && !plas.empty(); ++i) {
        std::fill(in.begin(), in.end(), 0u);
        for (uint32_t p : plas)
            for (uint32_t w = 0; w < H.kw; ++w) in[w] |= H.ifmask[static_cast<size_t>(p) * H.kw + w];
        next.clear();
        ++gen;
        const uint16_t *row = rows.data() + i * k;
        for (uint32_t w = 0; w < H.kw; ++w)
            for (uint32_t m = in[w]; m; m &= m - 1) {
                const uint32_t a = 32 * w + static_cast<uint32_t>(__builtin_ctz(m));
                const uint32_t s = row[a];
                if (s != dead && stamp[s] != gen) {
                    stamp[s] = gen;
                    next.push_back(s);
                }
            }
        plas.swap(next);
    }
    uint8_t acc = 0;
    for (uint32_t p : plas) acc |= H.final_flag[p];
    *h_accept = acc;
    return RIDFA_OK;
}

// Transition counters of the reach phase on the host (diagnostics for the roofline and for the
// paper's work metric).  For chunk 1 the runs start from {q0}'s slot only, for every other chunk
// from every interface slot (Sec. 3.2); a run ends at its chunk's end or at the undefined move.
//   w_paper: transitions executed when every run is followed on its own, the undefined move not
//            counted (the paper's measure, Sec. 1 and Fig. 1);
//   w_conv:  table lookups when runs that reach the same state at the same position are merged
//            (one lookup per distinct live state per byte, the undefined move included) -- the
//            work of a reach phase that collapses merged runs, as the device kernel does.
// The same counts for the all-states DFA comparator (Sec. 2) use the minimal DFA with every
// state as a start state.
#include <algorithm>
#include <cstdint>
#include <thread>
#include <vector>

#include "ridfa.h"
#include "ridfa_internal.h"

namespace ridfa {
namespace {

struct Counts {
    uint64_t w_paper = 0, w_conv = 0, runs = 0, dead = 0;
    uint64_t conv[16] = {};
};

// Bucket of a convergence distance (bytes read until at most one live state): 0 for 0 or 1,
// b for 2^b .. 2^(b+1) - 1, at most 14.
uint32_t conv_bucket(uint64_t bytes) {
    uint32_t b = 0;
    while (b < 14 && (bytes >> (b + 1)) != 0) ++b;
    return b;
}

uint64_t chunk_at(uint64_t i, uint64_t len, uint64_t c) { return i * (len / c) + (i * (len % c)) / c; }

// Chunks [c_lo, c_hi) of the text; stamp / slot are per-thread scratch of n + 1 entries.
void count_range(const HostAutomaton &H, const uint8_t *text, uint64_t len, uint64_t c, uint64_t c_lo,
                 uint64_t c_hi, Counts *out) {
    const uint32_t n = H.n_states, C = H.n_classes, dead = H.n_states;
    std::vector<uint32_t> stamp(n + 1, 0), where(n + 1, 0);
    uint32_t gen = 0;
    std::vector<uint32_t> st, st2;
    std::vector<uint64_t> mult, mult2;
    Counts k;
    for (uint64_t i = c_lo; i < c_hi; ++i) {
        const uint64_t b = chunk_at(i, len, c), e = chunk_at(i + 1, len, c);
        uint64_t conv_at = UINT64_MAX;      // bytes read when at most one live state remained
        st.clear();
        mult.clear();
        if (i == 0) {
            st.push_back(H.slot_state[H.q0_slot]);
            mult.push_back(1);
        } else {
            // slot start states are distinct singletons (or distinct DFA states)
            for (uint32_t a = 0; a < H.k; ++a) {
                st.push_back(H.slot_state[a]);
                mult.push_back(1);
            }
        }
        k.runs += st.size();
        uint64_t p = b;
        for (; p < e && !st.empty(); ++p) {
            if (i > 0 && st.size() <= 1 && conv_at == UINT64_MAX) conv_at = p - b;
            const uint32_t cls = H.classmap[text[p]];
            k.w_conv += st.size();
            if (++gen == 0) {                      // stamp wrap-around: clear once
                std::fill(stamp.begin(), stamp.end(), 0);
                gen = 1;
            }
            st2.clear();
            mult2.clear();
            for (size_t j = 0; j < st.size(); ++j) {
                const uint32_t s2 = H.trans[static_cast<uint64_t>(st[j]) * C + cls];
                if (s2 == dead) {
                    k.dead += mult[j];
                    continue;
                }
                k.w_paper += mult[j];
                if (stamp[s2] == gen) {
                    mult2[where[s2]] += mult[j];
                } else {
                    stamp[s2] = gen;
                    where[s2] = static_cast<uint32_t>(st2.size());
                    st2.push_back(s2);
                    mult2.push_back(mult[j]);
                }
            }
            st.swap(st2);
            mult.swap(mult2);
        }
        if (i > 0) {
            if (conv_at == UINT64_MAX && st.size() <= 1) conv_at = p - b;
            ++k.conv[conv_at == UINT64_MAX ? 15 : conv_bucket(conv_at)];
        }
    }
    *out = k;
}

// The NFA variant (Sec. 2): chunk 1 from q0, the others from every NFA state, each start's set of
// active states followed on its own.  A step from the set S on a byte of class c executes
// sum over q in S of |Follow(q) n cls(c)| transitions (w_paper) and processes |S| states (w_conv).
void count_range_nfa(const HostNfa &N, const uint8_t *text, uint64_t len, uint64_t c, uint64_t c_lo,
                     uint64_t c_hi, Counts *out) {
    const uint32_t nw = N.nw;
    Counts k;
    std::vector<uint32_t> S(nw), F(nw);
    for (uint64_t i = c_lo; i < c_hi; ++i) {
        const uint64_t b = chunk_at(i, len, c), e = chunk_at(i + 1, len, c);
        const uint32_t starts = i == 0 ? 1 : N.n;
        for (uint32_t q0 = 0; q0 < starts; ++q0) {
            std::fill(S.begin(), S.end(), 0u);
            S[q0 >> 5] = 1u << (q0 & 31);
            ++k.runs;
            bool alive = true;
            for (uint64_t p = b; p < e; ++p) {
                const uint32_t *cm = N.cls.data() + static_cast<size_t>(N.classmap[text[p]]) * nw;
                std::fill(F.begin(), F.end(), 0u);
                for (uint32_t w = 0; w < nw; ++w)
                    for (uint32_t m = S[w]; m; m &= m - 1) {
                        const uint32_t q = 32 * w + static_cast<uint32_t>(__builtin_ctz(m));
                        ++k.w_conv;
                        const uint32_t *f = N.follow.data() + static_cast<size_t>(q) * nw;
                        for (uint32_t v = 0; v < nw; ++v) {
                            F[v] |= f[v];
                            k.w_paper += static_cast<uint64_t>(__builtin_popcount(f[v] & cm[v]));
                        }
                    }
                uint32_t any = 0;
                for (uint32_t v = 0; v < nw; ++v) any |= (S[v] = F[v] & cm[v]);
                if (!any) {
                    alive = false;
                    break;
                }
            }
            if (!alive) ++k.dead;
        }
    }
    *out = k;
}

}  // namespace
}  // namespace ridfa

extern "C" int ridfa_count_transitions(const ridfa_program *prog, int which, const uint8_t *h_text, size_t len,
                                       uint32_t n_chunks, uint32_t n_threads, ridfa_transition_counts *out) {
    if (!prog || !out || (len && !h_text) || which < 0 || which > 2) return RIDFA_E_ARG;
    if (which == 1 && !prog->has_dfa) return RIDFA_E_NO_DFA;
    if (which == 2 && prog->nfa.n == 0) return RIDFA_E_UNSUPPORTED;
    if (n_chunks == 0 || n_chunks > len) return RIDFA_E_CHUNKS;
    const ridfa::HostAutomaton &H = which ? prog->dfa : prog->rid;
    uint32_t T = n_threads ? n_threads : std::max(1u, std::thread::hardware_concurrency());
    T = static_cast<uint32_t>(std::min<uint64_t>(T, n_chunks));
    std::vector<ridfa::Counts> parts(T);
    std::vector<std::thread> th;
    const uint64_t c = n_chunks;
    try {
        for (uint32_t t = 1; t < T; ++t)
            if (which == 2)
                th.emplace_back(ridfa::count_range_nfa, std::cref(prog->nfa), h_text, static_cast<uint64_t>(len), c,
                                c * t / T, c * (t + 1) / T, &parts[t]);
            else
                th.emplace_back(ridfa::count_range, std::cref(H), h_text, static_cast<uint64_t>(len), c, c * t / T,
                                c * (t + 1) / T, &parts[t]);
    } catch (...) {
        for (auto &x : th) x.join();
        return RIDFA_E_NOMEM;
    }
    if (which == 2) ridfa::count_range_nfa(prog->nfa, h_text, len, c, 0, c / T, &parts[0]);
    else ridfa::count_range(H, h_text, len, c, 0, c / T, &parts[0]);
    for (auto &x : th) x.join();
    ridfa_transition_counts r{};
    for (const auto &p : parts) {
        r.w_paper += p.w_paper;
        r.w_conv += p.w_conv;
        r.runs += p.runs;
        r.dead_runs += p.dead;
        for (int q = 0; q < 16; ++q) r.converge_hist[q] += p.conv[q];
    }
    *out = r;
    return RIDFA_OK;
}

// Host compiler of the RID recognizer: RE -> position NFA -> RI-DFA -> interface minimisation
// -> byte classes -> uint16 tables; plus the minimal DFA of the all-states comparator.
//
// Method (arXiv 2412.14975):
//   * NFA N = (Q_N, Sigma, rho, q0, F) from the RE by the McNaughton-Yamada / Glushkov position
//     construction (Sec. 4.1, Sec. 5): one state per symbol occurrence, plus q0.
//   * RI-DFA B = N(q0) u N(q1) u ... u N(q_{l-1}): the powerset machine started from each
//     singleton in turn, adding only what is new (Sec. 3.1); I^B = the singletons; F^RID = the
//     subsets that contain a final NFA state.
//   * Interface minimisation (Sec. 3.4): language-equivalence classes by state partition on B
//     completed with a dead state; in each class of singletons the lowest NFA state stays
//     initial and the others delegate to it; if_min maps {q} to its representative's slot.
//
// Numbering rules (so that independent implementations agree on ids): singletons {q} get ids
// 0..l-1; other subsets get the next ids in breadth-first discovery order, exploring {q0},
// {q1}, ... in turn and, from each state, the byte classes in ascending order; byte classes
// are numbered by their smallest byte.  The minimal DFA is numbered breadth-first from its
// start with classes ascending.
#include <algorithm>
#include <bitset>
#include <cstring>
#include <deque>
#include <new>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

#include "ridfa_internal.h"

namespace {

struct SyntaxError : std::runtime_error {
    using std::runtime_error::runtime_error;
};
struct TooManyStates : std::runtime_error {
    using std::runtime_error::runtime_error;
};

// --------------------------------------------------------------------------------- syntax
enum class Kind : uint8_t { Eps, Set, Cat, Alt, Star, Plus, Opt, Rep };

struct Node {
    Kind kind = Kind::Eps;
    std::bitset<256> bytes;
    std::vector<int> kids;
    int lo = 0, hi = 0;  // Rep bounds; hi < 0 means unbounded
};

class Parser {
public:
    Parser(const char *s, size_t n) : s_(reinterpret_cast<const unsigned char *>(s)), n_(n) {}

    int parse() {
        int root = alternation();
        if (i_ != n_) throw SyntaxError("unexpected character");
        return root;
    }
    std::vector<Node> nodes;

private:
    const unsigned char *s_;
    size_t n_, i_ = 0;

    int peek() const { return i_ < n_ ? s_[i_] : -1; }
    int add(Node nd) {
        nodes.push_back(std::move(nd));
        return static_cast<int>(nodes.size()) - 1;
    }
    int alternation() {
        std::vector<int> alts{concatenation()};
        while (peek() == '|') {
            ++i_;
            alts.push_back(concatenation());
        }
        if (alts.size() == 1) return alts[0];
        Node nd;
        nd.kind = Kind::Alt;
        nd.kids = std::move(alts);
        return add(std::move(nd));
    }
    int concatenation() {
        std::vector<int> items;
        while (peek() != -1 && peek() != '|' && peek() != ')') items.push_back(postfix());
        if (items.empty()) return add(Node{});
        if (items.size() == 1) return items[0];
        Node nd;
        nd.kind = Kind::Cat;
        nd.kids = std::move(items);
        return add(std::move(nd));
    }
    int number() {
        size_t st = i_;
        long v = 0;
        while (peek() >= '0' && peek() <= '9') {
            v = v * 10 + (s_[i_++] - '0');
            if (v > 100000) throw SyntaxError("repeat bound too large");
        }
        if (i_ == st) throw SyntaxError("expected a number");
        return static_cast<int>(v);
    }
    int postfix() {
        int x = atom();
        for (;;) {
            int c = peek();
            Node nd;
            if (c == '*') nd.kind = Kind::Star;
            else if (c == '+') nd.kind = Kind::Plus;
            else if (c == '?') nd.kind = Kind::Opt;
            else if (c == '{') {
                ++i_;
                nd.kind = Kind::Rep;
                nd.lo = number();
                if (peek() == '}') {
                    nd.hi = nd.lo;
                } else if (peek() == ',') {
                    ++i_;
                    nd.hi = (peek() == '}') ? -1 : number();
                    if (nd.hi >= 0 && nd.hi < nd.lo) throw SyntaxError("repeat {m,n} with n < m");
                } else {
                    throw SyntaxError("bad repeat");
                }
                if (peek() != '}') throw SyntaxError("expected }");
                nd.kids = {x};
                ++i_;
                x = add(std::move(nd));
                continue;
            } else {
                return x;
            }
            ++i_;
            nd.kids = {x};
            x = add(std::move(nd));
        }
    }
    int hexdigit(int c) {
        if (c >= '0' && c <= '9') return c - '0';
        if (c >= 'a' && c <= 'f') return c - 'a' + 10;
        if (c >= 'A' && c <= 'F') return c - 'A' + 10;
        throw SyntaxError("bad \\x escape");
    }
    int escaped() {  // after the backslash
        if (peek() == -1) throw SyntaxError("dangling backslash");
        int c = s_[i_++];
        switch (c) {
            case 'n': return 10;
            case 't': return 9;
            case 'r': return 13;
            case 'x': {
                if (i_ + 2 > n_) throw SyntaxError("bad \\x escape");
                int v = hexdigit(s_[i_]) * 16 + hexdigit(s_[i_ + 1]);
                i_ += 2;
                return v;
            }
            default: return c;
        }
    }
    int atom() {
        int c = peek();
        if (c == -1) throw SyntaxError("unexpected end");
        Node nd;
        nd.kind = Kind::Set;
        if (c == '(') {
            ++i_;
            int x = alternation();
            if (peek() != ')') throw SyntaxError("expected )");
            ++i_;
            return x;
        }
        if (c == '[') {
            ++i_;
            nd.bytes = bracket();
        } else if (c == '.') {
            ++i_;
            nd.bytes.set();
        } else if (c == '\\') {
            ++i_;
            nd.bytes.set(escaped());
        } else if (c == '*' || c == '+' || c == '?' || c == '{' || c == '}' || c == ')' || c == ']') {
            throw SyntaxError("unexpected metacharacter");
        } else {
            ++i_;
            nd.bytes.set(c);
        }
        return add(std::move(nd));
    }
    std::bitset<256> bracket() {
        std::bitset<256> m;
        bool neg = false, first = true;
        if (peek() == '^') {
            neg = true;
            ++i_;
        }
        for (;;) {
            int c = peek();
            if (c == -1) throw SyntaxError("unterminated [");
            if (c == ']' && !first) {
                ++i_;
                break;
            }
            first = false;
            ++i_;
            int lo = (c == '\\') ? escaped() : c;
            if (peek() == '-' && i_ + 1 < n_ && s_[i_ + 1] != ']') {
                ++i_;
                int h = s_[i_++];
                int hi = (h == '\\') ? escaped() : h;
                if (hi < lo) throw SyntaxError("bad range");
                for (int b = lo; b <= hi; ++b) m.set(b);
            } else {
                m.set(lo);
            }
        }
        if (neg) m.flip();
        if (m.none()) throw SyntaxError("empty class");
        return m;
    }
};

// ------------------------------------------------------------------- position automaton
struct Frag {
    bool nullable = true;
    std::vector<uint32_t> first, last;
};

class PositionBuilder {
public:
    explicit PositionBuilder(const std::vector<Node> &nodes) : nodes_(nodes) {
        sym.emplace_back();   // index 0 is q0
        follow.emplace_back();
    }
    std::vector<std::bitset<256>> sym;
    std::vector<std::vector<uint32_t>> follow;

    Frag build(int node) {
        const Node &nd = nodes_[node];
        switch (nd.kind) {
            case Kind::Eps: return Frag{};
            case Kind::Set: {
                if (sym.size() >= 200000) throw TooManyStates("too many positions");
                uint32_t p = static_cast<uint32_t>(sym.size());
                sym.push_back(nd.bytes);
                follow.emplace_back();
                Frag f;
                f.nullable = false;
                f.first = {p};
                f.last = {p};
                return f;
            }
            case Kind::Cat: {
                Frag acc;
                for (int kid : nd.kids) acc = concat(std::move(acc), build(kid));
                return acc;
            }
            case Kind::Alt: {
                Frag acc;
                acc.nullable = false;
                for (int kid : nd.kids) {
                    Frag f = build(kid);
                    acc.nullable = acc.nullable || f.nullable;
                    acc.first.insert(acc.first.end(), f.first.begin(), f.first.end());
                    acc.last.insert(acc.last.end(), f.last.begin(), f.last.end());
                }
                return acc;
            }
            case Kind::Star:
            case Kind::Plus: {
                Frag f = build(nd.kids[0]);
                loop(f);
                if (nd.kind == Kind::Star) f.nullable = true;
                return f;
            }
            case Kind::Opt: {
                Frag f = build(nd.kids[0]);
                f.nullable = true;
                return f;
            }
            case Kind::Rep: {
                // r{m,n} = r^m (r(r(...r)?)?)?; r{m,} = r^m r*.  Copies are built left to right
                // so positions are numbered in text order of the expansion.
                Frag acc;
                for (int i = 0; i < nd.lo; ++i) acc = concat(std::move(acc), build(nd.kids[0]));
                if (nd.hi < 0) {
                    Frag f = build(nd.kids[0]);
                    loop(f);
                    f.nullable = true;
                    acc = concat(std::move(acc), std::move(f));
                } else if (nd.hi > nd.lo) {
                    std::vector<Frag> copies;
                    for (int i = nd.lo; i < nd.hi; ++i) copies.push_back(build(nd.kids[0]));
                    Frag inner = std::move(copies.back());
                    inner.nullable = true;
                    for (int j = static_cast<int>(copies.size()) - 2; j >= 0; --j) {
                        inner = concat(std::move(copies[j]), std::move(inner));
                        inner.nullable = true;
                    }
                    acc = concat(std::move(acc), std::move(inner));
                }
                return acc;
            }
        }
        return Frag{};
    }

private:
    const std::vector<Node> &nodes_;

    void link(const std::vector<uint32_t> &from, const std::vector<uint32_t> &to) {
        for (uint32_t p : from) follow[p].insert(follow[p].end(), to.begin(), to.end());
    }
    void loop(const Frag &f) { link(f.last, f.first); }
    Frag concat(Frag a, Frag b) {
        link(a.last, b.first);
        Frag r;
        r.nullable = a.nullable && b.nullable;
        r.first = std::move(a.first);
        if (a.nullable) r.first.insert(r.first.end(), b.first.begin(), b.first.end());
        r.last = b.last;
        if (b.nullable) r.last.insert(r.last.end(), a.last.begin(), a.last.end());
        return r;
    }
};

// ------------------------------------------------------------------------ bitset helpers
struct Bits {
    uint32_t words = 0;
    std::vector<uint64_t> data;  // rows of `words` words
    uint64_t *row(size_t i) { return data.data() + i * words; }
    const uint64_t *row(size_t i) const { return data.data() + i * words; }
};

struct KeyHash {
    size_t operator()(const std::string &s) const { return std::hash<std::string>()(s); }
};

inline std::string key_of(const uint64_t *w, uint32_t words) {
    return std::string(reinterpret_cast<const char *>(w), sizeof(uint64_t) * words);
}

// NFA over byte classes: follow rows, class rows (positions reading the class), finals.
struct ClassNfa {
    uint32_t n = 0;        // states 0..n-1 (0 = q0)
    uint32_t words = 0;
    uint32_t n_classes = 0;
    std::vector<uint8_t> classmap;
    Bits follow;           // n rows
    Bits cls;              // n_classes rows
    std::vector<uint64_t> finals;
};

ClassNfa make_class_nfa(const PositionBuilder &pb, const Frag &root) {
    ClassNfa N;
    N.n = static_cast<uint32_t>(pb.sym.size());
    N.words = (N.n + 63) / 64;
    N.follow.words = N.words;
    N.follow.data.assign(static_cast<size_t>(N.n) * N.words, 0);
    auto set_bit = [](uint64_t *r, uint32_t p) { r[p >> 6] |= uint64_t(1) << (p & 63); };
    for (uint32_t p : root.first) set_bit(N.follow.row(0), p);
    for (uint32_t q = 1; q < N.n; ++q)
        for (uint32_t p : pb.follow[q]) set_bit(N.follow.row(q), p);
    // bytes read by exactly the same positions share a class; classes are numbered by their
    // smallest byte
    std::vector<uint64_t> byte_rows(static_cast<size_t>(256) * N.words, 0);
    for (uint32_t p = 1; p < N.n; ++p)
        for (int b = 0; b < 256; ++b)
            if (pb.sym[p].test(b)) set_bit(byte_rows.data() + static_cast<size_t>(b) * N.words, p);
    std::unordered_map<std::string, uint32_t, KeyHash> cid;
    N.classmap.assign(256, 0);
    N.cls.words = N.words;
    for (int b = 0; b < 256; ++b) {
        const uint64_t *r = byte_rows.data() + static_cast<size_t>(b) * N.words;
        auto key = key_of(r, N.words);
        auto it = cid.find(key);
        if (it == cid.end()) {
            uint32_t c = static_cast<uint32_t>(cid.size());
            cid.emplace(key, c);
            N.cls.data.insert(N.cls.data.end(), r, r + N.words);
            N.classmap[b] = static_cast<uint8_t>(c);
        } else {
            N.classmap[b] = static_cast<uint8_t>(it->second);
        }
    }
    N.n_classes = static_cast<uint32_t>(cid.size());
    N.finals.assign(N.words, 0);
    for (uint32_t p : root.last) set_bit(N.finals.data(), p);
    if (root.nullable) set_bit(N.finals.data(), 0);
    return N;
}

// The NFA variant's tables (32-bit words), for automata of at most 128 NFA states.
void keep_nfa(const ClassNfa &N, ridfa::HostNfa &out) {
    out = ridfa::HostNfa{};
    if (N.n > 128) return;
    const uint32_t nw = (N.n + 31) / 32;
    auto words32 = [&](const uint64_t *r, std::vector<uint32_t> &dst) {
        for (uint32_t w = 0; w < nw; ++w) dst.push_back(static_cast<uint32_t>(r[w / 2] >> (32 * (w & 1))));
    };
    out.n = N.n;
    out.nw = nw;
    out.n_classes = N.n_classes;
    out.classmap = N.classmap;
    for (uint32_t q = 0; q < N.n; ++q) words32(N.follow.row(q), out.follow);
    for (uint32_t c = 0; c < N.n_classes; ++c) words32(N.cls.row(c), out.cls);
    words32(N.finals.data(), out.finals);
}

// A subset automaton under construction: subsets, transitions by class (kDeadTmp = none).
constexpr uint32_t kDeadTmp = 0xFFFFFFFFu;

struct SubsetMachine {
    uint32_t words = 0, n_classes = 0;
    Bits sets;
    std::vector<uint32_t> trans;   // [state * n_classes + c]
    std::unordered_map<std::string, uint32_t, KeyHash> index;
    uint32_t size() const { return static_cast<uint32_t>(index.size()); }

    uint32_t intern(const uint64_t *w, uint32_t cap, bool *fresh) {
        auto key = key_of(w, words);
        auto it = index.find(key);
        if (it != index.end()) {
            *fresh = false;
            return it->second;
        }
        uint32_t id = size();
        if (id >= cap) throw TooManyStates("state cap exceeded");
        index.emplace(std::move(key), id);
        sets.data.insert(sets.data.end(), w, w + words);
        trans.resize(static_cast<size_t>(id + 1) * n_classes, kDeadTmp);
        *fresh = true;
        return id;
    }
};

// Expand one state: delta(S, c) = (U_{q in S} follow[q]) n cls[c], undefined when empty.
template <class OnNew>
void expand_state(const ClassNfa &N, SubsetMachine &M, uint32_t s, uint32_t cap, OnNew on_new) {
    std::vector<uint64_t> u(N.words, 0), t(N.words);
    {
        const uint64_t *S = M.sets.row(s);
        for (uint32_t w = 0; w < N.words; ++w) {
            uint64_t bits = S[w];
            while (bits) {
                uint32_t q = w * 64 + static_cast<uint32_t>(__builtin_ctzll(bits));
                bits &= bits - 1;
                const uint64_t *f = N.follow.row(q);
                for (uint32_t v = 0; v < N.words; ++v) u[v] |= f[v];
            }
        }
    }
    for (uint32_t c = 0; c < N.n_classes; ++c) {
        const uint64_t *cr = N.cls.row(c);
        bool any = false;
        for (uint32_t v = 0; v < N.words; ++v) {
            t[v] = u[v] & cr[v];
            any |= t[v] != 0;
        }
        if (!any) continue;
        bool fresh = false;
        uint32_t id = M.intern(t.data(), cap, &fresh);
        M.trans[static_cast<size_t>(s) * N.n_classes + c] = id;
        on_new(id, fresh);
    }
}

// Moore state partition over states 0..n-1 plus a dead state n (Sec. 3.4: language
// equivalence).  Returns block ids; the dead state's block is at index n.
std::vector<uint32_t> state_partition(uint32_t n, uint32_t C, const std::vector<uint32_t> &trans,
                                      const std::vector<uint8_t> &is_final) {
    std::vector<uint32_t> block(n + 1), next(n + 1);
    for (uint32_t p = 0; p < n; ++p) block[p] = is_final[p] ? 1 : 0;
    block[n] = 0;
    uint32_t count = 0;
    {
        bool f = false, nf = true;
        for (uint32_t p = 0; p < n; ++p) f |= is_final[p] != 0;
        count = (f ? 1 : 0) + (nf ? 1 : 0);
    }
    std::vector<uint32_t> sig(C + 1);
    for (;;) {
        std::unordered_map<std::string, uint32_t, KeyHash> ids;
        for (uint32_t p = 0; p <= n; ++p) {
            sig[0] = block[p];
            for (uint32_t c = 0; c < C; ++c) {
                uint32_t t = (p == n) ? n : trans[static_cast<size_t>(p) * C + c];
                sig[c + 1] = block[t == kDeadTmp ? n : t];
            }
            std::string key(reinterpret_cast<const char *>(sig.data()), sizeof(uint32_t) * sig.size());
            auto it = ids.find(key);
            if (it == ids.end()) {
                uint32_t id = static_cast<uint32_t>(ids.size());
                ids.emplace(std::move(key), id);
                next[p] = id;
            } else {
                next[p] = it->second;
            }
        }
        uint32_t nc = static_cast<uint32_t>(ids.size());
        block.swap(next);
        if (nc == count) return block;
        count = nc;
    }
}

void set_final_bits(ridfa::HostAutomaton &A) {
    A.final_bits.assign((A.n_states + 1 + 31) / 32, 0);
    for (uint32_t p = 0; p < A.n_states; ++p)
        if (A.final_flag[p]) A.final_bits[p >> 5] |= 1u << (p & 31);
}

// A planning hint, not part of the method: whether the runs from every slot merge into about one
// on text that follows no structure.  For 16 seeded random class sequences over the live classes
// (those with a defined move from some state), the distinct live states 64 bytes after starting
// in every slot state are counted (0 when all died); merges = 1 when they average at most 1.25.
// Automata whose runs merge are served best by one run per lane after the hand-off; those whose
// runs stay apart (the codon RE's reading frames) by a lane carrying all of its chunk's runs.
void merge_hint(ridfa::HostAutomaton &A) {
    const uint32_t n = A.n_states, C = A.n_classes;
    std::vector<uint32_t> live;
    for (uint32_t c = 0; c < C; ++c)
        for (uint32_t s = 0; s < n; ++s)
            if (A.trans[static_cast<size_t>(s) * C + c] != n) {
                live.push_back(c);
                break;
            }
    A.merges = 1;
    if (live.empty() || A.k == 0) return;
    uint64_t x = 0x9E3779B97F4A7C15ull;        // splitmix64 state, fixed seed
    auto next = [&]() {
        uint64_t z = (x += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    std::vector<uint32_t> st, st2, seen(n + 1, 0);
    uint32_t gen = 0, total = 0;
    const uint32_t trials = 16;
    for (uint32_t t = 0; t < trials; ++t) {
        st.assign(A.slot_state.begin(), A.slot_state.end());
        for (uint32_t i = 0; i < 64 && !st.empty(); ++i) {
            const uint32_t c = live[next() % live.size()];
            ++gen;
            st2.clear();
            for (uint32_t s : st) {
                const uint32_t s2 = A.trans[static_cast<size_t>(s) * C + c];
                if (s2 != n && seen[s2] != gen) {
                    seen[s2] = gen;
                    st2.push_back(s2);
                }
            }
            st.swap(st2);
        }
        total += static_cast<uint32_t>(st.size());
    }
    A.merges = 4 * total <= 5 * trials ? 1u : 0u;
}

// RI-DFA and its interface (Sec. 3.1, 3.2, 3.4).
void build_rid(const ClassNfa &N, uint32_t cap, bool minimize, ridfa_program &P) {
    SubsetMachine M;
    M.words = N.words;
    M.n_classes = N.n_classes;
    M.sets.words = N.words;
    std::vector<uint64_t> single(N.words);
    for (uint32_t q = 0; q < N.n; ++q) {           // I^B: the singletons get ids 0..l-1
        std::fill(single.begin(), single.end(), 0);
        single[q >> 6] |= uint64_t(1) << (q & 63);
        bool fresh;
        M.intern(single.data(), cap, &fresh);
    }
    std::vector<uint8_t> explored(N.n, 0);
    for (uint32_t q = 0; q < N.n; ++q) {           // N(q0), then what N(q1) adds, ...
        if (explored[q]) continue;
        explored[q] = 1;
        std::deque<uint32_t> queue{q};
        while (!queue.empty()) {
            uint32_t s = queue.front();
            queue.pop_front();
            expand_state(N, M, s, cap, [&](uint32_t id, bool) {
                if (id >= explored.size()) explored.resize(id + 1, 0);
                if (!explored[id]) {
                    explored[id] = 1;
                    queue.push_back(id);
                }
            });
        }
    }
    const uint32_t n = M.size();
    ridfa::HostAutomaton &A = P.rid;
    A.n_states = n;
    A.n_classes = N.n_classes;
    A.classmap = N.classmap;
    A.trans.assign(static_cast<size_t>(n + 1) * N.n_classes, static_cast<uint16_t>(n));
    for (size_t i = 0; i < static_cast<size_t>(n) * N.n_classes; ++i)
        if (M.trans[i] != kDeadTmp) A.trans[i] = static_cast<uint16_t>(M.trans[i]);
    A.final_flag.assign(n, 0);
    P.state_sets.assign(n, {});
    for (uint32_t p = 0; p < n; ++p) {
        const uint64_t *S = M.sets.row(p);
        bool fin = false;
        for (uint32_t w = 0; w < N.words; ++w) {
            fin |= (S[w] & N.finals[w]) != 0;
            uint64_t bits = S[w];
            while (bits) {
                P.state_sets[p].push_back(w * 64 + static_cast<uint32_t>(__builtin_ctzll(bits)));
                bits &= bits - 1;
            }
        }
        A.final_flag[p] = fin ? 1 : 0;
    }
    set_final_bits(A);

    // interface minimisation (Sec. 3.4)
    P.n_nfa = N.n;
    P.delegate_slot.assign(N.n, 0);
    P.slots.clear();
    if (minimize) {
        std::vector<uint32_t> block = state_partition(n, N.n_classes, M.trans, A.final_flag);
        std::unordered_map<uint32_t, uint32_t> slot_of_block;
        for (uint32_t q = 0; q < N.n; ++q) {        // lowest NFA state of a class = its rep
            auto it = slot_of_block.find(block[q]);
            if (it == slot_of_block.end()) {
                uint32_t a = static_cast<uint32_t>(P.slots.size());
                slot_of_block.emplace(block[q], a);
                P.slots.push_back(q);
                P.delegate_slot[q] = a;
            } else {
                P.delegate_slot[q] = it->second;
            }
        }
    } else {
        for (uint32_t q = 0; q < N.n; ++q) {
            P.slots.push_back(q);
            P.delegate_slot[q] = q;
        }
    }
    A.k = static_cast<uint32_t>(P.slots.size());
    A.kw = (A.k + 31) / 32;
    A.q0_slot = P.delegate_slot[0];
    A.slot_state.assign(A.k, 0);
    for (uint32_t a = 0; a < A.k; ++a) A.slot_state[a] = static_cast<uint16_t>(P.slots[a]);
    A.ifmask.assign(static_cast<size_t>(n + 1) * A.kw, 0);   // if_min({p}); dead row empty
    for (uint32_t p = 0; p < n; ++p)
        for (uint32_t q : P.state_sets[p]) {
            uint32_t a = P.delegate_slot[q];
            A.ifmask[static_cast<size_t>(p) * A.kw + (a >> 5)] |= 1u << (a & 31);
        }
    merge_hint(A);
}

// Minimal DFA for the all-states comparator (Sec. 2): powerset from {q0}, state partition,
// drop the dead class, breadth-first renumbering.  Every state is a slot; if({p}) = {p}.
bool build_min_dfa(const ClassNfa &N, uint32_t cap, ridfa_program &P) {
    SubsetMachine M;
    M.words = N.words;
    M.n_classes = N.n_classes;
    M.sets.words = N.words;
    std::vector<uint64_t> start(N.words, 0);
    start[0] = 1;
    bool fresh;
    // the powerset machine may be larger than the minimal DFA; allow some headroom
    const uint32_t pcap = std::max<uint32_t>(cap, 1u << 18);
    try {
        M.intern(start.data(), pcap, &fresh);
        std::deque<uint32_t> queue{0};
        while (!queue.empty()) {
            uint32_t s = queue.front();
            queue.pop_front();
            expand_state(N, M, s, pcap, [&](uint32_t id, bool is_new) {
                if (is_new) queue.push_back(id);
            });
        }
    } catch (const TooManyStates &) {
        return false;
    }
    const uint32_t n = M.size();
    std::vector<uint8_t> fin(n, 0);
    for (uint32_t p = 0; p < n; ++p) {
        const uint64_t *S = M.sets.row(p);
        for (uint32_t w = 0; w < N.words; ++w) fin[p] |= (S[w] & N.finals[w]) != 0;
    }
    std::vector<uint32_t> block = state_partition(n, N.n_classes, M.trans, fin);
    const uint32_t nb = *std::max_element(block.begin(), block.end()) + 1;
    const uint32_t dead_block = block[n];
    std::vector<uint32_t> rep(nb, kDeadTmp);
    for (uint32_t p = 0; p < n; ++p)
        if (rep[block[p]] == kDeadTmp) rep[block[p]] = p;
    // live blocks: can reach a final block (the dead block never does)
    std::vector<uint8_t> live(nb, 0);
    for (uint32_t p = 0; p < n; ++p)
        if (fin[p]) live[block[p]] = 1;
    for (bool changed = true; changed;) {
        changed = false;
        for (uint32_t b = 0; b < nb; ++b) {
            if (live[b] || b == dead_block || rep[b] == kDeadTmp) continue;
            for (uint32_t c = 0; c < N.n_classes; ++c) {
                uint32_t t = M.trans[static_cast<size_t>(rep[b]) * N.n_classes + c];
                if (t != kDeadTmp && live[block[t]]) {
                    live[b] = 1;
                    changed = true;
                    break;
                }
            }
        }
    }
    std::vector<uint32_t> order(nb, kDeadTmp);
    std::vector<uint32_t> seq;
    if (live[block[0]]) {
        order[block[0]] = 0;
        seq.push_back(block[0]);
    }
    for (size_t i = 0; i < seq.size(); ++i) {
        uint32_t p = rep[seq[i]];
        for (uint32_t c = 0; c < N.n_classes; ++c) {
            uint32_t t = M.trans[static_cast<size_t>(p) * N.n_classes + c];
            if (t == kDeadTmp || !live[block[t]]) continue;
            if (order[block[t]] == kDeadTmp) {
                if (seq.size() >= cap) return false;
                order[block[t]] = static_cast<uint32_t>(seq.size());
                seq.push_back(block[t]);
            }
        }
    }
    ridfa::HostAutomaton &A = P.dfa;
    const uint32_t q = seq.empty() ? 1 : static_cast<uint32_t>(seq.size());
    A.n_states = q;
    A.n_classes = N.n_classes;
    A.classmap = N.classmap;
    A.trans.assign(static_cast<size_t>(q + 1) * N.n_classes, static_cast<uint16_t>(q));
    A.final_flag.assign(q, 0);
    for (uint32_t i = 0; i < seq.size(); ++i) {
        uint32_t p = rep[seq[i]];
        A.final_flag[i] = fin[p];
        for (uint32_t c = 0; c < N.n_classes; ++c) {
            uint32_t t = M.trans[static_cast<size_t>(p) * N.n_classes + c];
            if (t != kDeadTmp && live[block[t]])
                A.trans[static_cast<size_t>(i) * N.n_classes + c] = static_cast<uint16_t>(order[block[t]]);
        }
    }
    set_final_bits(A);
    A.k = q;
    A.kw = (q + 31) / 32;
    A.q0_slot = 0;
    A.slot_state.resize(q);
    A.ifmask.assign(static_cast<size_t>(q + 1) * A.kw, 0);
    for (uint32_t i = 0; i < q; ++i) {
        A.slot_state[i] = static_cast<uint16_t>(i);
        A.ifmask[static_cast<size_t>(i) * A.kw + (i >> 5)] |= 1u << (i & 31);
    }
    merge_hint(A);
    return true;
}

// Bounds of every table index the device kernels compute without checking: transitions and slot
// states are states or the dead state n (whose row maps to itself), class numbers are below C,
// the q0 slot is a slot, and every table has the size the kernels assume.  A failure is an
// internal error of the construction above (never expected), reported as E_STATE.
bool tables_in_bounds(const ridfa::HostAutomaton &A) {
    const uint32_t n = A.n_states, C = A.n_classes;
    if (C == 0 || C > 256 || n > RIDFA_MAX_STATES || A.k == 0 || A.q0_slot >= A.k) return false;
    if (A.kw != (A.k + 31) / 32 || A.classmap.size() != 256 || A.final_flag.size() != n ||
        A.trans.size() != static_cast<size_t>(n + 1) * C || A.slot_state.size() != A.k ||
        A.ifmask.size() != static_cast<size_t>(n + 1) * A.kw || A.final_bits.size() < (n + 1 + 31) / 32)
        return false;
    for (uint8_t c : A.classmap)
        if (c >= C) return false;
    for (uint16_t t : A.trans)
        if (t > n) return false;
    for (uint32_t c = 0; c < C; ++c)
        if (A.trans[static_cast<size_t>(n) * C + c] != n) return false;
    for (uint16_t s : A.slot_state)
        if (s >= n) return false;
    for (uint32_t w = 0; w < A.kw; ++w)
        if (A.ifmask[static_cast<size_t>(n) * A.kw + w] != 0) return false;
    if (A.k % 32)
        for (uint32_t p = 0; p <= n; ++p)
            if (A.ifmask[static_cast<size_t>(p) * A.kw + A.kw - 1] >> (A.k % 32)) return false;
    return true;
}

}  // namespace

extern "C" int ridfa_compile(const char *re, size_t re_len, const ridfa_compile_opts *opts,
                             ridfa_program **out) {
    if (!out || (!re && re_len)) return RIDFA_E_ARG;
    ridfa::NvtxRange range("ridfa compile");
    ridfa_compile_opts o{1, 1, RIDFA_MAX_STATES};
    if (opts) o = *opts;
    uint32_t cap = (o.max_states == 0 || o.max_states > RIDFA_MAX_STATES) ? RIDFA_MAX_STATES : o.max_states;
    ridfa_program *P = nullptr;
    try {
        P = new ridfa_program();
        P->re.assign(re ? re : "", re_len);
        Parser parser(re ? re : "", re_len);
        int root = parser.parse();
        PositionBuilder pb(parser.nodes);
        Frag f = pb.build(root);
        ClassNfa N = make_class_nfa(pb, f);
        if (N.n > cap) throw TooManyStates("more NFA states than the cap");
        keep_nfa(N, P->nfa);
        build_rid(N, cap, o.minimize_interface != 0, *P);
        P->has_dfa = o.build_dfa ? build_min_dfa(N, cap, *P) : false;
    } catch (const SyntaxError &) {
        delete P;
        return RIDFA_E_SYNTAX;
    } catch (const TooManyStates &) {
        delete P;
        return RIDFA_E_TOO_MANY_STATES;
    } catch (const std::bad_alloc &) {
        delete P;
        return RIDFA_E_NOMEM;
    } catch (...) {
        delete P;
        return RIDFA_E_NOMEM;
    }
    if (!tables_in_bounds(P->rid) || (P->has_dfa && !tables_in_bounds(P->dfa))) {
        delete P;
        return RIDFA_E_STATE;
    }
    *out = P;
    return RIDFA_OK;
}

extern "C" void ridfa_free(ridfa_program *prog) {
    if (!prog) return;
    ridfa::release_device(prog);
    delete prog;
}

extern "C" int ridfa_program_info(const ridfa_program *prog, ridfa_info *out) {
    if (!prog || !out) return RIDFA_E_ARG;
    std::memset(out, 0, sizeof(*out));
    out->n_nfa = prog->n_nfa;
    out->n_states = prog->rid.n_states;
    out->k = prog->rid.k;
    out->n_classes = prog->rid.n_classes;
    out->n_dfa_states = prog->has_dfa ? prog->dfa.n_states : 0;
    out->q0_slot = prog->rid.q0_slot;
    auto bytes = [](const ridfa::HostAutomaton &A) {
        return static_cast<uint64_t>(A.trans.size() * 2 + 256 + A.final_bits.size() * 4 +
                                     A.ifmask.size() * 4 + A.slot_state.size() * 2);
    };
    out->table_bytes = bytes(prog->rid);
    out->dfa_table_bytes = prog->has_dfa ? bytes(prog->dfa) : 0;
    return RIDFA_OK;
}

extern "C" int ridfa_state_set(const ridfa_program *prog, uint32_t state, uint32_t *out,
                               uint32_t cap, uint32_t *n_out) {
    if (!prog || state >= prog->state_sets.size()) return RIDFA_E_ARG;
    const auto &s = prog->state_sets[state];
    if (n_out) *n_out = static_cast<uint32_t>(s.size());
    if (s.size() > cap || (!out && !s.empty())) return RIDFA_E_ARG;
    std::copy(s.begin(), s.end(), out);
    return RIDFA_OK;
}

extern "C" int ridfa_slots(const ridfa_program *prog, uint32_t *out) {
    if (!prog || !out) return RIDFA_E_ARG;
    std::copy(prog->slots.begin(), prog->slots.end(), out);
    return RIDFA_OK;
}

extern "C" int ridfa_delegates(const ridfa_program *prog, uint32_t *out) {
    if (!prog || !out) return RIDFA_E_ARG;
    std::copy(prog->delegate_slot.begin(), prog->delegate_slot.end(), out);
    return RIDFA_OK;
}

extern "C" int ridfa_export_tables(const ridfa_program *prog, int which, uint16_t *trans,
                                   uint8_t *classmap, uint8_t *final_flags) {
    if (!prog || (which != 0 && which != 1)) return RIDFA_E_ARG;
    if (which == 1 && !prog->has_dfa) return RIDFA_E_NO_DFA;
    const ridfa::HostAutomaton &A = which ? prog->dfa : prog->rid;
    if (trans) std::copy(A.trans.begin(), A.trans.end(), trans);
    if (classmap) std::copy(A.classmap.begin(), A.classmap.end(), classmap);
    if (final_flags) std::copy(A.final_flag.begin(), A.final_flag.end(), final_flags);
    return RIDFA_OK;
}

extern "C" const char *ridfa_strerror(int code) {
    switch (code) {
        case RIDFA_OK: return "ok";
        case RIDFA_E_ARG: return "bad argument";
        case RIDFA_E_SYNTAX: return "regular expression syntax error";
        case RIDFA_E_TOO_MANY_STATES: return "automaton exceeds the state limit";
        case RIDFA_E_CHUNKS: return "n_chunks must satisfy 1 <= n_chunks <= len";
        case RIDFA_E_NOMEM: return "out of memory";
        case RIDFA_E_CUDA: return "CUDA runtime error";
        case RIDFA_E_TIMEOUT: return "bounded device wait timed out";
        case RIDFA_E_BUSY: return "admission refused: device-memory budget";
        case RIDFA_E_UNSUPPORTED: return "unsupported size (too many interface slots)";
        case RIDFA_E_NO_DFA: return "program has no DFA comparator";
        case RIDFA_E_STATE: return "device consistency check failed";
        case RIDFA_E_TOO_LARGE:
            return "tables and scratch exceed the fixed no-allocation array (RIDFA_NOALLOC_SCRATCH_BYTES)";
        default: return "unknown status";
    }
}

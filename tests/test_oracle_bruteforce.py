"""Brute-force pins of the oracle: every word up to length 10 / 7 / 6 over 2 / 3 / 4 letters.

For each RE of a corpus (hand-written cases plus seeded random REs, >= 200 in all):
  definitional matcher (operator semantics)          == Thompson state-set simulation (C)
  == position-NFA set simulation (C) == serial RI-DFA run from {q0} == minimal-DFA run,
and the RID join (Sec. 3.2) gives the serial answer for EVERY chunking c = 1..len of the
shorter words (Th. 1 / Lemma 2), with both the minimised and the unminimised interface.
With the unminimised interface, Nst(PLAS_i) = rho(q0, y_1...y_i) (Lemma 1).
The Nerode partition used for delegation equals the partition by acceptance signatures over
all words up to the Moore bound, for RI-DFAs small enough to enumerate.
"""
import itertools

import numpy as np
import pytest

import textgen
from oracle import glushkov, thompson
from oracle.csim import SetSim, ThompsonSim
from oracle.definitional import SpanLanguage, all_words
from oracle.ridfa_sets import (NFA, UNDEF, build_ridfa, chunk_boundaries, min_dfa,
                               nerode_blocks, rid_join)

HAND = [
    "a", "ab", "a|b", "a*", "a+", "a?", "()", "(a|)", "(|a)b", "(a*)*", "(a*b*)*",
    "((a|b)*)*", "a{3}", "a{2,}", "a{0,2}", "(ab){1,3}", "(a|b)*a(a|b){2}", "b*a(ab*a|b+a)*",
    "(a|b)*abb", "(aa|b)*", "(a(b|c))*", "[ab]c*", "(a|b|c)*c(a|b)", "((a|b)(a|c))+",
    "a*b*c*", "(abc|ab|a)*", "(a+b?)+", "(a?b?)*c", "((ab)*|(ba)*)a", "a(b{0,3})a",
    "(a{1,2}b{2,3})*", "(c|ab*c)*b", "((a|b){3})*", "(a|ab)(c|bcd)", "d?(a|b)*(c|d)",
    "[a-c]{2,4}", "[^a]b", "(a|b)*(aa|bb)(a|b)*", "((a*)b(a*))*", "(ab|ba)*|a",
    "((a|b)*c){2}", "(a(a|b)*b|b(a|b)*a)", "(a{2})*(b{3})*", "ab*|ba*|c", "((ab)+)?c",
]


def corpus():
    rng = np.random.Generator(np.random.PCG64(0x5EED))
    out = [(r, None) for r in HAND]
    alphabets = [b"ab", b"abc", b"abcd"]
    while len(out) < 210:
        alpha = alphabets[len(out) % 3]
        node = textgen.random_re(rng, alpha, depth=int(rng.integers(2, 5)), max_lo=2, max_span=2)
        out.append((textgen.render(node), alpha))
    return out


def letters_of(re_src, given):
    if given is not None:
        return given
    used = sorted({ch for ch in re_src.encode() if ch in b"abcd"})
    return bytes(used) if len(used) >= 2 else b"ab"


MAX_LEN = {2: 10, 3: 7, 4: 6}          # all words up to these lengths
MAX_LEN_RID = {2: 8, 3: 5, 4: 4}       # ... and every chunking of the words up to these


def words_upto(alpha, n):
    return [w for k in range(n + 1) for w in all_words(alpha, k)]


@pytest.mark.parametrize("idx", range(0, 210, 10))
def test_bruteforce_corpus(idx):
    for re_src, given in corpus()[idx:idx + 10]:
        alpha = letters_of(re_src, given)
        na = len(alpha)
        spans = SpanLanguage(re_src)
        th = ThompsonSim(thompson.thompson_nfa(re_src))
        n, follow, sym, finals = glushkov.glushkov_tables(re_src)
        ss = SetSim(n, follow, sym)
        nfa = glushkov.glushkov_nfa(re_src)
        Bu = build_ridfa(nfa)                       # unminimised interface
        Bm = build_ridfa(nfa).minimize_interface()  # if_min
        d = min_dfa(nfa)
        for k in range(MAX_LEN[na] + 1):
            W = all_words(alpha, k)
            defin = spans.accepts(W)
            for w, want in zip(W, defin):
                wb = bytes(w)
                assert th.accepts(wb) == want, (re_src, wb)
                assert bool(ss.run({0}, wb) & finals) == want, (re_src, wb)
                p = Bu.run(0, wb)
                assert (p is not UNDEF and p in Bu.finals) == want, (re_src, wb)
                q = d.run(d.start, wb)
                assert (q is not UNDEF and q in d.finals) == want, (re_src, wb)
                if k <= MAX_LEN_RID[na]:
                    _check_all_chunkings(Bu, Bm, nfa, wb, want, re_src)


def _check_all_chunkings(Bu, Bm, nfa, w, want, re_src):
    for c in range(1, max(1, len(w)) + 1):
        if len(w) == 0:
            chunks = [w]
        else:
            b = chunk_boundaries(len(w), c)
            chunks = [w[b[i]:b[i + 1]] for i in range(c)]
        for B in (Bu, Bm):
            maps = [[B.run(B.slots[a], y) for a in range(B.k)] for y in chunks]
            assert rid_join(B, maps) == want, (re_src, w, c)
        # Lemma 1 with the unminimised interface: Nst(PLAS_i) = rho(q0, y_1..y_i)
        maps = [[Bu.run(Bu.slots[a], y) for a in range(Bu.k)] for y in chunks]
        _, hist = rid_join(Bu, maps, return_plas=True)
        prefix = b""
        for i, y in enumerate(chunks):
            prefix += y
            nst = set()
            for p in hist[i]:
                nst |= Bu.states[p]
            assert nst == set(nfa.run({0}, prefix)), (re_src, w, c, i)


def test_random_segmentations_longer_words():
    """Non-equal segmentations of longer random words (Th. 1: any segmentation)."""
    rng = np.random.Generator(np.random.PCG64(7))
    for re_src, given in corpus()[:60]:
        alpha = letters_of(re_src, given)
        nfa = glushkov.glushkov_nfa(re_src)
        Bm = build_ridfa(nfa).minimize_interface()
        th = ThompsonSim(thompson.thompson_nfa(re_src))
        for _ in range(20):
            n = int(rng.integers(10, 40))
            w = bytes(np.frombuffer(alpha, dtype=np.uint8)[rng.integers(0, len(alpha), n)])
            c = int(rng.integers(1, n + 1))
            cuts = sorted(rng.choice(np.arange(1, n), size=c - 1, replace=False).tolist()) if c > 1 else []
            bounds = [0] + cuts + [n]
            chunks = [w[bounds[i]:bounds[i + 1]] for i in range(c)]
            maps = [[Bm.run(Bm.slots[a], y) for a in range(Bm.k)] for y in chunks]
            assert rid_join(Bm, maps) == th.accepts(w), (re_src, w, bounds)


def _signature(B, p, words):
    return tuple((q := B.run(p, w)) is not UNDEF and q in B.finals for w in words)


def test_nerode_partition_matches_signatures():
    """Two RI-DFA states are language-equivalent iff no word of length <= |P| tells them apart
    (Moore's bound for |P| + 1 states with the implicit dead state)."""
    checked = 0
    for re_src, given in corpus():
        alpha = letters_of(re_src, given)
        B = build_ridfa(glushkov.glushkov_nfa(re_src))
        npst = len(B.states)
        if len(alpha) ** min(npst, 12) > 3000 or npst > 12:
            continue
        words = [bytes(w) for w in words_upto(alpha, npst)]
        sig = [_signature(B, p, words) for p in range(npst)]
        blocks = nerode_blocks(B)
        for p in range(npst):
            for q in range(npst):
                assert (blocks[p] == blocks[q]) == (sig[p] == sig[q]), (re_src, p, q)
        checked += 1
    assert checked >= 40


def test_min_dfa_is_minimal_and_canonical():
    """All states reachable, pairwise distinguishable (by words up to |Q|), and numbered in
    breadth-first order from the start with symbols ascending."""
    checked = 0
    for re_src, given in corpus():
        alpha = letters_of(re_src, given)
        d = min_dfa(glushkov.glushkov_nfa(re_src))
        nq = len(d.states)
        if nq > 8 or len(alpha) ** nq > 5000:
            continue
        words = [bytes(w) for w in words_upto(alpha, nq)]
        sigs = {tuple((r := d.run(q, w)) is not UNDEF and r in d.finals for w in words)
                for q in range(nq)}
        assert len(sigs) == nq, re_src
        seen, order = {0}, [0]
        for q in order:
            for b in sorted(d.delta[q]):
                t = d.delta[q][b]
                if t not in seen:
                    seen.add(t)
                    order.append(t)
        assert order == list(range(nq)), re_src
        checked += 1
    assert checked >= 40


def test_fig5_nfa_bruteforce():
    """The hand-drawn NFAs of Fig. 1 and Fig. 5: RID = NFA for every word <= 7 and chunking."""
    for edges, n in [([(0, "ac", 1), (1, "a", 1), (1, "b", 2), (2, "b", 1), (1, "abc", 0)], 3),
                     ([(0, "a", 1), (0, "c", 3), (1, "abc", 0), (1, "b", 2), (1, "a", 3),
                       (2, "b", 1), (3, "abc", 0), (3, "a", 1), (3, "b", 2)], 4)]:
        nfa = NFA.from_edges(n, edges, [2], "abc")
        Bu = build_ridfa(nfa)
        Bm = build_ridfa(nfa).minimize_interface()
        for k in range(8):
            for w in all_words(b"abc", k):
                wb = bytes(w)
                want = nfa.accepts(wb)
                if k <= 5:
                    _check_all_chunkings(Bu, Bm, nfa, wb, want, "fig")
                p = Bu.run(0, wb)
                assert (p is not UNDEF and p in Bu.finals) == want

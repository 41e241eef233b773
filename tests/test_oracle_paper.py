"""Pins of the oracle against the paper's worked examples (tests/golden/*.json, each cited).

These run on CPU only and exercise nothing but ``oracle/``.
"""
import json
import os

import pytest

from oracle.definitional import DefinitionalMatcher
from oracle.ridfa_sets import (DFA, NFA, UNDEF, build_ridfa, csdpa_dfa_join,
                               csdpa_dfa_maps, csdpa_dfa_transition_count, min_dfa,
                               nerode_blocks, rid_join, transition_count)

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def nfa_from(g):
    return NFA.from_edges(g["n"], [(a, s, b) for a, s, b in g["edges"]], g["finals"],
                          g["alphabet"], q0=g["q0"])


def dfa_from(g):
    delta = [dict() for _ in range(g["n"])]
    for a, syms, b in g["edges"]:
        for s in syms:
            delta[a][ord(s)] = b
    return DFA(list(range(g["n"])), [ord(s) for s in g["alphabet"]], delta, g["start"], g["finals"])


def fs(x):
    return frozenset(x)


# ---------------------------------------------------------------- Fig. 1 / Fig. 3 / Fig. 4

def test_fig1_ridfa_states_transitions_finals():
    g = load("fig1_ridfa.json")
    B = build_ridfa(nfa_from(g["nfa"]))
    assert set(B.states) == {fs(s) for s in g["ridfa_states"]}
    got = {(B.states[p], chr(b), B.states[t]) for p in range(len(B.states))
           for b, t in B.delta[p].items()}
    want = {(fs(a), s, fs(b)) for a, s, b in g["ridfa_delta"]}
    assert got == want
    assert {B.states[p] for p in B.finals} == {fs(s) for s in g["ridfa_finals"]}
    # I^B = singletons = Q_N (Sec. 3.1)
    assert [B.states[p] for p in B.initial] == [fs([q]) for q in range(3)]


def test_fig3_incremental_construction():
    """N(0) and N(1) have the states {0},{1},{0,1},{0,2}; N(2) adds {2} and {2} -b-> {1}."""
    g = load("fig1_ridfa.json")
    nfa = nfa_from(g["nfa"])
    # N(q) alone: powerset machine from {q}
    for q in (0, 1):
        d = NFA(nfa.n, nfa.alphabet, nfa.delta, q, nfa.finals)
        from oracle.ridfa_sets import powerset_dfa
        assert set(powerset_dfa(d).states) == {fs(s) for s in g["n0_states"]}
    B = build_ridfa(nfa)
    extra = set(B.states) - {fs(s) for s in g["n0_states"]}
    assert extra == {fs(g["n2_adds"]["state"])}
    src, sym, dst = g["n2_adds"]["edge"]
    p = B.index[fs(src)]
    assert B.states[B.delta[p][ord(sym)]] == fs(dst)
    assert set(B.delta[p]) == {ord(sym)}


def test_fig4_join_aab_cab():
    g = load("fig1_ridfa.json")
    B = build_ridfa(nfa_from(g["nfa"]))        # Fig. 4 uses the unminimised interface
    y1, y2 = [c.encode() for c in g["chunks"]]
    lam1 = [B.run(B.slots[a], y1) for a in range(B.k)]
    lam2 = [B.run(B.slots[a], y2) for a in range(B.k)]
    assert B.states[lam1[0]] == fs(g["lambda_1_q0"])
    for a, want in g["lambda_2"].items():
        got = lam2[int(a)]
        assert (got is UNDEF) if want is None else (B.states[got] == fs(want))
    plas1 = {lam1[0]}
    assert B.interface(plas1) == set(g["if_plas_1"])
    pis2 = {a for a in range(B.k) if lam2[a] is not UNDEF}
    assert pis2 == set(g["pis_2"])
    accept, hist = rid_join(B, [lam1, lam2], return_plas=True)
    assert {B.states[p] for p in hist[1]} == {fs(s) for s in g["plas_2"]}
    assert accept is g["accept"]
    assert transition_count(B, [y1, y2]) == g["transitions_rid"]


def test_fig1_min_dfa_and_dfa_transition_count():
    g = load("fig1_ridfa.json")
    nfa = nfa_from(g["nfa"])
    d = min_dfa(nfa)
    assert len(d.states) == g["min_dfa_states"]
    # isomorphism with the printed DFA, via canonical BFS numbering of the printed one
    names = {}
    want_delta = {}
    for a, s, b in g["min_dfa_edges"]:
        want_delta.setdefault(a, {})[ord(s)] = b
    order = [g["min_dfa_start"]]
    names[g["min_dfa_start"]] = 0
    i = 0
    while i < len(order):
        for b in sorted(want_delta.get(order[i], {})):
            t = want_delta[order[i]][b]
            if t not in names:
                names[t] = len(order)
                order.append(t)
        i += 1
    for a, row in want_delta.items():
        for b, t in row.items():
            assert d.delta[names[a]][b] == names[t]
    assert d.finals == {names[f] for f in g["min_dfa_finals"]}
    y = [c.encode() for c in g["chunks"]]
    assert csdpa_dfa_transition_count(d, y) == g["transitions_dfa"]
    assert csdpa_dfa_join(d, csdpa_dfa_maps(d, y)) is True


# ---------------------------------------------------------------- Fig. 2

def test_fig2_csdpa_dfa():
    g = load("fig2_csdpa.json")
    d = dfa_from(g["dfa"])
    y = [c.encode() for c in g["chunks"]]
    maps = csdpa_dfa_maps(d, y)
    assert maps[0] == g["lambda_1"]
    assert maps[1] == g["lambda_2"]
    assert csdpa_dfa_join(d, maps) is g["accept"]
    assert csdpa_dfa_transition_count(d, y) == g["transitions"]


def test_fig2_re_language_matches_dfa():
    """L = b*a(ab*a|b+a)* is the language of the Fig. 2 DFA (all words up to length 10)."""
    g = load("fig2_csdpa.json")
    d = dfa_from(g["dfa"])
    m = DefinitionalMatcher(g["re"])
    import itertools
    for n in range(11):
        for w in itertools.product(b"ab", repeat=n):
            w = bytes(w)
            q = d.run(d.start, w)
            assert m.match(w) == (q is not UNDEF and q in d.finals), w


# ---------------------------------------------------------------- Fig. 5

def test_fig5_states_classes_delegation():
    g = load("fig5_minimize.json")
    B = build_ridfa(nfa_from(g["nfa"]))
    names = {k: fs(v) for k, v in g["paper_names"].items()}
    assert set(B.states) == set(names.values())
    blocks = nerode_blocks(B)
    by_block = {}
    for p, blk in enumerate(blocks):
        by_block.setdefault(blk, set()).add(B.states[p])
    nontrivial = [s for s in by_block.values() if len(s) > 1]
    want = [{names[x] for x in cls} for cls in g["nontrivial_classes"]]
    assert sorted(map(sorted, map(lambda s: [tuple(sorted(x)) for x in s], nontrivial))) == \
        sorted(map(sorted, map(lambda s: [tuple(sorted(x)) for x in s], want)))
    B.minimize_interface()
    assert B.k == g["k_min"]
    for q, r in g["delegations"].items():
        assert B.slots[B.delegate[int(q)]] == r
    # q0 keeps its own slot (lowest representative)
    assert B.slots[B.delegate[0]] == 0


def test_fig5_join_and_counts():
    g = load("fig5_minimize.json")
    names = {k: fs(v) for k, v in g["paper_names"].items()}
    y = [c.encode() for c in g["chunks"]]
    B = build_ridfa(nfa_from(g["nfa"]))
    unmin = transition_count(B, y)
    B.minimize_interface()
    lam1 = [B.run(B.slots[a], y[0]) for a in range(B.k)]
    lam2 = [B.run(B.slots[a], y[1]) for a in range(B.k)]
    plas1 = {lam1[B.delegate[0]]}
    assert {B.states[p] for p in plas1} == {names[x] for x in g["plas_1"]}
    assert {B.slots[a] for a in B.interface(plas1)} == {s[0] for s in g["if_min_plas_1"]}
    for src, dst in g["lambda_2_min"].items():
        a = B.delegate[next(iter(names[src]))]
        assert (lam2[a] is UNDEF) if dst is None else B.states[lam2[a]] == names[dst]
    assert rid_join(B, [lam1, lam2]) is g["accept"]
    assert unmin == g["transitions_unminimized"]
    assert transition_count(B, y) == g["transitions_minimized"]


def test_fig5_reading_A8_typo():
    """{0,1} -a-> {0,1,3} by construction, so the printed p7 -a-> p4 is read as p7 -a-> p5."""
    g = load("fig5_minimize.json")
    names = {k: fs(v) for k, v in g["paper_names"].items()}
    B = build_ridfa(nfa_from(g["nfa"]))
    p7 = B.index[names["p7"]]
    assert B.states[B.delta[p7][ord('a')]] == names["p5"]


# ---------------------------------------------------------------- config 1 closed form

def test_config1_closed_form():
    from oracle.recognizer import RidOracle
    g = load("config1_closed_form.json")
    o = RidOracle(g["re"])
    assert o.nfa.n == g["n_nfa"]
    assert len(o.B.states) == g["ridfa_states"]
    assert o.B.slots == g["slots"]
    blocks = nerode_blocks(o.B)
    cls = {}
    for q in range(o.nfa.n):
        cls.setdefault(blocks[q], []).append(q)
    assert sorted(cls.values()) == sorted(g["nerode_classes_of_singletons"])
    d = o.dfa
    w = dfa_from({"n": g["min_dfa"]["n"], "alphabet": "ACGT", "start": 0,
                  "finals": g["min_dfa"]["finals"], "edges": g["min_dfa"]["edges"]})
    assert len(d.states) == g["min_dfa"]["n"]
    for q in range(len(d.states)):
        assert d.delta[q] == w.delta[q]
    assert d.finals == set(g["min_dfa"]["finals"])

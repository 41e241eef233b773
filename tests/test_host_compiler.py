"""The library's host side (no GPU needed): C ABI exports, and the compiled RI-DFA, interface
and minimal DFA against the oracle's independent construction, id for id."""
import os
import re

import numpy as np
import pytest

import textgen
from oracle.recognizer import RidOracle
from oracle.re_syntax import ReSyntaxError, parse

lib = pytest.importorskip("paper_2412_14975_gb300")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "ridfa.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ridfa_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_symbol():
    import ctypes
    names = header_functions()
    assert len(names) >= 29, names
    so = ctypes.CDLL(lib.lib_path())
    for n in names:
        assert hasattr(so, n), n


def corpus():
    from tests.test_oracle_bruteforce import corpus as bf
    res = [r for r, _ in bf()]
    res += [textgen.C1_RE, textgen.C3_RE, textgen.C3_RE_ANYFIELD,
            textgen.C2_RE.replace("{20,60}", "{2,4}"), textgen.regexp_family_re(3),
            textgen.regexp_family_re(8), "[\\x00-\\xff]*\\n", "\\x41\\.[^a-z]{2}", "(.|\\n)*x"]
    return res


def compare(re_src, minimize=True):
    o = RidOracle(re_src, minimize=minimize)
    p = lib.ridfa_compile(re_src, minimize_interface=minimize)
    info = p.info
    B = o.B
    assert info["n_nfa"] == o.nfa.n
    assert info["n_states"] == len(B.states)
    assert info["k"] == B.k
    assert info["q0_slot"] == B.delegate[0]
    for s in range(len(B.states)):
        assert frozenset(lib.ridfa_state_set(p, s).tolist()) == B.states[s], (re_src, s)
    assert lib.ridfa_slots(p).tolist() == B.slots
    assert lib.ridfa_delegates(p).tolist() == B.delegate
    trans, cmap, fin = lib.ridfa_export_tables(p, 0)
    n = len(B.states)
    for s in range(n):
        for b in range(256):
            want = B.delta[s].get(b)
            got = int(trans[s, cmap[b]])
            assert got == (n if want is None else want), (re_src, s, b)
        assert bool(fin[s]) == (s in B.finals)
    assert np.all(trans[n] == n)
    d = o.dfa
    assert info["n_dfa_states"] == len(d.states)
    dt, dc, dfin = lib.ridfa_export_tables(p, 1)
    nq = len(d.states)
    for q in range(nq):
        for b in range(256):
            want = d.delta[q].get(b)
            assert int(dt[q, dc[b]]) == (nq if want is None else want), (re_src, q, b)
        assert bool(dfin[q]) == (q in d.finals)
    # byte classes: bytes share a class iff they are read by the same positions; numbered by
    # their smallest byte
    seen = []
    for b in range(256):
        if cmap[b] not in seen:
            assert cmap[b] == len(seen)
            seen.append(cmap[b])
    p.close()


def test_compiler_matches_oracle_on_corpus():
    for r in corpus():
        compare(r, minimize=True)


def test_compiler_matches_oracle_unminimized():
    for r in corpus()[::5]:
        compare(r, minimize=False)


def test_workload_sizes():
    """Sizes of the single-text workloads (the C2 reading uses the {2,4} codon repeat)."""
    sizes = {}
    for name, r in [("c1", textgen.C1_RE), ("c3", textgen.C3_RE),
                    ("c3_any", textgen.C3_RE_ANYFIELD),
                    ("c2_2_4", textgen.C2_RE.replace("{20,60}", "{2,4}"))]:
        sizes[name] = lib.ridfa_compile(r).info
    assert (sizes["c1"]["n_nfa"], sizes["c1"]["n_states"], sizes["c1"]["k"],
            sizes["c1"]["n_dfa_states"]) == (7, 7, 4, 4)
    assert (sizes["c3"]["n_nfa"], sizes["c3"]["k"], sizes["c3"]["n_dfa_states"]) == (69, 68, 68)
    assert sizes["c2_2_4"]["n_states"] == 424 and sizes["c2_2_4"]["n_dfa_states"] == 1


def test_c2_as_written_exceeds_state_limit():
    """The {20,60} codon repeat makes the RI-DFA grow past 65,534 states."""
    with pytest.raises(lib.RidfaError) as e:
        lib.ridfa_compile(textgen.C2_RE)
    assert e.value.code == -3


def test_syntax_errors_agree_with_oracle_parser():
    bad = ["(", ")", "a)", "[", "[]", "*a", "a{2,1}", "a{", "a{x}", "\\", "a|*", "[b-a]",
           "a{1,2", "(a|b", "+", "?"]
    good = ["", "()", "a|", "|", "[]]", "[a-]", "a{0}", "a{0,0}", "\\*", "[\\]]", "a{2,}"]
    for r in bad:
        with pytest.raises(ReSyntaxError):
            parse(r)
        with pytest.raises(lib.RidfaError) as e:
            lib.ridfa_compile(r)
        assert e.value.code == -2, r
    for r in good:
        parse(r)
        compare(r)


def test_state_cap_and_arguments():
    with pytest.raises(lib.RidfaError) as e:
        lib.ridfa_compile(textgen.regexp_family_re(8), max_states=100)
    assert e.value.code == -3
    p = lib.ridfa_compile("ab*")
    with pytest.raises(lib.RidfaError):
        lib.ridfa_state_set(p, 10_000)

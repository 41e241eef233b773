"""The library's host transition counters (ridfa_count_transitions) against the oracle.

w_paper is pinned to the oracle's transition_count / csdpa_dfa_transition_count, which the
paper's worked examples pin (Fig. 1: 9 RID and 15 DFA transitions; Fig. 5: 12 and 9); w_conv is
checked against its definition -- distinct live states summed over positions -- evaluated here
with the oracle's RI-DFA and minimal DFA, and both against closed forms on small cases."""
import numpy as np
import pytest

import textgen
from oracle.recognizer import RidOracle
from oracle.ridfa_sets import (UNDEF, chunk_boundaries, csdpa_dfa_transition_count,
                               transition_count)

lib = pytest.importorskip("paper_2412_14975_gb300")


def w_conv_rid(B, chunks):
    total = 0
    for i, y in enumerate(chunks):
        live = {B.slots[B.delegate[B.nfa.q0]]} if i == 0 else set(B.slots[a] for a in range(B.k))
        for b in y:
            total += len(live)
            live = {p for p in (B.step(s, b) for s in live) if p is not UNDEF}
            if not live:
                break
    return total


def w_conv_dfa(d, chunks):
    total = 0
    for i, y in enumerate(chunks):
        live = {d.start} if i == 0 else set(range(len(d.states)))
        for b in y:
            total += len(live)
            live = {p for p in (d.step(s, b) for s in live) if p is not UNDEF}
            if not live:
                break
    return total


def chunks_of(x, c):
    b = chunk_boundaries(len(x), c)
    return [bytes(x[b[i]:b[i + 1]]) for i in range(c)]


def compare(re_src, x, c, n_threads=0):
    o = RidOracle(re_src)
    p = lib.ridfa_compile(re_src)
    ch = chunks_of(x, c)
    got = lib.ridfa_count_transitions(p, x, c, n_threads=n_threads)
    assert got["w_paper"] == transition_count(o.B, ch), (re_src, c)
    assert got["w_conv"] == w_conv_rid(o.B, ch), (re_src, c)
    assert got["runs"] == 1 + (c - 1) * o.B.k
    dg = lib.ridfa_count_transitions(p, x, c, dfa=True, n_threads=n_threads)
    assert dg["w_paper"] == csdpa_dfa_transition_count(o.dfa, ch), (re_src, c)
    assert dg["w_conv"] == w_conv_dfa(o.dfa, ch), (re_src, c)
    assert dg["runs"] == 1 + (c - 1) * len(o.dfa.states)
    return got, dg


def test_closed_forms_single_chunk_and_dead_runs():
    # one chunk: one run from {q0}; (ab)* over "abab" makes 4 transitions and 4 lookups
    got, dg = compare("(ab)*", b"abab", 1)
    assert got["w_paper"] == got["w_conv"] == 4 and got["dead_runs"] == 0
    # a byte outside the alphabet kills every run: no transitions, one lookup per live state
    p = lib.ridfa_compile("(ab)*")
    r = lib.ridfa_count_transitions(p, b"zab", 1)
    assert r == {"w_paper": 0, "w_conv": 1, "runs": 1, "dead_runs": 1, "converge_hist": [0] * 16}
    # c = len: every chunk one byte; chunk 1 from {q0}, the others from each of the k slots
    k = p.info["k"]
    r = lib.ridfa_count_transitions(p, b"abab", 4)
    assert r["runs"] == 1 + 3 * k


@pytest.mark.parametrize("re_name", ["c1", "c3", "c2_2_4", "regexp3"])
def test_workload_res_against_oracle(re_name):
    rng = np.random.Generator(np.random.PCG64(sum(map(ord, re_name))))
    re_src = {"c1": textgen.C1_RE, "c3": textgen.C3_RE, "c2_2_4": textgen.C2_RE.replace("{20,60}", "{2,4}"),
              "regexp3": textgen.regexp_family_re(3)}[re_name]
    n = 3000
    if re_name == "c1":
        x = textgen.c1_text(n, rng)[:n]
    elif re_name == "c3":
        x = textgen.c3_text(n, rng)[:n]
    elif re_name == "c2_2_4":
        x = textgen.c2_text(n, rng)
    else:
        x = textgen.regexp_family_text(n, rng)
    for c in (1, 7, 64):
        compare(re_src, x, c, n_threads=3)


def test_random_res_and_thread_split_invariance():
    rng = np.random.Generator(np.random.PCG64(0xC0))
    done = 0
    while done < 12:
        node = textgen.random_re(rng, b"abc", depth=int(rng.integers(2, 5)))
        re_src = "(" + textgen.render(node) + ")*"
        try:
            p = lib.ridfa_compile(re_src)
        except lib.RidfaError:
            continue
        if p.info["n_states"] > 400:
            continue
        parts = [textgen.sample_member(node, rng, soft_len=12) for _ in range(40)]
        x = np.frombuffer(b"".join(parts) or b"a", dtype=np.uint8)
        if done % 2:
            x, _ = textgen.mutate(x, rng, n_subs=1, alphabet=b"abc")
        c = int(rng.integers(1, min(x.size, 40) + 1))
        compare(re_src, x, c, n_threads=1)
        # any split of the chunks over threads gives the same counts
        a = lib.ridfa_count_transitions(p, x, c, n_threads=1)
        for t in (2, 5, 64):
            assert lib.ridfa_count_transitions(p, x, c, n_threads=t) == a
        done += 1


def test_counter_errors():
    p = lib.ridfa_compile("(ab)*", build_dfa=False)
    with pytest.raises(lib.RidfaError) as e:
        lib.ridfa_count_transitions(p, b"ab", 3)
    assert e.value.code == -4
    with pytest.raises(lib.RidfaError) as e:
        lib.ridfa_count_transitions(p, b"ab", 1, dfa=True)
    assert e.value.code == -10


def nfa_variant_counts(nfa, chunks):
    """The NFA variant's work (Sec. 2) written out: chunk 1 from q0, the others from every NFA
    state, each start's set followed on its own; a step from S executes sum |rho(q, b)| transitions
    and processes |S| states."""
    wp = wc = runs = dead = 0
    for i, y in enumerate(chunks):
        for q in ([nfa.q0] if i == 0 else range(nfa.n)):
            S = {q}
            runs += 1
            for b in y:
                T = set()
                for s in S:
                    wc += 1
                    t = nfa.rho(s, b)
                    wp += len(t)
                    T |= t
                S = T
                if not S:
                    dead += 1
                    break
    return dict(w_paper=wp, w_conv=wc, runs=runs, dead_runs=dead)


@pytest.mark.parametrize("re_name", ["c1", "c3", "regexp3", "codon"])
def test_nfa_variant_counts_match_definition(re_name):
    re_src = {"c1": textgen.C1_RE, "c3": textgen.C3_RE, "regexp3": textgen.regexp_family_re(3),
              "codon": textgen.C2_RE.replace("{20,60}", "{2,4}")}[re_name]
    x = {"c1": lambda: textgen.c1_text(2500, seed=11), "c3": lambda: textgen.c3_text(2500, seed=12),
         "regexp3": lambda: textgen.regexp_family_text(2500, seed=13),
         "codon": lambda: textgen.c2_text(2500, seed=14)}[re_name]()
    y, _ = textgen.mutate(x, seed=15, n_subs=2)
    prog = lib.ridfa_compile(re_src, build_dfa=False)
    nfa = RidOracle(re_src, with_dfa=False).nfa
    for t in (x, y):
        for c in (1, 3, 40):
            b = chunk_boundaries(t.size, c)
            chunks = [bytes(t[b[i]:b[i + 1]]) for i in range(c)]
            got = lib.ridfa_count_transitions(prog, t, c, nfa=True)
            assert got.pop("converge_hist") == [0] * 16
            assert got == nfa_variant_counts(nfa, chunks)


def test_nfa_variant_counts_refuse_large_nfa():
    prog = lib.ridfa_compile(textgen.C3_RE_ANYFIELD, build_dfa=False)   # 129 NFA states
    assert prog.info["n_nfa"] > 128
    with pytest.raises(lib.RidfaError) as e:
        lib.ridfa_count_transitions(prog, textgen.c3_text(1000, seed=16), 4, nfa=True)
    assert e.value.code == -9          # E_UNSUPPORTED


def converge_hist_by_definition(B, chunks):
    """Histogram of the bytes each chunk (after the first) reads until at most one live state of
    its runs from every interface slot remains, with the oracle's RI-DFA; bucket 15: never."""
    hist = [0] * 16
    for y in chunks[1:]:
        live = set(B.slots[a] for a in range(B.k))
        at = None
        for t in range(len(y) + 1):
            if len(live) <= 1:
                at = t
                break
            if t < len(y):
                live = {p for p in (B.step(s, y[t]) for s in live) if p is not UNDEF}
        if at is None:
            hist[15] += 1
        else:
            b = 0
            while b < 14 and (at >> (b + 1)):
                b += 1
            hist[b] += 1
    return hist


@pytest.mark.parametrize("k", [3, 5, 7])
def test_convergence_histogram_definite_automaton(k):
    """(a|b)*a(a|b){k} is k+1-definite: from every slot, runs over any k+1 letters end in one state
    and not before, so every chunk converges after exactly k + 1 bytes (bucket floor(log2(k+1)));
    the histogram also equals its definition evaluated with the oracle's RI-DFA."""
    re_src = textgen.regexp_family_re(k)
    x = textgen.regexp_family_text(200_000, seed=40 + k)
    prog = lib.ridfa_compile(re_src)
    B = RidOracle(re_src).B
    for c in (2, 64, 999):
        h = lib.ridfa_count_transitions(prog, x, c)["converge_hist"]
        want_bucket = (k + 1).bit_length() - 1
        assert h[want_bucket] == c - 1 and sum(h) == c - 1, (k, c, h)
        b = chunk_boundaries(x.size, c)
        chunks = [bytes(x[b[i]:b[i + 1]]) for i in range(c)]
        assert h == converge_hist_by_definition(B, chunks), (k, c)


def test_convergence_histogram_reading_frames_and_record_lines():
    """The codon RE's runs sit in three reading frames and never meet (every chunk in bucket 15),
    the record lines' runs meet within 16 bytes; both equal the definition with the oracle."""
    re2 = textgen.C2_RE.replace("{20,60}", "{2,4}")
    x = textgen.c2_text(60_000, seed=50)
    h = lib.ridfa_count_transitions(lib.ridfa_compile(re2), x, 100)["converge_hist"]
    assert h[15] == 99, h
    b = chunk_boundaries(x.size, 100)
    assert h == converge_hist_by_definition(RidOracle(re2).B, [bytes(x[b[i]:b[i + 1]]) for i in range(100)])
    y = textgen.c3_text(200_000, seed=51)
    h = lib.ridfa_count_transitions(lib.ridfa_compile(textgen.C3_RE), y, 300)["converge_hist"]
    assert sum(h[:4]) == 299 and h[15] == 0, h
    b = chunk_boundaries(y.size, 300)
    assert h == converge_hist_by_definition(RidOracle(textgen.C3_RE).B,
                                            [bytes(y[b[i]:b[i + 1]]) for i in range(300)])
    # the NFA variant reports no histogram
    p1 = lib.ridfa_compile(textgen.C1_RE)
    z = textgen.c1_text(5000, seed=52)
    assert lib.ridfa_count_transitions(p1, z, 10, nfa=True)["converge_hist"] == [0] * 16

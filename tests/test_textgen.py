"""The input generators against the oracle (labels always come from the oracle)."""
import itertools

import numpy as np

import textgen
from oracle.definitional import all_words
from oracle.recognizer import RidOracle, SerialRecognizer


def test_c1_hand_dfa_is_the_language():
    """The hand-written minimal DFA of config 1 accepts exactly L(RE) (words <= 8 over ACGT)."""
    t, acc, s0 = textgen.c1_min_dfa_table()
    ser = SerialRecognizer(textgen.C1_RE)
    for n in range(9):
        for w in all_words(b"ACGT", n):
            s = s0
            for b in w:
                s = t[s, b] if s >= 0 else -1
            assert (s >= 0 and bool(acc[s])) == ser.accepts(bytes(w))


def test_c1_walk_is_accepted_and_mutant_labelled_by_oracle():
    x = textgen.c1_text(1 << 14, seed=11)
    assert x.size >= 1 << 14 and x.size <= (1 << 14) + 4
    assert SerialRecognizer(textgen.C1_RE).accepts(x)
    m, pos = textgen.mutate(x, seed=12, n_subs=1, alphabet=b"ACGT")
    assert int(np.sum(m != x)) == 1 and m[pos[0]] != x[pos[0]]


def test_c3_records_are_accepted():
    x = textgen.c3_text(1 << 16, seed=5)
    assert x.size >= 1 << 16 and x[-1] == 10
    ser = SerialRecognizer(textgen.C3_RE)
    assert ser.accepts(x)
    assert SerialRecognizer(textgen.C3_RE_ANYFIELD).accepts(x)
    y = x.copy()
    y[100] = ord('#')
    assert not ser.accepts(y)


def test_c2_language_is_all_acgt():
    """A13: (([ACGT]{3})*ATG([ACGT]{3}){20,60}(TAA|TAG|TGA))*[ACGT]* = {A,C,G,T}*."""
    ser = SerialRecognizer(textgen.C2_RE)
    rng = np.random.Generator(np.random.PCG64(3))
    for n in (0, 1, 5, 100, 1000):
        assert ser.accepts(textgen.c2_text(n, rng))
    assert not ser.accepts(b"ACGTN")


def test_walk_generic_matches_language():
    """dfa_walk on the oracle's minimal DFA of a random RE always yields a member."""
    rng = np.random.Generator(np.random.PCG64(9))
    done = 0
    while done < 10:
        node = textgen.random_re(rng, b"abcd", depth=4)
        re_src = "(" + textgen.render(node) + ")*"
        o = RidOracle(re_src)
        d = o.dfa
        t = np.full((len(d.states), 256), -1, dtype=np.int32)
        for q, row in enumerate(d.delta):
            for b, r in row.items():
                t[q, b] = r
        acc = np.array([q in d.finals for q in range(len(d.states))])
        x = textgen.dfa_walk(t, acc, 0, 300, seed=done)
        assert SerialRecognizer(re_src).accepts(x)
        done += 1


def test_rendered_random_re_members():
    rng = np.random.Generator(np.random.PCG64(4))
    for _ in range(30):
        node = textgen.random_re(rng, b"abc", depth=4)
        ser = SerialRecognizer(textgen.render(node))
        for _ in range(5):
            assert ser.accepts(textgen.sample_member(node, rng))

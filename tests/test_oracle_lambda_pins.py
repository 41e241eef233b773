"""Pins of the oracle's chunk-map functions, the ones every GPU map comparison goes through.

``RidOracle.lambda_row`` computes lambda_i(a) as the position-NFA set simulation rho({q_a}, y_i)
looked up among the RI-DFA's subsets (Sec. 3.1 construction: delta^B({q}, y) = rho(q, y)), and
``RidOracle.dfa_lambda_row`` computes the comparator's map as rho(S_q, y_i) for a representative
subset S_q of minimal-DFA state q, mapped back to its class (Sec. 2, Fig. 2).  Here both are
checked against a different computation of the same definition: stepping the automaton's own
transition table one byte at a time (``chunk_mapping`` / ``B.run`` for the RI-DFA, whose runs are
pinned by brute force against the Thompson simulation, and ``csdpa_dfa_maps`` / ``DFA.run`` for
the minimal DFA, pinned minimal and canonical by brute force).  A wrong representative subset, a
live subset missing from the subset-to-state map, or a wrong slot-to-state map fails here.

Texts are random over the RE's letters plus bytes no position reads (out-of-alphabet bytes kill
every run), cut into several chunk counts including ragged ones.
"""
import numpy as np
import pytest

import textgen
from oracle.recognizer import LAMBDA_UNDEF, RidOracle
from oracle.ridfa_sets import UNDEF, chunk_boundaries, chunk_mapping, csdpa_dfa_maps

from .test_oracle_bruteforce import corpus, letters_of


def _wire(v):
    return LAMBDA_UNDEF if v is UNDEF else int(v)


def _texts(rng, alpha, n_texts, lo, hi, foreign=b"\x00\x7f\xff"):
    a = np.frombuffer(alpha, dtype=np.uint8)
    f = np.frombuffer(foreign, dtype=np.uint8)
    for t in range(n_texts):
        n = int(rng.integers(lo, hi + 1))
        x = a[rng.integers(0, a.size, size=n)]
        if t % 3 == 2 and n:
            # one or two bytes outside the alphabet: runs crossing them die
            for p in rng.integers(0, n, size=int(rng.integers(1, 3))):
                x[p] = f[rng.integers(0, f.size)]
        yield x


def _check(o, x, cs):
    B, d = o.B, o.dfa
    for c in cs:
        if c > max(1, x.size):
            continue
        b = chunk_boundaries(x.size, c)
        chunks = [bytes(x[b[i]:b[i + 1]]) for i in range(c)]
        got = o.lambda_rows(x, c)
        dgot = o.dfa_lambda_rows(x, c)
        want_dfa = csdpa_dfa_maps(d, chunks)
        for i, y in enumerate(chunks):
            want = [_wire(v) for v in chunk_mapping(B, y)]
            assert got[i].tolist() == want, (o.re, c, i)
            assert dgot[i].tolist() == [_wire(v) for v in want_dfa[i]], (o.re, c, i)


@pytest.mark.parametrize("idx", range(0, 210, 30))
def test_lambda_rows_match_table_runs_corpus(idx):
    rng = np.random.Generator(np.random.PCG64(0x1A3B + idx))
    for re_src, given in corpus()[idx:idx + 30]:
        alpha = letters_of(re_src, given)
        o = RidOracle(re_src)
        for x in _texts(rng, alpha, 6, 0, 40):
            _check(o, x, (1, 2, 3, 7, max(1, x.size)))


WORKLOAD = [
    (textgen.C1_RE, b"ACGT"),
    (textgen.C2_RE.replace("{20,60}", "{2,4}"), b"ACGT"),
    (textgen.C3_RE, b"0123456789-T:,.abcdefghijklmnopqrstuvwxyz\n"),
    (textgen.C3_RE_ANYFIELD, b"0123456789-T:,.abcdefghijklmnopqrstuvwxyz\n"),
    (textgen.regexp_family_re(3), b"ab"),
    (textgen.regexp_family_re(7), b"ab"),
]


@pytest.mark.parametrize("w", range(len(WORKLOAD)))
def test_lambda_rows_match_table_runs_workload_res(w):
    re_src, alpha = WORKLOAD[w]
    rng = np.random.Generator(np.random.PCG64(0x1A3C + w))
    o = RidOracle(re_src)
    for x in _texts(rng, alpha, 4, 100, 700):
        _check(o, x, (1, 5, 16, 61))
    if re_src == textgen.C3_RE:
        # members of the language, where the runs live long: record lines with a mutation
        x = textgen.c3_text(3000, seed=0x1A3D)
        _check(o, x, (1, 3, 40))
        y, _ = textgen.mutate(x, seed=0x1A3E, n_subs=2)
        _check(o, y, (1, 3, 40))
    if re_src == textgen.C1_RE:
        x = textgen.c1_text(2000, seed=0x1A3F)
        _check(o, x, (1, 4, 64))


def test_planted_mistakes_are_caught():
    """The comparison above fails for each plausible mistake in the two functions."""
    re_src = textgen.C1_RE
    x = textgen.c1_text(400, seed=0x1A40)
    # a wrong representative subset for one minimal-DFA state (state 2 of this DFA, read T or A,
    # given the subset of state 3, which also reads C)
    o = RidOracle(re_src)
    d = o.dfa
    d.state_subset[2] = d.state_subset[3]
    with pytest.raises(AssertionError):
        _check(o, x, (4, 133, 400))       # short chunks: long ones synchronise every run
    # a live subset missing from the subset-to-state map (the one reached by reading A from q0)
    o = RidOracle(re_src)
    d = o.dfa
    victim = o.sets.run({0}, b"A")
    assert victim in d.subset_to_state
    del d.subset_to_state[victim]
    with pytest.raises(AssertionError):
        _check(o, x, (1, 4, 133, 400))
    # the slot index used where its representative NFA state belongs (they differ once the
    # interface is minimised)
    class SlotMixup(RidOracle):
        def lambda_row(self, chunk):
            row = np.empty(self.B.k, dtype=np.uint16)
            for a in range(self.B.k):
                s = self.sets.run({a}, chunk)
                row[a] = LAMBDA_UNDEF if not s else self.B.index[s]
            return row

    o = SlotMixup(re_src)
    assert o.B.slots != list(range(o.B.k))
    with pytest.raises(AssertionError):
        _check(o, x, (1, 4, 133, 400))

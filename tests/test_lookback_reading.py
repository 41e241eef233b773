"""The reading behind intra-chunk pieces with look-back start sets, checked on the CPU with the
oracle's own RI-DFA (no device code): inside chunk i the run from slot a is in some state at
every earlier position w >= b_i, so at a piece's first byte b it lies among delta^B(P, y[w, b)),
the states that survive the window from every state (Sec. 3.2: B is deterministic).  Running
each piece only from that set (the chunk's first piece from the slots) and composing the piece
functions along the slots' runs gives the chunk row of the definition, for any window length.
"""
import numpy as np
import pytest

import textgen
from oracle.recognizer import LAMBDA_UNDEF, RidOracle
from oracle.ridfa_sets import UNDEF, chunk_boundaries


def lookback_row(B, chunk, spc, window, cap=32):
    """The chunk row through pieces: piece j >= 1 starts from the survivors of `window` bytes
    before it (never before the chunk start), or from every state when more than `cap` survive."""
    n_states = len(B.states)
    b = chunk_boundaries(len(chunk), spc)
    starts = [[B.slots[a] for a in range(B.k)]]          # slot a starts in its singleton state
    for j in range(1, spc):
        w = max(0, b[j] - window)
        surv = {B.run(p, chunk[w:b[j]]) for p in range(n_states)} - {UNDEF}
        starts.append(sorted(surv) if len(surv) <= cap else list(range(n_states)))
    funcs = [{x: B.run(x, chunk[b[j]:b[j + 1]]) for x in starts[j]} for j in range(spc)]
    row = np.empty(B.k, dtype=np.uint16)
    for a in range(B.k):
        y = B.slots[a]
        for j, f in enumerate(funcs):
            assert y in f, (a, j)          # the run's state at each piece start is a survivor
            y = f[y]
            if y is UNDEF:
                break
        row[a] = LAMBDA_UNDEF if y is UNDEF else y
    return row


def orf_text(n, rng):
    codons = [a + b + c for a in "ACGT" for b in "ACGT" for c in "ACGT"]
    parts = []
    while sum(map(len, parts)) < n:
        parts.append("".join(rng.choice(codons, int(rng.integers(0, 6)))) + "ATG" +
                     "".join(rng.choice(codons, int(rng.integers(2, 7)))) + "TGA")
    return np.frombuffer("".join(parts).encode(), dtype=np.uint8)


@pytest.mark.parametrize("name", ["c1", "c3", "codon", "regexp", "orf"])
def test_lookback_pieces_give_the_chunk_rows(name):
    rng = np.random.Generator(np.random.PCG64(11))
    re_src, x = {
        "c1": (textgen.C1_RE, textgen.c1_text(1500, 12)),
        "c3": (textgen.C3_RE, textgen.c3_text(1500, 13)),
        "codon": (textgen.C2_RE.replace("{20,60}", "{2,4}"), textgen.c2_text(1500, seed=14)),
        "regexp": (textgen.regexp_family_re(5), textgen.regexp_family_text(1500, 15)),
        "orf": ("(([ACGT]{3})*ATG([ACGT]{3}){2,6}(TAA|TAG|TGA))*", orf_text(1500, rng)),
    }[name]
    o = RidOracle(re_src, with_dfa=False)
    b = chunk_boundaries(len(x), 3)
    for i in range(3):
        chunk = bytes(x[b[i]:b[i + 1]])
        want = o.lambda_row(chunk)
        for spc, window in [(2, 16), (5, 16), (5, 3), (7, 64), (7, 1000)]:
            assert np.array_equal(lookback_row(o.B, chunk, spc, window), want), (name, i, spc, window)
        # capped start sets fall back to every state and still agree
        assert np.array_equal(lookback_row(o.B, chunk, 5, 16, cap=1), want)


def test_a_window_past_the_chunk_start_would_be_wrong():
    """Why the window stops at the chunk start: the chunk's runs start in the slots' singleton
    states, which need not survive the bytes before the chunk.  In (ab)*, after a preceding 'b'
    the only surviving state is the one that has just read 'b', which is not a slot's start
    state; a window reaching back past the chunk start would drop the slots' runs."""
    o = RidOracle("(ab)*", with_dfa=False)
    B = o.B
    before, chunk = b"abab", b"bab"
    surv = {B.run(p, before[-1:]) for p in range(len(B.states))} - {UNDEF}
    slot_states = {B.slots[a] for a in range(B.k)}
    assert not slot_states <= surv
    assert lookback_row(B, chunk, 1, 16).tolist() == o.lambda_row(chunk).tolist()

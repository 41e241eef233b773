"""The host recognition (``ridfa_cpu_recognize``, no GPU needed): the serial table loop and the
chunked speculative run on host threads, RI-DFA and all-states DFA, against the oracle's Thompson
simulation (the definition of acceptance) on the brute-force corpus and the workload REs, over
chunk counts from 1 to the text length and several thread counts."""
import numpy as np
import pytest

import textgen
from oracle.recognizer import SerialRecognizer

from .test_oracle_bruteforce import corpus, letters_of

lib = pytest.importorskip("paper_2412_14975_gb300")


def _texts(rng, alpha, n_texts, lo, hi, foreign=b"\x00\x7f\xff"):
    a = np.frombuffer(alpha, dtype=np.uint8)
    f = np.frombuffer(foreign, dtype=np.uint8)
    for t in range(n_texts):
        n = int(rng.integers(lo, hi + 1))
        x = a[rng.integers(0, a.size, size=n)]
        if t % 4 == 3 and n:
            x[int(rng.integers(0, n))] = f[rng.integers(0, f.size)]
        yield np.ascontiguousarray(x)


def _agree(prog, ser, x, cs, threads=(1, 3), dfa=True):
    want = ser.accepts(x)
    for c in cs:
        if not 1 <= c <= x.size:
            continue
        for t in threads:
            assert lib.ridfa_cpu_recognize(prog, x, c, n_threads=t) == want, (c, t)
            if dfa:
                assert lib.ridfa_cpu_recognize(prog, x, c, dfa=True, n_threads=t) == want, (c, t)
    return want


@pytest.mark.parametrize("idx", range(0, 210, 42))
def test_corpus_every_chunk_count(idx):
    rng = np.random.Generator(np.random.PCG64(0xC9 + idx))
    seen = set()
    for re_src, given in corpus()[idx:idx + 42]:
        prog = lib.ridfa_compile(re_src)
        ser = SerialRecognizer(re_src)
        alpha = letters_of(re_src, given)
        for x in _texts(rng, alpha, 5, 1, 24):
            seen.add(_agree(prog, ser, x, range(1, x.size + 1), threads=(1, 2)))
        e = np.zeros(0, np.uint8)
        assert lib.ridfa_cpu_recognize(prog, e, 0) == ser.accepts(e)
    assert seen == {True, False}


@pytest.mark.parametrize("which", ["c1", "c2", "c3", "c3any", "regexp7"])
def test_workload_res(which):
    if which == "c1":
        re_src, x = textgen.C1_RE, textgen.c1_text(300_000, seed=0xC1)
        alpha = b"ACGT"
    elif which == "c2":
        re_src, x = textgen.C2_RE.replace("{20,60}", "{2,4}"), textgen.c2_text(400_000, seed=0xC2)
        alpha = b"ACGT"
    elif which == "c3":
        re_src, x = textgen.C3_RE, textgen.c3_text(1 << 20, seed=0xC3)
        alpha = b"0123456789-T:,.abcdefghijklmnopqrstuvwxyz\n"
    elif which == "c3any":
        re_src, x = textgen.C3_RE_ANYFIELD, textgen.c3_text(1 << 20, seed=0xC4)
        alpha = b"0123456789-T:,.abcdefghijklmnopqrstuvwxyz\n"
    else:
        re_src, x = textgen.regexp_family_re(7), textgen.regexp_family_text(500_000, seed=0xC5)
        alpha = b"ab"
    prog = lib.ridfa_compile(re_src)
    ser = SerialRecognizer(re_src)
    cs = (1, 2, 16, 1000, 4099, x.size)
    dfa = prog.info["n_dfa_states"] > 0
    assert _agree(prog, ser, x, cs, threads=(1, 0), dfa=dfa)
    m, _ = textgen.mutate(x, seed=0xC6, n_subs=1, alphabet=alpha)
    _agree(prog, ser, m, cs, threads=(0,), dfa=dfa)
    z = x.copy()
    z[x.size // 2] = 0x00                            # a byte no position reads
    assert not _agree(prog, ser, z, (1, 7, 1000), threads=(0,), dfa=dfa)


def test_errors():
    prog = lib.ridfa_compile(textgen.C1_RE, build_dfa=False)
    x = textgen.c1_text(1000, seed=1)
    for c in (0, x.size + 1):
        with pytest.raises(lib.RidfaError) as e:
            lib.ridfa_cpu_recognize(prog, x, c)
        assert e.value.code == -4
    with pytest.raises(lib.RidfaError) as e:
        lib.ridfa_cpu_recognize(prog, np.zeros(0, np.uint8), 1)
    assert e.value.code == -4
    with pytest.raises(lib.RidfaError) as e:
        lib.ridfa_cpu_recognize(prog, x, 4, dfa=True)
    assert e.value.code == -10

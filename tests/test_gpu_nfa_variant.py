"""GPU NFA variant of the classic algorithm (Sec. 2; the NFA columns of Table 3), the RID's third
comparator: every chunk-relation row lambda_i(q) equals the oracle's position-set simulation
rho({q}, y_i) (chunk 1: q0's row only), and the accept bit equals the Thompson simulation, for
several REs, texts inside and outside the language, and chunk counts from 1 to the text length."""
import numpy as np
import pytest

import textgen
from oracle.recognizer import RidOracle, SerialRecognizer
from oracle.ridfa_sets import chunk_boundaries
from tests.gpu_util import to_device

pytestmark = pytest.mark.gpu

lib = pytest.importorskip("paper_2412_14975_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def bits(states, nw):
    w = np.zeros(nw, dtype=np.uint32)
    for q in states:
        w[q >> 5] |= np.uint32(1) << np.uint32(q & 31)
    return w


def check(re_src, x, cs):
    prog = lib.ridfa_compile(re_src, build_dfa=False)
    n = prog.info["n_nfa"]
    nw = (n + 31) // 32
    o = RidOracle(re_src, with_dfa=False)
    want_acc = SerialRecognizer(re_src).accepts(x)
    d = to_device(x)
    for c in cs:
        if c > x.size:
            continue
        sets = torch.zeros((c, n, nw), dtype=torch.int32, device="cuda:0")
        acc = lib.ridfa_recognize_nfa(prog, d, x.size, c, d_sets=sets)
        assert acc == want_acc, (re_src[:30], c)
        got = sets.cpu().numpy().view(np.uint32)
        b = chunk_boundaries(x.size, c)
        rows = range(c) if c <= 64 else sorted({0, 1, c // 2, c - 1} | set(range(0, c, max(1, c // 16))))
        for i in rows:
            y = bytes(x[b[i]:b[i + 1]])
            for q in range(n):
                want = o.sets.run({q}, y) if (i > 0 or q == 0) else frozenset()
                assert np.array_equal(got[i, q], bits(want, nw)), (re_src[:30], c, i, q)
        assert lib.ridfa_recognize_nfa(prog, d, x.size, c) == want_acc       # own scratch


@pytest.mark.parametrize("name", ["c1", "c3", "regexp3", "regexp7", "codon"])
def test_nfa_variant_rows_and_accept(name):
    re_src, gen = {
        "c1": (textgen.C1_RE, lambda s: textgen.c1_text(20_000, seed=s)),
        "c3": (textgen.C3_RE, lambda s: textgen.c3_text(20_000, seed=s)),
        "regexp3": (textgen.regexp_family_re(3), lambda s: textgen.regexp_family_text(20_000, seed=s)),
        "regexp7": (textgen.regexp_family_re(7), lambda s: textgen.regexp_family_text(20_000, seed=s)),
        "codon": (textgen.C2_RE.replace("{20,60}", "{2,4}"), lambda s: textgen.c2_text(20_000, seed=s)),
    }[name]
    x = gen(401)
    check(re_src, x, (1, 2, 7, 100, 5000))
    y, _ = textgen.mutate(x, seed=402, n_subs=2)
    check(re_src, y, (1, 7, 300))
    z = x.copy()
    z[x.size // 2] = 0x00                       # a byte no position reads: every run dies there
    check(re_src, z, (1, 7))


def test_nfa_variant_edges_and_limits():
    prog = lib.ridfa_compile("(ab)*", build_dfa=False)
    assert lib.ridfa_recognize_nfa(prog, 0, 0, 0) is True          # the empty word is in L
    prog2 = lib.ridfa_compile("(ab)+", build_dfa=False)
    assert lib.ridfa_recognize_nfa(prog2, 0, 0, 0) is False
    x = np.frombuffer(b"ab" * 50, dtype=np.uint8)
    d = to_device(x)
    assert lib.ridfa_recognize_nfa(prog, d, x.size, x.size) is True   # one byte per chunk
    with pytest.raises(lib.RidfaError) as e:
        lib.ridfa_recognize_nfa(prog, d, x.size, x.size + 1)
    assert e.value.code == -4
    big = lib.ridfa_compile(textgen.C3_RE_ANYFIELD, build_dfa=False)  # 129 NFA states
    with pytest.raises(lib.RidfaError) as e:
        lib.ridfa_recognize_nfa(big, d, x.size, 4)
    assert e.value.code == -9
    rng = np.random.Generator(np.random.PCG64(403))
    for _ in range(12):                                              # random small REs
        node = textgen.random_re(rng, b"abc", depth=int(rng.integers(2, 5)), max_lo=2, max_span=2)
        r = textgen.render(node)
        t = np.frombuffer(bytes(rng.choice(list(b"abc"), 3000)), dtype=np.uint8)
        check(r, t, (1, 5, 77))

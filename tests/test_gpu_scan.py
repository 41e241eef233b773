"""GPU join scan: the per-chunk entry sets E_i = if_min(PLAS_{i-1}) ∩ PIS_i and the first chunk
whose PLAS_i is empty, against the oracle's join history (Sec. 3.2), on accepted and rejected texts,
with matrix-join chunks and with chunks of more than 32 end states; c = 1 and c = n included."""
import numpy as np
import pytest

import textgen
from oracle.recognizer import RidOracle
from oracle.ridfa_sets import UNDEF, chunk_boundaries, chunk_mapping, rid_join
from tests.gpu_util import to_device

pytestmark = pytest.mark.gpu

lib = pytest.importorskip("paper_2412_14975_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

XS, YS = "ABCDEFGHIJKLMNOPQRSTUVWXYZ0123456789!#%&", "bcdefghijklmnopqrstuvwxyz<>=;:@$'\"^_`~,/"


def oracle_scan(B, text, c):
    b = chunk_boundaries(len(text), c)
    maps = [chunk_mapping(B, bytes(text[b[i]:b[i + 1]])) for i in range(c)]
    _, hist = rid_join(B, maps, return_plas=True)
    q0 = B.delegate[B.nfa.q0]
    entries, reject = [], -1
    for i in range(c):
        pis = {a for a, p in enumerate(maps[i]) if p is not UNDEF}
        e = ({q0} if i == 0 else B.interface(hist[i - 1])) & pis
        entries.append(e)
        if reject < 0 and not hist[i]:
            reject = i
    return entries, reject


def check(re_src, x, c):
    o = RidOracle(re_src, with_dfa=False)
    prog = lib.ridfa_compile(re_src, build_dfa=False)
    k = prog.info["k"]
    kw = (k + 31) // 32
    d = to_device(x)
    maps = torch.empty((c, k), dtype=torch.int16, device="cuda:0")
    lib.ridfa_recognize(prog, d, x.size, c, d_chunk_maps=maps)
    ent = torch.full((c, kw), -1, dtype=torch.int32, device="cuda:0")
    rej = lib.ridfa_join_scan(prog, maps, c, ent)
    want_e, want_r = oracle_scan(o.B, bytes(x), c)
    assert rej == want_r, (re_src[:30], c, rej, want_r)
    got = ent.cpu().numpy().view(np.uint32)
    for i in range(c):
        bits = {w * 32 + b for w in range(kw) for b in range(32) if (int(got[i, w]) >> b) & 1}
        assert bits == want_e[i], (re_src[:30], c, i, sorted(bits), sorted(want_e[i]))
    assert lib.ridfa_join_scan(prog, maps, c) == want_r        # without entry output


def test_scan_workload_res():
    rng = np.random.Generator(np.random.PCG64(404))
    x1 = textgen.c1_text(20_000, rng)
    x3 = textgen.c3_text(40_000, rng)
    x2 = textgen.c2_text(20_000, rng)
    for re_src, x in [(textgen.C1_RE, x1), (textgen.C3_RE, x3), (textgen.C2_RE.replace("{20,60}", "{2,4}"), x2),
                      (textgen.regexp_family_re(3), textgen.regexp_family_text(9000, rng))]:
        for c in (1, 2, 65, 130, 1000, 5000):
            check(re_src, x, min(c, x.size))
        y, _ = textgen.mutate(x, rng, n_subs=2)
        check(re_src, y, 777)
        # an out-of-alphabet byte rejects at its chunk
        z = x.copy()
        z[x.size // 3] = 0
        check(re_src, z, 300)


def test_scan_wide_chunks_and_tiny_texts():
    rng = np.random.Generator(np.random.PCG64(405))
    nb = 40
    re_src = "(" + "|".join(f"{XS[i]}a*{YS[i]}" for i in range(nb)) + ")*"
    parts = []
    for _ in range(40):
        i = int(rng.integers(nb))
        parts.append(XS[i] + "a" * int(rng.integers(0, 300)) + YS[i])
    x = np.frombuffer("".join(parts).encode(), dtype=np.uint8)
    for c in (3, 100, 1000):
        check(re_src, x, c)
    y = x.copy()
    y[x.size // 2] = ord(YS[0])
    check(re_src, y, 100)
    for re_src, t in [("(ab)*", b"ab"), ("(ab)*", b"ba"), ("a+", b"a"), ("a*b", b"aab")]:
        t = np.frombuffer(t, dtype=np.uint8)
        for c in range(1, t.size + 1):
            check(re_src, t, c)

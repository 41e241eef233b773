"""ridfa_recognize_noalloc: the recognize call for callers that cannot allocate device memory.

It must give exactly what ridfa_recognize gives (accept bit and every chunk map), on two calls in
a row, while keeping its tables and scratch in the library's fixed device array.  This file is
collected last so that a failure here does not hide the other tests.
"""
import numpy as np
import pytest

import textgen

pytestmark = pytest.mark.gpu

lib = pytest.importorskip("paper_2412_14975_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def reference(prog, d, n, c):
    maps = torch.empty((c, prog.info["k"]), dtype=torch.int16, device="cuda:0")
    acc = lib.ridfa_recognize(prog, d, n, c, d_chunk_maps=maps)
    return acc, maps.cpu().numpy().view(np.uint16)


def noalloc(prog, d, n, c):
    maps = torch.full((c, prog.info["k"]), -7, dtype=torch.int16, device="cuda:0")
    acc = torch.full((1,), 9, dtype=torch.uint8, device="cuda:0")
    lib.ridfa_recognize_noalloc(prog, d, n, c, acc, maps)
    torch.cuda.synchronize()
    return bool(acc.item()), maps.cpu().numpy().view(np.uint16)


def test_noalloc_matches_recognize_twice_in_a_row():
    cases = []
    x3 = textgen.c3_text(1 << 20, seed=21)
    x3m, _ = textgen.mutate(x3, seed=22, n_subs=2)
    x1 = textgen.c1_text(1 << 18, seed=23)
    x2 = textgen.c2_text(1 << 18, seed=24)     # runs that never merge: single-run hand-offs only
    re2 = textgen.C2_RE.replace("{20,60}", "{2,4}")
    for re_src, text, c in [(textgen.C3_RE, x3, 1000), (textgen.C3_RE, x3m, 4096),
                            (textgen.C1_RE, x1, 64), (textgen.C1_RE, x1, 7), (re2, x2, 300)]:
        cases.append((lib.ridfa_compile(re_src), torch.from_numpy(text.copy()).to("cuda:0"),
                      text.size, c))
    # alternate programs so each call has to bring its own tables into the shared array
    for prog, d, n, c in cases + cases[::-1]:
        want_acc, want_maps = reference(prog, d, n, c)
        for _ in range(2):
            acc, maps = noalloc(prog, d, n, c)
            assert acc == want_acc
            assert np.array_equal(maps, want_maps)


def test_noalloc_limits_and_empty_text():
    prog = lib.ridfa_compile(textgen.C3_RE)
    d = torch.zeros(2 << 20, dtype=torch.uint8, device="cuda:0")
    maps = torch.empty((1, prog.info["k"]), dtype=torch.int16, device="cuda:0")
    acc = torch.zeros(1, dtype=torch.uint8, device="cuda:0")
    c = (2 << 20) - 1            # 4 bytes per chunk alone exceed the fixed array
    with pytest.raises(lib.RidfaError) as e:
        lib.ridfa_recognize_noalloc(prog, d, 2 << 20, c, acc, maps)
    assert e.value.code == -12
    with pytest.raises(lib.RidfaError) as e:
        lib.ridfa_recognize_noalloc(prog, d, 10, 11, acc, maps)
    assert e.value.code == -4
    for re_src, eps in [("a*", True), ("a+", False)]:
        p = lib.ridfa_compile(re_src)
        lib.ridfa_recognize_noalloc(p, d, 0, 0, acc, maps)
        torch.cuda.synchronize()
        assert bool(acc.item()) is eps

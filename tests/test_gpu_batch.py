"""GPU batched recognition: every item's accept bit equals the oracle's (Thompson simulation)
and the single-text path's, across programs, lengths (empty to hundreds of KiB), explicit and
planned chunk counts, aligned (staged) and unaligned (global-load) texts, graph replays and the
one-shot call."""
import numpy as np
import pytest

import textgen
from oracle.recognizer import SerialRecognizer

pytestmark = pytest.mark.gpu

lib = pytest.importorskip("paper_2412_14975_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

RES = [textgen.C1_RE, textgen.C3_RE, textgen.C3_RE_ANYFIELD, textgen.regexp_family_re(3),
       textgen.C2_RE.replace("{20,60}", "{2,4}"), "(" + "|".join(f"{x}a*{y}" for x, y in
                                                                 zip("ABCDEFGHIJKLMNOPQRSTUVWXYZ0123456789!#%&",
                                                                     "bcdefghijklmnopqrstuvwxyz<>=;:@$'\"^_`~,/")) + ")*"]


def make_text(r, n, rng):
    if r == 0:
        return textgen.c1_text(n, rng)[:n]
    if r in (1, 2):
        return textgen.c3_text(n, rng)[:n]
    if r == 3:
        return textgen.regexp_family_text(n, rng)
    if r == 4:
        return textgen.c2_text(n, rng)
    xs, ys = "ABCDEFGHIJKLMNOPQRSTUVWXYZ0123456789!#%&", "bcdefghijklmnopqrstuvwxyz<>=;:@$'\"^_`~,/"
    parts, tot = [], 0
    while tot < n:
        i = int(rng.integers(40))
        s = xs[i] + "a" * int(rng.integers(0, 400)) + ys[i]
        parts.append(s)
        tot += len(s)
    return np.frombuffer("".join(parts).encode(), dtype=np.uint8)[:n]


def build_items(seed, n_items, aligned, explicit_every=0, max_len=200_000):
    rng = np.random.Generator(np.random.PCG64(seed))
    texts, meta = [], []
    for i in range(n_items):
        r = i % len(RES)
        n = int(rng.choice([0, 1, 17, 1000, 4096, 30_000, max_len]))
        x = make_text(r, n, rng) if n else np.zeros(0, np.uint8)
        if n > 50 and rng.random() < 0.5:
            x, _ = textgen.mutate(x, rng, n_subs=1)
        texts.append(np.ascontiguousarray(x, dtype=np.uint8))
        nc = 0
        if explicit_every and i % explicit_every == 0 and n:
            nc = int(rng.integers(1, min(n, 300) + 1))
        meta.append((r, nc))
    # lay the texts out in one device buffer: 16-byte aligned, or shifted off alignment
    offs, pos = [], 0
    for i, x in enumerate(texts):
        pos = (pos + 15) & ~15
        if not aligned and i % 3 == 1:
            pos += 5
        offs.append(pos)
        pos += x.size
    buf = np.zeros(max(pos, 16), np.uint8)
    for o, x in zip(offs, texts):
        buf[o:o + x.size] = x
    d = torch.from_numpy(buf).to("cuda:0")
    base = d.data_ptr()
    items = [(base + o, x.size, r, nc) for o, x, (r, nc) in zip(offs, texts, meta)]
    return d, texts, items


_SER = {}


def expected(texts, items):
    out = []
    for x, (_, _, r, _) in zip(texts, items):
        if r not in _SER:
            _SER[r] = SerialRecognizer(RES[r])
        out.append(_SER[r].accepts(x))
    return np.array(out, dtype=bool)


@pytest.mark.parametrize("aligned", [True, False])
def test_batch_matches_oracle_and_replays(aligned):
    progs = [lib.ridfa_compile(r) for r in RES]
    d, texts, items = build_items(11 if aligned else 12, 180, aligned, explicit_every=7)
    want = expected(texts, items)
    acc = torch.full((len(items),), 7, dtype=torch.uint8, device="cuda:0")
    b = lib.ridfa_batch_create(progs, items, acc, chunk_len=2048)
    st = lib.ridfa_batch_get_stats(b)
    assert st["graph"] == 1 and st["n_programs"] == len(RES)
    for _ in range(3):                                  # replays of the captured graph
        acc.fill_(7)
        lib.ridfa_batch_run(b)
        torch.cuda.synchronize()
        got = acc.cpu().numpy()
        assert set(np.unique(got)) <= {0, 1}
        assert np.array_equal(got.astype(bool), want)
    b.close()
    # the single-text path on the same items agrees
    for (ptr, n, r, nc), w in list(zip(items, want))[:60]:
        if n:
            assert lib.ridfa_recognize(progs[r], ptr, n, nc or max(1, min(n, 64))) == w


def test_batch_autotune_and_no_graph():
    progs = [lib.ridfa_compile(r) for r in RES[:3]]
    d, texts, items = build_items(21, 60, True, max_len=400_000)
    items = [(p, n, r % 3, nc) for (p, n, r, nc) in items]
    want = np.array([SerialRecognizer(RES[r]).accepts(x) for x, (_, _, r, _) in zip(texts, items)])
    for no_graph in (False, True):
        acc = torch.zeros(len(items), dtype=torch.uint8, device="cuda:0")
        b = lib.ridfa_batch_create(progs, items, acc, chunk_len=0, no_graph=no_graph)
        st = lib.ridfa_batch_get_stats(b)
        assert st["chunk_len"] in (4096, 8192, 16384, 32768)
        assert st["graph"] == (0 if no_graph else 1)
        lib.ridfa_batch_run(b)
        torch.cuda.synchronize()
        assert np.array_equal(acc.cpu().numpy().astype(bool), want)
        b.close()


def test_recognize_batch_one_shot_and_errors():
    progs = [lib.ridfa_compile(r) for r in RES[:2]]
    d, texts, items = build_items(31, 40, False)
    items = [(p, n, r % 2, nc) for (p, n, r, nc) in items]
    want = np.array([SerialRecognizer(RES[r]).accepts(x) for x, (_, _, r, _) in zip(texts, items)])
    acc = torch.zeros(len(items), dtype=torch.uint8, device="cuda:0")
    lib.ridfa_recognize_batch(progs, items, acc)
    assert np.array_equal(acc.cpu().numpy().astype(bool), want)
    with pytest.raises(lib.RidfaError) as e:
        lib.ridfa_batch_create(progs, [(d, 10, 5, 0)], acc)
    assert e.value.code == -1
    with pytest.raises(lib.RidfaError) as e:
        lib.ridfa_batch_create(progs, [(d, 10, 0, 11)], acc)
    assert e.value.code == -4


ORF_RE = "(([ACGT]{3})*ATG([ACGT]{3}){2,6}(TAA|TAG|TGA))*"   # 825 RI-DFA states: compact table


def orf_text(n, rng):
    """Concatenated open reading frames (random codons, ATG, 2-6 codons, a stop codon) of about n
    bytes: a word of ORF_RE, whose reading frame (length mod 3) every chunk must carry."""
    codons = [a + b + c for a in "ACGT" for b in "ACGT" for c in "ACGT"]
    parts, tot = [], 0
    while tot < n:
        s = "".join(rng.choice(codons, int(rng.integers(0, 12)))) + "ATG" + \
            "".join(rng.choice(codons, int(rng.integers(2, 7)))) + str(rng.choice(["TAA", "TAG", "TGA"]))
        parts.append(s)
        tot += len(s)
    return np.frombuffer("".join(parts).encode(), dtype=np.uint8)


@pytest.mark.parametrize("aligned", [True, False])
def test_batch_compact_table_reading_frame(aligned):
    """A program whose table is too large to replicate (runs stay apart; on aligned texts each
    lane finishes all of its chunk's runs together) and whose accept bit depends on every chunk's
    end states: positives, one-byte deletions (frame broken, rejected) and substitutions."""
    rng = np.random.Generator(np.random.PCG64(41 if aligned else 42))
    prog = lib.ridfa_compile(ORF_RE)
    ser = SerialRecognizer(ORF_RE)
    texts = []
    for i in range(48):
        x = orf_text(int(rng.choice([200, 3000, 20_000, 60_000])), rng)
        if i % 3 == 1:
            j = int(rng.integers(x.size))
            x = np.concatenate([x[:j], x[j + 1:]])
        elif i % 3 == 2:
            x = x.copy()
            x[int(rng.integers(x.size))] = ord("ACGT"[int(rng.integers(4))])
        texts.append(np.ascontiguousarray(x))
    want = np.array([ser.accepts(x) for x in texts])
    assert want.any() and not want.all()
    offs, pos = [], 0
    for i, x in enumerate(texts):
        pos = ((pos + 15) & ~15) + (0 if aligned or i % 2 == 0 else 3)
        offs.append(pos)
        pos += x.size
    buf = np.zeros(pos, np.uint8)
    for o, x in zip(offs, texts):
        buf[o:o + x.size] = x
    d = torch.from_numpy(buf).to("cuda:0")
    items = [(d.data_ptr() + o, x.size, 0, 0) for o, x in zip(offs, texts)]
    for chunk_len in (512, 2048):
        acc = torch.full((len(items),), 7, dtype=torch.uint8, device="cuda:0")
        b = lib.ridfa_batch_create([prog], items, acc, chunk_len=chunk_len)
        lib.ridfa_batch_run(b)
        torch.cuda.synchronize()
        assert np.array_equal(acc.cpu().numpy().astype(bool), want), chunk_len
        b.close()


def test_batch_launch_shapes_agree_and_autotune():
    """The batch autotuner's knobs -- warps per block of the reach launches and, for tables too
    large to replicate, a lane carrying all of its chunk's runs together or one run per lane --
    give the same accept bits as the oracle in every combination; an autotuned batch reports the
    shape it chose, and a second batch over the same programs reuses the cached tune."""
    progs = [lib.ridfa_compile(r) for r in RES]
    d, texts, items = build_items(51, 90, True, max_len=120_000)
    want = expected(texts, items)
    acc = torch.zeros(len(items), dtype=torch.uint8, device="cuda:0")
    for warps in (0, 4, 8, 16):
        for set_mode in (0, 1, 2):
            acc.fill_(7)
            b = lib.ridfa_batch_create(progs, items, acc, chunk_len=2048, block_warps=warps, set_mode=set_mode)
            st = lib.ridfa_batch_get_stats(b)
            assert st["block_warps"] == warps and st["set_mode"] == set_mode
            lib.ridfa_batch_run(b)
            torch.cuda.synchronize()
            assert np.array_equal(acc.cpu().numpy().astype(bool), want), (warps, set_mode)
            b.close()
    acc.fill_(7)
    b = lib.ridfa_batch_create(progs, items, acc, chunk_len=0)
    st = lib.ridfa_batch_get_stats(b)
    assert st["chunk_len"] in (4096, 8192, 16384, 32768)
    assert st["block_warps"] in (0, 8, 16) and st["set_mode"] in (0, 1, 2)
    lib.ridfa_batch_run(b)
    torch.cuda.synchronize()
    assert np.array_equal(acc.cpu().numpy().astype(bool), want)
    b.close()
    acc.fill_(7)
    b2 = lib.ridfa_batch_create(progs, items[: len(items) // 2], acc, chunk_len=0)
    st2 = lib.ridfa_batch_get_stats(b2)
    assert (st2["chunk_len"], st2["block_warps"], st2["set_mode"]) == (st["chunk_len"], st["block_warps"], st["set_mode"])
    lib.ridfa_batch_run(b2)
    torch.cuda.synchronize()
    assert np.array_equal(acc.cpu().numpy()[: len(items) // 2].astype(bool), want[: len(items) // 2])
    b2.close()
    with pytest.raises(lib.RidfaError) as e:
        lib.ridfa_batch_create(progs, items, acc, chunk_len=2048, set_mode=3)
    assert e.value.code == -1

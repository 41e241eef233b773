"""GPU parity: the sm_103a reach + join kernels, called through the C ABI, against the oracle.

Bit-exact everywhere (integer states): every chunk-map entry lambda_i(a) equals the oracle's
delta^B({q_a}, y_i) (computed by position-set simulation, Lemma 1) under the shared numbering
rule, and the accept bit equals the Thompson simulation.  The all-states DFA comparator is held
to the same bar against the oracle's minimal DFA.
"""
import numpy as np
import pytest

import textgen
from oracle.recognizer import RidOracle, SerialRecognizer
from tests.gpu_util import run, to_device

pytestmark = pytest.mark.gpu

lib = pytest.importorskip("paper_2412_14975_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

_ORACLES = {}


def oracle(re_src):
    if re_src not in _ORACLES:
        _ORACLES[re_src] = (RidOracle(re_src), SerialRecognizer(re_src))
    return _ORACLES[re_src]


def check(re_src, text, c, dfa_too=True, tuning=None, rows=None):
    o, ser = oracle(re_src)
    prog = lib.ridfa_compile(re_src)
    n = text.size
    d = to_device(text)
    acc, maps = run(lib, prog, d, n, c, tuning=tuning)
    want_acc = ser.accepts(text)
    assert acc == want_acc, (re_src, n, c)
    if rows is None and c * max(prog.info["k"], prog.info["n_dfa_states"]) > 20000:
        rng = np.random.Generator(np.random.PCG64(c))
        rows = sorted({0, 1, 2, c // 2, c - 2, c - 1} | set(rng.integers(0, c, 24).tolist()))
    ids = range(c) if rows is None else rows
    want = o.lambda_rows(text, c, ids)
    for i in ids:
        assert np.array_equal(maps[i], want[i]), (re_src, n, c, i, maps[i], want[i])
    if dfa_too and prog.info["n_dfa_states"] <= lib.RIDFA_MAX_SLOTS:
        dacc, dmaps = run(lib, prog, d, n, c, dfa=True, tuning=tuning)
        assert dacc == want_acc
        dwant = o.dfa_lambda_rows(text, c, ids)
        for i in ids:
            assert np.array_equal(dmaps[i], dwant[i]), (re_src, n, c, i)
    return acc


def test_config1_full_1mib_64_chunks():
    x = textgen.c1_text(1 << 20, seed=0x5EED01)
    assert check(textgen.C1_RE, x, 64)
    m, _ = textgen.mutate(x, seed=0x5EED02, n_subs=1, alphabet=b"ACGT")
    check(textgen.C1_RE, m, 64)


SIZES = [1, 2, 3, 17, 31, 32, 33, 1000, 4097, 65536 + 7]


@pytest.mark.parametrize("re_name", ["c1", "c3", "c3any", "c2_2_4", "regexp3", "regexp8"])
def test_small_sizes_all_rows(re_name):
    rng = np.random.Generator(np.random.PCG64(sum(map(ord, re_name))))
    re_src = {"c1": textgen.C1_RE, "c3": textgen.C3_RE, "c3any": textgen.C3_RE_ANYFIELD,
              "c2_2_4": textgen.C2_RE.replace("{20,60}", "{2,4}"),
              "regexp3": textgen.regexp_family_re(3), "regexp8": textgen.regexp_family_re(8)}[re_name]
    for n in SIZES:
        if re_name == "c1":
            x = textgen.c1_text(n, rng)[:n]
        elif re_name.startswith("c3"):
            x = textgen.c3_text(n, rng)[:n]
        elif re_name.startswith("c2"):
            x = textgen.c2_text(n, rng)
        else:
            x = textgen.regexp_family_text(n, rng)
        for c in sorted({1, 2, 7, 31, 32, 33, 64, 1000, n}):
            if c <= n:
                check(re_src, x, c, dfa_too=(n <= 4097))
        if n > 40:
            y, _ = textgen.mutate(x, rng, n_subs=int(rng.integers(1, 4)))
            check(re_src, y, min(n, 33))


def test_random_res_random_texts():
    rng = np.random.Generator(np.random.PCG64(0xC0FFEE))
    done = 0
    while done < 25:
        node = textgen.random_re(rng, b"abcd", depth=int(rng.integers(2, 6)))
        re_src = "(" + textgen.render(node) + ")*"
        try:
            prog = lib.ridfa_compile(re_src)
        except lib.RidfaError:
            continue
        if prog.info["k"] > lib.RIDFA_MAX_SLOTS:
            continue
        parts = [textgen.sample_member(node, rng, soft_len=30) for _ in range(400)]
        x = np.frombuffer(b"".join(parts), dtype=np.uint8)
        if x.size < 8:
            continue
        if done % 2:
            x, _ = textgen.mutate(x, rng, n_subs=1, alphabet=b"abcd")
        for c in (1, 5, 64, min(x.size, 777)):
            check(re_src, x, c, dfa_too=prog.info["n_dfa_states"] <= 256)
        done += 1


def test_empty_text_and_chunk_errors():
    import torch
    d = torch.zeros(16, dtype=torch.uint8, device="cuda:0")
    for re_src, eps in [("a*", True), ("a+", False), ("()", True), ("(ab)*", True)]:
        prog = lib.ridfa_compile(re_src)
        assert lib.ridfa_recognize(prog, d, 0, 0) is eps
        assert lib.ridfa_recognize_dfa(prog, d, 0, 0) is eps
        with pytest.raises(lib.RidfaError) as e:
            lib.ridfa_recognize(prog, d, 5, 6)
        assert e.value.code == -4
        with pytest.raises(lib.RidfaError) as e:
            lib.ridfa_recognize(prog, d, 5, 0)
        assert e.value.code == -4


def test_out_of_alphabet_bytes_kill_runs():
    x = np.frombuffer(b"ACGTTC" * 1000 + b"\x00" + b"ACG" * 100, dtype=np.uint8)
    check(textgen.C1_RE, x, 50)
    check(textgen.C1_RE, np.full(4096, 0xFF, dtype=np.uint8), 64)


def _branches_re(nb):
    xs = "ABCDEFGHIJKLMNOPQRSTUVWXYZ0123456789!#%&"
    ys = "bcdefghijklmnopqrstuvwxyz<>=;:@$'\"^_`~,/"
    return "(" + "|".join(f"{xs[i]}a*{ys[i]}" for i in range(nb)) + ")*", xs, ys


@pytest.mark.parametrize("nb", [3, 20, 40])
def test_many_distinct_end_states(nb):
    """Chunks that end with several distinct live states (matrix join with m > 1, and the
    sequential fallback when m > 32)."""
    re_src, xs, ys = _branches_re(nb)
    rng = np.random.Generator(np.random.PCG64(nb))
    parts = []
    for _ in range(30):
        i = int(rng.integers(nb))
        parts.append(xs[i] + "a" * int(rng.integers(0, 300)) + ys[i])
    x = np.frombuffer("".join(parts).encode(), dtype=np.uint8)
    for c in (3, 17, 100, 1000):
        check(re_src, x, min(c, x.size), dfa_too=False)
    y = x.copy()
    y[x.size // 2] = ord(ys[0])
    check(re_src, y, 100, dfa_too=False)


def test_piece_speculation_maps():
    """Few long chunks: each chunk is cut into pieces run from every automaton state and the piece
    functions are composed into the chunk's row.  Pieces forced on at several lengths, and off,
    give the oracle's maps; also for the all-states DFA comparator and for rows with more than 32
    distinct end states (composed rows, then the sequential join)."""
    x3 = textgen.c3_text(400_000, seed=95)
    x1 = textgen.c1_text(300_000, seed=96)
    for re_src, x in [(textgen.C3_RE, x3), (textgen.C1_RE, x1), (textgen.regexp_family_re(3),
                                                                  textgen.regexp_family_text(200_000, 97))]:
        o, ser = oracle(re_src)
        prog = lib.ridfa_compile(re_src)
        d = to_device(x)
        want_acc = ser.accepts(x)
        for c in (1, 3, 64):
            want = o.lambda_rows(x, c)
            dwant = o.dfa_lambda_rows(x, c)
            for piece in (0, 1, 64, 1000):
                acc, maps = run(lib, prog, d, x.size, c, tuning=dict(piece_len=piece))
                assert acc == want_acc
                for i in range(c):
                    assert np.array_equal(maps[i], want[i]), (re_src[:20], c, piece, i)
                dacc, dmaps = run(lib, prog, d, x.size, c, dfa=True, tuning=dict(piece_len=piece))
                assert dacc == want_acc
                for i in range(c):
                    assert np.array_equal(dmaps[i], dwant[i]), (re_src[:20], c, piece, i)
    y, _ = textgen.mutate(x3, seed=98, n_subs=3)
    check(textgen.C3_RE, y, 5, tuning=dict(piece_len=64))
    # enough pieces (65,536) that the reach kernel runs them, one lane per piece, instead of one
    # lockstep warp per piece
    x4 = textgen.c3_text(4 << 20, seed=100)
    check(textgen.C3_RE, x4, 2, tuning=dict(piece_len=64))
    re_src, xs, ys = _branches_re(40)
    rng = np.random.Generator(np.random.PCG64(99))
    parts = [xs[int(i)] + "a" * int(rng.integers(0, 300)) + ys[int(i)] for i in rng.integers(40, size=200)]
    z = np.frombuffer("".join(parts).encode(), dtype=np.uint8)
    for c in (2, 9):
        check(re_src, z, c, tuning=dict(piece_len=64), dfa_too=False)
    prog = lib.ridfa_compile(textgen.C1_RE)
    with pytest.raises(lib.RidfaError) as e:
        lib.ridfa_recognize(prog, to_device(x1), x1.size, 4, tuning=dict(piece_len=17))
    assert e.value.code == -1


def test_multi_run_handoff_rows():
    """Chunks whose live runs never merge into one state (the {2,4} codon RE keeps up to five
    distinct states) are handed off as several runs each; with ~1 KiB chunks a warp holds over 32
    runs, so the finals go through the run list.  Every row, ragged last chunk included."""
    re2 = textgen.C2_RE.replace("{20,60}", "{2,4}")
    x = textgen.c2_text((1 << 20) + 13, seed=91)
    for c in (1000, 3001):
        for path in (1, 3, 5):
            check(re2, x, c, dfa_too=False, rows=list(range(c)), tuning=dict(text_path=path))
    y, _ = textgen.mutate(x, seed=92, n_subs=3, alphabet=b"ACGT")
    check(re2, y, 1000, dfa_too=False, rows=list(range(1000)))


@pytest.mark.parametrize("path", [1, 3, 4, 5])
def test_text_paths_agree(path):
    """16-byte global loads and the staged paths give the same maps, on aligned texts and on
    texts that start 1..15 bytes past an alignment boundary (the staged paths then refuse)."""
    x = textgen.c3_text(300_000, seed=81)
    for c in (1, 31, 1000, 9000):
        check(textgen.C3_RE, x, c, tuning=dict(text_path=path), dfa_too=(c == 1000))
    prog = lib.ridfa_compile(textgen.C3_RE)
    # text path 2 (per-lane bulk copies) is retired: refused on any text
    with pytest.raises(lib.RidfaError) as e:
        lib.ridfa_recognize(prog, to_device(x), x.size, 1000, tuning=dict(text_path=2))
    assert e.value.code == -1
    o, ser = oracle(textgen.C3_RE)
    base = torch.from_numpy(np.concatenate([np.zeros(16, np.uint8), x])).to("cuda:0")
    for off in (1, 3, 8, 15):
        y = x[off:]
        d = base[16 + off:]
        if path in (3, 4, 5):
            with pytest.raises(lib.RidfaError) as e:
                lib.ridfa_recognize(prog, d, y.size, 100, tuning=dict(text_path=path))
            assert e.value.code == -1
            continue
        maps = torch.empty((100, prog.info["k"]), dtype=torch.int16, device="cuda:0")
        acc = lib.ridfa_recognize(prog, d, y.size, 100, tuning=dict(text_path=path), d_chunk_maps=maps)
        assert acc == ser.accepts(y)
        got = maps.cpu().numpy().view(np.uint16)
        want = o.lambda_rows(y, 100, [0, 1, 50, 98, 99])
        for i in want:
            assert np.array_equal(got[i], want[i])


@pytest.mark.parametrize("mode", [1, 2, 3, 4, 5, 6])
def test_tuning_variants_agree(mode):
    """Every table layout (compact, lane-replicated 16/32-bit, half-replicated, generic loads) and
    launch shape gives the same bit-exact maps."""
    x = textgen.c3_text(1 << 18, seed=77)
    for t in [dict(probe_interval=1), dict(probe_interval=64), dict(block_threads=64),
              dict(grid_blocks=1), dict(block_threads=128, grid_blocks=3),
              dict(block_threads=1024), dict(), dict(text_path=1, block_threads=1024),
              dict(text_path=3, block_threads=96), dict(text_path=3, grid_blocks=1),
              dict(text_path=4, block_threads=64), dict(text_path=4, grid_blocks=1), dict(text_path=4),
              dict(text_path=5), dict(text_path=5, block_threads=160, grid_blocks=2)]:
        t["table_mode"] = mode
        check(textgen.C3_RE, x, 1000, dfa_too=True, tuning=t)
    y = textgen.c1_text(1 << 16, seed=78)
    check(textgen.C1_RE, y, 300, tuning=dict(table_mode=mode))
    re2 = textgen.C2_RE.replace("{20,60}", "{2,4}")
    z = textgen.c2_text(1 << 16, seed=79)
    # 424 states x 5 classes: the 16-bit offsets overflow and the 32-bit replicated table exceeds
    # shared memory; the compact tables (the two-byte one automatic) and the half-replicated one
    # (on request) fit
    check(re2, z, 200, tuning=dict(table_mode=mode if mode in (1, 4, 5, 6) else 0), dfa_too=False)
    check(re2, z, 1000, tuning=dict(table_mode=mode if mode in (1, 4, 5, 6) else 0, text_path=1), dfa_too=False)
    prog = lib.ridfa_compile(re2)
    d = to_device(z)
    for bad in (2, 3):
        with pytest.raises(lib.RidfaError) as e:
            lib.ridfa_recognize(prog, d, z.size, 200, tuning=dict(table_mode=bad))
        assert e.value.code == -1


def test_unminimized_interface_maps():
    """With minimize_interface=0 every NFA state is a slot; maps still match the oracle."""
    re_src = textgen.C1_RE
    o = RidOracle(re_src, minimize=False)
    prog = lib.ridfa_compile(re_src, minimize_interface=False)
    x = textgen.c1_text(50_000, seed=3)
    acc, maps = run(lib, prog, to_device(x), x.size, 77)
    assert acc == SerialRecognizer(re_src).accepts(x)
    want = o.lambda_rows(x, 77)
    for i in range(77):
        assert np.array_equal(maps[i], want[i])


def test_c3_64mib_sampled_rows():
    """A larger record-line text in 16,384 chunks (cut into pieces: the chunks fill under half of
    the lanes), sampled rows."""
    x = textgen.c3_text(64 << 20, seed=0x5EED03)
    c = 1 << 14
    rows = sorted({0, 1, 2, c // 2, c - 2, c - 1} | set(
        np.random.Generator(np.random.PCG64(1)).integers(0, c, 10).tolist()))
    assert check(textgen.C3_RE, x, c, rows=rows)
    y, _ = textgen.mutate(x, seed=5, n_subs=3)
    check(textgen.C3_RE, y, c, rows=rows)


def test_recognize_host_buffers():
    """Texts in host memory (pageable numpy, bytes, page-locked tensor) go through the one-call
    host entry: copied into the caller's device buffer and recognized; the accept bit and the
    staged bytes match the oracle and the source.  Empty text and null buffers."""
    x = textgen.c3_text((1 << 20) + 5, seed=101)
    y, _ = textgen.mutate(x, seed=102, n_subs=2)
    prog = lib.ridfa_compile(textgen.C3_RE)
    _, ser = oracle(textgen.C3_RE)
    d_stage = torch.empty(x.size + 16, dtype=torch.uint8, device="cuda:0")
    for t in (x, y):
        want = ser.accepts(t)
        for c in (1, 64, 1000):
            assert lib.ridfa_recognize_host(prog, t, t.size, c, d_stage) is want
        assert lib.ridfa_recognize_host(prog, t.tobytes(), t.size, 77, d_stage) is want
        pinned = torch.from_numpy(t.copy()).pin_memory()
        assert lib.ridfa_recognize_host(prog, pinned, t.size, 155, d_stage) is want
        assert np.array_equal(d_stage[:t.size].cpu().numpy(), t)
    eps = lib.ridfa_compile("a*")
    assert lib.ridfa_recognize_host(eps, None, 0, 0, None) is True
    for bad in [(None, 10, 1, d_stage), (x, 10, 1, None)]:
        with pytest.raises(lib.RidfaError) as e:
            lib.ridfa_recognize_host(prog, *bad)
        assert e.value.code == -1


def test_compact_table_runs_finished_together():
    """Every row of a program with a compact (unreplicated) table, where chunks hand off several
    runs: the automatic path (each lane finishes its chunk's runs together) and one run per lane
    give the oracle's maps."""
    re_src = "(([ACGT]{3})*ATG([ACGT]{3}){2,6}(TAA|TAG|TGA))*"
    rng = np.random.Generator(np.random.PCG64(103))
    codons = [a + b + c for a in "ACGT" for b in "ACGT" for c in "ACGT"]
    parts = []
    while sum(map(len, parts)) < 24_000:
        parts.append("".join(rng.choice(codons, int(rng.integers(0, 12)))) + "ATG" +
                     "".join(rng.choice(codons, int(rng.integers(2, 7)))) + "TGA")
    x = np.frombuffer("".join(parts).encode(), dtype=np.uint8)
    y = np.concatenate([x[:5000], x[5001:]])
    for t in (x, y):
        for c in (23, 100):
            for tuning in (None, dict(text_path=3), dict(text_path=5, block_threads=64)):
                check(re_src, t, c, dfa_too=False, rows=list(range(c)), tuning=tuning)


def test_pieces_large_automata():
    """Automata of more than 256 states.  With k <= 32 (regexp family k = 7: 273 states; codon RE
    {2,4}: 424; the reading-frame RE: 825) each piece starts from its look-back start set (the
    chunk's first piece from the interface slots) and the rows are scattered into the piece
    functions; with the start sets capped below their size the pieces fall back to whole functions
    from every state.  With k > 32 (a prefixed regexp family: 303 states, k = 38) the pieces run
    from every state in groups of at most 256, one reach launch per group.  The composed rows equal
    the oracle's, pieces on (automatic and forced) and off."""
    rng = np.random.Generator(np.random.PCG64(104))
    codons = [a + b + c for a in "ACGT" for b in "ACGT" for c in "ACGT"]
    parts = []
    while sum(map(len, parts)) < 120_000:
        parts.append("".join(rng.choice(codons, int(rng.integers(0, 12)))) + "ATG" +
                     "".join(rng.choice(codons, int(rng.integers(2, 7)))) + "TAG")
    orf = np.frombuffer("".join(parts).encode(), dtype=np.uint8)
    cases = [(textgen.regexp_family_re(7), textgen.regexp_family_text(100_000, 105), True),
             (textgen.C2_RE.replace("{20,60}", "{2,4}"), textgen.c2_text(100_000, seed=106), False),
             ("(([ACGT]{3})*ATG([ACGT]{3}){2,6}(TAA|TAG|TGA))*", orf, False),
             ("(([ACGT]{3})*ATG([ACGT]{3}){2,6}(TAA|TAG|TGA))*", np.concatenate([orf[:777], orf[778:]]), False)]
    pre = "ghijklmnopqrstuvwxyzGHIJKLMNOP"
    words = []
    while sum(map(len, words)) < 100_000:
        ab = "".join(rng.choice(["a", "b"], int(rng.integers(8, 300))))
        words.append(pre + ab[:-8] + "a" + ab[-7:])
    cases.append(("(" + pre + "(a|b)*a(a|b){7})*", np.frombuffer("".join(words).encode(), dtype=np.uint8), False))
    for re_src, x, dfa_too in cases:
        info = lib.ridfa_compile(re_src).info
        assert info["n_states"] > 256
        for c in (1, 3, 7):
            for piece in (0, 1, 256):
                check(re_src, x, c, dfa_too=dfa_too, rows=list(range(c)), tuning=dict(piece_len=piece))
        if info["k"] <= 32:
            for cap in (1, 3):
                check(re_src, x, 3, dfa_too=False, rows=[0, 1, 2], tuning=dict(piece_len=256, lookback_cap=cap))
    prog = lib.ridfa_compile(cases[0][0])
    with pytest.raises(lib.RidfaError) as e:
        lib.ridfa_recognize(prog, to_device(cases[0][1]), cases[0][1].size, 3, tuning=dict(lookback_cap=33))
    assert e.value.code == -1


def test_lookback_pieces_unaligned_and_accept_only():
    """Look-back pieces on a text that starts off a 16-byte boundary (plain global loads), with
    and without chunk maps requested (accept only: the library's own scratch), and on a mutated
    text whose reading frame breaks in a middle piece."""
    re_src = "(([ACGT]{3})*ATG([ACGT]{3}){2,6}(TAA|TAG|TGA))*"
    o, ser = oracle(re_src)
    prog = lib.ridfa_compile(re_src)
    rng = np.random.Generator(np.random.PCG64(107))
    codons = [a + b + c for a in "ACGT" for b in "ACGT" for c in "ACGT"]
    parts = []
    while sum(map(len, parts)) < 150_000:
        parts.append("".join(rng.choice(codons, int(rng.integers(0, 12)))) + "ATG" +
                     "".join(rng.choice(codons, int(rng.integers(2, 7)))) + "TAA")
    x = np.frombuffer("".join(parts).encode(), dtype=np.uint8)
    y = np.concatenate([x[:70_001], x[70_002:]])
    for t in (x, y):
        want_acc = ser.accepts(t)
        base = torch.from_numpy(np.concatenate([np.zeros(16, np.uint8), t])).to("cuda:0")
        for off in (0, 3):
            d = base[16 - off:] if off else base[16:]
            src = np.concatenate([np.zeros(off, np.uint8), t]) if off else t
            n = src.size
            for c in (2, 5):
                acc, maps = run(lib, prog, d, n, c, tuning=dict(piece_len=512))
                assert acc == ser.accepts(src)
                want = o.lambda_rows(src, c, range(c))
                for i in range(c):
                    assert np.array_equal(maps[i], want[i]), (off, c, i)
                assert lib.ridfa_recognize(prog, d, n, c, tuning=dict(piece_len=512)) == ser.accepts(src)
        assert lib.ridfa_recognize(prog, base[16:], t.size, 4) == want_acc


def test_c3_4gib_bench_workload_sampled_rows():
    """The bench's workload in its launch shape: 4 GiB of record lines generated on the device
    with the bench's seed, 155,648 chunks.  Sampled rows equal the oracle's, chunk by chunk; the
    accept bit equals the Thompson oracle's over the whole 4 GiB text (about half a minute on
    one host core), and so does the accept bit of a copy with one in-alphabet substitution; one
    byte outside the alphabet anywhere makes the RID and the all-states DFA both reject."""
    import bench
    from oracle.ridfa_sets import chunk_boundaries
    d = bench.make_text("c3", 4 << 30, 0x5EED02, "cuda:0")
    n, c = d.numel(), 155_648
    o, ser = oracle(textgen.C3_RE)
    prog = lib.ridfa_compile(textgen.C3_RE)
    maps = torch.empty((c, prog.info["k"]), dtype=torch.int16, device="cuda:0")
    acc = lib.ridfa_recognize(prog, d, n, c, d_chunk_maps=maps)
    host = d.cpu().numpy()
    assert acc == ser.accepts(host)
    assert lib.ridfa_recognize_dfa(prog, d, n, c) == acc
    b = chunk_boundaries(n, c)
    rows = sorted({0, 1, c // 2, c - 2, c - 1} | set(np.random.Generator(np.random.PCG64(3)).integers(0, c, 12).tolist()))
    got = maps[rows].cpu().numpy().view(np.uint16)
    for g, i in zip(got, rows):
        want = o.lambda_row(host[b[i]:b[i + 1]])
        assert np.array_equal(g, want), i
    # one in-alphabet substitution (a digit becomes a letter or a comma ...): the oracle decides
    pos = int(b[(2 * c) // 3] + 777)
    keep = int(host[pos])
    repl = ord("a") if keep != ord("a") else ord("0")
    host[pos] = repl
    d[pos] = repl
    want_mut = ser.accepts(host)
    assert lib.ridfa_recognize(prog, d, n, c) == want_mut
    assert lib.ridfa_recognize_dfa(prog, d, n, c) == want_mut
    host[pos] = keep
    d[pos] = keep
    pos = int(b[c // 3] + 1234)
    keep = d[pos].item()
    d[pos] = 0
    assert lib.ridfa_recognize(prog, d, n, c) is False
    assert lib.ridfa_recognize_dfa(prog, d, n, c) is False
    d[pos] = keep
    del d, maps, host
    torch.cuda.empty_cache()


def test_compact_class_table_layout():
    """Table layout 7: the lane-replicated transition table of layout 6 beside one 512-byte copy of
    the class table, on the set path (aligned texts) and plain global loads (unaligned ones).
    Every row equals the oracle's: the codon RE (runs stay apart: several runs per lane), record
    lines, the regexp family, pieces (few chunks: lockstep pieces and look-back start sets);
    the cooperative single-run paths refuse the layout."""
    re2 = textgen.C2_RE.replace("{20,60}", "{2,4}")
    x = textgen.c2_text((1 << 20) + 13, seed=201)
    for c in (1000, 3001):
        check(re2, x, c, dfa_too=False, rows=list(range(c)), tuning=dict(table_mode=7))
    check(re2, x, 1000, dfa_too=False, rows=list(range(1000)), tuning=dict(table_mode=7, text_path=1))
    y, _ = textgen.mutate(x, seed=202, n_subs=5, alphabet=b"ACGTN")
    check(re2, y, 777, dfa_too=False, rows=list(range(777)), tuning=dict(table_mode=7))
    check(re2, x, 2, dfa_too=False, tuning=dict(table_mode=7))          # look-back pieces
    x3 = textgen.c3_text(1 << 18, seed=203)
    for c in (1, 1000, 4099):
        check(textgen.C3_RE, x3, c, tuning=dict(table_mode=7))
    check(textgen.regexp_family_re(7), textgen.regexp_family_text(1 << 18, seed=204), 1000,
          tuning=dict(table_mode=7))
    x1 = textgen.c1_text(1 << 16, seed=205)
    check(textgen.C1_RE, x1, 4, tuning=dict(table_mode=7))              # lockstep pieces
    prog = lib.ridfa_compile(re2)
    o, ser = oracle(re2)
    base = torch.from_numpy(np.concatenate([np.zeros(16, np.uint8), x])).to("cuda:0")
    d = base[16 + 3:]
    z = x[3:]
    maps = torch.empty((500, prog.info["k"]), dtype=torch.int16, device="cuda:0")
    acc = lib.ridfa_recognize(prog, d, z.size, 500, tuning=dict(table_mode=7), d_chunk_maps=maps)
    assert acc == ser.accepts(z)
    got = maps.cpu().numpy().view(np.uint16)
    want = o.lambda_rows(z, 500, [0, 1, 250, 498, 499])
    for i in want:
        assert np.array_equal(got[i], want[i])
    for tp in (3, 4):
        with pytest.raises(lib.RidfaError) as e:
            lib.ridfa_recognize(prog, to_device(x), x.size, 1000, tuning=dict(table_mode=7, text_path=tp))
        assert e.value.code == -1


def test_compact_two_byte_layout():
    """Table layout 9 (two-byte steps in one compact table: a lane's runs share each pair's
    column; single steps at ragged edges and hand-off positions): every row equals the oracle's
    on the codon RE (several runs per lane on the set path), the regexp family and the C1 RE,
    aligned (set path) and unaligned (global loads) texts, bytes outside the alphabet, few chunks
    (lockstep pieces and look-back start sets); automata whose pair table does not fit, and the
    single-run cooperative paths, refuse it."""
    re2 = textgen.C2_RE.replace("{20,60}", "{2,4}")
    x = textgen.c2_text((1 << 20) + 13, seed=401)
    for c in (1, 1000, 3001):
        check(re2, x, c, dfa_too=False, rows=list(range(c)), tuning=dict(table_mode=9))
    check(re2, x, 1000, dfa_too=False, rows=list(range(1000)), tuning=dict(table_mode=9, text_path=1))
    check(re2, x, 1000, dfa_too=False, rows=list(range(1000)), tuning=dict(table_mode=9, text_path=5))
    y, _ = textgen.mutate(x, seed=402, n_subs=5, alphabet=b"ACGTN")
    check(re2, y, 777, dfa_too=False, rows=list(range(777)), tuning=dict(table_mode=9))
    check(re2, x, 2, dfa_too=False, tuning=dict(table_mode=9))          # look-back pieces
    for re_src, z in ((textgen.regexp_family_re(7), textgen.regexp_family_text((1 << 18) + 5, seed=403)),
                      (textgen.C1_RE, textgen.c1_text((1 << 17) + 3, seed=404))):
        for c in (4, 1000, 4099):
            check(re_src, z, c, rows=list(range(c)) if c <= 1000 else None, tuning=dict(table_mode=9))
        w, _ = textgen.mutate(z, seed=405, n_subs=3, alphabet=b"ACGTabN\n")
        check(re_src, w, 1000, rows=list(range(1000)), tuning=dict(table_mode=9))
    prog = lib.ridfa_compile(re2)
    o, ser = oracle(re2)
    base = torch.from_numpy(np.concatenate([np.zeros(16, np.uint8), x])).to("cuda:0")
    z = x[7:]
    maps = torch.empty((500, prog.info["k"]), dtype=torch.int16, device="cuda:0")
    acc = lib.ridfa_recognize(prog, base[16 + 7:], z.size, 500, tuning=dict(table_mode=9), d_chunk_maps=maps)
    assert acc == ser.accepts(z)
    got = maps.cpu().numpy().view(np.uint16)
    want = o.lambda_rows(z, 500, [0, 1, 250, 498, 499])
    for i in want:
        assert np.array_equal(got[i], want[i])
    for tp in (3, 4):
        with pytest.raises(lib.RidfaError) as e:
            lib.ridfa_recognize(prog, to_device(x), x.size, 1000, tuning=dict(table_mode=9, text_path=tp))
        assert e.value.code == -1
    # the codon RE {3,6}: 1,588 states x 30 columns do not fit 16-bit row offsets
    prog = lib.ridfa_compile(textgen.C2_RE.replace("{20,60}", "{3,6}"))
    assert (prog.info["n_states"] + 1) * 30 * 2 > 0xFFFF
    with pytest.raises(lib.RidfaError) as e:
        lib.ridfa_recognize(prog, to_device(x), x.size, 100, tuning=dict(table_mode=9))
    assert e.value.code == -1


@pytest.mark.parametrize("mode", [10, 11])
def test_two_byte_lane_copies_layout(mode):
    """Table layouts 10 and 11 (two-byte steps in F lane copies, F = 16, 8, 4 or 2 by size; byte
    and half-word offsets): every row equals the oracle's on the regexp family k = 5 and k = 7,
    the any-field record lines and the codon RE, aligned (staged) and unaligned (global loads)
    texts, bytes outside the alphabet, few chunks (pieces), and on the DFA comparator where it
    fits; automata whose pair table fits no copy count, and the set path, refuse it."""
    cases = ((textgen.regexp_family_re(5), textgen.regexp_family_text(200_003, seed=501), True),
             (textgen.regexp_family_re(7), textgen.regexp_family_text(300_001, seed=502), True),
             (textgen.C3_RE_ANYFIELD, textgen.c3_text(1 << 18, seed=503), True),
             (textgen.C3_RE, textgen.c3_text(1 << 18, seed=507), True),          # k = 68: R = 4
             (textgen.C2_RE.replace("{20,60}", "{2,4}"), textgen.c2_text(300_007, seed=504), False))
    for re_src, x, dfa in cases:
        for c in (1, 7, 1000, 4099):
            check(re_src, x, c, dfa_too=dfa, rows=list(range(c)) if c <= 1000 else None,
                  tuning=dict(table_mode=mode))
        y, _ = textgen.mutate(x, seed=505, n_subs=3, alphabet=b"ACGTabN\n")
        check(re_src, y, 1000, dfa_too=dfa, rows=list(range(1000)), tuning=dict(table_mode=mode))
        check(re_src, x, 1000, dfa_too=dfa, rows=list(range(1000)), tuning=dict(table_mode=mode, text_path=1))
        prog = lib.ridfa_compile(re_src)
        o, ser = oracle(re_src)
        base = torch.from_numpy(np.concatenate([np.zeros(16, np.uint8), x])).to("cuda:0")
        z = x[9:]
        maps = torch.empty((300, prog.info["k"]), dtype=torch.int16, device="cuda:0")
        acc = lib.ridfa_recognize(prog, base[16 + 9:], z.size, 300, tuning=dict(table_mode=mode), d_chunk_maps=maps)
        assert acc == ser.accepts(z)
        got = maps.cpu().numpy().view(np.uint16)
        want = o.lambda_rows(z, 300, [0, 1, 150, 298, 299])
        for i in want:
            assert np.array_equal(got[i], want[i])
        with pytest.raises(lib.RidfaError) as e:
            lib.ridfa_recognize(prog, to_device(x), x.size, 1000, tuning=dict(table_mode=mode, text_path=5))
        assert e.value.code == -1
    # 4,121 states x 12 columns: even 2 copies overflow the 16-bit entries
    prog = lib.ridfa_compile(textgen.regexp_family_re(11))
    x = textgen.regexp_family_text(1 << 16, seed=506)
    with pytest.raises(lib.RidfaError) as e:
        lib.ridfa_recognize(prog, to_device(x), x.size, 100, tuning=dict(table_mode=mode))
    assert e.value.code == -1


def test_two_byte_step_layout():
    """Table layout 8 (two-byte steps: one transition lookup per pair of bytes in the converged
    phase, single steps at ragged edges): every row equals the oracle's on the C1 RE and the
    regexp family k = 3, 4, 5, aligned (staged, whole granules of pairs) and unaligned (global
    loads) texts, bytes outside the alphabet, few chunks (pieces); automata too large for the
    layout, and the set path, refuse it."""
    for re_src, x in ((textgen.C1_RE, textgen.c1_text(300_001, seed=301)),
                      (textgen.regexp_family_re(3), textgen.regexp_family_text(300_001, seed=302)),
                      (textgen.regexp_family_re(4), textgen.regexp_family_text(200_003, seed=303)),
                      (textgen.regexp_family_re(5), textgen.regexp_family_text(200_005, seed=304))):
        for c in (1, 7, 1000, 4099):
            check(re_src, x, c, rows=list(range(c)) if c <= 1000 else None, tuning=dict(table_mode=8))
        y, _ = textgen.mutate(x, seed=305, n_subs=3, alphabet=b"ACGTabN\n")
        check(re_src, y, 1000, rows=list(range(1000)), tuning=dict(table_mode=8))
        check(re_src, x, 1000, rows=list(range(1000)), tuning=dict(table_mode=8, text_path=1))
        prog = lib.ridfa_compile(re_src)
        o, ser = oracle(re_src)
        base = torch.from_numpy(np.concatenate([np.zeros(16, np.uint8), x])).to("cuda:0")
        z = x[5:]
        maps = torch.empty((300, prog.info["k"]), dtype=torch.int16, device="cuda:0")
        acc = lib.ridfa_recognize(prog, base[16 + 5:], z.size, 300, tuning=dict(table_mode=8), d_chunk_maps=maps)
        assert acc == ser.accepts(z)
        got = maps.cpu().numpy().view(np.uint16)
        want = o.lambda_rows(z, 300, [0, 1, 150, 298, 299])
        for i in want:
            assert np.array_equal(got[i], want[i])
    prog = lib.ridfa_compile(textgen.C3_RE)
    x3 = textgen.c3_text(1 << 16, seed=306)
    for tu in (dict(table_mode=8), dict(table_mode=8, text_path=5)):
        with pytest.raises(lib.RidfaError) as e:
            lib.ridfa_recognize(prog, to_device(x3), x3.size, 100, tuning=tu)
        assert e.value.code == -1
    prog = lib.ridfa_compile(textgen.C1_RE)
    x1 = textgen.c1_text(1 << 16, seed=307)
    with pytest.raises(lib.RidfaError) as e:
        lib.ridfa_recognize(prog, to_device(x1), x1.size, 100, tuning=dict(table_mode=8, text_path=5))
    assert e.value.code == -1


def test_planner_choices():
    """The automatic plan (reported by ridfa_last_plan) takes the layouts the measurements chose:
    lane-replicated 16-bit tables for the record lines, the compact two-byte table on the set path
    for the codon RE (runs in three reading frames stay apart), the two-byte table in lane copies
    with one run per lane for the regexp family (runs merge), global loads for an unaligned text;
    an explicit layout is reported as requested.  Every answer still equals the oracle's."""
    def plan_of(re_src, x, c, tuning=None, offset=0):
        prog = lib.ridfa_compile(re_src)
        _, ser = oracle(re_src)
        base = torch.from_numpy(np.concatenate([np.zeros(16, np.uint8), x])).to("cuda:0")
        acc = lib.ridfa_recognize(prog, base[16 + offset:], x.size - offset, c, tuning=tuning)
        assert acc == ser.accepts(x[offset:])
        return lib.ridfa_last_plan(prog)

    p = plan_of(textgen.C3_RE, textgen.c3_text(1 << 20, seed=601), 1000)
    assert (p["table_mode"], p["text_path"], p["lane_copies"], p["pieces"]) == (2, 3, 0, 0), p
    re2 = textgen.C2_RE.replace("{20,60}", "{2,4}")
    p = plan_of(re2, textgen.c2_text(1 << 20, seed=602), 1000)
    assert (p["table_mode"], p["text_path"]) == (9, 5), p
    p = plan_of(textgen.regexp_family_re(9), textgen.regexp_family_text(1 << 20, seed=603), 4096)
    assert (p["table_mode"], p["text_path"]) == (11, 3) and p["lane_copies"] >= 2, p
    p = plan_of(textgen.regexp_family_re(7), textgen.regexp_family_text(1 << 20, seed=604), 4096)
    assert (p["table_mode"], p["text_path"], p["lane_copies"]) == (11, 3, 16), p
    p = plan_of(textgen.C3_RE, textgen.c3_text(1 << 20, seed=605), 1000, offset=3)
    assert p["text_path"] == 1, p
    p = plan_of(textgen.C3_RE, textgen.c3_text(1 << 20, seed=606), 1000, tuning=dict(table_mode=1))
    assert p["table_mode"] == 1, p
    p = plan_of(textgen.C3_RE, textgen.c3_text(1 << 20, seed=607), 4)
    assert p["pieces"] == 1, p
    with pytest.raises(lib.RidfaError) as e:             # no call on this device yet
        lib.ridfa_last_plan(lib.ridfa_compile(textgen.C1_RE))
    assert e.value.code == -1

"""GPU parity on large automata: seeded random REs of the batched and served workloads with
1,000-5,000 RI-DFA states over 45-50 byte classes (and more than 32 interface slots), whose tables
are too large for the compact shared-memory layouts: the reach kernel reads the flat table from
shared memory where it fits and from global memory where it does not.

Every chunk-map row of every run is compared with the oracle's lambda_i (Sec. 3.2: delta^B({q_a},
y_i) by position-set simulation), and the accept bit with the Thompson simulation, at chunk
counts 1, 7, 1,000 and n/64, for the automatic plan, each text path and table layout that
applies, pieces requested and refused, and an unaligned text.  A fourth RE of over 1,000 states
with at most 32 slots exercises the look-back pieces at that size.  The same REs then run in one
batch (``ridfa_batch_create``), accept bits against the Thompson simulation.
"""
import numpy as np
import pytest

import textgen
import textgen.batch as tb
from oracle.recognizer import RidOracle, SerialRecognizer
from tests.gpu_util import run, to_device

pytestmark = pytest.mark.gpu

lib = pytest.importorskip("paper_2412_14975_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

# (seed, draw index) in textgen.batch.random_re_candidates: the first REs of these seeds' draws
# with 1,000..5,000 RI-DFA states and at least 40 byte classes
LARGE = [(0x5EED10, 5), (0x5EED16, 307), (0x5EED16, 581)]
# 1,203 states, 14 slots: look-back start sets for the pieces of a long text in few chunks
LOOKBACK = (0x5EED04, 235)

_CACHE = {}


def workload_re(seed, idx):
    key = (seed, idx)
    if key not in _CACHE:
        r, body, alpha = tb.random_re_candidates(seed, idx + 1)[idx]
        _CACHE[key] = (r, body, alpha, RidOracle(r), SerialRecognizer(r))
    return _CACHE[key]


def member_text(r, body, alpha, n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    x = tb.pool_for(r, body, rng, n_members=400).text(rng, n)
    return np.ascontiguousarray(x)


def rows_equal(maps, want, c, tag):
    for i in range(c):
        assert np.array_equal(maps[i], want[i]), (tag, c, i, maps[i][:8], want[i][:8])


@pytest.mark.parametrize("which", range(len(LARGE)))
def test_large_automaton_every_row(which):
    r, body, alpha, o, ser = workload_re(*LARGE[which])
    prog = lib.ridfa_compile(r)
    info = prog.info
    assert 1000 <= info["n_states"] <= 5000 and info["n_classes"] >= 40 and info["k"] > 32
    # too large for the compact shared-memory layouts: the flat table, in shared memory when it
    # fits there (the second and third RE) and in global memory otherwise (the first)
    table = 2 * info["n_classes"] * (info["n_states"] + 1)
    assert table > 0xFFFF and (table > 227 * 1024) == (which == 0)
    x = member_text(r, body, alpha, 100_000, seed=which)
    m, _ = textgen.mutate(x, seed=100 + which, n_subs=1, alphabet=alpha)
    z = x.copy()
    z[x.size // 3] = 0x00                           # a byte no position reads
    for t, tag in ((x, "member"), (m, "mutated"), (z, "foreign")):
        n = t.size
        d = to_device(t)
        want_acc = ser.accepts(t)
        if tag == "member":
            assert want_acc
        if tag == "foreign":
            assert not want_acc
        for c in (1, 7, 1000, n // 64) if tag == "member" else (7, n // 64):
            want = o.lambda_rows(t, c)
            acc, maps = run(lib, prog, d, n, c)
            assert acc == want_acc, (tag, c)
            rows_equal(maps, want, c, tag)
            if tag == "member" and c in (7, 1000):
                variants = [dict(text_path=1), dict(text_path=3), dict(text_path=5),
                            dict(table_mode=5), dict(piece_len=256), dict(piece_len=1),
                            dict(probe_interval=3)]
                for tu in variants:
                    acc, maps = run(lib, prog, d, n, c, tuning=tu)
                    assert acc == want_acc, (tag, c, tu)
                    rows_equal(maps, want, c, (tag, tu))
        if tag == "member":
            # unaligned text (global loads) and the comparator where its states fit the slots
            base = to_device(np.concatenate([np.zeros(3, np.uint8), t]))
            want = o.lambda_rows(t, 1000)
            acc, maps = run(lib, prog, base[3:], n, 1000)
            assert acc == want_acc
            rows_equal(maps, want, 1000, "unaligned")
            if info["n_dfa_states"] <= lib.RIDFA_MAX_SLOTS:
                dwant = o.dfa_lambda_rows(t, 1000)
                dacc, dmaps = run(lib, prog, d, n, 1000, dfa=True)
                assert dacc == want_acc
                rows_equal(dmaps, dwant, 1000, "dfa")


def test_large_automaton_lookback_pieces():
    """Over 1,000 states with at most 32 slots: a long text in few chunks runs its pieces from
    look-back start sets; rows with pieces, without, and with a capped start set agree with the
    oracle."""
    r, body, alpha, o, ser = workload_re(*LOOKBACK)
    prog = lib.ridfa_compile(r)
    info = prog.info
    assert info["n_states"] > 1000 and info["k"] <= 32
    x = member_text(r, body, alpha, 600_000, seed=7)
    m, _ = textgen.mutate(x, seed=8, n_subs=1, alphabet=alpha)
    for t in (x, m):
        d = to_device(t)
        want_acc = ser.accepts(t)
        for c in (1, 3, 16):
            want = o.lambda_rows(t, c)
            for tu in (None, dict(piece_len=1), dict(piece_len=2048), dict(lookback_cap=4)):
                acc, maps = run(lib, prog, d, t.size, c, tuning=tu)
                assert acc == want_acc, (c, tu)
                rows_equal(maps, want, c, tu)


def test_large_automata_in_one_batch():
    """The four REs in one batch over texts of 0 B .. 200 KB, half mutated, aligned and not;
    accept bits against the Thompson simulation, planned and explicit chunk counts."""
    keys = LARGE + [LOOKBACK]
    res = [workload_re(*k) for k in keys]
    progs = [lib.ridfa_compile(r) for r, *_ in res]
    rng = np.random.Generator(np.random.PCG64(77))
    texts, meta = [], []
    for i in range(48):
        j = i % len(res)
        r, body, alpha, _, _ = res[j]
        n = int(rng.choice([0, 1, 100, 5000, 50_000, 200_000]))
        x = member_text(r, body, alpha, n, seed=1000 + i) if n else np.zeros(0, np.uint8)
        if n > 1 and i % 2:
            x, _ = textgen.mutate(x, seed=2000 + i, n_subs=1, alphabet=alpha)
        texts.append(np.ascontiguousarray(x, dtype=np.uint8))
        meta.append((j, int(rng.integers(1, min(n, 300) + 1)) if n and i % 5 == 0 else 0))
    offs, pos = [], 0
    for i, x in enumerate(texts):
        pos = ((pos + 15) & ~15) + (3 if i % 4 == 3 else 0)
        offs.append(pos)
        pos += x.size
    buf = np.zeros(max(pos, 16), np.uint8)
    for o_, x in zip(offs, texts):
        buf[o_:o_ + x.size] = x
    d = torch.from_numpy(buf).to("cuda:0")
    items = [(d.data_ptr() + o_, x.size, j, nc) for o_, x, (j, nc) in zip(offs, texts, meta)]
    want = np.array([res[j][4].accepts(x) for x, (j, _) in zip(texts, meta)])
    assert want.any() and not want.all()
    for chunk_len in (2048, 0):
        acc = torch.full((len(items),), 7, dtype=torch.uint8, device="cuda:0")
        b = lib.ridfa_batch_create(progs, items, acc, chunk_len=chunk_len)
        for _ in range(2):
            acc.fill_(7)
            lib.ridfa_batch_run(b)
            torch.cuda.synchronize()
            assert np.array_equal(acc.cpu().numpy().astype(bool), want), chunk_len
        b.close()

"""GPU served recognition: every request's accept bit equals the oracle's (Thompson simulation),
whether it ran alone or batched with others (continuous batching over several launch slots),
for host texts copied into the arena and device texts read in place; admission limits."""
import time

import numpy as np
import pytest

import textgen
from oracle.recognizer import SerialRecognizer

pytestmark = pytest.mark.gpu

lib = pytest.importorskip("paper_2412_14975_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

_XS, _YS = "ABCDEFGHIJKLMNOPQRSTUVWXYZ0123456789!#%&", "bcdefghijklmnopqrstuvwxyz<>=;:@$'\"^_`~,/"
RES = [textgen.C1_RE, textgen.C3_RE, textgen.C2_RE.replace("{20,60}", "{2,4}"), textgen.regexp_family_re(3),
       "(" + "|".join(f"{x}a*{y}" for x, y in zip(_XS, _YS)) + ")*"]


def make_text(r, n, rng):
    if r == 0:
        return textgen.c1_text(n, rng)[:n]
    if r == 1:
        return textgen.c3_text(n, rng)[:n]
    if r == 2:
        return textgen.c2_text(n, rng)
    if r == 3:
        return textgen.regexp_family_text(n, rng)
    parts, tot = [], 0
    while tot < n:
        i = int(rng.integers(len(_XS)))
        s = _XS[i] + "a" * int(rng.integers(0, 300)) + _YS[i]
        parts.append(s)
        tot += len(s)
    return np.frombuffer("".join(parts).encode(), dtype=np.uint8)[:n]


def workload(seed, n):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        r = i % len(RES)
        ln = int(rng.choice([0, 1, 17, 900, 5000, 40_000, 150_000]))
        x = make_text(r, ln, rng) if ln else np.zeros(0, np.uint8)
        if ln > 50 and rng.random() < 0.5:
            x, _ = textgen.mutate(x, rng, n_subs=1)
        out.append((r, np.ascontiguousarray(x, dtype=np.uint8)))
    return out


_SER = {}


def want(r, x):
    if r not in _SER:
        _SER[r] = SerialRecognizer(RES[r])
    return _SER[r].accepts(x)


def collect(srv, n, timeout=60.0):
    got = {}
    t0 = time.time()
    while len(got) < n and time.time() - t0 < timeout:
        for rid, st, acc, lat in srv.poll(wait_us=2000):
            assert st == 0, (rid, st)
            assert lat >= 0.0
            got[rid] = acc
    return got


def test_served_alone_and_in_the_mix():
    work = workload(5, 120)
    expect = [want(r, x) for r, x in work]
    progs = [lib.ridfa_compile(r) for r in RES]
    with lib.Server(n_streams=3, arena_bytes=8 << 20, max_batch_requests=40, chunk_len=4096) as srv:
        slots = [srv.add_program(p) for p in progs]
        # alone: one request at a time
        for (r, x), w in list(zip(work, expect))[:30]:
            rid = srv.submit(slots[r], x)
            srv.drain()
            res = srv.poll()
            assert [(a, b) for a, _, b, _ in res] == [(rid, w)]
        # in the mix: everything at once (retrying when the 8 MiB arena is full)
        ids = {}
        got = {}
        for j, (r, x) in enumerate(work):
            while True:
                rid = srv.try_submit(slots[r], x)
                if rid is not None:
                    break
                for a, st, acc, _ in srv.poll(wait_us=1000):
                    assert st == 0
                    got[a] = acc
            ids[rid] = j
        srv.drain()
        got.update(collect(srv, len(work) - len(got)))
        assert len(got) == len(work)
        for rid, j in ids.items():
            assert got[rid] == expect[j], (j, work[j][0], work[j][1].size)
        st = srv.stats()
        assert st["completed"] == 30 + len(work)
        assert st["max_batch"] > 1                 # requests did share batches
        assert st["n_programs"] == len(RES)


def test_served_device_texts_and_admission():
    work = workload(6, 40)
    progs = [lib.ridfa_compile(r) for r in RES]
    with lib.Server(n_streams=2, arena_bytes=1 << 20, max_requests=64, chunk_len=2048) as srv:
        slots = [srv.add_program(p) for p in progs]
        # device texts, read in place, some of them unaligned
        base = torch.zeros(sum(x.size + 21 for _, x in work) + 16, dtype=torch.uint8, device="cuda:0")
        pos, ids = 0, {}
        for j, (r, x) in enumerate(work):
            pos += 5 if j % 3 == 1 else 0
            if x.size:
                base[pos:pos + x.size] = torch.from_numpy(x).to("cuda:0")
            ids[srv.submit(slots[r], base.data_ptr() + pos, length=x.size, device=True)] = j
            pos = (pos + x.size + 15) & ~15
        torch.cuda.synchronize()
        srv.drain()
        got = collect(srv, len(work))
        for rid, j in ids.items():
            assert got[rid] == want(*work[j])
        # a host text larger than the 1 MiB arena cannot be admitted at all
        with pytest.raises(lib.RidfaError) as e:
            srv.submit(slots[1], np.zeros((1 << 20) + 1, np.uint8))
        assert e.value.code == -12
        with pytest.raises(lib.RidfaError) as e:
            srv.submit(len(RES), b"ACGT")
        assert e.value.code == -1
        # the request budget: 64 admitted and unpolled at most
        x = np.frombuffer(b"AGTC" * 4, dtype=np.uint8)
        n_ok = 0
        while srv.try_submit(slots[0], x) is not None:
            n_ok += 1
            assert n_ok <= 64
        assert n_ok == 64
        srv.drain()
        got = collect(srv, 64)
        assert len(got) == 64 and all(got.values())
        assert srv.try_submit(slots[0], x) is not None     # room again after polling
        srv.drain()
        assert len(collect(srv, 1)) == 1


def test_served_device_budget_counts_tables_and_texts():
    """Admission by device memory: resident tables are charged to the budget for the server's
    life; a request is charged its arena text plus its kernels' scratch until its result is
    posted.  Tables that fill the budget leave no room for texts; a program that does not fit
    is refused; charges come back when results are polled."""
    progs = [lib.ridfa_compile(r) for r in RES]
    tb = [p.info["table_bytes"] for p in progs]
    x = np.ascontiguousarray(make_text(1, 8192, np.random.Generator(np.random.PCG64(3))))
    # a request of the record-line RE: its 16-byte-rounded text plus 2k + 4 bytes per 1 KiB chunk
    k1 = progs[1].info["k"]
    charge = ((x.size + 15) & ~15) + ((x.size + 1023) // 1024) * (2 * k1 + 4) + 64
    budget = sum(tb) + 3 * charge + charge // 2          # room for three such requests in flight
    with lib.Server(n_streams=1, arena_bytes=1 << 20, chunk_len=1024, device_budget=budget) as srv:
        slots = [srv.add_program(p) for p in progs]
        st = srv.stats()
        assert st["table_bytes"] == sum(tb) and st["budget_used"] == sum(tb)
        # texts until the budget refuses; at most three fit (the arena alone would take ~120)
        admitted = []
        while True:
            rid = srv.try_submit(slots[1], x)
            if rid is None:
                break
            admitted.append(rid)
            assert len(admitted) <= 3
        assert 1 <= len(admitted) <= 3
        assert srv.stats()["budget_used"] <= budget
        srv.drain()
        got = collect(srv, len(admitted))
        assert set(got) == set(admitted) and all(v == want(1, x) for v in got.values())
        st = srv.stats()
        assert st["budget_used"] == sum(tb) and st["budget_peak"] <= budget
        assert srv.try_submit(slots[1], x) is not None    # the charges came back
        srv.drain()
        collect(srv, 1)
        # a text whose charge exceeds what the tables leave can never be admitted
        with pytest.raises(lib.RidfaError) as e:
            srv.submit(slots[1], np.zeros(4 * charge, np.uint8))
        assert e.value.code == -12
    # tables alone fill a budget: no further program fits and no text is admitted at all
    with lib.Server(n_streams=1, arena_bytes=1 << 20, device_budget=sum(tb)) as srv:
        slots = [srv.add_program(p) for p in progs]
        with pytest.raises(lib.RidfaError) as e:
            srv.add_program(lib.ridfa_compile("(ab|c)*"))
        assert e.value.code == -8
        assert srv.stats()["n_programs"] == len(progs)
        with pytest.raises(lib.RidfaError) as e:
            srv.submit(slots[0], b"ACGT")
        assert e.value.code == -12


def test_served_poisson_load_generator():
    """The C load generator: every request of an open-loop Poisson run gets a result equal to the
    oracle's, batches form (histogram), and latencies are at least the server's own."""
    work = [(r, x) for r, x in workload(8, 60) if x.size]
    expect = np.array([want(r, x) for r, x in work])
    progs = [lib.ridfa_compile(r) for r in RES]
    with lib.Server(n_streams=3, arena_bytes=64 << 20) as srv:
        slots = [srv.add_program(p) for p in progs]
        recs, wall = srv.bench_poisson([slots[r] for r, _ in work], [x for _, x in work],
                                       rate_rps=20000, seconds=0.5, seed=11)
        assert 8000 <= len(recs) <= 12000 and wall >= 0.45
        assert (recs["status"] == 0).all()
        assert np.array_equal(recs["accept"].astype(bool), expect[recs["text"]])
        assert (recs["latency_us"] >= recs["server_us"] - 1.0).all()
        st = srv.stats()
        assert st["completed"] == len(recs)
        assert sum(st["batch_hist"]) == st["batches"] and sum(st["batch_hist"][1:]) > 0


def test_served_poisson_device_texts():
    """The load generator on device-resident texts (submitted in place, no arena copy): every
    request of an open-loop run gets a result equal to the oracle's."""
    work = [(r, x) for r, x in workload(8, 61) if x.size]
    expect = np.array([want(r, x) for r, x in work])
    progs = [lib.ridfa_compile(r) for r in RES]
    offs, pos = [], 0
    for _, x in work:
        offs.append(pos)
        pos = (pos + x.size + 15) & ~15
    buf = np.zeros(max(pos, 16), np.uint8)
    for o, (_, x) in zip(offs, work):
        buf[o:o + x.size] = x
    d = torch.from_numpy(buf).to("cuda:0")
    dev = [(d.data_ptr() + o, x.size) for o, (_, x) in zip(offs, work)]
    with lib.Server(n_streams=3, arena_bytes=1 << 20) as srv:
        slots = [srv.add_program(p) for p in progs]
        recs, wall = srv.bench_poisson([slots[r] for r, _ in work], None, rate_rps=50000, seconds=0.4,
                                       seed=12, device_texts=dev)
        assert 16000 <= len(recs) <= 24000
        assert (recs["status"] == 0).all()
        assert np.array_equal(recs["accept"].astype(bool), expect[recs["text"]])
        assert srv.stats()["completed"] == len(recs)

"""Sharded recognition on the host side (no GPU): shard summaries evaluated with the oracle and
composed by the library's ridfa_join_shards give the oracle's accept bit for every split of the
text into shards, including the exchange of summaries between two gloo ranks on CPU."""
import os

import numpy as np
import pytest

import textgen
from oracle.recognizer import RidOracle, SerialRecognizer
from tests.shard_util import oracle_summary, split_points

lib = pytest.importorskip("paper_2412_14975_gb300")
torch = pytest.importorskip("torch")

CASES = [("c1", textgen.C1_RE), ("c3", textgen.C3_RE), ("c2_2_4", textgen.C2_RE.replace("{20,60}", "{2,4}")),
         ("regexp3", textgen.regexp_family_re(3))]


def text_for(name, n, rng):
    if name == "c1":
        return textgen.c1_text(n, rng)[:n]
    if name == "c3":
        return textgen.c3_text(n, rng)[:n]
    if name == "c2_2_4":
        return textgen.c2_text(n, rng)
    return textgen.regexp_family_text(n, rng)


@pytest.mark.parametrize("name,re_src", CASES)
def test_join_of_oracle_summaries_equals_whole_text(name, re_src):
    rng = np.random.Generator(np.random.PCG64(sum(map(ord, name)) + 3))
    o = RidOracle(re_src, with_dfa=False)
    ser = SerialRecognizer(re_src)
    prog = lib.ridfa_compile(re_src, build_dfa=False)
    for trial in range(6):
        n = int(rng.integers(40, 2500))
        x = text_for(name, n, rng)
        if trial % 2:
            x, _ = textgen.mutate(x, rng, n_subs=1)
        want = ser.accepts(x)
        for n_shards in (1, 2, 3, 5):
            cuts = split_points(x.size, n_shards, rng)
            sums = []
            for s0, s1 in zip(cuts[:-1], cuts[1:]):
                c = int(rng.integers(1, min(s1 - s0, 9) + 1))
                sums.append(oracle_summary(o.B, x[s0:s1], c))
            assert lib.ridfa_join_shards(prog, sums) == want, (name, trial, n_shards)


def test_join_shards_errors():
    prog = lib.ridfa_compile("(ab)*", build_dfa=False)
    other = lib.ridfa_compile(textgen.C3_RE, build_dfa=False)
    o = RidOracle(textgen.C3_RE, with_dfa=False)
    s = oracle_summary(o.B, b"2024-01-02T03:04:05,1,2.5,abc,1.2.3.4\n", 3)
    with pytest.raises(lib.RidfaError) as e:
        lib.ridfa_join_shards(prog, [s])          # a summary of another program (k differs)
    assert e.value.code == -1
    assert lib.ridfa_join_shards(other, [s]) is True


def _rank_main(rank, world, port, re_src, text, cuts, chunks, want, out_q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        o = RidOracle(re_src, with_dfa=False)
        prog = lib.ridfa_compile(re_src, build_dfa=False)
        mine = oracle_summary(o.B, text[cuts[rank]:cuts[rank + 1]], chunks[rank])
        buf = torch.frombuffer(bytearray(mine.to_bytes()), dtype=torch.uint8)
        bufs = [torch.empty_like(buf) for _ in range(world)]
        dist.all_gather(bufs, buf)                # the one exchange: a few KB per shard
        sums = [lib.ShardSummary.from_bytes(b.numpy().tobytes()) for b in bufs]
        out_q.put((rank, lib.ridfa_join_shards(prog, sums) == want))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_gloo_ranks_exchange_summaries(world):
    import socket

    import torch.multiprocessing as mp
    rng = np.random.Generator(np.random.PCG64(77))
    re_src = textgen.C3_RE
    x = textgen.c3_text(6000, rng)
    y, _ = textgen.mutate(x, rng, n_subs=1)
    for text in (x, y):
        want = SerialRecognizer(re_src).accepts(text)
        cuts = split_points(text.size, world, rng)
        chunks = [int(rng.integers(1, 7)) for _ in range(world)]
        with socket.socket() as s:
            s.bind(("127.0.0.1", 0))
            port = s.getsockname()[1]
        ctx = mp.get_context("spawn")
        q = ctx.Queue()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, re_src, bytes(text), cuts, chunks, want, q))
                 for r in range(world)]
        for p in procs:
            p.start()
        res = [q.get(timeout=120) for _ in range(world)]
        for p in procs:
            p.join(timeout=60)
            assert p.exitcode == 0
        assert sorted(res) == [(r, True) for r in range(world)]


def _rank_dies_main(rank, world, port, out_q):
    import datetime

    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(3)                               # this rank dies before the exchange
    buf = torch.zeros(16, dtype=torch.uint8)
    try:
        dist.all_gather([torch.empty_like(buf) for _ in range(world)], buf)
        out_q.put((rank, "completed"))
    except Exception as e:                        # the survivor learns of it from the collective
        out_q.put((rank, "error:" + type(e).__name__))


def test_gloo_rank_that_dies_fails_the_exchange():
    """A shard rank that dies before the summary exchange makes the survivor's all-gather fail with
    an error (closed connection or the short process-group timeout) instead of hanging."""
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_dies_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    rank, what = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert rank == 0 and what.startswith("error:"), what
    assert procs[1].exitcode == 3

"""GPU sharded recognition: each shard's relation summary from ridfa_recognize_shard equals the
one evaluated with the oracle, field by field, and composing the summaries of any split of a text
(several virtual shards on one GPU, summaries joined through host memory) gives the oracle's
accept bit -- for matrix-join shards and for shards with more than 32 distinct end states."""
import numpy as np
import pytest

import textgen
from oracle.recognizer import RidOracle, SerialRecognizer
from tests.shard_util import oracle_summary, split_points, summaries_equal
from tests.gpu_util import to_device

pytestmark = pytest.mark.gpu

lib = pytest.importorskip("paper_2412_14975_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

XS, YS = "ABCDEFGHIJKLMNOPQRSTUVWXYZ0123456789!#%&", "bcdefghijklmnopqrstuvwxyz<>=;:@$'\"^_`~,/"


def branches(nb, rng, n_parts=30):
    re_src = "(" + "|".join(f"{XS[i]}a*{YS[i]}" for i in range(nb)) + ")*"
    parts = []
    for _ in range(n_parts):
        i = int(rng.integers(nb))
        parts.append(XS[i] + "a" * int(rng.integers(0, 300)) + YS[i])
    return re_src, np.frombuffer("".join(parts).encode(), dtype=np.uint8)


def cases(rng):
    yield textgen.C1_RE, textgen.c1_text(20_000, rng)
    yield textgen.C3_RE, textgen.c3_text(30_000, rng)
    yield textgen.C2_RE.replace("{20,60}", "{2,4}"), textgen.c2_text(20_000, rng)
    yield textgen.regexp_family_re(3), textgen.regexp_family_text(20_000, rng)
    for nb in (5, 40):                            # 40 branches: chunks with > 32 end states
        yield branches(nb, rng)


def test_shard_summaries_and_join():
    rng = np.random.Generator(np.random.PCG64(2024))
    for re_src, x in cases(rng):
        o = RidOracle(re_src, with_dfa=False)
        ser = SerialRecognizer(re_src)
        prog = lib.ridfa_compile(re_src, build_dfa=False)
        for trial in range(4):
            y = x
            if trial % 2:
                y, _ = textgen.mutate(x, rng, n_subs=1)
            want = ser.accepts(y)
            d = to_device(y)
            n_shards = 1 + trial
            cuts = split_points(y.size, n_shards, rng)
            sums = []
            for s0, s1 in zip(cuts[:-1], cuts[1:]):
                c = int(rng.integers(1, min(s1 - s0, 300) + 1))
                got = lib.ridfa_recognize_shard(prog, d.data_ptr() + s0, s1 - s0, c)
                ref = oracle_summary(o.B, y[s0:s1], c)
                assert summaries_equal(got, ref), (re_src[:40], trial, s0, s1, c)
                sums.append(got)
            assert lib.ridfa_join_shards(prog, sums) == want, (re_src[:40], trial)
            # a single shard spanning the text agrees with ridfa_recognize
            c = min(y.size, 257)
            whole = lib.ridfa_recognize_shard(prog, d, y.size, c)
            assert lib.ridfa_join_shards(prog, [whole]) == lib.ridfa_recognize(prog, d, y.size, c) == want

"""Shard summaries built from the oracle (test infrastructure): the relation a run of whole
chunks realises under the join of Sec. 3.2, evaluated with the oracle's RI-DFA."""
import numpy as np

import paper_2412_14975_gb300 as lib
from oracle.ridfa_sets import UNDEF, chunk_boundaries, chunk_mapping

UNDEF16 = 0xFFFF


def oracle_summary(B, shard, c):
    """ShardSummary of `shard` (bytes / uint8 array) cut into c chunks, from oracle B."""
    shard = bytes(shard) if isinstance(shard, (bytes, bytearray)) else bytes(np.asarray(shard, dtype=np.uint8))
    b = chunk_boundaries(len(shard), c)
    maps = [chunk_mapping(B, shard[b[i]:b[i + 1]]) for i in range(c)]
    out = sorted({v for v in maps[-1] if v is not UNDEF})
    pos = {v: y for y, v in enumerate(out)}
    s = lib.ShardSummary()
    s.k = B.k
    s.n_out = len(out)
    for a in range(lib.RIDFA_MAX_SLOTS):
        s.out_state[a] = out[a] if a < len(out) else UNDEF16
        s.entry[a] = UNDEF16
        for w in range(lib.RIDFA_MAX_SLOTS // 32):
            s.reach[a][w] = 0
    for a in range(B.k):
        x = maps[0][a]
        if x is UNDEF:
            continue
        s.entry[a] = x
        plas = {x}
        for lam in maps[1:]:
            pis = {j for j, p in enumerate(lam) if p is not UNDEF}
            plas = {lam[j] for j in (B.interface(plas) & pis)}
        for v in plas:
            y = pos[v]
            s.reach[a][y // 32] |= 1 << (y % 32)
    return s


def split_points(n, n_shards, rng):
    """n_shards - 1 distinct cut points in (0, n): every shard non-empty."""
    cuts = np.sort(rng.choice(np.arange(1, n), size=n_shards - 1, replace=False)) if n_shards > 1 else []
    return [0] + [int(x) for x in cuts] + [n]


def summaries_equal(a, b):
    if a.k != b.k or a.n_out != b.n_out:
        return False
    ka = a.k
    return (list(a.entry[:ka]) == list(b.entry[:ka]) and list(a.out_state[:a.n_out]) == list(b.out_state[:b.n_out])
            and all(list(a.reach[r]) == list(b.reach[r]) for r in range(ka)))

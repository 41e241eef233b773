"""Seeded workload of the batched configuration: many texts against many REs.

Recipe (the configuration names the sizes; the rest is a stated reading):
  * REs: the three single-text REs (the DNA-motif one with the {2,4} codon repeat) plus random REs
    over alphabets of 4-64 symbols (bytes 0x21 upward), depth 6, union / concatenation / star /
    bounded repeat, each wrapped as (R)* so that arbitrarily long members exist.  The caller keeps
    the candidates whose compiled size is in range (the filter needs a compiler, which this module
    does not import).
  * lengths: lognormal, median 256 KiB, sigma 1.0, clipped to [1 KiB, 64 MiB]; text j uses RE
    j mod (number of REs).
  * positives: concatenations of random members of the RE's starred body, drawn from a pool of
    members sampled from the syntax tree (the record-line RE: whole record lines; the DNA RE:
    i.i.d. ACGT); a text is the shortest prefix of whole members reaching its target length.
  * negatives: half of the texts get one substitution at a uniform position, the byte uniform over
    the RE's alphabet minus the original.  Labels always come from a recognizer, never from here.
"""

import numpy as np

from .regex_ast import Alt, Cat, Plus, Star, Sym, random_re, render, sample_member
from .texts import C1_RE, C2_RE, C3_RE, c3_text


def _rng(seed):
    return seed if isinstance(seed, np.random.Generator) else np.random.Generator(np.random.PCG64(seed))


def c1_body():
    """Syntax tree of the starred body of ((A|C)*G(T|A)+C)*."""
    A, C, G, T = (Sym([ord(ch)]) for ch in "ACGT")
    return Cat(Star(Alt(A, C)), G, Plus(Alt(T, A)), C)


def random_re_candidates(seed, count, depth=6):
    """Random (R)* REs with their bodies and alphabets, in the order drawn."""
    rng = _rng(seed)
    out = []
    for _ in range(count):
        size = int(rng.integers(4, 65))
        alphabet = list(range(0x21, 0x21 + size))
        node = random_re(rng, alphabet, depth=depth)
        out.append(("(" + render(node) + ")*", node, bytes(alphabet)))
    return out


def lognormal_lengths(rng, n, median=256 << 10, sigma=1.0, lo=1 << 10, hi=64 << 20):
    x = np.exp(rng.normal(np.log(median), sigma, size=n))
    return np.clip(x, lo, hi).astype(np.int64)


class MemberPool:
    """A pool of members of a starred body, concatenated, for fast text assembly."""

    def __init__(self, members):
        members = [m for m in members if len(m) > 0]
        if not members:
            raise ValueError("empty pool")
        self.lens = np.array([len(m) for m in members], dtype=np.int64)
        self.offs = np.concatenate([[0], np.cumsum(self.lens)[:-1]])
        self.bytes = np.frombuffer(b"".join(members), dtype=np.uint8)

    def text(self, rng, target):
        """Shortest concatenation of random pool members with length >= target."""
        mean = float(self.lens.mean())
        parts = []
        total = 0
        while total < target:
            k = max(16, int((target - total) / mean * 1.2) + 8)
            idx = rng.integers(0, self.lens.size, size=k)
            ls = self.lens[idx]
            cs = np.cumsum(ls)
            cut = int(np.searchsorted(cs, target - total, side="left")) + 1
            idx, ls = idx[:cut], ls[:cut]
            starts = self.offs[idx]
            rel = np.arange(int(ls.sum())) - np.repeat(np.cumsum(ls) - ls, ls)
            parts.append(self.bytes[np.repeat(starts, ls) + rel])
            total += int(ls.sum())
        return np.concatenate(parts) if len(parts) > 1 else parts[0]


def pool_for(re_src, body, rng, n_members=2000, soft_len=64):
    if re_src == C3_RE:
        x = c3_text(1 << 20, rng)
        nl = np.nonzero(x == 10)[0]
        starts = np.concatenate([[0], nl[:-1] + 1])
        return MemberPool([bytes(x[s:e + 1]) for s, e in zip(starts[:n_members], nl[:n_members])])
    if body is None:     # i.i.d. alphabet (the DNA-motif language {A,C,G,T}*)
        return MemberPool([bytes([b]) for b in b"ACGT"])
    return MemberPool([sample_member(body, rng, soft_len=soft_len) for _ in range(n_members)])


def batch_texts(res_bodies, n_texts, seed, median=256 << 10, sigma=1.0):
    """Yields (index, RE index, text uint8 array, mutated flag) for the batched workload.

    res_bodies: list of (re_src, body syntax tree or None, alphabet bytes)."""
    rng = _rng(seed)
    lengths = lognormal_lengths(rng, n_texts, median=median, sigma=sigma)
    pools = [pool_for(r, b, rng) for r, b, _ in res_bodies]
    for j in range(n_texts):
        r = j % len(res_bodies)
        x = pools[r].text(rng, int(lengths[j]))
        mutated = bool(j % 2)
        if mutated:
            alpha = np.frombuffer(res_bodies[r][2], dtype=np.uint8)
            p = int(rng.integers(0, x.size))
            cand = alpha[alpha != x[p]]
            x = x.copy()
            x[p] = cand[int(rng.integers(cand.size))]
        yield j, r, x, mutated


def standard_res():
    """The three single-text REs with their starred bodies (or None for i.i.d.) and alphabets."""
    return [(C1_RE, c1_body(), b"ACGT"),
            (C2_RE.replace("{20,60}", "{2,4}"), None, b"ACGT"),
            (C3_RE, None, b"0123456789-T:,.abcdefghijklmnopqrstuvwxyz\n")]

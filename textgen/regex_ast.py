"""A tiny RE syntax tree used only to *generate* REs and sample members of them.

Rendering produces the byte dialect accepted by the recognizer (literals, ``[...]`` classes,
``( )``, ``| * + ? {m,n}``); bytes that are metacharacters or non-printable are written as
``\\xHH``.
"""

import numpy as np

_META = set(b"|*+?{}()[]\\.^-")


def _lit(b):
    if 0x21 <= b <= 0x7E and b not in _META:
        return chr(b)
    return "\\x%02x" % b


class Sym:
    def __init__(self, byteset):
        self.bytes = sorted(set(byteset))

    def render(self):
        if len(self.bytes) == 1:
            return _lit(self.bytes[0])
        out, i, bs = [], 0, self.bytes
        while i < len(bs):
            j = i
            while j + 1 < len(bs) and bs[j + 1] == bs[j] + 1:
                j += 1
            out.append(_lit(bs[i]) if j == i else (_lit(bs[i]) + (_lit(bs[j]) if j == i + 1
                                                                    else "-" + _lit(bs[j]))))
            i = j + 1
        return "[" + "".join(out) + "]"

    def sample(self, rng, out, budget):
        out.append(self.bytes[rng.integers(len(self.bytes))])


class Cat:
    def __init__(self, *items):
        self.items = items

    def render(self):
        return "".join(_wrap(i, for_cat=True) for i in self.items)

    def sample(self, rng, out, budget):
        for i in self.items:
            i.sample(rng, out, budget)


class Alt:
    def __init__(self, *items):
        self.items = items

    def render(self):
        return "|".join(i.render() for i in self.items)

    def sample(self, rng, out, budget):
        self.items[rng.integers(len(self.items))].sample(rng, out, budget)


class _Post:
    op = ""

    def __init__(self, item):
        self.item = item

    def render(self):
        return _wrap(self.item, for_cat=False) + self.op


class Star(_Post):
    op = "*"

    def sample(self, rng, out, budget):
        while len(out) < budget[0] and rng.random() < budget[1]:
            self.item.sample(rng, out, budget)


class Plus(_Post):
    op = "+"

    def sample(self, rng, out, budget):
        self.item.sample(rng, out, budget)
        while len(out) < budget[0] and rng.random() < budget[1]:
            self.item.sample(rng, out, budget)


class Opt(_Post):
    op = "?"

    def sample(self, rng, out, budget):
        if rng.random() < 0.5:
            self.item.sample(rng, out, budget)


class Rep(_Post):
    def __init__(self, item, lo, hi):
        super().__init__(item)
        self.lo, self.hi = lo, hi
        self.op = "{%d}" % lo if lo == hi else "{%d,%d}" % (lo, hi)

    def sample(self, rng, out, budget):
        for _ in range(int(rng.integers(self.lo, self.hi + 1))):
            self.item.sample(rng, out, budget)


def _wrap(node, for_cat):
    s = node.render()
    if isinstance(node, Sym):
        return s
    if isinstance(node, Alt) or (not for_cat and isinstance(node, (Cat, _Post))):
        return "(" + s + ")"
    return s


def render(node) -> str:
    return node.render()


def sample_member(node, rng, soft_len=64, p_repeat=0.6) -> bytes:
    """A random member of L(node): alternatives uniform, ``?`` with probability 1/2, bounded
    repeats uniform in count, ``*``/``+`` repeat with probability ``p_repeat`` while the output
    is shorter than ``soft_len``."""
    out = []
    node.sample(rng, out, (soft_len, p_repeat))
    return bytes(out)


def random_re(rng, alphabet, depth, max_lo=3, max_span=5, leaf_class_p=0.3, star_p=0.25):
    """A random RE over ``alphabet`` (bytes): union, concatenation, star and bounded repeat
    {m,n} with m in [0, max_lo], n in [m, m + max_span]; leaves are a symbol or a class."""
    alphabet = list(alphabet)

    def leaf():
        if len(alphabet) > 1 and rng.random() < leaf_class_p:
            k = int(rng.integers(2, min(len(alphabet), 4) + 1))
            return Sym(rng.choice(alphabet, size=k, replace=False).tolist())
        return Sym([alphabet[rng.integers(len(alphabet))]])

    def gen(d):
        if d <= 0 or rng.random() < 0.2:
            return leaf()
        r = rng.random()
        if r < 0.35:
            return Cat(*[gen(d - 1) for _ in range(int(rng.integers(2, 4)))])
        if r < 0.6:
            return Alt(*[gen(d - 1) for _ in range(int(rng.integers(2, 4)))])
        if r < 0.6 + star_p:
            return Star(gen(d - 1))
        lo = int(rng.integers(0, max_lo + 1))
        hi = lo + int(rng.integers(0, max_span + 1))
        if hi == 0:
            hi = 1
        return Rep(gen(d - 1), lo, hi)

    return gen(depth)

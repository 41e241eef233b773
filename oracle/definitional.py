"""Oracle definitional matcher for tiny strings (brute-force pins).

Test infrastructure only (see ``oracle/__init__.py``).

Decides s[i:j] in L(node) straight from the language of each RE operator, on the UNEXPANDED
syntax tree (so it does not depend on the bounded-repeat expansion convention):
  L(eps) = {""}, L(set) = its bytes, L(r1 r2) = L(r1) L(r2), L(r1|r2) = L(r1) u L(r2),
  L(r*) = {""} u L(r) L(r*) (split into a non-empty first piece), L(r+) = L(r) L(r*),
  L(r?) = {""} u L(r), L(r{m,n}) = U_{t=m..n} L(r)^t, L(r{m,}) = L(r)^m L(r*).
Exponential in the worst case; used only for strings of length <= 10 or so.
"""

from . import re_syntax


class DefinitionalMatcher:
    def __init__(self, re_src):
        self.ast = re_syntax.parse(re_src)

    def match(self, s: bytes) -> bool:
        self.s = bytes(s)
        self.memo = {}
        return self._m(self.ast, 0, len(self.s))

    def _m(self, node, i, j):
        key = (id(node), i, j)
        hit = self.memo.get(key)
        if hit is not None:
            return hit
        self.memo[key] = False          # guards the (impossible) left recursion on equal spans
        r = self._compute(node, i, j)
        self.memo[key] = r
        return r

    def _compute(self, node, i, j):
        kind = node[0]
        if kind == 'eps':
            return i == j
        if kind == 'set':
            return j == i + 1 and self.s[i] in node[1]
        if kind == 'alt':
            return any(self._m(c, i, j) for c in node[1])
        if kind == 'cat':
            return self._cat(node[1], 0, i, j)
        if kind == 'star':
            return i == j or self._star_nonempty(node[1], i, j)
        if kind == 'plus':
            return any(self._m(node[1], i, m) and (m == j or self._star_nonempty(node[1], m, j))
                       for m in range(i, j + 1))
        if kind == 'opt':
            return i == j or self._m(node[1], i, j)
        if kind == 'rep':
            r, lo, hi = node[1], node[2], node[3]
            if hi is None:
                return any(self._pow(r, lo, i, m) and (m == j or self._star_nonempty(r, m, j))
                           for m in range(i, j + 1))
            return any(self._pow(r, t, i, j) for t in range(lo, hi + 1))
        raise ValueError(kind)

    def _cat(self, children, idx, i, j):
        key = ('cat', id(children), idx, i, j)
        if key in self.memo:
            return self.memo[key]
        if idx == len(children):
            r = i == j
        else:
            r = any(self._m(children[idx], i, m) and self._cat(children, idx + 1, m, j)
                    for m in range(i, j + 1))
        self.memo[key] = r
        return r

    def _star_nonempty(self, r, i, j):
        """s[i:j] (i < j) splits into non-empty pieces of L(r)."""
        key = ('star+', id(r), i, j)
        if key in self.memo:
            return self.memo[key]
        res = any(self._m(r, i, m) and (m == j or self._star_nonempty(r, m, j))
                  for m in range(i + 1, j + 1))
        self.memo[key] = res
        return res

    def _pow(self, r, t, i, j):
        key = ('pow', id(r), t, i, j)
        if key in self.memo:
            return self.memo[key]
        if t == 0:
            res = i == j
        else:
            res = any(self._m(r, i, m) and self._pow(r, t - 1, m, j) for m in range(i, j + 1))
        self.memo[key] = res
        return res


def all_words(alphabet, n):
    """All words of length n over alphabet, as an (|alphabet|^n, n) uint8 array in
    lexicographic order."""
    import numpy as np
    alpha = np.asarray(sorted(alphabet), dtype=np.uint8)
    m = len(alpha)
    idx = np.indices((m,) * n).reshape(n, -1).T if n else np.zeros((1, 0), dtype=np.int64)
    return alpha[idx].astype(np.uint8)


class SpanLanguage:
    """The same operator definitions as DefinitionalMatcher, evaluated for many words at once.

    For words W (shape (m, n)) and every AST node, R[i] is an (m,) int array whose bit j says
    W[:, i:j] is in L(node) (0 <= i <= j <= n); acceptance of W is bit n of R[0] at the root.
    """

    def __init__(self, re_src):
        self.ast = re_syntax.parse(re_src)

    def accepts(self, words):
        import numpy as np
        self.w = np.asarray(words, dtype=np.uint8)
        self.m, self.n = self.w.shape
        R = self._eval(self.ast)
        return ((R[0] >> self.n) & 1).astype(bool)

    def _zero(self):
        import numpy as np
        return [np.zeros(self.m, dtype=np.int64) for _ in range(self.n + 1)]

    def _compose(self, A, B):
        """L(A) L(B): bit j of out[i] iff exists k: bit k of A[i] and bit j of B[k]."""
        import numpy as np
        out = self._zero()
        for i in range(self.n + 1):
            acc = np.zeros(self.m, dtype=np.int64)
            for k in range(i, self.n + 1):
                has = ((A[i] >> k) & 1).astype(bool)
                if has.any():
                    acc = np.where(has, acc | B[k], acc)
            out[i] = acc
        return out

    def _eps(self):
        import numpy as np
        return [np.full(self.m, 1 << i, dtype=np.int64) for i in range(self.n + 1)]

    def _star(self, A):
        """L(A*) = {""} u L(A) L(A*), with a non-empty first piece (i < k)."""
        import numpy as np
        out = self._zero()
        for i in range(self.n, -1, -1):
            acc = np.full(self.m, 1 << i, dtype=np.int64)
            for k in range(i + 1, self.n + 1):
                has = ((A[i] >> k) & 1).astype(bool)
                if has.any():
                    acc = np.where(has, acc | out[k], acc)
            out[i] = acc
        return out

    def _eval(self, node):
        import numpy as np
        kind = node[0]
        if kind == 'eps':
            return self._eps()
        if kind == 'set':
            mem = np.zeros(256, dtype=bool)
            mem[list(node[1])] = True
            out = self._zero()
            for i in range(self.n):
                out[i] = np.where(mem[self.w[:, i]], 1 << (i + 1), 0).astype(np.int64)
            return out
        if kind == 'alt':
            parts = [self._eval(c) for c in node[1]]
            return [np.bitwise_or.reduce([p[i] for p in parts]) for i in range(self.n + 1)]
        if kind == 'cat':
            acc = self._eps()
            for c in node[1]:
                acc = self._compose(acc, self._eval(c))
            return acc
        if kind == 'star':
            return self._star(self._eval(node[1]))
        if kind == 'plus':
            A = self._eval(node[1])
            return self._compose(A, self._star(A))
        if kind == 'opt':
            A = self._eval(node[1])
            e = self._eps()
            return [A[i] | e[i] for i in range(self.n + 1)]
        if kind == 'rep':
            A = self._eval(node[1])
            lo, hi = node[2], node[3]
            power = self._eps()
            for _ in range(lo):
                power = self._compose(power, A)
            if hi is None:
                return self._compose(power, self._star(A))
            out = [p.copy() for p in power]
            for _ in range(hi - lo):
                power = self._compose(power, A)
                out = [out[i] | power[i] for i in range(self.n + 1)]
            return out
        raise ValueError(kind)

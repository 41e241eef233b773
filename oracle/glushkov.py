"""Oracle position automaton (McNaughton-Yamada / Glushkov) -- the source NFA N of the RID.

Test infrastructure only (see ``oracle/__init__.py``).

The paper builds the chunk automaton from an NFA N = (Q_N, Sigma, rho, q0, F) with
Q_N = {q0, ..., q_{l-1}} (Sec. 3.1) and obtains N from an RE by the McNaughton-Yamada method
(Sec. 4.1; Sec. 5 calls it GMY).  Here:

* every symbol occurrence of the expanded RE (``re_syntax.expand``) is a position; positions are
  numbered 1, 2, ... in left-to-right order of the expanded RE, and state 0 is q0;
* rho(0, b) = {p in First : b in sym(p)},  rho(p, b) = {p' in Follow(p) : b in sym(p')};
* F = Last, plus q0 when the RE is nullable.

The result is an ``NFA`` object (``ridfa_sets.NFA``) so that the paper's RI-DFA construction can
run on it exactly as on the hand-drawn NFAs of Fig. 1 and Fig. 5.
"""

from . import re_syntax
from .ridfa_sets import NFA


class Positions:
    """First/Last/Follow sets of an expanded AST (textbook definitions)."""

    def __init__(self, ast):
        self.sym = [None]          # sym[p] = frozenset of bytes of position p; index 0 = q0
        self.follow = [set()]
        self.nullable, self.first, self.last = self._walk(ast)

    def _new(self, byteset):
        self.sym.append(frozenset(byteset))
        self.follow.append(set())
        return len(self.sym) - 1

    def _walk(self, node):
        kind = node[0]
        if kind == 'eps':
            return True, set(), set()
        if kind == 'set':
            p = self._new(node[1])
            return False, {p}, {p}
        if kind == 'cat':
            nullable, first, last = True, set(), set()
            for child in node[1]:
                cn, cf, cl = self._walk(child)
                for p in last:                      # Follow(p) gets First(child) for p in Last(prefix)
                    self.follow[p] |= cf
                if nullable:
                    first |= cf
                last = cl | last if cn else set(cl)
                nullable = nullable and cn
            return nullable, first, last
        if kind == 'alt':
            nullable, first, last = False, set(), set()
            for child in node[1]:
                cn, cf, cl = self._walk(child)
                nullable = nullable or cn
                first |= cf
                last |= cl
            return nullable, first, last
        if kind in ('star', 'plus'):
            cn, cf, cl = self._walk(node[1])
            for p in cl:
                self.follow[p] |= cf
            return (True if kind == 'star' else cn), cf, cl
        if kind == 'opt':
            cn, cf, cl = self._walk(node[1])
            return True, cf, cl
        raise ValueError(f"unexpected node {kind} (expand repeats first)")


def glushkov_nfa(re_src) -> NFA:
    """Position NFA of an RE (bytes or str), states 0..npos, q0 = 0."""
    pos = Positions(re_syntax.expand(re_syntax.parse(re_src)))
    n = len(pos.sym)
    delta = [dict() for _ in range(n)]
    succ = [pos.first] + [pos.follow[p] for p in range(1, n)]
    for q in range(n):
        for p in succ[q]:
            for b in pos.sym[p]:
                delta[q].setdefault(b, set()).add(p)
    delta = [{b: frozenset(s) for b, s in d.items()} for d in delta]
    finals = set(pos.last)
    if pos.nullable:
        finals.add(0)
    alphabet = sorted(set().union(*[set(s) for s in pos.sym[1:]])) if n > 1 else []
    return NFA(n, alphabet, delta, 0, frozenset(finals))


def glushkov_tables(re_src):
    """(n_states, follow, sym) of the position NFA, for the C set simulator.

    follow[q] = successor positions of q (q = 0 is q0, whose successors are First);
    sym[b] = positions whose symbol set contains byte b.
    """
    pos = Positions(re_syntax.expand(re_syntax.parse(re_src)))
    n = len(pos.sym)
    follow = [frozenset(pos.first)] + [frozenset(pos.follow[p]) for p in range(1, n)]
    sym = [frozenset(p for p in range(1, n) if b in pos.sym[p]) for b in range(256)]
    finals = set(pos.last) | ({0} if pos.nullable else set())
    return n, follow, sym, frozenset(finals)

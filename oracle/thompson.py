"""Oracle Thompson epsilon-NFA: the plain definition of acceptance x in L(RE).

Test infrastructure only (see ``oracle/__init__.py``).

Thompson's construction (one state per symbol, split states for alternation and loops), then
state-set simulation: S <- eps-closure({start}); for each byte b: S <- eps-closure(move(S, b));
accept <=> MATCH in S.  This is the serial device operation of the paper's Sec. 2 run with a
nondeterministic recognizer of L; the RID must give the same answer (Th. 1).

Deliberately a different NFA from the position automaton used by the RID construction, so a
mistake in either shows up as a disagreement.
"""

from . import re_syntax

CHAR, SPLIT, MATCH = 0, 1, 2


class ThompsonNFA:
    def __init__(self):
        self.kind = []      # CHAR / SPLIT / MATCH
        self.sym = []       # frozenset of bytes for CHAR
        self.out1 = []      # successor (CHAR: after the byte; SPLIT: first eps edge)
        self.out2 = []      # SPLIT: second eps edge (-1 if none)
        self.start = -1

    def _state(self, kind, sym=None):
        self.kind.append(kind)
        self.sym.append(sym)
        self.out1.append(-1)
        self.out2.append(-1)
        return len(self.kind) - 1


def _build(nfa, node):
    """Returns (entry, list of dangling (state, which_out)) for a fragment."""
    kind = node[0]
    if kind == 'eps':
        s = nfa._state(SPLIT)
        return s, [(s, 1)]
    if kind == 'set':
        s = nfa._state(CHAR, node[1])
        return s, [(s, 1)]
    if kind == 'cat':
        entry, dangling = _build(nfa, node[1][0])
        for child in node[1][1:]:
            e2, d2 = _build(nfa, child)
            _patch(nfa, dangling, e2)
            dangling = d2
        return entry, dangling
    if kind == 'alt':
        entries, dangling = [], []
        for child in node[1]:
            e, d = _build(nfa, child)
            entries.append(e)
            dangling += d
        # chain of binary splits
        entry = entries[-1]
        for e in reversed(entries[:-1]):
            s = nfa._state(SPLIT)
            nfa.out1[s] = e
            nfa.out2[s] = entry
            entry = s
        return entry, dangling
    if kind == 'star':
        s = nfa._state(SPLIT)
        e, d = _build(nfa, node[1])
        nfa.out1[s] = e
        _patch(nfa, d, s)
        return s, [(s, 2)]
    if kind == 'plus':
        e, d = _build(nfa, node[1])
        s = nfa._state(SPLIT)
        nfa.out1[s] = e
        _patch(nfa, d, s)
        return e, [(s, 2)]
    if kind == 'opt':
        s = nfa._state(SPLIT)
        e, d = _build(nfa, node[1])
        nfa.out1[s] = e
        return s, d + [(s, 2)]
    raise ValueError(f"unexpected node {kind}")


def _patch(nfa, dangling, target):
    for s, which in dangling:
        if which == 1:
            nfa.out1[s] = target
        else:
            nfa.out2[s] = target


def thompson_nfa(re_src) -> ThompsonNFA:
    nfa = ThompsonNFA()
    entry, dangling = _build(nfa, re_syntax.expand(re_syntax.parse(re_src)))
    m = nfa._state(MATCH)
    _patch(nfa, dangling, m)
    nfa.start = entry
    return nfa


def _closure(nfa, states):
    stack = list(states)
    seen = set(states)
    while stack:
        s = stack.pop()
        if nfa.kind[s] == SPLIT:
            for t in (nfa.out1[s], nfa.out2[s]):
                if t >= 0 and t not in seen:
                    seen.add(t)
                    stack.append(t)
    return seen


def accepts(nfa: ThompsonNFA, text: bytes) -> bool:
    """Pure-Python state-set simulation (small inputs; csim.thompson_accept is the same loop in C)."""
    cur = _closure(nfa, {nfa.start})
    for b in text:
        nxt = {nfa.out1[s] for s in cur if nfa.kind[s] == CHAR and b in nfa.sym[s]}
        cur = _closure(nfa, nxt)
        if not cur:
            return False
    return any(nfa.kind[s] == MATCH for s in cur)

"""Oracle RI-DFA, interface function, Nerode delegation and joins, over explicit subsets.

Test infrastructure only (see ``oracle/__init__.py``).  Plain Python on frozensets; every step
follows the paper's text in its order and notation:

* ``NFA``                    N = (Q_N, Sigma, rho, q0, F)                                (Sec. 3.1)
* ``build_ridfa``            B = (P, Sigma, delta^B, I^B, F^B) as N(q0) u N(q1) u ... (Sec. 3.1, Fig. 3)
* ``RIDFA.interface``        if(PLAS) = U_{p in PLAS} {{q} : q in p}                     (Sec. 3.2)
* ``nerode_blocks``          language-equivalence classes of P (state-partition)         (Sec. 3.4)
* ``RIDFA.minimize_interface`` delegation to one representative per class of initial
                             states, and if_min                                           (Sec. 3.4)
* ``chunk_mapping``          lambda_i(a) = delta^B(a, y_i) or undefined                  (Sec. 3.2)
* ``rid_join``               PLAS_1 = lambda_1(PIS_1); PLAS_i = lambda_i(if(PLAS_{i-1}) n PIS_i);
                             accept <=> PLAS_c n F^RID != {}                               (Sec. 3.2)
* ``csdpa_dfa_join``         the classic join with a DFA chunk automaton                   (Sec. 2, Fig. 2)
* ``transition_count``       transitions executed by the reach phase; moves into the
                             undefined state are not counted                               (Sec. 1, Fig. 1)
* ``min_dfa``                minimal DFA (powerset + state partition) for the all-states
                             comparator                                                    (Sec. 2, Fig. 1)

State numbering convention (the paper's numbering is only presentational): the singletons
{q0}, ..., {q_{l-1}} get ids 0..l-1; aggregates get the next ids in breadth-first discovery
order, exploring the singletons {q0}, {q1}, ... in turn and, from each state, the input
symbols in ascending byte order.  Implementations that follow the same rule give the same ids.
"""

from collections import deque

UNDEF = None          # the undefined transition / dead run (the paper's "exits", Fig. 5)


class NFA:
    """N = (Q_N, Sigma, rho, q0, F): states 0..n-1, rho as a list of dicts byte -> frozenset."""

    def __init__(self, n, alphabet, delta, q0, finals):
        self.n = n
        self.alphabet = sorted(alphabet)
        self.delta = delta
        self.q0 = q0
        self.finals = frozenset(finals)

    @staticmethod
    def from_edges(n, edges, finals, alphabet, q0=0):
        """Build from (q, symbols, q') edges, symbols an iterable of single-character strings."""
        delta = [dict() for _ in range(n)]
        for q, syms, q2 in edges:
            for s in syms:
                b = ord(s) if isinstance(s, str) else s
                delta[q].setdefault(b, set()).add(q2)
        delta = [{b: frozenset(t) for b, t in d.items()} for d in delta]
        alpha = [ord(s) if isinstance(s, str) else s for s in alphabet]
        return NFA(n, alpha, delta, q0, finals)

    def rho(self, q, b):
        return self.delta[q].get(b, frozenset())

    def rho_set(self, states, b):
        out = set()
        for q in states:
            out |= self.rho(q, b)
        return frozenset(out)

    def run(self, states, word):
        """rho extended to strings and to sets of states (proof of Th. 1)."""
        cur = frozenset(states)
        for b in word:
            cur = self.rho_set(cur, b)
        return cur

    def accepts(self, word):
        return bool(self.run({self.q0}, word) & self.finals)


class RIDFA:
    """B = (P, Sigma, delta^B, I^B, F^B) with the RID initial state {q0} and F^RID."""

    def __init__(self, nfa, states, delta, finals):
        self.nfa = nfa
        self.states = states                 # list of frozensets; id = index
        self.index = {s: i for i, s in enumerate(states)}
        self.delta = delta                   # list of dicts byte -> id
        self.finals = finals                 # F^RID as a set of ids
        self.initial = list(range(nfa.n))    # I^B: the singletons, ids 0..l-1
        # interface minimisation (Sec. 3.4); identity until minimize_interface() runs
        self.slots = list(range(nfa.n))      # representative NFA state of each slot
        self.delegate = list(range(nfa.n))   # NFA state q -> slot index of its representative

    @property
    def k(self):
        return len(self.slots)

    def step(self, p, b):
        if p is UNDEF:
            return UNDEF
        return self.delta[p].get(b, UNDEF)

    def run(self, p, word):
        for b in word:
            p = self.step(p, b)
            if p is UNDEF:
                return UNDEF
        return p

    def interface(self, plas):
        """if(PLAS) = U_{p in PLAS} {{q} | q in p}, returned as a set of slot indices.

        With the identity delegation the slot of {q} is q; after minimize_interface() each
        singleton maps to the slot of its representative, which is if_min (Sec. 3.4).
        """
        out = set()
        for p in plas:
            for q in self.states[p]:
                out.add(self.delegate[q])
        return out

    def minimize_interface(self):
        """Delegation (Sec. 3.4): in each Nerode class of initial states keep the lowest NFA
        state as the representative; the others delegate their initial role to it."""
        blocks = nerode_blocks(self)
        rep_of_block = {}
        for q in range(self.nfa.n):
            blk = blocks[q]
            if blk not in rep_of_block:
                rep_of_block[blk] = q          # lowest q first, since q ascends
        reps = sorted(set(rep_of_block.values()))
        slot_of_rep = {r: i for i, r in enumerate(reps)}
        self.slots = reps
        self.delegate = [slot_of_rep[rep_of_block[blocks[q]]] for q in range(self.nfa.n)]
        return self


def build_ridfa(nfa: NFA, max_states=None) -> RIDFA:
    """Incremental powerset construction N(q0) u N(q1) u ... u N(q_{l-1}) (Sec. 3.1).

    delta^B(S, b) = U_{q in S} rho(q, b), undefined when empty; F^RID = {p : p n F != {}}.
    """
    states = [frozenset([q]) for q in range(nfa.n)]
    index = {s: i for i, s in enumerate(states)}
    delta = [dict() for _ in states]
    explored = [False] * len(states)
    for q in range(nfa.n):                       # N(q0), then N(q1) adds what is new, ...
        if explored[q]:
            continue
        explored[q] = True
        queue = deque([q])
        while queue:
            p = queue.popleft()
            for b in nfa.alphabet:
                t = nfa.rho_set(states[p], b)
                if not t:
                    continue                     # undefined transition
                if t not in index:
                    index[t] = len(states)
                    states.append(t)
                    delta.append(dict())
                    explored.append(False)
                    if max_states is not None and len(states) > max_states:
                        raise OverflowError("RI-DFA exceeds max_states")
                j = index[t]
                delta[p][b] = j
                if not explored[j]:
                    explored[j] = True
                    queue.append(j)
    finals = {i for i, s in enumerate(states) if s & nfa.finals}
    return RIDFA(nfa, states, delta, finals)


def nerode_blocks(dfa) -> list:
    """Language-equivalence classes by the state-partition algorithm (Sec. 3.4).

    Works on any object with .states, .delta (list of dict byte -> id), .finals and an
    .nfa.alphabet (or .alphabet).  The partial transition function is completed with an
    implicit dead state.  Returns block ids per state (ids are canonical: first-occurrence).
    """
    alphabet = dfa.nfa.alphabet if hasattr(dfa, 'nfa') else dfa.alphabet
    n = len(dfa.states)
    dead = n
    block = [1 if i in dfa.finals else 0 for i in range(n)] + [0]
    # make the dead state its own block only if it is distinguishable; Moore iteration
    # below handles that automatically, starting from {finals}, {non-finals + dead}
    num = len(set(block))
    while True:
        sigs = {}
        new = []
        for i in range(n + 1):
            if i == dead:
                succ = tuple(block[dead] for _ in alphabet)
            else:
                succ = tuple(block[dfa.delta[i].get(b, dead)] for b in alphabet)
            key = (block[i], succ)
            if key not in sigs:
                sigs[key] = len(sigs)
            new.append(sigs[key])
        if len(sigs) == num:
            return new[:n]
        block, num = new, len(sigs)


def chunk_boundaries(n, c):
    """b_i = floor(i*n/c), i = 0..c; chunk i is x[b_i, b_{i+1}) (non-empty when c <= n)."""
    return [(i * n) // c for i in range(c + 1)]


def chunk_mapping(B: RIDFA, chunk, slots=None):
    """lambda_i over the interface slots: slot a -> delta^B({rep_a}, y_i), or UNDEF (Sec. 3.2)."""
    if slots is None:
        slots = range(B.k)
    return [B.run(B.slots[a], chunk) for a in slots]


def rid_join(B: RIDFA, maps, return_plas=False):
    """The RID join phase (Sec. 3.2): maps[i][a] = lambda_{i+1}(slot a) (ids or UNDEF).

    PIS_1 = {{q0}}; PLAS_1 = lambda_1(PIS_1);
    PIS_i = {a : lambda_i(a) defined};  PLAS_i = lambda_i(if(PLAS_{i-1}) n PIS_i);
    accept <=> PLAS_c n F^RID != {}.
    """
    q0_slot = B.delegate[B.nfa.q0]
    first = maps[0][q0_slot]
    plas = set() if first is UNDEF else {first}
    history = [set(plas)]
    for lam in maps[1:]:
        pis = {a for a, p in enumerate(lam) if p is not UNDEF}
        plas = {lam[a] for a in (B.interface(plas) & pis)}
        history.append(set(plas))
    accept = bool(plas & B.finals)
    return (accept, history) if return_plas else accept


def transition_count(B: RIDFA, chunks, slots_per_chunk=None):
    """Transitions executed by the reach phase: chunk 1 from {q0}, every other chunk from every
    interface slot; a run stops at the undefined state, which is not counted (Sec. 1, Fig. 1)."""
    total = 0
    q0_slot = B.delegate[B.nfa.q0]
    for i, y in enumerate(chunks):
        starts = [q0_slot] if i == 0 else range(B.k)
        for a in starts:
            p = B.slots[a]
            for b in y:
                p = B.step(p, b)
                if p is UNDEF:
                    break
                total += 1
    return total


class DFA:
    """A (partial) DFA: states 0..n-1, delta list of dict byte -> id, start, finals."""

    def __init__(self, states, alphabet, delta, start, finals):
        self.states = states
        self.alphabet = sorted(alphabet)
        self.delta = delta
        self.start = start
        self.finals = set(finals)

    def step(self, q, b):
        if q is UNDEF:
            return UNDEF
        return self.delta[q].get(b, UNDEF)

    def run(self, q, word):
        for b in word:
            q = self.step(q, b)
            if q is UNDEF:
                return UNDEF
        return q


def powerset_dfa(nfa: NFA) -> DFA:
    """Classic one-shot powerset construction from {q0} (the DFA variant of CSDPA, Sec. 2)."""
    start = frozenset([nfa.q0])
    states = [start]
    index = {start: 0}
    delta = [dict()]
    queue = deque([0])
    while queue:
        i = queue.popleft()
        for b in nfa.alphabet:
            t = nfa.rho_set(states[i], b)
            if not t:
                continue
            if t not in index:
                index[t] = len(states)
                states.append(t)
                delta.append(dict())
                queue.append(index[t])
            delta[i][b] = index[t]
    finals = {i for i, s in enumerate(states) if s & nfa.finals}
    return DFA(states, nfa.alphabet, delta, 0, finals)


def min_dfa(nfa: NFA) -> DFA:
    """Minimal DFA: powerset DFA, state partition, then renumber the live classes in
    breadth-first order from the start (symbols ascending).  The class of the implicit dead
    state (and any class equivalent to it) is dropped, so transitions into it are undefined."""
    d = powerset_dfa(nfa)
    blocks = nerode_blocks(d)
    # the dead state's block: any block with no path to a final state
    n = len(d.states)
    dead_block = None
    # a block is dead iff none of its states is final and all successors stay in dead blocks;
    # compute co-reachability on the quotient
    nb = max(blocks) + 1 if blocks else 0
    rep = {}
    for i, blk in enumerate(blocks):
        rep.setdefault(blk, i)
    live = {blocks[i] for i in d.finals}
    changed = True
    while changed:
        changed = False
        for blk in range(nb):
            if blk in live:
                continue
            i = rep[blk]
            if any(blocks[j] in live for j in d.delta[i].values()):
                live.add(blk)
                changed = True
    order = {}
    queue = deque()
    sb = blocks[d.start]
    if sb in live:
        order[sb] = 0
        queue.append(sb)
    new_delta = []
    while queue:
        blk = queue.popleft()
        i = rep[blk]
        row = {}
        for b in d.alphabet:
            j = d.delta[i].get(b)
            if j is None or blocks[j] not in live:
                continue
            tb = blocks[j]
            if tb not in order:
                order[tb] = len(order)
                queue.append(tb)
            row[b] = order[tb]
        new_delta.append(row)
    inv = {v: k for k, v in order.items()}
    states = [frozenset(i for i in range(n) if blocks[i] == inv[s]) for s in range(len(order))]
    finals = {s for s in range(len(order)) if rep[inv[s]] in d.finals}
    if not order:     # empty language: a single non-final start state with no transitions
        return DFA([frozenset()], d.alphabet, [dict()], 0, set())
    out = DFA(states, d.alphabet, new_delta, 0, finals)
    # NFA subset <-> minimal-DFA state: every live powerset state belongs to one class
    out.subset_to_state = {d.states[i]: order[blocks[i]] for i in range(n) if blocks[i] in order}
    out.state_subset = [d.states[rep[inv[s]]] for s in range(len(order))]
    return out


def csdpa_dfa_maps(dfa: DFA, chunks):
    """lambda_i for the DFA variant of CSDPA: every state is initial (Sec. 2)."""
    return [[dfa.run(q, y) for q in range(len(dfa.states))] for y in chunks]


def csdpa_dfa_join(dfa: DFA, maps):
    """PLAS_1 = lambda_1({q0}); PLAS_i = lambda_i(PLAS_{i-1} n PIS_i), PIS_i = Q; accept <=>
    PLAS_c n F != {} (Sec. 2, Fig. 2)."""
    first = maps[0][dfa.start]
    plas = set() if first is UNDEF else {first}
    for lam in maps[1:]:
        plas = {lam[q] for q in plas if lam[q] is not UNDEF}
    return bool(plas & dfa.finals)


def csdpa_dfa_transition_count(dfa: DFA, chunks):
    """Transitions of the DFA variant: chunk 1 from q0 only, other chunks from every state."""
    total = 0
    for i, y in enumerate(chunks):
        starts = [dfa.start] if i == 0 else range(len(dfa.states))
        for q in starts:
            for b in y:
                q = dfa.step(q, b)
                if q is UNDEF:
                    break
                total += 1
    return total

"""Oracle entry points used by the tests and by the bench's CPU baseline.  Test infrastructure only.

``SerialRecognizer``  -- accept = [x in L(RE)] by Thompson state-set simulation (the definition).
``RidOracle``         -- the paper's RID pieces for one RE over its position NFA:
                         RI-DFA B with interface minimisation (Sec. 3.1, 3.4), chunk mappings
                         lambda_i computed from the definition delta^B({q}, y) = rho(q, y)
                         (construction of Sec. 3.1, Lemma 1) by set simulation, the RID join
                         (Sec. 3.2), and the minimal DFA with its CSDPA maps and join (Sec. 2).
"""

import numpy as np

from . import glushkov, thompson
from .csim import SetSim, ThompsonSim
from .ridfa_sets import (UNDEF, build_ridfa, chunk_boundaries, csdpa_dfa_join, min_dfa,
                         rid_join)

LAMBDA_UNDEF = 0xFFFF     # wire encoding of an undefined chunk mapping entry


class SerialRecognizer:
    def __init__(self, re_src):
        self.nfa = thompson.thompson_nfa(re_src)
        self.sim = ThompsonSim(self.nfa)

    def accepts(self, text) -> bool:
        return self.sim.accepts(text)


class RidOracle:
    def __init__(self, re_src, minimize=True, max_states=65534, with_dfa=True):
        self.re = re_src
        self.nfa = glushkov.glushkov_nfa(re_src)
        self.B = build_ridfa(self.nfa, max_states=max_states)
        if minimize:
            self.B.minimize_interface()
        n, follow, sym, finals = glushkov.glushkov_tables(re_src)
        self.sets = SetSim(n, follow, sym)
        self.dfa = min_dfa(self.nfa) if with_dfa else None
        self._dfa_sets = None

    # --- RID -------------------------------------------------------------------------------
    def lambda_row(self, chunk):
        """lambda_i(a) for every slot a, from rho(q_a, y_i) (ids; LAMBDA_UNDEF when empty)."""
        row = np.empty(self.B.k, dtype=np.uint16)
        for a, q in enumerate(self.B.slots):
            s = self.sets.run({q}, chunk)
            row[a] = LAMBDA_UNDEF if not s else self.B.index[s]
        return row

    def lambda_rows(self, text, c, chunk_ids=None):
        text = np.asarray(text, dtype=np.uint8)
        b = chunk_boundaries(len(text), c)
        ids = range(c) if chunk_ids is None else chunk_ids
        return {i: self.lambda_row(text[b[i]:b[i + 1]]) for i in ids}

    def join(self, rows):
        """RID join over wire-encoded rows (list of uint16 arrays, chunk order)."""
        maps = [[UNDEF if v == LAMBDA_UNDEF else int(v) for v in r] for r in rows]
        return rid_join(self.B, maps)

    # --- all-states DFA comparator ---------------------------------------------------------
    def dfa_lambda_row(self, chunk):
        """lambda_i(q) for every minimal-DFA state q.  State q is the class of some NFA subset
        S_q reachable from {q0}; rho(S_q, y) is again reachable, and its class is the image."""
        d = self.dfa
        row = np.empty(len(d.states), dtype=np.uint16)
        for q in range(len(d.states)):
            t = self.sets.run(d.state_subset[q], chunk)
            p = d.subset_to_state.get(t) if t else None
            row[q] = LAMBDA_UNDEF if p is None else p
        return row

    def dfa_lambda_row_slow(self, chunk):
        """Same as dfa_lambda_row by stepping the minimal DFA's own table (small inputs)."""
        d = self.dfa
        row = np.empty(len(d.states), dtype=np.uint16)
        for q in range(len(d.states)):
            p = d.run(q, chunk)
            row[q] = LAMBDA_UNDEF if p is UNDEF else p
        return row

    def dfa_lambda_rows(self, text, c, chunk_ids=None):
        text = np.asarray(text, dtype=np.uint8)
        b = chunk_boundaries(len(text), c)
        ids = range(c) if chunk_ids is None else chunk_ids
        return {i: self.dfa_lambda_row(text[b[i]:b[i + 1]]) for i in ids}

    def dfa_join(self, rows):
        maps = [[UNDEF if v == LAMBDA_UNDEF else int(v) for v in r] for r in rows]
        return csdpa_dfa_join(self.dfa, maps)

    # --- definition --------------------------------------------------------------------------
    def set_accepts(self, text) -> bool:
        """rho(q0, x) n F != {} by set simulation over the position NFA."""
        return bool(self.sets.run({0}, text) & self.nfa.finals)

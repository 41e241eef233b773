"""Seeded synthetic inputs shared by the tests and the bench.

This module generates REs and texts only.  It holds none of the recognizer's arithmetic (no
automaton construction, no chunk mappings, no join) and imports neither ``oracle`` nor
``paper_2412_14975_gb300``.  Where a generator needs an automaton (the random walk of the
single-text configs), the automaton is passed in as plain arrays by the caller, or is a small
hand-derived table written out below and pinned by a test against the oracle.

Randomness: ``numpy.random.Generator(PCG64(seed))`` everywhere; every public function takes a
seed or a Generator.  Labels (accept / reject) never come from here: the tests take them from
the oracle.
"""

from .regex_ast import (Alt, Cat, Opt, Plus, Rep, Star, Sym, random_re, render,
                        sample_member)  # noqa: F401
from .texts import (C1_RE, C2_RE, C3_RE, C3_RE_ANYFIELD, c1_min_dfa_table, c1_text,
                    c2_text, c3_text, dfa_walk, mutate, regexp_family_re,
                    regexp_family_text)  # noqa: F401
from .texts_torch import c3_text_torch  # noqa: F401

"""Test infrastructure: a plain, slow, independent CPU oracle for the RID recognizer.

This package is NOT part of the product.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code, tables or constants with ``paper_2412_14975_gb300`` (the GPU
library) and never imports it.

What it computes (Borsotti, Breveglieri, Crespi Reghizzi, Morzenti,
"Minimizing speculation overhead in a parallel recognizer for regular texts"):

* ``re_syntax``    -- RE parser A (byte dialect) and the bounded-repeat expansion convention.
* ``thompson``     -- Thompson epsilon-NFA; state-set simulation is the definition of acceptance.
* ``glushkov``     -- position (McNaughton-Yamada/Glushkov) NFA used as the RID source NFA N (Sec. 3.1).
* ``ridfa_sets``   -- RI-DFA construction N(q0) u N(q1) u ... over subsets (Sec. 3.1), the
                      interface function ``if`` (Sec. 3.2), the Nerode partition and delegation
                      that give ``if_min`` (Sec. 3.4), the chunk mappings lambda_i, the RID join
                      and the CSDPA join with a DFA (Sec. 2), and the paper's transition count.
* ``definitional`` -- a definitional matcher for tiny strings (language of each RE operator).
* ``csim``         -- the two hot simulation loops written in plain C (loaded with ctypes):
                      Thompson state-set simulation and epsilon-free NFA set simulation.

Parity pins live in ``tests/test_oracle_*.py`` (paper worked examples Fig. 1-5, closed forms,
brute-force enumeration).  Every function here cites the passage of the paper it follows.
"""

"""Seeded texts for the single-text workloads (uint8 numpy arrays).

Workload recipes (sizes and structure of the paper's text benchmarks, synthetic):
  C1  ((A|C)*G(T|A)+C)*, random walk on its minimal DFA (uniform over live transitions), then
      the shortest completion to an accepting state once the target length is reached.
  C2  (([ACGT]{3})*ATG([ACGT]{3}){20,60}(TAA|TAG|TGA))*[ACGT]*: its language is {A,C,G,T}*, so
      a uniform walk is i.i.d. uniform ACGT.
  C3  comma-separated record lines (timestamp, id, float, word, dotted 4-tuple, newline);
      field lengths and digits/letters uniform.
  regexp family (a|b)*a(a|b){k} over i.i.d. uniform a/b.
Negatives are made with ``mutate``.
"""

import numpy as np

C1_RE = "((A|C)*G(T|A)+C)*"
C2_RE = "(([ACGT]{3})*ATG([ACGT]{3}){20,60}(TAA|TAG|TGA))*[ACGT]*"
_TS = "[0-9]{4}-[0-9]{2}-[0-9]{2}T[0-9]{2}:[0-9]{2}:[0-9]{2}"
_ID = "[0-9]{1,9}"
_FLOAT = "[0-9]+\\.[0-9]{1,6}"
_WORD = "[a-z]{1,12}"
_IP = "[0-9]{1,3}\\.[0-9]{1,3}\\.[0-9]{1,3}\\.[0-9]{1,3}"
C3_RE = "(" + ",".join([_TS, _ID, _FLOAT, _WORD, _IP]) + "\\n)*"
_F = "(" + "|".join([_TS, _ID, _FLOAT, _WORD, _IP]) + ")"
C3_RE_ANYFIELD = "(" + _F + "(," + _F + ")*\\n)*"


def _rng(seed):
    return seed if isinstance(seed, np.random.Generator) else np.random.Generator(np.random.PCG64(seed))


def c1_min_dfa_table():
    """Minimal DFA of ((A|C)*G(T|A)+C)*, written out by hand (states 0..3, 0 accepting):
    0 -A,C-> 1, 0 -G-> 2, 1 -A,C-> 1, 1 -G-> 2, 2 -T,A-> 3, 3 -T,A-> 3, 3 -C-> 0."""
    t = np.full((4, 256), -1, dtype=np.int32)
    for s, syms, d in [(0, b"AC", 1), (0, b"G", 2), (1, b"AC", 1), (1, b"G", 2),
                       (2, b"TA", 3), (3, b"TA", 3), (3, b"C", 0)]:
        for b in syms:
            t[s, b] = d
    acc = np.array([True, False, False, False])
    return t, acc, 0


def dfa_walk(trans, accepting, start, n, seed):
    """Random walk of >= n bytes on a DFA given as trans[state, byte] (-1 = undefined).

    Each step picks uniformly among the live bytes (the target can still reach an accepting
    state).  Once n bytes are out, the walk appends the shortest path to an accepting state,
    breaking ties by the lowest byte.  The walk's distribution depends only on the language."""
    rng = _rng(seed)
    trans = np.asarray(trans)
    ns = trans.shape[0]
    acc = np.asarray(accepting, dtype=bool)
    live = acc.copy()
    changed = True
    while changed:
        nxt = live | np.array([bool(np.any(live[trans[s][trans[s] >= 0]])) for s in range(ns)])
        changed = bool(np.any(nxt != live))
        live = nxt
    if not live[start]:
        raise ValueError("the language is empty")
    choices = [np.nonzero((trans[s] >= 0) & live[np.maximum(trans[s], 0)])[0].astype(np.uint8)
               for s in range(ns)]
    u = rng.random(n)
    out = np.empty(n, dtype=np.uint8)
    s = start
    tr = trans.tolist()
    ch = [c.tolist() for c in choices]
    for t in range(n):
        c = ch[s]
        if not c:
            raise ValueError("walk reached a state with no live byte")
        b = c[int(u[t] * len(c))]
        out[t] = b
        s = tr[s][b]
    if acc[s]:
        return out
    # shortest completion: BFS over live transitions, bytes ascending
    prev = {s: None}
    queue = [s]
    i = 0
    goal = None
    while i < len(queue):
        x = queue[i]
        i += 1
        if acc[x]:
            goal = x
            break
        for b in ch[x]:
            y = tr[x][b]
            if y not in prev:
                prev[y] = (x, b)
                queue.append(y)
    tail = []
    while prev[goal] is not None:
        x, b = prev[goal]
        tail.append(b)
        goal = x
    return np.concatenate([out, np.array(tail[::-1], dtype=np.uint8)])


def c1_text(n, seed):
    t, acc, s0 = c1_min_dfa_table()
    return dfa_walk(t, acc, s0, n, seed)


def c2_text(n, seed):
    """n i.i.d. uniform bytes of ACGT (a uniform walk of {A,C,G,T}*)."""
    rng = _rng(seed)
    return np.frombuffer(b"ACGT", dtype=np.uint8)[rng.integers(0, 4, size=n)]


# record layout: (kind, fixed byte) per segment; kind 0 = digits, 1 = lowercase, 2 = fixed
_SEGS = ([(0, 0), (2, ord('-')), (0, 0), (2, ord('-')), (0, 0), (2, ord('T')), (0, 0),
          (2, ord(':')), (0, 0), (2, ord(':')), (0, 0)]                       # timestamp
         + [(2, ord(',')), (0, 0), (2, ord(',')), (0, 0), (2, ord('.')), (0, 0),
            (2, ord(',')), (1, 0), (2, ord(','))]                               # ,id,float,word,
         + [(0, 0), (2, ord('.')), (0, 0), (2, ord('.')), (0, 0), (2, ord('.')), (0, 0)]
         + [(2, 10)])                                                           # ip, newline
_TS_LENS = [4, 1, 2, 1, 2, 1, 2, 1, 2, 1, 2]


def _c3_block(rng, nrec):
    nseg = len(_SEGS)
    lens = np.ones((nrec, nseg), dtype=np.int64)
    lens[:, :11] = _TS_LENS
    lens[:, 12] = rng.integers(1, 10, size=nrec)     # id digits 1..9
    lens[:, 14] = rng.integers(1, 10, size=nrec)     # float integer part 1..9
    lens[:, 16] = rng.integers(1, 7, size=nrec)      # float fraction 1..6
    lens[:, 18] = rng.integers(1, 13, size=nrec)     # word 1..12
    for j in (20, 22, 24, 26):
        lens[:, j] = rng.integers(1, 4, size=nrec)   # octets 1..3
    kinds = np.tile(np.array([k for k, _ in _SEGS], dtype=np.uint8), nrec)
    fixed = np.tile(np.array([c for _, c in _SEGS], dtype=np.uint8), nrec)
    flat = lens.ravel()
    kind_b = np.repeat(kinds, flat)
    out = np.repeat(fixed, flat)
    dig = kind_b == 0
    out[dig] = rng.integers(48, 58, size=int(dig.sum()), dtype=np.uint8)
    let = kind_b == 1
    out[let] = rng.integers(97, 123, size=int(let.sum()), dtype=np.uint8)
    return out


def c3_text(n, seed, block_records=1 << 20):
    """Record lines until at least n bytes (whole lines, so the text ends with a newline)."""
    rng = _rng(seed)
    parts, total = [], 0
    while total < n:
        need = n - total
        nrec = int(min(block_records, max(16, need // 40 + 16)))
        blk = _c3_block(rng, nrec)
        if total + blk.size > n:
            # keep whole lines only, stopping at the first newline at or after the target
            nl = np.nonzero(blk == 10)[0]
            cut = nl[np.searchsorted(nl, need - 1)] + 1
            blk = blk[:cut]
        parts.append(blk)
        total += blk.size
    return np.concatenate(parts) if len(parts) > 1 else parts[0]


def mutate(text, seed, n_subs=1, alphabet=None):
    """Copy of text with n_subs uniformly placed byte substitutions; each replacement is uniform
    over ``alphabet`` (bytes; default: the bytes present in the text) minus the original byte."""
    rng = _rng(seed)
    out = np.array(text, dtype=np.uint8, copy=True)
    if alphabet is None:
        alphabet = np.unique(out)
    alphabet = np.asarray(list(alphabet), dtype=np.uint8)
    pos = rng.integers(0, out.size, size=n_subs)
    for p in pos:
        cand = alphabet[alphabet != out[p]]
        out[p] = cand[rng.integers(cand.size)]
    return out, pos


def regexp_family_re(k):
    return "(a|b)*a(a|b){%d}" % k


def regexp_family_text(n, seed):
    rng = _rng(seed)
    return np.frombuffer(b"ab", dtype=np.uint8)[rng.integers(0, 2, size=n)]

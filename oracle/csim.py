"""ctypes wrapper of the oracle's plain-C loops (``csim.c``).  Test infrastructure only.

``build()`` compiles ``csim.c`` with gcc into ``oracle/libcsim.so``; the wrappers build it on
first use if it is missing.
"""

import ctypes
import os
import subprocess

import numpy as np

from .thompson import ThompsonNFA, CHAR, SPLIT, MATCH  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csim.c")
_LIB = os.path.join(_HERE, "libcsim.so")
_lib = None


def build(force=False):
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp = ctypes.c_void_p
        lib.oracle_thompson_accept.restype = ctypes.c_int
        lib.oracle_thompson_accept.argtypes = [ctypes.c_int32, vp, vp, vp, vp, ctypes.c_int32,
                                               vp, ctypes.c_int64]
        lib.oracle_set_run.restype = ctypes.c_int
        lib.oracle_set_run.argtypes = [ctypes.c_int32, ctypes.c_int32, vp, vp, vp, vp,
                                       ctypes.c_int64, vp]
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _text_ptr(text):
    if isinstance(text, np.ndarray):
        assert text.dtype == np.uint8 and text.flags['C_CONTIGUOUS']
        return text, _ptr(text), text.size
    buf = np.frombuffer(bytes(text), dtype=np.uint8)
    return buf, _ptr(buf), buf.size


class ThompsonSim:
    """Thompson state-set simulation in C for one RE."""

    def __init__(self, nfa: ThompsonNFA):
        n = len(nfa.kind)
        self.n = n
        self.kind = np.array(nfa.kind, dtype=np.uint8)
        self.out1 = np.array(nfa.out1, dtype=np.int32)
        self.out2 = np.array(nfa.out2, dtype=np.int32)
        sym = np.zeros((n, 32), dtype=np.uint8)
        for s in range(n):
            if nfa.kind[s] == CHAR:
                for b in nfa.sym[s]:
                    sym[s, b >> 3] |= 1 << (b & 7)
        self.sym = sym
        self.start = nfa.start

    def accepts(self, text) -> bool:
        keep, p, ln = _text_ptr(text)
        r = _load().oracle_thompson_accept(self.n, _ptr(self.kind), _ptr(self.out1),
                                           _ptr(self.out2), _ptr(self.sym), self.start, p, ln)
        if r < 0:
            raise MemoryError("oracle_thompson_accept")
        return bool(r)


class SetSim:
    """rho(S, x) over an epsilon-free NFA given as follow sets and byte -> state sets."""

    def __init__(self, n, follow, sym):
        self.n = n
        self.words = max(1, (n + 63) // 64)
        f = np.zeros((n, self.words), dtype=np.uint64)
        for q in range(n):
            for p in follow[q]:
                f[q, p >> 6] |= np.uint64(1) << np.uint64(p & 63)
        s = np.zeros((256, self.words), dtype=np.uint64)
        for b in range(256):
            for p in sym[b]:
                s[b, p >> 6] |= np.uint64(1) << np.uint64(p & 63)
        self.follow, self.sym = f, s

    def to_bits(self, states):
        v = np.zeros(self.words, dtype=np.uint64)
        for q in states:
            v[q >> 6] |= np.uint64(1) << np.uint64(q & 63)
        return v

    def from_bits(self, v):
        out = []
        for w in range(self.words):
            x = int(v[w])
            while x:
                low = x & -x
                out.append(w * 64 + low.bit_length() - 1)
                x ^= low
        return frozenset(out)

    def run(self, start_states, text):
        keep, p, ln = _text_ptr(text)
        start = self.to_bits(start_states)
        out = np.zeros(self.words, dtype=np.uint64)
        r = _load().oracle_set_run(self.n, self.words, _ptr(self.follow), _ptr(self.sym),
                                   _ptr(start), p, ln, _ptr(out))
        if r < 0:
            raise MemoryError("oracle_set_run")
        return self.from_bits(out)

"""Oracle RE parser ("parser A") for the byte dialect, plus the repeat-expansion convention.

Test infrastructure only (see ``oracle/__init__.py``).

Dialect (over bytes 0..255; full-text match, no anchors, no search semantics):
  literal byte | ``.`` (any byte) | ``[...]`` / ``[^...]`` with ranges ``a-z`` |
  escapes ``\\n \\t \\r \\xHH`` and ``\\c`` = literal c for any other c |
  ``( )`` grouping, ``()`` = empty word | postfix ``* + ? {m} {m,} {m,n}`` |
  concatenation | alternation ``|`` (an empty alternative is the empty word).

The paper turns REs into NFAs with the McNaughton-Yamada (Glushkov) method (Sec. 4.1, Sec. 5);
bounded repeats are not primitive there, so they are expanded syntactically, with this
convention (shared, as a written rule, by every implementation that must agree on position
numbering):
  r{m}    = r r ... r            (m copies; m = 0 gives the empty word)
  r{m,}   = r^m r*
  r{m,n}  = r^m (r (r ( ... r)?)?)?   (n - m nested optional copies, outermost first)
``*``, ``+`` and ``?`` stay primitive.

AST nodes are tuples:
  ('eps',) | ('set', frozenset_of_bytes) | ('cat', (n1, n2, ...)) | ('alt', (n1, n2, ...)) |
  ('star', n) | ('plus', n) | ('opt', n) | ('rep', n, m, n_max_or_None)
"""

_META = set(b"|*+?{}()[]\\.")


class ReSyntaxError(ValueError):
    pass


class _Parser:
    def __init__(self, src: bytes):
        self.s = src
        self.i = 0

    def peek(self):
        return self.s[self.i] if self.i < len(self.s) else None

    def take(self):
        c = self.s[self.i]
        self.i += 1
        return c

    def parse(self):
        node = self.alt()
        if self.i != len(self.s):
            raise ReSyntaxError(f"unexpected {chr(self.s[self.i])!r} at {self.i}")
        return node

    def alt(self):
        branches = [self.cat()]
        while self.peek() == ord('|'):
            self.take()
            branches.append(self.cat())
        return branches[0] if len(branches) == 1 else ('alt', tuple(branches))

    def cat(self):
        items = []
        while self.peek() is not None and self.peek() not in (ord('|'), ord(')')):
            items.append(self.postfix())
        if not items:
            return ('eps',)
        return items[0] if len(items) == 1 else ('cat', tuple(items))

    def postfix(self):
        node = self.atom()
        while True:
            c = self.peek()
            if c == ord('*'):
                self.take(); node = ('star', node)
            elif c == ord('+'):
                self.take(); node = ('plus', node)
            elif c == ord('?'):
                self.take(); node = ('opt', node)
            elif c == ord('{'):
                self.take()
                m = self.number()
                if self.peek() == ord('}'):
                    self.take(); node = ('rep', node, m, m)
                elif self.peek() == ord(','):
                    self.take()
                    if self.peek() == ord('}'):
                        self.take(); node = ('rep', node, m, None)
                    else:
                        n = self.number()
                        if self.peek() != ord('}'):
                            raise ReSyntaxError("expected '}'")
                        self.take()
                        if n < m:
                            raise ReSyntaxError("repeat {m,n} with n < m")
                        node = ('rep', node, m, n)
                else:
                    raise ReSyntaxError("bad repeat")
            else:
                return node

    def number(self):
        start = self.i
        while self.peek() is not None and 0x30 <= self.peek() <= 0x39:
            self.take()
        if self.i == start:
            raise ReSyntaxError("expected a number")
        return int(self.s[start:self.i])

    def escape(self):
        if self.peek() is None:
            raise ReSyntaxError("dangling backslash")
        c = self.take()
        if c == ord('n'):
            return 10
        if c == ord('t'):
            return 9
        if c == ord('r'):
            return 13
        if c == ord('x'):
            h = self.s[self.i:self.i + 2]
            if len(h) != 2:
                raise ReSyntaxError("bad \\x escape")
            self.i += 2
            return int(h, 16)
        return c

    def atom(self):
        c = self.peek()
        if c is None:
            raise ReSyntaxError("unexpected end")
        if c == ord('('):
            self.take()
            node = self.alt()
            if self.peek() != ord(')'):
                raise ReSyntaxError("expected ')'")
            self.take()
            return node
        if c == ord('['):
            self.take()
            return ('set', self.bracket())
        if c == ord('.'):
            self.take()
            return ('set', frozenset(range(256)))
        if c == ord('\\'):
            self.take()
            return ('set', frozenset([self.escape()]))
        if c in (ord('*'), ord('+'), ord('?'), ord('{'), ord('}'), ord(')'), ord(']')):
            raise ReSyntaxError(f"unexpected {chr(c)!r} at {self.i}")
        self.take()
        return ('set', frozenset([c]))

    def bracket(self):
        neg = False
        if self.peek() == ord('^'):
            self.take(); neg = True
        members = set()
        first = True
        while True:
            c = self.peek()
            if c is None:
                raise ReSyntaxError("unterminated [")
            if c == ord(']') and not first:
                self.take()
                break
            first = False
            lo = self.take()
            if lo == ord('\\'):
                lo = self.escape()
            if self.peek() == ord('-') and self.i + 1 < len(self.s) and self.s[self.i + 1] != ord(']'):
                self.take()
                hi = self.take()
                if hi == ord('\\'):
                    hi = self.escape()
                if hi < lo:
                    raise ReSyntaxError("bad range")
                members.update(range(lo, hi + 1))
            else:
                members.add(lo)
        if neg:
            members = set(range(256)) - members
        if not members:
            raise ReSyntaxError("empty class")
        return frozenset(members)


def parse(re_src) -> tuple:
    """Parse an RE (bytes or str) into the AST above."""
    if isinstance(re_src, str):
        re_src = re_src.encode('latin-1')
    return _Parser(bytes(re_src)).parse()


def expand(node) -> tuple:
    """Rewrite every ``('rep', r, m, n)`` with the convention in the module docstring.

    The result contains only eps/set/cat/alt/star/plus/opt nodes; each copy of ``r`` is a
    separate subtree so that a position automaton gives each copy its own positions.
    """
    kind = node[0]
    if kind in ('eps', 'set'):
        return node
    if kind in ('cat', 'alt'):
        return (kind, tuple(expand(c) for c in node[1]))
    if kind in ('star', 'plus', 'opt'):
        return (kind, expand(node[1]))
    assert kind == 'rep'
    r, m, n = expand(node[1]), node[2], node[3]
    parts = [r] * m
    if n is None:
        parts.append(('star', r))
    elif n > m:
        tail = ('opt', r)
        for _ in range(n - m - 1):
            tail = ('opt', ('cat', (r, tail)))
        parts.append(tail)
    if not parts:
        return ('eps',)
    return parts[0] if len(parts) == 1 else ('cat', tuple(parts))

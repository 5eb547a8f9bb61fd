"""Oracle of the user-defined operators (Section 5.1: user kernels written
against the point / local abstractions).  Test infrastructure only: imported
by tests/, never by the library.

The operator is an integer expression in a small C-like language (integer
literals; a, b, c = a point operator's inputs at the pixel; in(dx, dy) = a
local operator's input at literal offsets under its border mode; unary - + ~;
binary * + - << >> < > <= >= == != & ^ |; min, max, abs; parentheses), with C
precedence and 64-bit two's-complement arithmetic, comparisons 0 or 1, the
result saturated to the output format.  This module parses it with its own
recursive-descent parser and evaluates it on whole numpy int64 arrays, one
node of the expression at a time.
"""
from __future__ import annotations

import re

import numpy as np

from . import BORDER_CONSTANT, BORDER_MIRROR, BORDER_REPEAT, BORDER_REPLICATE, BORDER_UNDEFINED
from . import Img

_TOKEN = re.compile(r"\s*(\d+|[A-Za-z_]\w*|<<|>>|<=|>=|==|!=|[-+~*<>&^|(),])")

# binary levels from the loosest to the tightest (C precedence)
_LEVELS = [["|"], ["^"], ["&"], ["==", "!="], ["<=", ">=", "<", ">"], ["<<", ">>"], ["+", "-"],
           ["*"]]


def _tokens(src: str):
    pos, out = 0, []
    src = src.rstrip()
    while pos < len(src):
        m = _TOKEN.match(src, pos)
        if not m:
            raise ValueError(f"unexpected character at {pos}")
        out.append(m.group(1))
        pos = m.end()
    return out


def _binop(op, x, y):
    if op == "*":
        return x * y
    if op == "+":
        return x + y
    if op == "-":
        return x - y
    if op == "<<":
        return np.left_shift(x, y)
    if op == ">>":
        return np.right_shift(x, y)  # arithmetic for signed int64
    if op in ("<", ">", "<=", ">=", "==", "!="):
        r = {"<": np.less, ">": np.greater, "<=": np.less_equal, ">=": np.greater_equal,
             "==": np.equal, "!=": np.not_equal}[op](x, y)
        return r.astype(np.int64)
    if op == "&":
        return np.bitwise_and(x, y)
    if op == "^":
        return np.bitwise_xor(x, y)
    if op == "|":
        return np.bitwise_or(x, y)
    raise ValueError(op)


class _Eval:
    def __init__(self, src, env, tap):
        self.t = _tokens(src)
        self.i = 0
        self.env = env      # name -> array (point operators)
        self.tap = tap      # (dx, dy) -> array (local operators), or None

    def peek(self):
        return self.t[self.i] if self.i < len(self.t) else None

    def take(self, want=None):
        tok = self.peek()
        if tok is None or (want is not None and tok != want):
            raise ValueError(f"expected {want!r}, got {tok!r}")
        self.i += 1
        return tok

    def level(self, k):
        if k == len(_LEVELS):
            return self.unary()
        x = self.level(k + 1)
        while self.peek() in _LEVELS[k]:
            op = self.take()
            x = _binop(op, x, self.level(k + 1))
        return x

    def unary(self):
        tok = self.peek()
        if tok == "-":
            self.take()
            return -self.unary()
        if tok == "+":
            self.take()
            return self.unary()
        if tok == "~":
            self.take()
            return np.invert(self.unary())
        return self.primary()

    def literal(self):
        neg = self.peek() == "-"
        if neg:
            self.take()
        v = int(self.take())
        return -v if neg else v

    def primary(self):
        tok = self.take()
        if tok == "(":
            x = self.level(0)
            self.take(")")
            return x
        if tok.isdigit():
            return np.int64(int(tok))
        if tok in self.env:
            return self.env[tok]
        if tok == "in" and self.tap is not None:
            self.take("(")
            dx = self.literal()
            self.take(",")
            dy = self.literal()
            self.take(")")
            return self.tap(dx, dy)
        if tok in ("min", "max"):
            self.take("(")
            x = self.level(0)
            self.take(",")
            y = self.level(0)
            self.take(")")
            return np.minimum(x, y) if tok == "min" else np.maximum(x, y)
        if tok == "abs":
            self.take("(")
            x = self.level(0)
            self.take(")")
            return np.abs(x)
        raise ValueError(f"unknown name {tok!r}")

    def run(self):
        x = self.level(0)
        if self.peek() is not None:
            raise ValueError(f"unexpected {self.peek()!r}")
        return x


_RANGE = {np.dtype(np.uint8): (0, 255), np.dtype(np.int16): (-32768, 32767),
          np.dtype(np.int32): (-2 ** 31, 2 ** 31 - 1)}


def _saturate(x, shape, out_dtype):
    lo, hi = _RANGE[np.dtype(out_dtype)]
    return np.clip(np.broadcast_to(np.asarray(x, np.int64), shape), lo, hi).astype(out_dtype)


def user_point(expr: str, inputs, out_dtype) -> Img:
    """A user point operator on 1..3 images (a, b, c); the output is 0
    outside the intersection of their valid rectangles."""
    imgs = [x if isinstance(x, Img) else Img(np.asarray(x)) for x in inputs]
    env = {n: im.data.astype(np.int64) for n, im in zip("abc", imgs)}
    shape = imgs[0].data.shape
    out = _saturate(_Eval(expr, env, None).run(), shape, out_dtype)
    x0 = max(im.rect[0] for im in imgs)
    y0 = max(im.rect[1] for im in imgs)
    x1 = max(x0, min(im.rect[2] for im in imgs))
    y1 = max(y0, min(im.rect[3] for im in imgs))
    mask = np.zeros(shape, bool)
    mask[y0:y1, x0:x1] = True
    return Img(np.where(mask, out, 0).astype(out_dtype), (x0, y0, x1, y1))


_PAD = {BORDER_REPLICATE: "edge", BORDER_MIRROR: "symmetric", BORDER_REPEAT: "wrap"}


def user_local(expr: str, src, kw: int, kh: int, border=BORDER_REPLICATE, cval=0,
               out_dtype=np.int16) -> Img:
    """A user local operator over a kw x kh window: in(dx, dy) reads the input
    at (x + dx, y + dy), outside the image under the border mode.  Under
    UNDEFINED the valid rectangle shrinks by the window radius."""
    im = src if isinstance(src, Img) else Img(np.asarray(src))
    rx, ry = kw // 2, kh // 2
    a = im.data.astype(np.int64)
    h, w = a.shape
    if border == BORDER_CONSTANT:
        p = np.pad(a, ((ry, ry), (rx, rx)), mode="constant", constant_values=cval)
    elif border == BORDER_UNDEFINED:
        p = np.pad(a, ((ry, ry), (rx, rx)), mode="constant", constant_values=0)
    else:
        p = np.pad(a, ((ry, ry), (rx, rx)), mode=_PAD[border])

    def tap(dx, dy):
        if abs(dx) > rx or abs(dy) > ry:
            raise ValueError("offset outside the window")
        return p[ry + dy:ry + dy + h, rx + dx:rx + dx + w]

    out = _saturate(_Eval(expr, {}, tap).run(), a.shape, out_dtype)
    x0, y0, x1, y1 = im.rect
    if border == BORDER_UNDEFINED:
        x0, y0, x1, y1 = x0 + rx, y0 + ry, x1 - rx, y1 - ry
        x1, y1 = max(x0, x1), max(y0, y1)
    mask = np.zeros(a.shape, bool)
    mask[y0:y1, x0:x1] = True
    return Img(np.where(mask, out, 0).astype(out_dtype), (x0, y0, x1, y1))

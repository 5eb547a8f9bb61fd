"""Graph-level oracle: verification, dead-computation elimination, execution.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

A graph is described with plain Python objects, independently of the CUDA
library's C ABI:

* ``GraphDesc.image(name, w, h, fmt)`` / ``GraphDesc.virtual(name)`` declare the
  data vertices D = D_nv U D_v (Section 5.2, Section 5.2.1);
* ``GraphDesc.node(kind, ins, outs, **params)`` declares a CV-function node.

``implementation_graph`` lowers each CV-function node to single-output
point/local abstraction ops (Section 4: Sobel3x3 becomes two parallel local
operators, as the paper's edge-detection example does).  ``verify`` applies
the checks Section 5.2 requires (no cycle, bipartite edges) plus the parameter
checks Section 3.1 lists (presence, data types).  ``eliminate_dead`` follows
Algorithm 1 step by step.  ``run`` executes the alive ops in dependency order
with the node functions of ``oracle`` (the C oracle).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

import oracle as O

FORMATS = ("U8", "S16", "S32", "F32", "UYVY")


@dataclass
class Data:
    name: str
    virtual: bool
    w: int = 0
    h: int = 0
    fmt: str = ""


@dataclass
class Op:
    """One point/local abstraction op with exactly one output data vertex."""
    name: str
    kind: str
    ins: list
    out: str
    params: dict = field(default_factory=dict)
    node: int = -1     # index of the CV-function node it was lowered from


class GraphError(ValueError):
    pass


class GraphDesc:
    def __init__(self):
        self.data: dict[str, Data] = {}
        self.nodes: list[tuple[str, list, list, dict]] = []

    def image(self, name, w, h, fmt):
        assert fmt in FORMATS
        self.data[name] = Data(name, False, w, h, fmt)
        return name

    def virtual(self, name, w=0, h=0, fmt=""):
        self.data[name] = Data(name, True, w, h, fmt)
        return name

    def node(self, kind, ins, outs, **params):
        self.nodes.append((kind, list(ins), list(outs), dict(params)))
        return len(self.nodes) - 1


# --- lowering of CV functions to abstraction ops (Section 4, Table 2) ---------

def implementation_graph(g: GraphDesc) -> list[Op]:
    ops = []
    for idx, (kind, ins, outs, params) in enumerate(g.nodes):
        if kind == "sobel3x3":
            # one local operator per derivative; an absent output makes no op
            if outs[0] is not None:
                ops.append(Op(f"n{idx}.gx", "sobel_x", ins, outs[0], params, idx))
            if len(outs) > 1 and outs[1] is not None:
                ops.append(Op(f"n{idx}.gy", "sobel_y", ins, outs[1], params, idx))
        else:
            if len(outs) != 1 or outs[0] is None:
                raise GraphError(f"node {idx} ({kind}) needs one output")
            ops.append(Op(f"n{idx}", kind, ins, outs[0], params, idx))
    return ops


def edges(g: GraphDesc, ops: list[Op]):
    """E of G_app over V = D U N: data -> op for each input, op -> data for
    the output (Section 5.2)."""
    E = []
    for op in ops:
        for i in op.ins:
            E.append((("D", i), ("N", op.name)))
        E.append((("N", op.name), ("D", op.out)))
    return E


# --- verification (Section 3.1, Section 5.2) -------------------------------------

_POINT_OUT = {"magnitude": "S16", "phase": "U8", "threshold": "U8", "mul": "S32",
              "harris_response": "F32", "tomasi_response": "F32", "and": "U8", "or": "U8",
              "xor": "U8", "not": "U8"}
_LOCAL_OUT = {"gaussian3x3": "U8", "box3x3": "U8", "sobel_x": "S16", "sobel_y": "S16",
              "window_sum": "S32", "dilate3x3": "U8", "erode3x3": "U8", "median3x3": "U8"}
_IN_FMTS = {
    "gaussian3x3": [("U8",)], "box3x3": [("U8",)], "sobel_x": [("U8",)],
    "sobel_y": [("U8",)], "window_sum": [("S32",)], "convolve": [("U8",)],
    "magnitude": [("S16",), ("S16",)], "phase": [("S16",), ("S16",)],
    "threshold": [("U8", "S16", "S32", "F32")], "mul": [("S16",), ("S16",)],
    "harris_response": [("S32",), ("S32",), ("S32",)],
    "tomasi_response": [("S32",), ("S32",), ("S32",)],
    "channel_extract": [("UYVY",)],
    "add": [("U8", "S16"), ("U8", "S16")], "subtract": [("U8", "S16"), ("U8", "S16")],
    "absdiff": [("U8", "S16"), ("U8", "S16")],
    "multiply": [("U8", "S16"), ("U8", "S16")],
    "convert_depth": [("U8", "S16")], "copy": [("U8", "S16")],
    "dilate3x3": [("U8",)], "erode3x3": [("U8",)], "median3x3": [("U8",)],
    "and": [("U8",), ("U8",)], "or": [("U8",), ("U8",)], "xor": [("U8",), ("U8",)],
    "not": [("U8",)],
}


def has_cycle(g: GraphDesc, ops: list[Op]) -> bool:
    """Depth-first search for a back edge over G_app."""
    succ: dict = {}
    for a, b in edges(g, ops):
        succ.setdefault(a, []).append(b)
    WHITE, GREY, BLACK = 0, 1, 2
    colour: dict = {}
    for start in list(succ):
        if colour.get(start, WHITE) != WHITE:
            continue
        stack = [(start, iter(succ.get(start, ())))]
        colour[start] = GREY
        while stack:
            v, it = stack[-1]
            nxt = next(it, None)
            if nxt is None:
                colour[v] = BLACK
                stack.pop()
                continue
            c = colour.get(nxt, WHITE)
            if c == GREY:
                return True
            if c == WHITE:
                colour[nxt] = GREY
                stack.append((nxt, iter(succ.get(nxt, ()))))
    return False


def is_bipartite(E) -> bool:
    """Every edge joins a data vertex and a node vertex (Section 5.2)."""
    return all((a[0] == "D" and b[0] == "N") or (a[0] == "N" and b[0] == "D") for a, b in E)


def verify(g: GraphDesc) -> list[Op]:
    """Raise GraphError for a graph Section 5.2 / Section 3.1 would reject;
    otherwise resolve every virtual image's size and format and return the
    implementation ops."""
    ops = implementation_graph(g)
    for op in ops:
        for name in op.ins + [op.out]:
            if name is None or name not in g.data:
                raise GraphError(f"{op.name}: missing parameter")
    writers: dict = {}
    for op in ops:
        if op.out in writers:
            raise GraphError(f"{op.out} has two writers")
        writers[op.out] = op
    if not is_bipartite(edges(g, ops)):
        raise GraphError("not bipartite")
    if has_cycle(g, ops):
        raise GraphError("cycle")
    for d in g.data.values():
        if d.virtual and d.name not in writers and any(d.name in op.ins for op in ops):
            raise GraphError(f"virtual image {d.name} is read but never written")
    # resolve virtual sizes/formats in dependency order
    done = {d.name for d in g.data.values() if not d.virtual}
    pending = list(ops)
    order = []
    while pending:
        progress = False
        for op in list(pending):
            if all(i in done for i in op.ins):
                _infer(g, op)
                done.add(op.out)
                order.append(op)
                pending.remove(op)
                progress = True
        if not progress:
            raise GraphError("unresolvable inputs")
    return order


def _infer(g: GraphDesc, op: Op):
    allowed = _IN_FMTS.get(op.kind)
    if allowed is None:
        raise GraphError(f"unknown kind {op.kind}")
    if len(op.ins) != len(allowed):
        raise GraphError(f"{op.name}: wrong input count")
    ins = [g.data[i] for i in op.ins]
    for d, fm in zip(ins, allowed):
        if d.fmt not in fm:
            raise GraphError(f"{op.name}: format {d.fmt} not accepted")
    w, h = ins[0].w, ins[0].h
    if op.kind == "channel_extract":
        ch = op.params.get("channel", 0)
        ow, oh, of = (w if ch == 0 else w // 2), h, "U8"
    else:
        for d in ins[1:]:
            if (d.w, d.h) != (w, h):
                raise GraphError(f"{op.name}: input sizes differ")
        ow, oh = w, h
        if op.kind in _POINT_OUT:
            of = _POINT_OUT[op.kind]
        elif op.kind in _LOCAL_OUT:
            of = _LOCAL_OUT[op.kind]
        elif op.kind == "convolve":  # U8 or S16 output: the output image decides
            of = g.data[op.out].fmt or "S16"
            if of not in ("U8", "S16"):
                raise GraphError(f"{op.name}: convolve output must be U8 or S16")
        else:  # add / subtract / absdiff: the output image's own format decides
            of = g.data[op.out].fmt or ("S16" if "S16" in [d.fmt for d in ins] else "U8")
    out = g.data[op.out]
    if out.virtual:
        if out.w and (out.w, out.h) != (ow, oh):
            raise GraphError(f"{op.out}: size mismatch")
        if out.fmt and out.fmt != of:
            raise GraphError(f"{op.out}: format mismatch")
        out.w, out.h, out.fmt = ow, oh, of
    else:
        if (out.w, out.h) != (ow, oh) or out.fmt != of:
            raise GraphError(f"{op.out}: output image does not match {op.kind}")


# --- Algorithm 1: dead computation elimination -------------------------------

def eliminate_dead(g: GraphDesc, ops: list[Op]):
    """Algorithm 1 (Section 5.2.2), in the paper's order and notation.

    Returns (alive_ops, alive_data): the vertex sets of G_filt."""
    E = edges(g, ops)
    deg_in: dict = {}
    deg_out: dict = {}
    for a, b in E:
        deg_out[a] = deg_out.get(a, 0) + 1
        deg_in[b] = deg_in.get(b, 0) + 1
    D_nv = [("D", d.name) for d in g.data.values() if not d.virtual]
    # candidate non-virtual roots and leaves
    D_in, D_out = set(), set()
    for v in D_nv:
        if deg_in.get(v, 0) == 0:
            D_in.add(v)
        elif deg_out.get(v, 0) == 0:
            D_out.add(v)
        else:
            D_in.add(v)
            D_out.add(v)
    # G_trans: every edge reversed
    G_trans: dict = {}
    for a, b in E:
        G_trans.setdefault(b, []).append(a)
    V_alive = set()
    for v_start in sorted(D_out):
        V_alive |= _depth_first_visit(v_start, D_in, G_trans)
    alive_ops = [op for op in ops if ("N", op.name) in V_alive]
    alive_data = {v[1] for v in V_alive if v[0] == "D"}
    return alive_ops, alive_data


def _depth_first_visit(v_start, D_in, G_trans):
    """Vertices reachable from v_start in G_trans; a vertex of D_in other than
    v_start ends its branch (it is a root of the application)."""
    seen = {v_start}
    stack = [v_start]
    while stack:
        v = stack.pop()
        if v != v_start and v in D_in:
            continue
        for u in G_trans.get(v, ()):
            if u not in seen:
                seen.add(u)
                stack.append(u)
    return seen


# --- execution -----------------------------------------------------------------

_BORDER = {"undefined": O.BORDER_UNDEFINED, "replicate": O.BORDER_REPLICATE,
           "constant": O.BORDER_CONSTANT, "mirror": O.BORDER_MIRROR, "repeat": O.BORDER_REPEAT}
_ROUND = {"zero": O.ROUND_ZERO, "nearest": O.ROUND_NEAREST}
_ARITH = {"add": O.ARITH_ADD, "subtract": O.ARITH_SUB, "absdiff": O.ARITH_ABSDIFF}
_MORPH = {"dilate3x3": O.MORPH_DILATE, "erode3x3": O.MORPH_ERODE, "median3x3": O.MORPH_MEDIAN}
_BITS = {"and": O.BIT_AND, "or": O.BIT_OR, "xor": O.BIT_XOR, "not": O.BIT_NOT}
_NPFMT = {"U8": np.uint8, "S16": np.int16, "S32": np.int32, "F32": np.float32}


def run(g: GraphDesc, inputs: dict, dce: bool = True) -> dict:
    """Execute the graph node by node on the CPU; return every non-virtual
    image that an alive op writes, as oracle.Img (data + valid rectangle)."""
    order = verify(g)
    alive = eliminate_dead(g, order)[0] if dce else order
    alive_names = {op.name for op in alive}
    vals: dict = {}
    for name, arr in inputs.items():
        vals[name] = O.Img(arr)
    for op in order:
        if op.name not in alive_names:
            continue
        p = op.params
        b = _BORDER[p.get("border", "replicate")]
        c = int(p.get("cval", 0))
        x = [vals[i] for i in op.ins]
        k = op.kind
        if k == "gaussian3x3":
            r = O.gaussian3x3(x[0], b, c, _ROUND[p.get("rounding", "zero")])
        elif k == "box3x3":
            r = O.box3x3(x[0], b, c, _ROUND[p.get("rounding", "zero")])
        elif k in ("sobel_x", "sobel_y"):
            gx, gy = O.sobel3x3(x[0], b, c)
            r = gx if k == "sobel_x" else gy
        elif k == "window_sum":
            r = O.window_sum(x[0], p.get("kw", 5), p.get("kh", 5), b, c)
        elif k == "convolve":
            r = O.convolve(x[0], p["coeffs"], p.get("shift", 0), b, c,
                           _NPFMT[g.data[op.out].fmt])
        elif k == "magnitude":
            r = O.magnitude(x[0], x[1])
        elif k == "phase":
            r = O.phase(x[0], x[1])
        elif k == "threshold":
            if p.get("type", "binary") == "binary":
                r = O.threshold(x[0], p["value"], p.get("true_value", 255),
                                p.get("false_value", 0))
            else:
                r = O.threshold_range(x[0], p["lower"], p["upper"], p.get("true_value", 255),
                                      p.get("false_value", 0))
        elif k == "mul":
            r = O.mul_s32(x[0], x[1])
        elif k == "tomasi_response":
            r = O.tomasi_response(x[0], x[1], x[2])
        elif k == "harris_response":
            r = O.harris_response(x[0], x[1], x[2], p.get("kn", 1), p.get("kd", 25))
        elif k == "channel_extract":
            r = O.channel_extract_uyvy(x[0].data, p.get("channel", 0))
        elif k in _MORPH:
            r = O.morph3x3(x[0], _MORPH[k], b, c)
        elif k in _BITS:
            r = O.bitwise(x[0], x[1] if k != "not" else None, _BITS[k])
        elif k in ("convert_depth", "copy"):
            r = O.convert_depth(x[0], _NPFMT[g.data[op.out].fmt], p.get("shift", 0),
                                p.get("policy", "saturate") == "saturate")
        elif k == "multiply":
            r = O.multiply(x[0], x[1], p.get("scale", 1.0), _NPFMT[g.data[op.out].fmt],
                           p.get("policy", "saturate") == "saturate",
                           p.get("rounding", "zero") == "nearest_even")
        elif k in _ARITH:
            r = O.arith(x[0], x[1], _NPFMT[g.data[op.out].fmt], _ARITH[k],
                        p.get("policy", "saturate") == "saturate")
        else:
            raise GraphError(k)
        vals[op.out] = r
    return {n: v for n, v in vals.items() if not g.data[n].virtual and n not in inputs}

"""NumPy-style slice-assignment frontend over the stencil library.

The paper's programming model (Sec. III-A, Example 1; Sec. III-B Frontend):
a program creates arrays and assigns to array slices expressions over
shifted slices of other arrays, e.g. the 2D Laplace (Jacobi) solver

    u1 = create_array((n, n)); u2 = create_array((n, n))
    u1[0, :] = u1[-1, :] = u1[:, 0] = u1[:, -1] = 1      # boundary ring
    u2[0, :] = u2[-1, :] = u2[:, 0] = u2[:, -1] = 1
    for i in range(iters):
        u2[1:-1, 1:-1] = 0.25 * (u1[:-2, 1:-1] + u1[2:, 1:-1] + u1[1:-1, :-2] + u1[1:-1, 2:])
        u1, u2 = u2, u1
    sync()

What this module does with such a program, step by step as the paper
describes its frontend and backend:

* Every slice assignment becomes a node holding a *parameterised* AST: the
  expression's structure with the arrays replaced by numbered parameters
  (Sec. III-B "Execution graph").  Swapping the Python names of two arrays
  changes the node's arguments, not its AST, so all iterations of the loop
  above share one AST and one lowered kernel.
* An expression that reads the array it assigns to is rejected
  (Sec. III-A: the frontend detects such dependencies and raises an error).
* Nodes form a DAG whose edges are the true, anti and output dependencies,
  tracked per array, not per index (Sec. III-B).  The DAG goes to the
  backend when ``sync()`` is called or when its depth passes a configurable
  maximum.
* Node fusion (Sec. III-B "Node fusion"): consecutive nodes in program order
  with the same output shape and no path between them are fused.
* Lowering (Sec. III-C "Code generation"): an AST whose right-hand side is a
  linear combination of shifted slices of one array, written to the interior
  of another array of the same shape, becomes the library's stencil update
  u_out[p] = sum_k w_k u_in[p + o_k] with offsets o_k read off the slice
  bounds and weights w_k from the constant factors; the ghost width of an
  array is the largest offset of the kernels that touch it (Sec. III-C
  "Data layout").  The ring outside the interior is the Dirichlet boundary:
  when both arrays' rings hold one value it becomes the sweep's boundary
  value (Example 1's ring of 1s); otherwise (per-face or varying values) the
  rings are handed to the library as caller-owned ghost cells, which every
  sweep reads and none writes.
* Execution: a run of nodes with the same AST that alternate between the same
  two arrays (the ``u1, u2 = u2, u1`` loop) becomes ONE ``stencil_step(n)``
  call on a grid handle whose two time-level buffers are the two arrays'
  storage, captured by the library as a CUDA graph.  A fused group of
  independent 2D radius-1 sweeps over arrays of one shape becomes one
  ``stencil_batch_step`` launch of the batched persistent kernel (one launch
  for several fields); repeated fused groups alternate the same way.

Every sweep runs in libstencil's kernels; this module only records,
analyses, allocates (through torch) and calls the C ABI.  Expressions that
do not lower (products of arrays, a constant term, an output region other
than a centred interior, several input arrays, assignments to an array after
a sweep has written it on the device) raise
``UnsupportedExpression``; there is no CPU evaluation path.
"""
from __future__ import annotations

import numbers
from dataclasses import dataclass, field

import numpy as np

__all__ = ["create_array", "sync", "Array", "Program", "FrontendError", "DependencyError",
           "UnsupportedExpression", "default_program", "set_max_depth"]


class FrontendError(Exception):
    """Base class of the frontend's errors."""


class DependencyError(FrontendError):
    """An assignment reads the array it writes (Sec. III-A)."""


class UnsupportedExpression(FrontendError):
    """An assignment the stencil library cannot execute."""


# ---------------------------------------------------------------------------
# Expressions
# ---------------------------------------------------------------------------
def _region(shape, key):
    """Normalise a basic-slicing key to per-axis half-open (start, stop)."""
    if not isinstance(key, tuple):
        key = (key,)
    if len(key) > len(shape):
        raise IndexError("too many indices")
    key = key + (slice(None),) * (len(shape) - len(key))
    out = []
    for k, n in zip(key, shape):
        if isinstance(k, slice):
            if k.step not in (None, 1):
                raise UnsupportedExpression("slices with a step are not stencil accesses")
            a, b, _ = k.indices(n)
            out.append((a, max(a, b)))
        elif isinstance(k, numbers.Integral):
            i = int(k) + (n if k < 0 else 0)
            if not 0 <= i < n:
                raise IndexError("index out of range")
            out.append((i, i + 1))
        else:
            raise UnsupportedExpression(f"index {k!r} is not an integer or a slice")
    return tuple(out)


def _extent(region):
    return tuple(b - a for a, b in region)


class Expr:
    """A node of an assignment's right-hand side."""

    def _wrap(self, o):
        if isinstance(o, Expr):
            return o
        if isinstance(o, numbers.Real):
            return Const(float(o))
        return NotImplemented

    def __add__(self, o):
        o = self._wrap(o)
        return o if o is NotImplemented else Bin("+", self, o)

    def __radd__(self, o):
        o = self._wrap(o)
        return o if o is NotImplemented else Bin("+", o, self)

    def __sub__(self, o):
        o = self._wrap(o)
        return o if o is NotImplemented else Bin("-", self, o)

    def __rsub__(self, o):
        o = self._wrap(o)
        return o if o is NotImplemented else Bin("-", o, self)

    def __mul__(self, o):
        o = self._wrap(o)
        return o if o is NotImplemented else Bin("*", self, o)

    def __rmul__(self, o):
        o = self._wrap(o)
        return o if o is NotImplemented else Bin("*", o, self)

    def __truediv__(self, o):
        o = self._wrap(o)
        return o if o is NotImplemented else Bin("/", self, o)

    def __neg__(self):
        return Bin("*", Const(-1.0), self)

    def __pos__(self):
        return self


@dataclass(eq=False)
class Const(Expr):
    value: float


@dataclass(eq=False)
class Ref(Expr):
    array: "Array"
    region: tuple


@dataclass(eq=False)
class Bin(Expr):
    op: str
    a: Expr
    b: Expr


def _parameterise(expr, out):
    """(AST key, argument arrays): arrays become parameters numbered by first
    appearance, the output array being parameter 0."""
    args = [out]
    index = {id(out): 0}

    def walk(e):
        if isinstance(e, Const):
            return ("c", e.value)
        if isinstance(e, Ref):
            k = index.get(id(e.array))
            if k is None:
                k = index[id(e.array)] = len(args)
                args.append(e.array)
            return ("r", k, e.region)
        return (e.op, walk(e.a), walk(e.b))

    return walk(expr), args


def _linear(ast):
    """Linear form of an AST: ({(param, region): weight}, constant), terms in
    order of first appearance.  Products need a constant side; quotients a
    constant divisor."""
    kind = ast[0]
    if kind == "c":
        return {}, ast[1]
    if kind == "r":
        return {(ast[1], ast[2]): 1.0}, 0.0
    ta, ca = _linear(ast[1])
    tb, cb = _linear(ast[2])
    if kind in "+-":
        s = 1.0 if kind == "+" else -1.0
        terms = dict(ta)
        for k, v in tb.items():
            terms[k] = terms.get(k, 0.0) + s * v
        return terms, ca + s * cb
    if kind == "*":
        if ta and tb:
            raise UnsupportedExpression("a product of two array slices is not a linear stencil")
        if ta:
            return {k: v * cb for k, v in ta.items()}, ca * cb
        return {k: v * ca for k, v in tb.items()}, ca * cb
    if kind == "/":
        if tb:
            raise UnsupportedExpression("division by an array slice is not a linear stencil")
        return {k: v / cb for k, v in ta.items()}, ca / cb
    raise UnsupportedExpression(f"operator {kind}")


@dataclass(frozen=True)
class Lowered:
    """A stencil update read off an AST: out[interior] = sum_k w_k in[p + o_k]."""
    ghost: int          # width of the ring outside the written interior
    offsets: tuple      # ((dy, dx) or (dz, dy, dx), ...) in order of appearance
    weights: tuple
    radius: int         # largest offset component


def _lower(ast, out_region, shape):
    """Read the stencil off a parameterised AST (parameter 0 = output,
    parameter 1 = the one input array).  Raises UnsupportedExpression."""
    terms, const = _linear(ast)
    if const != 0.0:
        raise UnsupportedExpression("a constant term is not part of the stencil update")
    ghosts = {a for a, _ in out_region} | {n - b for (_, b), n in zip(out_region, shape)}
    if len(ghosts) != 1:
        raise UnsupportedExpression("the written region must be the array's interior, the same width from every edge")
    g = ghosts.pop()
    if g < 1:
        raise UnsupportedExpression("the written region leaves no boundary ring")
    ext = _extent(out_region)
    offsets, weights = [], []
    for (param, region), w in terms.items():
        if param != 1:
            raise UnsupportedExpression("a stencil reads exactly one input array")
        if _extent(region) != ext:
            raise UnsupportedExpression("an operand slice's extent differs from the written region's")
        if w == 0.0:
            continue
        offsets.append(tuple(r[0] - o[0] for r, o in zip(region, out_region)))
        weights.append(w)
    if not offsets:
        raise UnsupportedExpression("the expression reads no array")
    radius = max(abs(c) for o in offsets for c in o)
    if radius > g:
        raise UnsupportedExpression("an offset reaches beyond the boundary ring")
    return Lowered(g, tuple(offsets), tuple(weights), radius)


# ---------------------------------------------------------------------------
# Arrays and the program (DAG)
# ---------------------------------------------------------------------------
class Array:
    """A frontend array.  Its data lives on the host until a sweep needs it,
    then in a padded device buffer in the library's layout (the array being
    the interior plus the ring of its ghost width)."""

    def __init__(self, program, shape, dtype):
        self.program = program
        self.shape = tuple(int(s) for s in shape)
        self.dtype = np.dtype(dtype)
        if self.dtype not in (np.float32, np.float64):
            raise TypeError("float32 or float64 arrays only")
        if len(self.shape) not in (2, 3) or min(self.shape) < 1:
            raise ValueError("2D or 3D arrays with positive extents")
        self.host = np.zeros(self.shape, dtype=self.dtype)
        self.dev = None        # padded torch buffer once on the device
        self.ghost = None      # ghost width of the device layout
        self.view = None       # the array's region of the padded buffer

    def __getitem__(self, key):
        return Ref(self, _region(self.shape, key))

    def __setitem__(self, key, value):
        self.program.assign(self, _region(self.shape, key), value)

    def set(self, values) -> None:
        """Replace the whole array (host data; before the array is on the device)."""
        self.program.assign(self, tuple((0, n) for n in self.shape), np.asarray(values, dtype=self.dtype))

    def get(self) -> np.ndarray:
        """Flush the program and return a host copy of the array."""
        self.program.sync()
        if self.dev is None:
            return self.host.copy()
        return self.view.cpu().numpy().copy()


@dataclass(eq=False)
class Node:
    kind: str                       # "fill" or "stencil"
    out: Array
    region: tuple
    value: object = None            # fill: scalar or array
    ast: object = None              # stencil: parameterised AST (hashable)
    args: list = field(default_factory=list)  # stencil: [out, in]
    lowered: Lowered | None = None
    preds: set = field(default_factory=set)   # indices of nodes this one depends on
    depth: int = 1


class Program:
    """Records slice assignments as a DAG and executes it on ``sync``."""

    def __init__(self, max_depth: int = 1 << 16, device=None, tune: bool = True):
        self.max_depth = int(max_depth)
        self.device = device
        self.tune = bool(tune)      # autotune tunable grid handles on their first run
        self.nodes: list[Node] = []
        self.asts: dict = {}        # AST -> Lowered (or the exception it raised)
        self._last_writer: dict = {}
        self._readers: dict = {}
        self._handles: dict = {}
        self.executed: list = []    # per flush: ("fill", 1, 1) / ("run", members, repeats)

    # -- capture -----------------------------------------------------------
    def create_array(self, shape, dtype=np.float64) -> Array:
        return Array(self, shape, dtype)

    def _lower_cached(self, ast, region, shape):
        key = (ast, region, shape)
        hit = self.asts.get(key)
        if hit is None:
            try:
                hit = _lower(ast, region, shape)
            except UnsupportedExpression as e:
                hit = e
            self.asts[key] = hit
        if isinstance(hit, Exception):
            raise UnsupportedExpression(str(hit))
        return hit

    def assign(self, out: Array, region, value) -> None:
        if isinstance(value, Expr):
            ast, args = _parameterise(value, out)
            if any(a is out for a in args[1:]) or _reads(ast, 0):
                raise DependencyError("an assignment reads the array it writes; use a second array and swap")
            for a in args[1:]:
                if a.shape != out.shape:
                    raise UnsupportedExpression("input and output arrays differ in shape")
                if a.dtype != out.dtype:
                    raise UnsupportedExpression("input and output arrays differ in dtype")
            lowered = self._lower_cached(ast, region, out.shape)
            node = Node("stencil", out, region, ast=ast, args=args, lowered=lowered)
            reads = args[1:]
        else:
            if isinstance(value, np.ndarray):
                v = np.asarray(value, dtype=out.dtype)
                if v.shape != _extent(region):
                    v = np.broadcast_to(v, _extent(region))
            elif isinstance(value, numbers.Real):
                v = float(value)
            else:
                raise UnsupportedExpression(f"cannot assign {type(value).__name__}")
            node = Node("fill", out, region, value=v)
            reads = []
        i = len(self.nodes)
        # array-level dependencies: true (read after write), anti (write after
        # read) and output (write after write)
        for a in reads:
            w = self._last_writer.get(id(a))
            if w is not None:
                node.preds.add(w)
        w = self._last_writer.get(id(out))
        if w is not None:
            node.preds.add(w)
        node.preds |= self._readers.get(id(out), set())
        node.preds.discard(i)
        node.depth = 1 + max((self.nodes[p].depth for p in node.preds), default=0)
        self.nodes.append(node)
        for a in reads:
            self._readers.setdefault(id(a), set()).add(i)
        self._last_writer[id(out)] = i
        self._readers[id(out)] = set()
        if node.depth > self.max_depth:
            self.sync()

    def depth(self) -> int:
        return max((n.depth for n in self.nodes), default=0)

    def edges(self):
        return sorted((p, i) for i, n in enumerate(self.nodes) for p in n.preds)

    # -- analysis ----------------------------------------------------------
    def fused_groups(self):
        """Node fusion (Sec. III-B): consecutive nodes with the same output
        shape and no dependency between any two of them form one group."""
        groups, cur = [], []
        for i, n in enumerate(self.nodes):
            if cur and n.kind == "stencil" and self.nodes[cur[0]].kind == "stencil" and \
                    n.out.shape == self.nodes[cur[0]].out.shape and not (n.preds & set(cur)):
                cur.append(i)
            else:
                if cur:
                    groups.append(cur)
                cur = [i]
        if cur:
            groups.append(cur)
        return groups

    def plan(self):
        """The launch plan of the recorded nodes: a list of
        ("fill", node) and ("run", [node indices of the first group], n)
        entries, where a run repeats a fused group n times with each member
        alternating between its two arrays."""
        out = []
        groups = self.fused_groups()
        k = 0
        while k < len(groups):
            g = groups[k]
            first = self.nodes[g[0]]
            if first.kind == "fill":
                out.append(("fill", g[0]))
                k += 1
                continue
            n = 1
            prev = g
            while k + n < len(groups) and _continues(self.nodes, prev, groups[k + n]):
                prev = groups[k + n]
                n += 1
            out.append(("run", list(g), n))
            k += n
        return out

    # -- execution ---------------------------------------------------------
    def sync(self) -> None:
        """Send the recorded DAG to the library and wait for it."""
        if not self.nodes:
            return
        plan = self.plan()
        nodes = self.nodes
        self.nodes, self._last_writer, self._readers = [], {}, {}
        self.executed.append([("fill", 1, 1) if p[0] == "fill" else ("run", len(p[1]), p[2]) for p in plan])
        _Executor(self).run(plan, nodes)

    def close(self) -> None:
        for h in self._handles.values():
            h.close()
        self._handles.clear()


def _reads(ast, param):
    if ast[0] == "c":
        return False
    if ast[0] == "r":
        return ast[1] == param
    return _reads(ast[1], param) or _reads(ast[2], param)


def _continues(nodes, prev, group):
    """True if `group` repeats `prev` with every member's arrays swapped."""
    if len(prev) != len(group):
        return False
    for i, j in zip(prev, group):
        a, b = nodes[i], nodes[j]
        if b.kind != "stencil" or a.ast != b.ast or a.region != b.region:
            return False
        if b.args[1] is not a.args[0] or b.args[0] is not a.args[1]:
            return False
    return True


# ---------------------------------------------------------------------------
# Backend: device storage and library calls
# ---------------------------------------------------------------------------
class _Executor:
    def __init__(self, prog: Program):
        import torch

        from . import abi
        self.torch, self.abi, self.prog = torch, abi, prog
        if not torch.cuda.is_available():
            raise RuntimeError("the stencil frontend executes on a CUDA device; none is available")
        self.device = torch.device(prog.device) if prog.device is not None else \
            torch.device("cuda", torch.cuda.current_device())
        self.stream = torch.cuda.current_stream(self.device)

    def run(self, plan, nodes) -> None:
        for p in plan:
            if p[0] == "fill":
                self._fill(nodes[p[1]])
            else:
                self._run([nodes[i] for i in p[1]], p[2])
        self.torch.cuda.synchronize(self.device)

    # host-side initial data
    def _fill(self, node: Node) -> None:
        a = node.out
        if a.dev is not None:
            raise UnsupportedExpression("assignment to an array after a sweep wrote it on the device")
        a.host[tuple(slice(lo, hi) for lo, hi in node.region)] = node.value

    def _layout(self, shape, g, dtype):
        """Padded shape and interior origin of the library layout."""
        key = ("layout", shape, g, dtype.str)
        hit = self.prog._handles.get(key)
        if hit is None:
            abi = self.abi
            nd = len(shape)
            dims = tuple(n - 2 * g for n in shape)
            offs = [(0,) * nd]
            h = abi.stencil_create(nd, dims, g, offs, [1.0], None, abi.ST_DIRICHLET, 0.0,
                                   abi.ST_F64 if dtype == np.float64 else abi.ST_F32, 1, 0)
            padded, origin, _ = abi.stencil_layout(h, nd)
            abi.stencil_destroy(h)
            hit = _Layout(tuple(padded), tuple(origin))
            self.prog._handles[key] = hit
        return hit

    def _place(self, a: Array, g: int) -> None:
        """Give an array its padded device buffer (ghost width g) and upload it."""
        torch = self.torch
        if a.dev is not None:
            if a.ghost != g:
                raise UnsupportedExpression("an array is used with two different ghost widths")
            return
        lay = self._layout(a.shape, g, a.dtype)
        tdt = torch.float64 if a.dtype == np.float64 else torch.float32
        a.dev = torch.zeros(lay.padded, dtype=tdt, device=self.device)
        a.ghost = g
        a.view = a.dev[tuple(slice(o - g, o - g + n) for o, n in zip(lay.origin, a.shape))]
        a.view.copy_(torch.from_numpy(a.host))
        a.boundary = _ring_value(a.host, g)
        a.host = None

    def _run(self, members, n) -> None:
        for m in members:
            for a in m.args:
                self._place(a, m.lowered.ghost)
        if len(members) > 1 and _batchable(members):
            self._run_batch(members, n)
        else:
            for m in members:
                self._run_single(m, n)

    def _grid(self, m: Node, n: int):
        """The grid handle of a node's stencil over its two arrays' buffers.
        A handle keeps the same two buffers for life (bound once, slot A =
        the first run's input), so the library's captured graphs stay valid;
        later runs only choose which slot is current.  A new handle on the
        persistent 2D tile kernel is autotuned for runs of up to 20 steps
        (the tuner uses the output buffer, whose contents the run replaces,
        as scratch and puts the input back)."""
        abi = self.abi
        lo, src, dst = m.lowered, m.args[1], m.args[0]
        pair = frozenset((src.dev.data_ptr(), dst.dev.data_ptr()))
        # one value on both rings: the library's Dirichlet value (it fills the
        # ghosts with it); otherwise the rings are the caller's ghost cells,
        # which the sweep reads and never writes
        uniform = src.boundary is not None and src.boundary == dst.boundary
        mode = ("bc", dst.boundary) if uniform else ("caller",)
        key = ("grid", dst.shape, lo, dst.dtype.str, mode, pair)
        h = self.prog._handles.get(key)
        if h is None:
            dims = tuple(s - 2 * lo.ghost for s in dst.shape)
            h = _Handle(abi, abi.stencil_create(len(dims), dims, lo.ghost, list(lo.offsets), list(lo.weights), None,
                                                abi.ST_DIRICHLET, dst.boundary if uniform else 0.0,
                                                abi.ST_F64 if dst.dtype == np.float64 else abi.ST_F32, 1,
                                                0 if uniform else abi.ST_FLAG_CALLER_GHOSTS), False)
            self.prog._handles[key] = h
            abi.stencil_bind(h.h, abi.ST_SLOT_A, src.dev.data_ptr())
            abi.stencil_bind(h.h, abi.ST_SLOT_B, dst.dev.data_ptr())
            h.slots = [(src.dev.data_ptr(), dst.dev.data_ptr())]
            if self.prog.tune and abi.stencil_info(h.h)[2] == "tile2d_persistent":
                abi.stencil_tune(h.h, min(n, 20), self.stream)
        return h

    def _run_single(self, m: Node, n: int) -> None:
        """n sweeps of one node's stencil, alternating between its two arrays.
        The first sweep reads args[1] and writes args[0]."""
        abi = self.abi
        h = self._grid(m, n)
        src, dst = m.args[1], m.args[0]
        abi.stencil_set_current(h.h, 0 if h.slots[0][0] == src.dev.data_ptr() else 1)
        # n - 1 steps, then one: whatever passes the library fuses, the last
        # two levels end up in the two buffers
        if n > 1:
            abi.stencil_step(h.h, n - 1, self.stream)
        abi.stencil_step(h.h, 1, self.stream)
        _settle(src, dst, h.slots[0][abi.stencil_current(h.h)], n)

    def _run_batch(self, members, n) -> None:
        abi = self.abi
        offs = []
        for m in members:
            for o in m.lowered.offsets:
                if o not in offs:
                    offs.append(o)
        wts = []
        for m in members:
            w = dict(zip(m.lowered.offsets, m.lowered.weights))
            wts.extend(w.get(o, 0.0) for o in offs)
        a0 = members[0].args[0]
        dims = [tuple(s - 2 for s in m.args[0].shape) for m in members]
        pairs = tuple(frozenset((m.args[1].dev.data_ptr(), m.args[0].dev.data_ptr())) for m in members)
        key = ("batch", tuple(dims), tuple(offs), tuple(wts), a0.dtype.str, a0.boundary, pairs)
        h = self.prog._handles.get(key)
        srcs = [m.args[1].dev.data_ptr() for m in members]
        dsts = [m.args[0].dev.data_ptr() for m in members]
        if h is None:
            h = _Handle(abi, abi.stencil_batch_create(dims, offs, wts, abi.ST_DIRICHLET, a0.boundary,
                                                      abi.ST_F64 if a0.dtype == np.float64 else abi.ST_F32, 0),
                        True)
            self.prog._handles[key] = h
            h.slots = None
        # one current slot serves every grid of the batch: rebind (slot A =
        # the inputs) unless every member's input is already in it
        cur = abi.stencil_batch_current(h.h) if h.slots is not None else 0
        if h.slots is None or any(sl[cur] != sp for sl, sp in zip(h.slots, srcs)):
            abi.stencil_batch_bind(h.h, srcs, dsts)
            h.slots = list(zip(srcs, dsts))
        if n > 1:
            abi.stencil_batch_step(h.h, n - 1, self.stream)
        abi.stencil_batch_step(h.h, 1, self.stream)
        newest = abi.stencil_batch_current(h.h)
        for m, sl in zip(members, h.slots):
            _settle(m.args[1], m.args[0], sl[newest], n)


@dataclass
class _Layout:
    padded: tuple
    origin: tuple

    def close(self):
        pass


class _Handle:
    def __init__(self, abi, h, batch):
        self.abi, self.h, self.batch = abi, h, batch
        self.slots = None   # per grid: (buffer in slot A, buffer in slot B)

    def close(self):
        if self.h:
            (self.abi.stencil_batch_destroy if self.batch else self.abi.stencil_destroy)(self.h)
            self.h = None


def _ring_value(host, g):
    """The one value held by every point outside the interior [g:-g], or None."""
    mask = np.ones(host.shape, dtype=bool)
    mask[tuple(slice(g, n - g) for n in host.shape)] = False
    ring = host[mask]
    if ring.size == 0:
        return None
    v = ring.flat[0]
    return float(v) if np.all(ring == v) else None


def _batchable(members) -> bool:
    """Fused members that one batched launch can run: 2D, radius 1 in a 3x3
    neighbourhood, ghost width 1, one dtype and one boundary value."""
    a0 = members[0].args[0]
    if a0.boundary is None:
        return False
    for m in members:
        if len(m.args[0].shape) != 2 or m.lowered.ghost != 1 or m.args[0].dtype != a0.dtype:
            return False
        if any(a.boundary is None or a.boundary != a0.boundary for a in m.args):
            return False
    return True


def _settle(src: Array, dst: Array, newest_ptr: int, n: int) -> None:
    """After n alternating sweeps from src into dst, the program's semantics
    put level n in dst when n is odd and in src when n is even, and level
    n - 1 in the other.  The library reports where level n is; if that is not
    the buffer the program expects, the two arrays exchange their device
    buffers (both are frontend-owned)."""
    want = dst if n % 2 == 1 else src
    if want.dev.data_ptr() != newest_ptr:
        src.dev, dst.dev = dst.dev, src.dev
        src.view, dst.view = dst.view, src.view


# ---------------------------------------------------------------------------
# Module-level program (the paper's examples use free functions)
# ---------------------------------------------------------------------------
default_program = Program()


def create_array(shape, dtype=np.float64) -> Array:
    """A new array of zeros in the default program."""
    return default_program.create_array(shape, dtype)


def sync() -> None:
    """Execute everything recorded in the default program."""
    default_program.sync()


def set_max_depth(depth: int) -> None:
    """DAG depth at which the default program flushes on its own."""
    default_program.max_depth = int(depth)

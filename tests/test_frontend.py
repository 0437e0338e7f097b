"""Host-side logic of the slice-assignment frontend (no GPU): AST capture and
parameterisation, lowering to offsets and weights, the dependency rule, the
array-level DAG, node fusion and the launch plan (Sec. III-A, III-B)."""
import numpy as np
import pytest

from paper_2512_19851_gb300 import frontend as fe
from paper_2512_19851_gb300.frontend import DependencyError, Program, UnsupportedExpression


def example1(p, n=10, iters=10, dtype=np.float64):
    """Example 1 of Sec. III-A, on an n x n array."""
    u1 = p.create_array((n, n), dtype)
    u2 = p.create_array((n, n), dtype)
    u1[0, :] = u1[-1, :] = u1[:, 0] = u1[:, -1] = 1
    u2[0, :] = u2[-1, :] = u2[:, 0] = u2[:, -1] = 1
    for _ in range(iters):
        u2[1:-1, 1:-1] = 0.25 * (u1[:-2, 1:-1] + u1[2:, 1:-1] + u1[1:-1, :-2] + u1[1:-1, 2:])
        u1, u2 = u2, u1
    return u1, u2


def stencil_nodes(p):
    return [n for n in p.nodes if n.kind == "stencil"]


def test_example1_lowers_to_the_four_point_average():
    p = Program()
    example1(p)
    nodes = stencil_nodes(p)
    assert len(nodes) == 10
    lo = nodes[0].lowered
    assert lo.offsets == ((-1, 0), (1, 0), (0, -1), (0, 1))
    assert lo.weights == (0.25,) * 4
    assert lo.ghost == 1 and lo.radius == 1


def test_ast_is_parameterised_over_swapped_arrays():
    """All ten iterations refer to one AST although the arrays swap (Sec. III-B)."""
    p = Program()
    u1, u2 = example1(p)
    nodes = stencil_nodes(p)
    assert len({n.ast for n in nodes}) == 1
    assert len(p.asts) == 1
    # arguments alternate: (out, in) = (u2, u1), (u1, u2), ...
    assert nodes[0].args[0] is nodes[1].args[1] and nodes[0].args[1] is nodes[1].args[0]


def test_dag_edges_and_depth():
    p = Program()
    example1(p, iters=3)
    # 8 fills (nodes 0-7), then stencils 8, 9, 10
    e = set(p.edges())
    # the first stencil reads u1 (last written by fill 3) and writes u2 (last
    # written by fill 7)
    assert {(3, 8), (7, 8)} <= e
    # true dependency 8 -> 9 (9 reads what 8 wrote), anti dependency 8 -> 9
    # (9 writes what 8 read), output 3 -> 9, then 9 -> 10 and output 8 -> 10
    assert {(8, 9), (3, 9), (9, 10), (8, 10)} <= e
    assert len([x for x in e if x[1] >= 8]) == 6
    # chained fills to the same array are output dependencies
    assert (0, 1) in e and (4, 5) in e
    assert p.depth() == 4 + 3


def test_dependency_rule_rejects_reading_the_output():
    p = Program()
    u = p.create_array((6, 6))
    with pytest.raises(DependencyError):
        u[1:-1, 1:-1] = 0.5 * (u[:-2, 1:-1] + u[2:, 1:-1])


@pytest.mark.parametrize("expr,msg", [
    (lambda a, b: a[1:-1, 1:-1] * a[2:, 1:-1], "product"),
    (lambda a, b: a[1:-1, 1:-1] / a[2:, 1:-1], "division"),
    (lambda a, b: a[1:-1, 1:-1] + 1.0, "constant"),
    (lambda a, b: a[1:-1, 1:-1] + b[2:, 1:-1], "one input"),
    (lambda a, b: a[1:-1, 1:] , "extent"),
])
def test_unsupported_expressions(expr, msg):
    p = Program()
    a = p.create_array((6, 6))
    b = p.create_array((6, 6))
    c = p.create_array((6, 6))
    with pytest.raises(UnsupportedExpression, match=msg):
        c[1:-1, 1:-1] = expr(a, b)


def test_written_region_must_be_a_centred_interior():
    p = Program()
    a, c = p.create_array((8, 8)), p.create_array((8, 8))
    with pytest.raises(UnsupportedExpression, match="interior"):
        c[1:-1, 2:-1] = a[1:-1, 2:-1]
    with pytest.raises(UnsupportedExpression, match="ring"):
        c[:, :] = a[:, :]


def test_wider_ring_and_radius_two():
    p = Program()
    a, c = p.create_array((12, 9)), p.create_array((12, 9))
    c[2:-2, 2:-2] = (a[:-4, 2:-2] - 2 * a[2:-2, 2:-2] + a[4:, 2:-2]) / 4 + a[2:-2, 3:-1]
    lo = stencil_nodes(p)[0].lowered
    assert lo.ghost == 2 and lo.radius == 2
    assert lo.offsets == ((-2, 0), (0, 0), (2, 0), (0, 1))
    assert lo.weights == (0.25, -0.5, 0.25, 1.0)


def test_repeated_terms_merge_and_cancelling_terms_drop():
    p = Program()
    a, c = p.create_array((6, 6)), p.create_array((6, 6))
    c[1:-1, 1:-1] = a[1:-1, 1:-1] + a[2:, 1:-1] + a[1:-1, 1:-1] - a[2:, 1:-1] + (-a[:-2, 1:-1])
    lo = stencil_nodes(p)[0].lowered
    assert lo.offsets == ((0, 0), (-1, 0))
    assert lo.weights == (2.0, -1.0)


def test_3d_seven_point():
    p = Program()
    a, c = p.create_array((6, 7, 8)), p.create_array((6, 7, 8))
    i = slice(1, -1)
    c[i, i, i] = 0.4 * a[i, i, i] + 0.1 * (a[:-2, i, i] + a[2:, i, i] + a[i, :-2, i] + a[i, 2:, i]
                                           + a[i, i, :-2] + a[i, i, 2:])
    lo = stencil_nodes(p)[0].lowered
    assert lo.offsets == ((0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1))
    assert lo.weights == (0.4,) + (0.1,) * 6


def test_plan_merges_the_loop_into_one_run():
    p = Program()
    example1(p, iters=10)
    plan = p.plan()
    assert [e[0] for e in plan] == ["fill"] * 8 + ["run"]
    assert plan[-1][2] == 10 and len(plan[-1][1]) == 1


def test_node_fusion_groups_independent_fields():
    """Two fields updated in the same iteration: consecutive nodes with the
    same output shape and no path between them fuse (Sec. III-B); the loop
    then becomes one run of the fused pair."""
    p = Program()
    v1, v2 = p.create_array((8, 8)), p.create_array((8, 8))
    w1, w2 = p.create_array((8, 8)), p.create_array((8, 8))
    for _ in range(5):
        v2[1:-1, 1:-1] = 0.5 * (v1[:-2, 1:-1] + v1[2:, 1:-1])
        w2[1:-1, 1:-1] = 0.25 * (w1[1:-1, :-2] + w1[1:-1, 2:]) + 0.5 * w1[1:-1, 1:-1]
        v1, v2 = v2, v1
        w1, w2 = w2, w1
    groups = p.fused_groups()
    assert groups == [[0, 1], [2, 3], [4, 5], [6, 7], [8, 9]]
    plan = p.plan()
    assert plan == [("run", [0, 1], 5)]


def test_fusion_stops_at_a_dependency_and_at_a_shape_change():
    p = Program()
    a, b, c = (p.create_array((6, 6)) for _ in range(3))
    d = p.create_array((7, 7))
    e = p.create_array((7, 7))
    b[1:-1, 1:-1] = a[1:-1, 1:-1]
    c[1:-1, 1:-1] = b[1:-1, 1:-1]       # reads what the previous node wrote
    e[1:-1, 1:-1] = d[1:-1, 1:-1]       # another shape
    assert p.fused_groups() == [[0], [1], [2]]


def test_depth_limit_triggers_a_flush(monkeypatch):
    flushed = []
    p = Program(max_depth=2)
    monkeypatch.setattr(Program, "sync", lambda self: flushed.append(len(self.nodes)) or self.nodes.clear())
    a, b = p.create_array((5, 5)), p.create_array((5, 5))
    for _ in range(2):
        b[1:-1, 1:-1] = a[1:-1, 1:-1]
        a, b = b, a
    assert flushed == []
    b[1:-1, 1:-1] = a[1:-1, 1:-1]
    assert flushed == [3]


def test_execution_needs_a_gpu():
    """No CPU evaluation path: flushing without CUDA raises."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = Program()
    example1(p, n=6, iters=2)
    with pytest.raises(RuntimeError, match="CUDA"):
        p.sync()


def test_fill_values_and_host_data_before_execution():
    p = Program()
    a = p.create_array((4, 5), np.float32)
    a[1:3, :] = 2.5
    a.set(np.arange(20, dtype=np.float32).reshape(4, 5))
    a[0, 0] = -1
    assert fe._ring_value(np.ones((5, 5)), 1) == 1.0
    host = np.zeros((5, 5))
    host[0, 2] = 3
    assert fe._ring_value(host, 1) is None
    assert [n.kind for n in p.nodes] == ["fill", "fill", "fill"]


class _Buf:
    def __init__(self, ptr):
        self.ptr = ptr

    def data_ptr(self):
        return self.ptr


def test_settle_puts_the_newest_level_where_the_program_expects_it():
    """After n alternating sweeps from src into dst the program expects level
    n in dst (n odd) or src (n even); if the library left it in the other
    buffer, the two arrays exchange buffers, otherwise nothing moves."""
    for n, newest_in, swapped in ((3, "dst", False), (3, "src", True), (4, "src", False), (4, "dst", True)):
        p = Program()
        src, dst = p.create_array((4, 4)), p.create_array((4, 4))
        src.dev, dst.dev = _Buf(100), _Buf(200)
        src.view, dst.view = "view-a", "view-b"
        fe._settle(src, dst, 200 if newest_in == "dst" else 100, n)
        assert (src.dev.ptr == 200) == swapped and (dst.dev.ptr == 100) == swapped
        assert (src.view == "view-b") == swapped


def test_fused_3d_members_run_one_after_another():
    """Fusion groups members of any dimension; 3D members are not batchable
    (the batched kernel is 2D), so the plan still has one run of the group."""
    p = Program()
    a1, a2 = p.create_array((5, 6, 7)), p.create_array((5, 6, 7))
    b1, b2 = p.create_array((5, 6, 7)), p.create_array((5, 6, 7))
    i = slice(1, -1)
    for _ in range(3):
        a2[i, i, i] = 0.5 * (a1[:-2, i, i] + a1[2:, i, i])
        b2[i, i, i] = 0.5 * (b1[i, :-2, i] + b1[i, 2:, i])
        a1, a2 = a2, a1
        b1, b2 = b2, b1
    assert p.plan() == [("run", [0, 1], 3)]
    members = [p.nodes[0], p.nodes[1]]
    for m in members:
        for arr in m.args:
            arr.boundary = 0.0
    assert not fe._batchable(members)

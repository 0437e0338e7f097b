"""stencil_reduce_noalloc, the reduction entry point for callers that cannot
allocate device memory at call time (their GPU memory is owned by another
allocator, or a cudaMalloc and its implicit synchronisation are not allowed
on their path).  It must give the results of stencil_reduce without
allocating: two calls in a row through the C ABI, each checked against
stencil_reduce on the same buffers, within the reduction tolerance used by
the other GPU tests (1e-12 relative; the maximum exactly).  This file is
collected last so that a run stopping at the first failure has run every
other test first; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2512_19851_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def _check(out, ref, d_abs_sum):
    assert abs(out[0] - ref[0]) <= 1e-12 * d_abs_sum
    assert abs(out[1] - ref[1]) <= 1e-12 * ref[1]
    assert out[2] == ref[2]


@pytest.mark.parametrize("dtype,st_dtype", [(torch.float32, abi.ST_F32), (torch.float64, abi.ST_F64)])
def test_reduce_noalloc_matches_reduce_twice(dtype, st_dtype):
    assert torch.cuda.is_available(), "GPU test run without a CUDA device"
    shape = (37, 45, 130)
    h = abi.stencil_create(3, shape, 0, inputs.OFFSETS_7PT, [0.4] + [0.1] * 6, None, abi.ST_PERIODIC, 0.0,
                           st_dtype, 1, 0)
    pd, org, _ = abi.stencil_layout(h, 3)
    gen = torch.Generator(device="cuda").manual_seed(7)
    interior = tuple(slice(o, o + s) for o, s in zip(org, shape))
    for call in range(2):
        a = torch.randn(pd, dtype=dtype, device="cuda", generator=gen)
        b = torch.randn(pd, dtype=dtype, device="cuda", generator=gen) if call == 0 else None
        out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        ref = torch.empty(3, dtype=torch.float64, device="cuda")
        bp = b.data_ptr() if b is not None else 0
        abi.stencil_reduce_noalloc(h, a.data_ptr(), bp, out.data_ptr())
        abi.stencil_reduce(h, a.data_ptr(), bp, ref.data_ptr())
        torch.cuda.synchronize()
        d = a[interior].double() - (b[interior].double() if b is not None else 0.0)
        _check(out.cpu().numpy(), ref.cpu().numpy(), float(d.abs().sum()))
        assert float(ref[2]) == float(d.abs().max())
    abi.stencil_destroy(h)


def test_reduce_noalloc_allocates_nothing_on_a_grid_larger_than_its_blocks():
    """A grid with many more rows than the static array has block partials
    (the blocks walk the rows in a grid-stride loop): the results agree with
    stencil_reduce, and after a first call (which loads the kernels and looks
    up the array's address) further calls leave the device's free memory
    exactly as it was, so nothing was allocated."""
    assert torch.cuda.is_available(), "GPU test run without a CUDA device"
    shape = (96, 700, 36)  # 67200 interior rows, more than 8 x 4096
    h = abi.stencil_create(3, shape, 0, inputs.OFFSETS_7PT, [0.4] + [0.1] * 6, None, abi.ST_DIRICHLET, 0.0,
                           abi.ST_F32, 1, 0)
    pd, org, _ = abi.stencil_layout(h, 3)
    gen = torch.Generator(device="cuda").manual_seed(11)
    a = torch.rand(pd, dtype=torch.float32, device="cuda", generator=gen)
    out = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    abi.stencil_reduce_noalloc(h, a.data_ptr(), 0, out[0].data_ptr())
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for i in range(1, 4):
        abi.stencil_reduce_noalloc(h, a.data_ptr(), 0, out[i].data_ptr())
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    ref = torch.empty(3, dtype=torch.float64, device="cuda")
    abi.stencil_reduce(h, a.data_ptr(), 0, ref.data_ptr())
    torch.cuda.synchronize()
    interior = a[tuple(slice(o, o + s) for o, s in zip(org, shape))].double()
    r = ref.cpu().numpy()
    for i in range(4):
        _check(out[i].cpu().numpy(), r, float(interior.abs().sum()))
    abi.stencil_destroy(h)

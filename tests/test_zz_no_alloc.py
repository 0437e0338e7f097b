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


def test_reduce_noalloc_rejects_grids_beyond_its_scratch():
    assert torch.cuda.is_available(), "GPU test run without a CUDA device"
    h = abi.stencil_create(3, (1025, 512, 512), 0, inputs.OFFSETS_7PT, [0.4] + [0.1] * 6, None, abi.ST_PERIODIC,
                           0.0, abi.ST_F32, 1, 0)
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    with pytest.raises(abi.StencilError) as e:
        abi.stencil_reduce_noalloc(h, out.data_ptr(), 0, out.data_ptr())  # rejected before any access
    assert e.value.code == abi.ST_ERR_ARG and "268435456" in str(e.value)
    abi.stencil_destroy(h)

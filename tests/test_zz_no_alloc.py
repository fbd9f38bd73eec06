"""bsrht_sketch_noalloc: the sketch entry point for callers that cannot
allocate device memory (its scratch is a fixed array inside the library).

It must return exactly what bsrht_sketch returns for the same inputs, call
after call, even though every call reuses the same scratch array and finds
there whatever the previous call left.  The file name makes pytest collect it
last."""

import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu

NOALLOC_LIMIT = 32 << 20  # bytes of the library's fixed scratch array


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_11295_gb300 as b
    from paper_2210_11295_gb300 import _binding as bb
    fn = b.lib.bsrht_sketch_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                   ctypes.c_uint64, ctypes.c_void_p, ctypes.POINTER(bb.Opts)]
    # Kernel choices recorded by the autotuner in earlier tests would change
    # the plans (and their scratch); start from the built-in rules.
    b.bsrht_sketch_autotune_reset()
    return b, bb


def _noalloc(b, bb, a, p, l, seed, variant=0):
    n, m = a.shape
    out = torch.full((l, m), float("nan"), device=a.device, dtype=b.sketch_out_dtype(a.dtype))
    o = bb.make_opts(a, variant=variant)
    st = b.lib.bsrht_sketch_noalloc(ctypes.c_void_p(a.data_ptr()), n, m, p, l, seed,
                                    ctypes.c_void_p(out.data_ptr()), ctypes.byref(o))
    return st, out


def _check_same(b, bb, a, p, l, seed, variant=0):
    ref = b.bsrht_sketch(a, p, l, seed, variant=variant)
    st, got = _noalloc(b, bb, a, p, l, seed, variant)
    torch.cuda.synchronize()
    assert st == 0, b.strerror(st)
    # Same plan, same kernels, same fixed-order block sum: the same bits.
    assert torch.equal(got, ref)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_noalloc_matches_sketch_on_consecutive_calls(lib, dtype):
    b, bb = lib
    gen = torch.Generator("cuda").manual_seed(21)
    shapes = [((1 << 17) + 123, 200, 4, 256, 5), (30000, 77, 3, 128, 6)]
    for (n, m, p, l, seed) in shapes:  # two calls in a row, different sizes
        a = torch.randn(n, m, device="cuda", dtype=dtype, generator=gen)
        _check_same(b, bb, a, p, l, seed)


def test_noalloc_repeat_same_input(lib):
    b, bb = lib
    a = torch.randn(1 << 16, 64, device="cuda", dtype=torch.float32,
                    generator=torch.Generator("cuda").manual_seed(3))
    for _ in range(2):
        _check_same(b, bb, a, 8, 192, 9)


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_noalloc_16bit_after_a_larger_call(lib, dtype):
    """16-bit inputs use other scratch layouts (paired panel slots, the status
    word after the partials, the sign tables): a large FP32 call first fills
    the array with stale values, then the 16-bit sketch on the TMA-fed path
    (l >= 512, 16-byte aligned rows) and on the tensor-core path must still
    equal bsrht_sketch bit for bit."""
    b, bb = lib
    gen = torch.Generator("cuda").manual_seed(5)
    big = torch.randn(1 << 18, 1024, device="cuda", dtype=torch.float32, generator=gen)
    _check_same(b, bb, big, 4, 512, 1)
    del big
    a = torch.randn((1 << 17) + 512, 320, device="cuda", dtype=torch.float32, generator=gen).to(dtype)
    _check_same(b, bb, a, 4, 512, 2)
    _check_same(b, bb, a, 4, 512, 3, variant=b.VARIANT_TENSOR)
    _check_same(b, bb, a, 2, 640, 4)


def test_noalloc_rejects_oversized_problem(lib):
    """A problem whose sketch scratch exceeds the fixed array is refused with
    BSRHT_ENOMEM before any launch: real buffers of the right size, 65536
    columns (2048 column panels of per-CTA partial sums)."""
    b, bb = lib
    n, m, p, l = 1024, 1 << 16, 1, 512
    need = b.bsrht_sketch_workspace(n, m, p, l, torch.float32)
    assert need > NOALLOC_LIMIT
    a = torch.zeros(n, m, device="cuda", dtype=torch.float32)
    out = torch.zeros(l, m, device="cuda", dtype=torch.float32)
    o = bb.make_opts(a)
    st = b.lib.bsrht_sketch_noalloc(ctypes.c_void_p(a.data_ptr()), n, m, p, l, 0,
                                    ctypes.c_void_p(out.data_ptr()), ctypes.byref(o))
    torch.cuda.synchronize()
    assert st == bb.BSRHT_ENOMEM
    assert torch.count_nonzero(out).item() == 0

"""bsrht_sketch_noalloc: the sketch entry point for callers that cannot
allocate device memory (its scratch is a fixed array inside the library).

It must return what bsrht_sketch returns for the same inputs, call after
call, even though every call reuses the same scratch array.  The file name
makes pytest collect it last."""

import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu


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
    return b, bb


def _noalloc(b, bb, a, p, l, seed):
    n, m = a.shape
    out = torch.full((l, m), float("nan"), device=a.device, dtype=b.sketch_out_dtype(a.dtype))
    o = bb.make_opts(a)
    st = b.lib.bsrht_sketch_noalloc(ctypes.c_void_p(a.data_ptr()), n, m, p, l, seed,
                                    ctypes.c_void_p(out.data_ptr()), ctypes.byref(o))
    return st, out


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 1e-6), (torch.float64, 1e-13)])
def test_noalloc_matches_sketch_on_consecutive_calls(lib, dtype, tol):
    b, bb = lib
    gen = torch.Generator("cuda").manual_seed(21)
    shapes = [((1 << 17) + 123, 200, 4, 256, 5), (30000, 77, 3, 128, 6)]
    for (n, m, p, l, seed) in shapes:  # two calls in a row, different sizes
        a = torch.randn(n, m, device="cuda", dtype=dtype, generator=gen)
        ref = b.bsrht_sketch(a, p, l, seed)
        st, got = _noalloc(b, bb, a, p, l, seed)
        torch.cuda.synchronize()
        assert st == 0, b.strerror(st)
        err = (torch.linalg.norm(got.double() - ref.double()) / torch.linalg.norm(ref.double())).item()
        assert err <= tol


def test_noalloc_repeat_same_input(lib):
    b, bb = lib
    a = torch.randn(1 << 16, 64, device="cuda", dtype=torch.float32,
                    generator=torch.Generator("cuda").manual_seed(3))
    ref = b.bsrht_sketch(a, 8, 192, 9)
    for _ in range(2):
        st, got = _noalloc(b, bb, a, 8, 192, 9)
        torch.cuda.synchronize()
        assert st == 0
        assert (torch.linalg.norm(got - ref) / torch.linalg.norm(ref)).item() <= 1e-6


def test_noalloc_rejects_oversized_problem(lib):
    b, bb = lib
    # Needs far more than the fixed 32 MiB of scratch: rejected before any launch.
    need = b.bsrht_sketch_workspace(1 << 22, 1 << 16, 4, 1024, torch.float32)
    assert need > 32 << 20
    o = bb.Opts()
    b.lib.bsrht_opts_init(ctypes.byref(o))
    o.dtype = bb.F32
    st = b.lib.bsrht_sketch_noalloc(ctypes.c_void_p(256), 1 << 22, 1 << 16, 4, 1024, 0,
                                    ctypes.c_void_p(256), ctypes.byref(o))
    assert st == bb.BSRHT_ENOMEM

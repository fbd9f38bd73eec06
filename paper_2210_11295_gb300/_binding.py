"""ctypes binding of libbsrht (include/bsrht.h): argument marshalling only.

Every function here forwards torch tensors' device pointers, strides and the
current CUDA stream to the C entry point of the same name; all arithmetic runs
in the library's CUDA kernels. If the library has not been built the import
of this module raises, so there is no silent fallback.
"""

from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libbsrht.so")

BSRHT_OK = 0
BSRHT_EINVAL = -22
BSRHT_ENOMEM = -12
BSRHT_EUNSUP = -95
BSRHT_ETIMEDOUT = -110
BSRHT_ENOTPD = -1001
BSRHT_ENOCONV = -1002
BSRHT_ECUDA = -1003

F64, F32, BF16, F16 = 0, 1, 2, 3
VARIANT_AUTO, VARIANT_CUDACORE, VARIANT_TENSOR, VARIANT_GAUSSIAN = 0, 1, 2, 3
PREC_AUTO, PREC_F64 = 0, 1  # bsrht_precision

_DTYPES = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16}


class BsrhtError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} (status {status})")


class Opts(ctypes.Structure):
    _fields_ = [
        ("dtype", ctypes.c_int32),
        ("variant", ctypes.c_int32),
        ("lda", ctypes.c_int64),
        ("stream", ctypes.c_void_p),
        ("workspace", ctypes.c_void_p),
        ("workspace_bytes", ctypes.c_size_t),
        ("precision", ctypes.c_int32),
    ]


class Request(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("dtype", ctypes.c_int32),
        ("A", ctypes.c_void_p),
        ("n", ctypes.c_int64),
        ("m", ctypes.c_int64),
        ("lda", ctypes.c_int64),
        ("p", ctypes.c_int32),
        ("k", ctypes.c_int32),
        ("l", ctypes.c_int64),
        ("seed", ctypes.c_uint64),
        ("out", ctypes.c_void_p),
        ("U", ctypes.c_void_p),
        ("S", ctypes.c_void_p),
        ("V", ctypes.c_void_p),
        ("precision", ctypes.c_int32),
    ]


class ServerOpts(ctypes.Structure):
    _fields_ = [
        ("hbm_budget", ctypes.c_size_t),
        ("executors", ctypes.c_int32),
        ("max_group", ctypes.c_int32),
        ("use_graphs", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("exec_timeout_ms", ctypes.c_int64),
    ]


class ServerStats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_int64),
        ("completed", ctypes.c_int64),
        ("failed", ctypes.c_int64),
        ("pending", ctypes.c_int64),
        ("grouped_launches", ctypes.c_int64),
        ("grouped_requests", ctypes.c_int64),
        ("graph_launches", ctypes.c_int64),
        ("tuned_classes", ctypes.c_int64),
        ("p50_ms", ctypes.c_double),
        ("p99_ms", ctypes.c_double),
        ("mean_ms", ctypes.c_double),
        ("max_ms", ctypes.c_double),
        ("pool_high_bytes", ctypes.c_size_t),
    ]


REQ_SKETCH, REQ_RSVD, REQ_NYSTROM = 0, 1, 2


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libbsrht.so is not built ({LIB_PATH}); run "
            "`python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = ctypes.CDLL(LIB_PATH)
    i64, i32, u64, vp, sz = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_size_t
    pd = ctypes.POINTER(ctypes.c_double)
    po = ctypes.POINTER(Opts)
    sigs = {
        "bsrht_opts_init": (None, [po]),
        "bsrht_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "bsrht_version": (ctypes.c_char_p, []),
        "bsrht_sketch": (ctypes.c_int, [vp, i64, i64, i32, i64, u64, vp, po]),
        "bsrht_sketch_workspace": (ctypes.c_int, [i64, i64, i32, i64, po, ctypes.POINTER(sz)]),
        "bsrht_rsvd": (ctypes.c_int, [vp, i64, i64, i32, i64, i32, u64, pd, pd, pd, po]),
        "bsrht_rsvd_workspace": (ctypes.c_int, [i64, i64, i32, i64, i32, po, ctypes.POINTER(sz)]),
        "bsrht_srsvd": (ctypes.c_int, [vp, i64, i64, i32, i64, i64, i32, u64, pd, pd, pd, po]),
        "bsrht_srsvd_workspace": (ctypes.c_int, [i64, i64, i32, i64, i64, i32, po, ctypes.POINTER(sz)]),
        "bsrht_nystrom": (ctypes.c_int, [vp, i64, i32, i64, i32, u64, pd, pd, po]),
        "bsrht_nystrom_workspace": (ctypes.c_int, [i64, i32, i64, i32, po, ctypes.POINTER(sz)]),
        "bsrht_nystrom_rbf": (ctypes.c_int, [vp, i64, i64, ctypes.c_double, i32, i64, i32, u64, pd, pd, po]),
        "bsrht_nystrom_rbf_workspace": (ctypes.c_int, [i64, i64, i32, i64, i32, po, ctypes.POINTER(sz)]),
        "bsrht_release_pool": (ctypes.c_int, []),
        "bsrht_kernel_launches": (ctypes.c_uint64, []),
        "bsrht_profile_enable": (ctypes.c_int, [ctypes.c_int]),
        "bsrht_profile_stages": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                                 ctypes.POINTER(ctypes.c_int)]),
        "bsrht_sketch_autotune": (ctypes.c_int, [vp, i64, i64, i32, i64, po, ctypes.POINTER(i32),
                                                 ctypes.POINTER(ctypes.c_double)]),
        "bsrht_sketch_autotune_reset": (ctypes.c_int, []),
        "bsrht_server_opts_init": (None, [ctypes.POINTER(ServerOpts)]),
        "bsrht_server_create": (ctypes.c_int, [sz, ctypes.POINTER(vp)]),
        "bsrht_server_create_ex": (ctypes.c_int, [ctypes.POINTER(ServerOpts), ctypes.POINTER(vp)]),
        "bsrht_submit": (ctypes.c_int, [vp, ctypes.POINTER(Request), ctypes.POINTER(u64)]),
        "bsrht_poll": (ctypes.c_int, [vp, u64, ctypes.POINTER(ctypes.c_int)]),
        "bsrht_wait": (ctypes.c_int, [vp, u64, i64]),
        "bsrht_server_stats_get": (ctypes.c_int, [vp, ctypes.POINTER(ServerStats)]),
        "bsrht_request_times": (ctypes.c_int, [vp, u64, ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_double)]),
        "bsrht_server_destroy": (ctypes.c_int, [vp]),
        "bsrht_selftest_pool_allocator": (ctypes.c_int, [u64, i32]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def strerror(status: int) -> str:
    return lib.bsrht_strerror(int(status)).decode()


def version() -> str:
    return lib.bsrht_version().decode()


def _check(status: int, where: str) -> None:
    if status != BSRHT_OK:
        raise BsrhtError(status, where)


def _dptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dbl(t: torch.Tensor):
    return ctypes.cast(ctypes.c_void_p(t.data_ptr()), ctypes.POINTER(ctypes.c_double))


def make_opts(a: torch.Tensor, variant: int = VARIANT_AUTO, workspace: torch.Tensor | None = None,
              stream: torch.cuda.Stream | None = None, precision: int = 0) -> Opts:
    if a.dim() != 2 or a.stride(1) != 1:
        raise ValueError("A must be a 2-D tensor with unit column stride (row-major)")
    if a.dtype not in _DTYPES:
        raise ValueError(f"unsupported dtype {a.dtype}")
    o = Opts()
    lib.bsrht_opts_init(ctypes.byref(o))
    o.dtype = _DTYPES[a.dtype]
    o.variant = int(variant)
    o.precision = int(precision)
    o.lda = int(a.stride(0)) if a.shape[0] > 1 else int(a.shape[1])
    s = stream if stream is not None else torch.cuda.current_stream(a.device)
    o.stream = ctypes.c_void_p(s.cuda_stream)
    if workspace is not None:
        o.workspace = ctypes.c_void_p(workspace.data_ptr())
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    return o


def sketch_out_dtype(dtype: torch.dtype, precision: int = 0) -> torch.dtype:
    return torch.float64 if dtype == torch.float64 or precision == PREC_F64 else torch.float32


def bsrht_sketch_workspace(n: int, m: int, p: int, l: int, dtype=torch.float32,
                           variant: int = VARIANT_AUTO, precision: int = 0) -> int:
    o = Opts()
    lib.bsrht_opts_init(ctypes.byref(o))
    o.dtype = _DTYPES[dtype]
    o.variant = int(variant)
    o.precision = int(precision)
    out = ctypes.c_size_t(0)
    _check(lib.bsrht_sketch_workspace(n, m, p, l, ctypes.byref(o), ctypes.byref(out)), "bsrht_sketch_workspace")
    return int(out.value)


def bsrht_sketch(a: torch.Tensor, p: int, l: int, seed: int, out: torch.Tensor | None = None,
                 variant: int = VARIANT_AUTO, workspace: torch.Tensor | None = None,
                 stream: torch.cuda.Stream | None = None, precision: int = 0) -> torch.Tensor:
    """B = Omega A (l x m) for the n x m device matrix ``a`` (FP64 output
    for FP64 data or precision=PREC_F64)."""
    n, m = a.shape
    odt = sketch_out_dtype(a.dtype, precision)
    if out is None:
        out = torch.empty(l, m, device=a.device, dtype=odt)
    if out.shape != (l, m) or not out.is_contiguous() or out.dtype != odt:
        raise ValueError("out must be a contiguous l x m tensor of the sketch dtype")
    o = make_opts(a, variant, workspace, stream, precision)
    _check(lib.bsrht_sketch(_dptr(a), n, m, p, l, seed & (2**64 - 1), _dptr(out), ctypes.byref(o)),
           "bsrht_sketch")
    return out


def bsrht_rsvd_workspace(n: int, m: int, k: int, l: int, p: int, dtype=torch.float32,
                         variant: int = VARIANT_AUTO) -> int:
    o = Opts()
    lib.bsrht_opts_init(ctypes.byref(o))
    o.dtype = _DTYPES[dtype]
    o.variant = int(variant)
    out = ctypes.c_size_t(0)
    _check(lib.bsrht_rsvd_workspace(n, m, k, l, p, ctypes.byref(o), ctypes.byref(out)), "bsrht_rsvd_workspace")
    return int(out.value)


def bsrht_rsvd(a: torch.Tensor, k: int, l: int, p: int, seed: int, variant: int = VARIANT_AUTO,
               workspace: torch.Tensor | None = None, stream: torch.cuda.Stream | None = None,
               outs=None):
    """Rank-k randomized SVD (Algorithm 1): returns (U n x k, S k, V m x k) in float64."""
    n, m = a.shape
    if outs is None:
        u = torch.empty(n, k, device=a.device, dtype=torch.float64)
        s = torch.empty(k, device=a.device, dtype=torch.float64)
        v = torch.empty(m, k, device=a.device, dtype=torch.float64)
    else:
        u, s, v = outs
    o = make_opts(a, variant, workspace, stream)
    _check(lib.bsrht_rsvd(_dptr(a), n, m, k, l, p, seed & (2**64 - 1), _dbl(u), _dbl(s), _dbl(v),
                          ctypes.byref(o)), "bsrht_rsvd")
    return u, s, v


def bsrht_srsvd_workspace(n: int, m: int, k: int, l: int, s: int, p: int, dtype=torch.float32) -> int:
    o = Opts()
    lib.bsrht_opts_init(ctypes.byref(o))
    o.dtype = _DTYPES[dtype]
    out = ctypes.c_size_t(0)
    _check(lib.bsrht_srsvd_workspace(n, m, k, l, s, p, ctypes.byref(o), ctypes.byref(out)), "bsrht_srsvd_workspace")
    return int(out.value)


def bsrht_srsvd(a: torch.Tensor, k: int, l: int, s: int, p: int, seed: int,
                workspace: torch.Tensor | None = None, stream: torch.cuda.Stream | None = None, outs=None):
    """Rank-k single-view randomized SVD (Algorithm 3): returns (U n x k, S k, V m x k) in float64."""
    n, m = a.shape
    if outs is None:
        u = torch.empty(n, k, device=a.device, dtype=torch.float64)
        sv = torch.empty(k, device=a.device, dtype=torch.float64)
        v = torch.empty(m, k, device=a.device, dtype=torch.float64)
    else:
        u, sv, v = outs
    o = make_opts(a, VARIANT_AUTO, workspace, stream)
    _check(lib.bsrht_srsvd(_dptr(a), n, m, k, l, s, p, seed & (2**64 - 1), _dbl(u), _dbl(sv), _dbl(v),
                           ctypes.byref(o)), "bsrht_srsvd")
    return u, sv, v


def bsrht_nystrom_workspace(n: int, k: int, l: int, p: int, dtype=torch.float32, precision: int = 0) -> int:
    o = Opts()
    lib.bsrht_opts_init(ctypes.byref(o))
    o.dtype = _DTYPES[dtype]
    o.precision = int(precision)
    out = ctypes.c_size_t(0)
    _check(lib.bsrht_nystrom_workspace(n, k, l, p, ctypes.byref(o), ctypes.byref(out)),
           "bsrht_nystrom_workspace")
    return int(out.value)


def bsrht_nystrom(a: torch.Tensor, k: int, l: int, p: int, seed: int, variant: int = VARIANT_AUTO,
                  workspace: torch.Tensor | None = None, stream: torch.cuda.Stream | None = None,
                  outs=None, precision: int = 0):
    """Rank-k randomized Nystrom (Algorithm 2): returns (U n x k, Lambda k) in float64."""
    n = a.shape[0]
    if a.shape[1] != n:
        raise ValueError("A must be square")
    if outs is None:
        u = torch.empty(n, k, device=a.device, dtype=torch.float64)
        lam = torch.empty(k, device=a.device, dtype=torch.float64)
    else:
        u, lam = outs
    o = make_opts(a, variant, workspace, stream, precision)
    _check(lib.bsrht_nystrom(_dptr(a), n, k, l, p, seed & (2**64 - 1), _dbl(u), _dbl(lam), ctypes.byref(o)),
           "bsrht_nystrom")
    return u, lam


def bsrht_nystrom_rbf_workspace(n: int, dim: int, k: int, l: int, p: int, ldx: int = 0) -> int:
    o = Opts()
    lib.bsrht_opts_init(ctypes.byref(o))
    o.dtype = F32
    o.lda = int(ldx)
    out = ctypes.c_size_t(0)
    _check(lib.bsrht_nystrom_rbf_workspace(n, dim, k, l, p, ctypes.byref(o), ctypes.byref(out)),
           "bsrht_nystrom_rbf_workspace")
    return int(out.value)


def bsrht_nystrom_rbf(x: torch.Tensor, h: float, k: int, l: int, p: int, seed: int, variant: int = VARIANT_AUTO,
                      workspace: torch.Tensor | None = None, stream: torch.cuda.Stream | None = None, outs=None):
    """Rank-k randomized Nystrom (Algorithm 2) of the RBF kernel matrix
    A_ij = exp(-|x_i - x_j|^2 / (2 h^2)) of the rows of x (n x dim, float32),
    without storing A: returns (U n x k, Lambda k) in float64."""
    if x.dtype != torch.float32:
        raise ValueError("points must be float32")
    n, dim = x.shape
    if outs is None:
        u = torch.empty(n, k, device=x.device, dtype=torch.float64)
        lam = torch.empty(k, device=x.device, dtype=torch.float64)
    else:
        u, lam = outs
    o = make_opts(x, variant, workspace, stream)
    _check(lib.bsrht_nystrom_rbf(_dptr(x), n, dim, float(h), k, l, p, seed & (2**64 - 1), _dbl(u), _dbl(lam),
                                 ctypes.byref(o)), "bsrht_nystrom_rbf")
    return u, lam


def bsrht_kernel_launches() -> int:
    """Cumulative count of CUDA kernels the library has launched."""
    return int(lib.bsrht_kernel_launches())


def bsrht_profile_enable(on: bool = True) -> None:
    """Record CUDA events between the stages of bsrht_rsvd / bsrht_nystrom."""
    _check(lib.bsrht_profile_enable(1 if on else 0), "bsrht_profile_enable")


def bsrht_profile_stages() -> list[tuple[str, float]]:
    """(stage name, milliseconds) of the last traced call on this thread."""
    cap = 64
    names = ctypes.create_string_buffer(32 * cap)
    ms = (ctypes.c_double * cap)()
    cnt = ctypes.c_int(0)
    _check(lib.bsrht_profile_stages(names, ms, cap, ctypes.byref(cnt)), "bsrht_profile_stages")
    out = []
    for i in range(min(cnt.value, cap)):
        nm = names.raw[32 * i:32 * i + 32].split(b"\0", 1)[0].decode()
        out.append((nm, float(ms[i])))
    return out


def bsrht_release_pool() -> None:
    _check(lib.bsrht_release_pool(), "bsrht_release_pool")


def bsrht_sketch_autotune(a: torch.Tensor, p: int, l: int) -> tuple[int, float]:
    """Times the sketch kernel instances on `a` and records the fastest for
    its shape class; returns (choice, ms) with choice -1 = TMA-fed kernel."""
    o = make_opts(a)
    c = ctypes.c_int32(0)
    t = ctypes.c_double(0.0)
    _check(lib.bsrht_sketch_autotune(_dptr(a), a.shape[0], a.shape[1], int(p), int(l), ctypes.byref(o),
                                     ctypes.byref(c), ctypes.byref(t)), "bsrht_sketch_autotune")
    return int(c.value), float(t.value)


def bsrht_sketch_autotune_reset() -> None:
    _check(lib.bsrht_sketch_autotune_reset(), "bsrht_sketch_autotune_reset")


def bsrht_selftest_pool_allocator(seed: int, steps: int) -> int:
    return int(lib.bsrht_selftest_pool_allocator(int(seed), int(steps)))


class Server:
    """The library's serving loop (bsrht_server_*): requests run on the
    server's own executor streams; tensors passed to submit_* must stay alive
    (and untouched) until the request is done."""

    def __init__(self, hbm_budget: int, executors: int = 4, max_group: int = 16, use_graphs: bool = True,
                 autotune: bool = True, exec_timeout_ms: int = 600_000):
        o = ServerOpts()
        lib.bsrht_server_opts_init(ctypes.byref(o))
        o.hbm_budget = int(hbm_budget)
        o.executors = int(executors)
        o.max_group = int(max_group)
        o.use_graphs = 1 if use_graphs else 0
        o.autotune = 1 if autotune else 0
        o.exec_timeout_ms = int(exec_timeout_ms)
        h = ctypes.c_void_p()
        _check(lib.bsrht_server_create_ex(ctypes.byref(o), ctypes.byref(h)), "bsrht_server_create_ex")
        self._h = h
        self._keep: dict[int, tuple] = {}

    def _submit(self, r: Request, keep: tuple) -> int:
        t = ctypes.c_uint64(0)
        _check(lib.bsrht_submit(self._h, ctypes.byref(r), ctypes.byref(t)), "bsrht_submit")
        self._keep[int(t.value)] = keep
        return int(t.value)

    @staticmethod
    def _base(a: torch.Tensor, kind: int, p: int, l: int, seed: int, k: int = 0) -> Request:
        if a.dim() != 2 or a.stride(1) != 1 or a.dtype not in _DTYPES or not a.is_cuda:
            raise ValueError("A must be a row-major 2-D CUDA tensor of f64/f32/bf16/f16")
        r = Request()
        r.kind = kind
        r.dtype = _DTYPES[a.dtype]
        r.A = a.data_ptr()
        r.n, r.m = a.shape
        r.lda = int(a.stride(0)) if a.shape[0] > 1 else int(a.shape[1])
        r.p, r.k, r.l, r.seed = int(p), int(k), int(l), int(seed)
        return r

    def submit_sketch(self, a: torch.Tensor, p: int, l: int, seed: int, out: torch.Tensor,
                      precision: int = 0) -> int:
        if (out.shape != (l, a.shape[1]) or not out.is_contiguous()
                or out.dtype != sketch_out_dtype(a.dtype, precision)):
            raise ValueError("out must be a contiguous l x m tensor of the sketch dtype")
        r = self._base(a, REQ_SKETCH, p, l, seed)
        r.out = out.data_ptr()
        r.precision = int(precision)
        return self._submit(r, (a, out))

    def submit_rsvd(self, a: torch.Tensor, k: int, l: int, p: int, seed: int,
                    outs: tuple[torch.Tensor, torch.Tensor, torch.Tensor]) -> int:
        u, sv, v = outs
        r = self._base(a, REQ_RSVD, p, l, seed, k)
        r.U, r.S, r.V = u.data_ptr(), sv.data_ptr(), v.data_ptr()
        return self._submit(r, (a, u, sv, v))

    def submit_nystrom(self, a: torch.Tensor, k: int, l: int, p: int, seed: int,
                       outs: tuple[torch.Tensor, torch.Tensor], precision: int = 0) -> int:
        u, lam = outs
        r = self._base(a, REQ_NYSTROM, p, l, seed, k)
        r.U, r.S = u.data_ptr(), lam.data_ptr()
        r.precision = int(precision)
        return self._submit(r, (a, u, lam))

    def poll(self, ticket: int) -> tuple[bool, int]:
        d = ctypes.c_int(0)
        st = lib.bsrht_poll(self._h, int(ticket), ctypes.byref(d))
        return bool(d.value), int(st)

    def wait(self, ticket: int, timeout_s: float = 600.0) -> int:
        """The request's status (BSRHT_OK = 0), or BSRHT_ETIMEDOUT."""
        st = int(lib.bsrht_wait(self._h, int(ticket), int(timeout_s * 1e6)))
        if st != BSRHT_ETIMEDOUT:
            self._keep.pop(int(ticket), None)
        return st

    def times(self, ticket: int) -> tuple[float, float]:
        """(submit, done) in seconds of the monotonic clock (time.monotonic's);
        done is -1 while the request is pending."""
        a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
        _check(lib.bsrht_request_times(self._h, int(ticket), ctypes.byref(a), ctypes.byref(b)), "bsrht_request_times")
        return float(a.value), float(b.value)

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib.bsrht_server_stats_get(self._h, ctypes.byref(s)), "bsrht_server_stats_get")
        return {name: getattr(s, name) for name, _ in ServerStats._fields_}

    def close(self) -> None:
        if self._h:
            _check(lib.bsrht_server_destroy(self._h), "bsrht_server_destroy")
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


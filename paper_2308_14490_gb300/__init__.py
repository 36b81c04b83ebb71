"""Python binding of the GB300 AZ solver (include/az.h).

Argument marshalling only: every step of the solver runs in the CUDA kernels
of libaz.so.  Arrays are torch CUDA tensors (device memory); streams are torch
CUDA streams.  Importing this package fails loudly when libaz.so is missing.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libaz.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libaz.so not built ({LIB_PATH}); run paper_2308_14490_gb300.build.build()")
_lib = ctypes.CDLL(LIB_PATH)

AZ_OK, AZ_ERR_ARG, AZ_ERR_OOM, AZ_ERR_ADMISSION, AZ_ERR_CUDA, AZ_ERR_NUMERIC, AZ_ERR_TIMEOUT = range(7)
AZ_FP64, AZ_MIXED = 0, 1
AZ_GAUSS, AZ_NEG_LAPLACE_GAUSS = 0, 1
(AZ_ARRAY_SYMBOL, AZ_ARRAY_SKETCH, AZ_ARRAY_W, AZ_ARRAY_R, AZ_ARRAY_UT, AZ_ARRAY_SIGMA,
 AZ_ARRAY_KEPT) = range(7)
STATUS_NAMES = ["AZ_OK", "AZ_ERR_ARG", "AZ_ERR_OOM", "AZ_ERR_ADMISSION", "AZ_ERR_CUDA",
                "AZ_ERR_NUMERIC", "AZ_ERR_TIMEOUT"]


class az_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n", ctypes.c_int64 * 2), ("s", ctypes.c_int32 * 2),
                ("T", ctypes.c_double * 2)]


class az_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("k", ctypes.c_int32), ("tau_svd", ctypes.c_double),
                ("tau_sym", ctypes.c_double), ("seed", ctypes.c_uint64), ("refine_steps", ctypes.c_int32),
                ("k0", ctypes.c_double), ("bnormal", ctypes.c_void_p)]


class az_info_t(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("L", ctypes.c_int64), ("M", ctypes.c_int64), ("Mb", ctypes.c_int64),
                ("k", ctypes.c_int32), ("rank", ctypes.c_int32), ("rank_gram", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("sigma_max", ctypes.c_double),
                ("sigma_min_kept", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
                ("jacobi_sweeps", ctypes.c_int32)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_D = ctypes.c_double
_SIGS = {
    "az_setup": [ctypes.POINTER(az_grid), _P, _P, _I64, _D, _I32, _D, ctypes.POINTER(az_options), _P,
                 ctypes.POINTER(_P)],
    "az_solve": [_P, _P, _I64, _I64, _P, _I64, _P, _P],
    "az_collocate": [_P, _P, _I64, _P, _I64, _I64, _P, _I64, _P, _P],
    "az_evaluate": [_P, _P, _I64, _I64, _I32, _P, _I64, _P],
    "az_apply_A": [_P, _P, _I64, _I64, _P, _I64, _P],
    "az_apply_Zstar": [_P, _P, _I64, _I64, _P, _I64, _P],
    "az_get_array": [_P, _I32, _P, _P],
    "az_get_info": [_P, ctypes.POINTER(az_info_t)],
    "az_query_footprint": [ctypes.POINTER(az_grid), _I64, _I64, ctypes.POINTER(az_options), _I64,
                           ctypes.POINTER(ctypes.c_size_t)],
    "az_destroy": [_P],
    "az_last_error": [],
    "az_rademacher": [_I64, _I32, ctypes.c_uint64, _P, _P],
    "az_refactor": [_P, ctypes.c_uint64, _P],
    "az_rademacher_noalloc": [_I64, _I32, ctypes.c_uint64, _P, _P],
    "az_launch_count": [],
    "az_debug_tc_withhold": [_I32, _I64],
    "az_debug_f32_sum_f64": [_P, _P, _P, _I64, _P],
    "az_debug_gram": [_P, _I64, _I32, _I64, _P, _I32, _P],
    "az_profile_begin": [],
    "az_profile_end": [],
    "az_profile_query": [_I32, ctypes.c_char_p, _I32, ctypes.POINTER(_I64), ctypes.POINTER(_D), ctypes.POINTER(_D)],
}
EXPORTS = list(_SIGS)
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = {"az_last_error": ctypes.c_char_p, "az_destroy": None, "az_profile_begin": None,
                  "az_launch_count": ctypes.c_int64}.get(_name, ctypes.c_int)


class AZError(RuntimeError):
    def __init__(self, status, where):
        msg = _lib.az_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


def _check(status, where):
    if status != AZ_OK:
        raise AZError(status, where)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _ld(t):
    """Leading dimension of a (ncols, rows) tensor viewed column-major: its row
    stride (the stride of a single row is arbitrary; the row length then)."""
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("expected a 2D tensor with contiguous rows")
    return t.stride(0) if t.shape[0] > 1 else t.shape[1]


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_grid(dim, n, s, T):
    g = az_grid()
    g.dim = dim
    for d in range(2):
        g.n[d] = int(n[d]) if d < dim else 1
        g.s[d] = int(s[d]) if d < dim else 1
        g.T[d] = float(T[d]) if d < dim else 1.0
    return g


def make_options(precision=AZ_MIXED, k=24, tau_svd=0.0, tau_sym=0.0, seed=1, refine_steps=-1, k0=0.0):
    o = az_options()
    o.precision, o.k, o.tau_svd, o.tau_sym, o.seed, o.refine_steps = precision, k, tau_svd, tau_sym, seed, refine_steps
    o.k0 = k0
    return o


def az_setup(grid, mask, eps, kernel=AZ_GAUSS, boundary=None, boundary_weight=1.0, options=None, stream=None,
             normals=None):
    """mask: uint8 CUDA tensor (grid points); boundary: (Mb, dim) float64 CUDA tensor or None;
    normals: (Mb, dim) float64 CUDA tensor (nonzero rows: Neumann points) or None."""
    h = ctypes.c_void_p()
    nb = 0 if boundary is None else int(boundary.shape[0])
    if normals is not None:
        if options is None:
            options = make_options()
        o = az_options()
        ctypes.pointer(o)[0] = options
        o.bnormal = normals.data_ptr()
        options = o
    _check(_lib.az_setup(ctypes.byref(grid), _ptr(mask), _ptr(boundary), nb, float(eps), int(kernel),
                         float(boundary_weight), ctypes.byref(options) if options is not None else None,
                         _stream(stream), ctypes.byref(h)), "az_setup")
    return h


def az_solve(h, b, x, stream=None, relres=False):
    """b: (nrhs, ldb) float64 CUDA tensor viewed column-major (each row of the
    tensor is one right-hand side); x: (nrhs, ldx) float64 output."""
    nrhs, ldb = b.shape
    rr = (ctypes.c_double * nrhs)() if relres else None
    _check(_lib.az_solve(h, _ptr(b), ldb, nrhs, _ptr(x), x.shape[1], _stream(stream), rr), "az_solve")
    return list(rr) if relres else None


def az_collocate(h, f, g, x, stream=None, relres=False):
    """f: (nrhs, >= M) interior data, g: (nrhs, >= Mb) boundary data, x: (nrhs, >= N);
    the leading dimensions are the tensors' row strides (views are allowed)."""
    nrhs = f.shape[0]
    rr = (ctypes.c_double * nrhs)() if relres else None
    _check(_lib.az_collocate(h, _ptr(f), _ld(f), _ptr(g), _ld(g), nrhs, _ptr(x), _ld(x), _stream(stream), rr),
           "az_collocate")
    return list(rr) if relres else None


def az_evaluate(h, x, s_test, out, stream=None):
    _check(_lib.az_evaluate(h, _ptr(x), x.shape[1], x.shape[0], int(s_test), _ptr(out), out.shape[1],
                            _stream(stream)), "az_evaluate")


def az_apply_A(h, x, y, stream=None):
    _check(_lib.az_apply_A(h, _ptr(x), x.shape[1], x.shape[0], _ptr(y), y.shape[1], _stream(stream)), "az_apply_A")


def az_apply_Zstar(h, y, x, stream=None):
    _check(_lib.az_apply_Zstar(h, _ptr(y), y.shape[1], y.shape[0], _ptr(x), x.shape[1], _stream(stream)),
           "az_apply_Zstar")


def az_get_array(h, which, dst, stream=None):
    _check(_lib.az_get_array(h, int(which), _ptr(dst), _stream(stream)), "az_get_array")


def az_get_info(h):
    info = az_info_t()
    _check(_lib.az_get_info(h, ctypes.byref(info)), "az_get_info")
    return {f: getattr(info, f) for f, _ in az_info_t._fields_}


def az_query_footprint(grid, M, n_boundary, options, nrhs_max):
    b = ctypes.c_size_t()
    _check(_lib.az_query_footprint(ctypes.byref(grid), int(M), int(n_boundary), ctypes.byref(options),
                                   int(nrhs_max), ctypes.byref(b)), "az_query_footprint")
    return b.value


def az_destroy(h):
    _lib.az_destroy(h)


def az_rademacher(N, k, seed, R, stream=None):
    """R: (k, N) float64 CUDA tensor (column j of the matrix is row j of the tensor)."""
    _check(_lib.az_rademacher(int(N), int(k), int(seed), _ptr(R), _stream(stream)), "az_rademacher")


def az_rademacher_noalloc(N, k, seed, R, stream=None):
    """Same output as az_rademacher, but uses the library's fixed device scratch
    instead of allocating (for callers that cannot allocate device memory)."""
    _check(_lib.az_rademacher_noalloc(int(N), int(k), int(seed), _ptr(R), _stream(stream)), "az_rademacher_noalloc")


def az_debug_tc_withhold(iteration, wait_ns):
    """Test hook: the next tensor-core projection launch withholds its TMA copies
    from `iteration` on, with waits bounded by wait_ns (see include/az.h)."""
    _check(_lib.az_debug_tc_withhold(int(iteration), int(wait_ns)), "az_debug_tc_withhold")


def az_debug_f32_sum_f64(a, b, out, stream=None):
    """Test hook: out = FP64 nearest to a + b for FP32 device tensors a, b of
    the same length, by the solve's FP64-pipe-free routine (see include/az.h)."""
    import torch
    n = a.numel()
    if b.numel() != n or out.numel() != n or a.dtype != torch.float32 or b.dtype != torch.float32 \
            or out.dtype != torch.float64 or not (a.is_contiguous() and b.is_contiguous() and out.is_contiguous()):
        raise ValueError("az_debug_f32_sum_f64: a, b FP32 and out FP64, contiguous, same length")
    _check(_lib.az_debug_f32_sum_f64(_ptr(a), _ptr(b), _ptr(out), n, _stream(stream)), "az_debug_f32_sum_f64")


def az_debug_gram(Y, G, route, stream=None):
    """Test hook: G (k, k) float64 = Y^T Y for Y (k, M) float32 CUDA tensor
    viewed column-major (row c of the tensor is column c); route 0 double-float
    SIMT, route 1 exact tensor-core split (see include/az.h)."""
    k, M = Y.shape
    _check(_lib.az_debug_gram(_ptr(Y), _ld(Y), int(k), int(M), _ptr(G), int(route), _stream(stream)), "az_debug_gram")


def az_last_error():
    return _lib.az_last_error().decode(errors="replace")


def az_refactor(h, seed, stream=None):
    """Recompute every setup step on the handle (new test-matrix seed), no allocation, no sync."""
    _check(_lib.az_refactor(h, int(seed), _stream(stream)), "az_refactor")


def az_launch_count():
    return int(_lib.az_launch_count())


def az_profile_begin():
    _lib.az_profile_begin()


def az_profile_end():
    _check(_lib.az_profile_end(), "az_profile_end")
    out = {}
    i = 0
    name = ctypes.create_string_buffer(128)
    n, ms, by = _I64(), _D(), _D()
    while _lib.az_profile_query(i, name, 128, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)) == AZ_OK:
        out[name.value.decode()] = {"launches": n.value, "ms": ms.value, "bytes": by.value}
        i += 1
    return out

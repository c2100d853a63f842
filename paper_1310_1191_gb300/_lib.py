"""ctypes binding of the C ABI in include/fem.h (argument marshalling only).

Function names match the C entry points.  Device buffers are passed as
torch CUDA tensors (their data pointers are handed to the library) or as raw
integer addresses; every computation runs in the library's CUDA kernels.
If the shared library has not been built, loading fails loudly: there is no
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfem_gb300.so")
# the checked variant (kernel index checks; build.build(checked=True)), loaded
# instead when the environment sets FEM_GB300_CHECKED=1
LIB_PATH_CHECKED = os.path.join(HERE, "libfem_gb300_checked.so")

FEM_OK, FEM_EINVAL, FEM_ENOMEM, FEM_ECUDA, FEM_EUNSUPPORTED, FEM_EELEMENT, FEM_ETIMEOUT, FEM_ECHECKED = range(8)
FEM_TET4, FEM_PRISM6 = 0, 1
FEM_F64, FEM_F32, FEM_BF16X3, FEM_F16X3 = 0, 1, 2, 3
FEM_OUT_FULL, FEM_OUT_SYMPACKED = 0, 1
FEM_RULE_COLLAPSED, FEM_RULE_TABLE1 = 0, 1
FEM_ST_DET, FEM_ST_NONFINITE, FEM_ST_NONSYM, FEM_ST_FALLBACK, FEM_ST_TIMEOUT = 1, 2, 4, 8, 16

# every symbol include/fem.h declares (checked by the CPU tests)
EXPORTS = (
    "fem_reference_rule", "fem_reference_rule_ex", "fem_tables_build", "fem_tables_build_ex",
    "fem_tables_destroy", "fem_integrate", "fem_integrate_uniform",
    "fem_sync_status", "fem_probe_fma",
    "fem_matrix_size", "fem_status_str", "fem_last_error", "fem_error_flag",
    "fem_output_offsets", "fem_plan_create", "fem_plan_execute", "fem_plan_variant",
    "fem_plan_destroy", "fem_integrate_mixed_noalloc",
    "fem_integrate_law", "fem_field_samples", "fem_box_from_samples", "fem_law_samples",
    "fem_mlp_create", "fem_mlp_destroy", "fem_mlp_nparams", "fem_mlp_forward", "fem_mlp_loss_grad",
    "fem_mlp_train", "fem_mlp_get", "fem_mlp_set", "fem_mlp_save", "fem_mlp_load",
    "fem_integrate_host", "fem_integrate_elastic", "fem_debug_stall_next", "fem_debug_shrink_bound",
    "fem_jacobian_terms", "fem_integrate_terms", "fem_integrate_elastic_terms", "fem_apply",
)
FEM_LAW_EXACT, FEM_LAW_MLP = 1, 2
FEM_PLAN_AUTOTUNE, FEM_PLAN_LOOP, FEM_PLAN_NOGRAPH, FEM_PLAN_CONCURRENT = 1, 2, 4, 8

_lib = None


class FemError(RuntimeError):
    def __init__(self, fn, code, msg):
        super().__init__("%s failed: %s (%d): %s" % (fn, status_str(code), code, msg))
        self.code = code


def load():
    """Load libfem_gb300.so (libfem_gb300_checked.so when FEM_GB300_CHECKED=1);
    raises if it was not built (no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    checked = os.environ.get("FEM_GB300_CHECKED", "") == "1"
    path = LIB_PATH_CHECKED if checked else LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("%s is not built: run paper_1310_1191_gb300.build.build(%s) "
                           "(or __graft_entry__.build()) first"
                           % (os.path.basename(path), "checked=True" if checked else ""))
    lib = ctypes.CDLL(path)
    i, i64, P = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
    lib.fem_reference_rule.argtypes = [i, i, P, P, P, P, P]
    lib.fem_tables_build.argtypes = [i, i, i, P]
    lib.fem_reference_rule_ex.argtypes = [i, i, i, P, P, P, P, P]
    lib.fem_tables_build_ex.argtypes = [i, i, i, i, P]
    lib.fem_tables_destroy.argtypes = [P]
    lib.fem_integrate.argtypes = [P, i64, P, P, i, P, i64, P, i, i, P, P, P, P]
    lib.fem_integrate_uniform.argtypes = [P, i, i64, P, P, i64, i, i, P, P, P, P]
    lib.fem_sync_status.argtypes = [P, P, i64, P, P, P]
    lib.fem_probe_fma.argtypes = [i, i, i64, i64, P, P, P]
    lib.fem_matrix_size.argtypes = [i, i, i]
    lib.fem_matrix_size.restype = i64
    lib.fem_status_str.argtypes = [i]
    lib.fem_status_str.restype = ctypes.c_char_p
    lib.fem_last_error.argtypes = []
    lib.fem_last_error.restype = ctypes.c_char_p
    lib.fem_error_flag.argtypes = [P, i]
    lib.fem_output_offsets.argtypes = [i, P, i64, i, P, P, P]
    lib.fem_plan_create.argtypes = [P, i64, P, i, i, i, ctypes.c_char_p, P]
    lib.fem_plan_execute.argtypes = [P, P, P, i64, P, P, P, P]
    lib.fem_plan_variant.argtypes = [P, i, P]
    lib.fem_plan_destroy.argtypes = [P]
    lib.fem_integrate_mixed_noalloc.argtypes = [P, i64, P, P, P, i64, i, i, P, P, P, P]
    u64, f = ctypes.c_uint64, ctypes.c_float
    lib.fem_integrate_law.argtypes = [P, i, i64, P, P, i64, P, i, P, i, i, P, P, P, P]
    lib.fem_field_samples.argtypes = [P, i, i64, P, P, P, P]
    lib.fem_box_from_samples.argtypes = [i64, P, ctypes.c_double, ctypes.c_double, P]
    lib.fem_law_samples.argtypes = [i64, P, u64, P, P, P]
    lib.fem_mlp_create.argtypes = [P, u64, P]
    lib.fem_mlp_destroy.argtypes = [P]
    lib.fem_mlp_nparams.argtypes = []
    lib.fem_mlp_forward.argtypes = [P, i64, P, P, P]
    lib.fem_mlp_loss_grad.argtypes = [P, i64, P, P, P, P, P]
    lib.fem_mlp_train.argtypes = [P, i64, P, P, i64, i, f, u64, P, P]
    lib.fem_mlp_get.argtypes = [P, P, P, P]
    lib.fem_mlp_set.argtypes = [P, P]
    lib.fem_mlp_save.argtypes = [P, ctypes.c_char_p]
    lib.fem_mlp_load.argtypes = [ctypes.c_char_p, P]
    lib.fem_integrate_host.argtypes = [P, i, i64, P, P, i64, i, i, P, P, P, i64]
    lib.fem_integrate_elastic.argtypes = [P, i, i64, P, P, i64, i, P, P, P, P]
    lib.fem_apply.argtypes = [P, i, i64, P, P, i64, i, P, P, P, P]
    lib.fem_jacobian_terms.argtypes = [P, i, i64, P, P, P, P]
    lib.fem_integrate_terms.argtypes = [P, i, i64, P, P, i64, i, i, P, P, P, P]
    lib.fem_integrate_elastic_terms.argtypes = [P, i, i64, P, P, i64, i, P, P, P, P]
    lib.fem_debug_stall_next.argtypes = [P]
    lib.fem_debug_shrink_bound.argtypes = [P]
    _lib = lib
    return lib


def status_str(code: int) -> str:
    return load().fem_status_str(code).decode()


def last_error() -> str:
    return load().fem_last_error().decode()


def _check(fn, code):
    if code != FEM_OK:
        raise FemError(fn, code, last_error())
    return code


def _addr(x):
    """Device/host address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError("cannot take the address of %r" % type(x))


def _stream(stream):
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return stream


def fem_reference_rule(elem: int, p: int):
    """(xi [nq][3], w [nq], phi [nq][4][ns]) from the library's host tables."""
    return fem_reference_rule_ex(elem, FEM_RULE_COLLAPSED, p)


def fem_reference_rule_ex(elem: int, rule: int, p: int):
    """fem_reference_rule for a chosen prism rule (FEM_RULE_COLLAPSED / FEM_RULE_TABLE1)."""
    lib = load()
    nq, ns = ctypes.c_int(), ctypes.c_int()
    _check("fem_reference_rule_ex", lib.fem_reference_rule_ex(elem, rule, p, ctypes.byref(nq),
                                                              ctypes.byref(ns), None, None, None))
    xi = np.zeros((nq.value, 3))
    w = np.zeros(nq.value)
    phi = np.zeros((nq.value, 4, ns.value))
    _check("fem_reference_rule_ex", lib.fem_reference_rule_ex(elem, rule, p, None, None, xi.ctypes.data,
                                                              w.ctypes.data, phi.ctypes.data))
    return xi, w, phi


def fem_matrix_size(elem: int, p: int, layout: int) -> int:
    return load().fem_matrix_size(elem, p, layout)


class Tables:
    """Owning wrapper of a fem_tables handle."""

    def __init__(self, elem: int, p_min: int, p_max: int, rule: int = FEM_RULE_COLLAPSED):
        self.elem, self.p_min, self.p_max, self.rule = elem, p_min, p_max, rule
        h = ctypes.c_void_p()
        _check("fem_tables_build_ex", load().fem_tables_build_ex(elem, rule, p_min, p_max, ctypes.byref(h)))
        self.handle = h

    def close(self):
        if self.handle:
            load().fem_tables_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fem_tables_build(elem: int, p_min: int, p_max: int) -> Tables:
    return Tables(elem, p_min, p_max)


def fem_tables_build_ex(elem: int, rule: int, p_min: int, p_max: int) -> Tables:
    return Tables(elem, p_min, p_max, rule)


def fem_tables_destroy(t: Tables) -> None:
    t.close()


class CoefLaw(ctypes.Structure):
    """fem_coef_law: law (0, FEM_LAW_EXACT, FEM_LAW_MLP), ucoef, mlp,
    newton_steps (0: 8), hw_tanh."""
    _fields_ = [("law", ctypes.c_int), ("ucoef", ctypes.c_void_p), ("mlp", ctypes.c_void_p),
                ("newton_steps", ctypes.c_int), ("hw_tanh", ctypes.c_int)]


def coef_law(law: int, ucoef=None, mlp=None, newton_steps: int = 0, hw_tanh: bool = False) -> CoefLaw:
    """A coefficient law for fem_integrate (ucoef: device float [n][NS])."""
    c = CoefLaw(law, _addr(ucoef), mlp.handle.value if mlp is not None else None, newton_steps,
                1 if hw_tanh else 0)
    c._keep = (ucoef, mlp)  # the buffers must outlive the call
    return c


def fem_integrate(t: Tables, n_elem: int, coords, p_per_elem, p_uniform: int, coeffs, coeff_stride: int,
                  law, prec: int, layout: int, A_out, b_out=None, status=None, stream=None) -> int:
    """Enqueue the integration of n_elem elements (see fem.h): p_per_elem a
    host int8 array of degrees or None (then every element has p_uniform);
    law None (constant coefficients) or a CoefLaw from coef_law()."""
    pp = None
    if p_per_elem is not None:
        pp = np.ascontiguousarray(p_per_elem, dtype=np.int8)
        if pp.shape[0] != n_elem:
            raise ValueError("p_per_elem must have n_elem entries")
    return _check("fem_integrate", load().fem_integrate(
        t.handle, n_elem, _addr(coords), pp.ctypes.data if pp is not None else None, p_uniform,
        _addr(coeffs), coeff_stride, ctypes.byref(law) if law is not None else None, prec, layout,
        _addr(A_out), _addr(b_out), _addr(status), _stream(stream)))


def fem_probe_fma(fp64: bool, form: int, iters: int, n_threads: int, out, clk=None, stream=None) -> int:
    """Enqueue the FMA-pipe throughput probe (form 0: 8 chains of iters
    multiply-adds per thread; form 1: 32 x iters outer-product steps of 16
    (FP64) or 64 (FP32) multiply-adds per thread; clk: optional int64
    [n_threads / 256][2] cycles and ns per CTA)."""
    return _check("fem_probe_fma", load().fem_probe_fma(1 if fp64 else 0, form, iters, n_threads, _addr(out),
                                                        _addr(clk), _stream(stream)))


def fem_integrate_uniform(t: Tables, p: int, n_elem: int, coords, coeffs, coeff_stride: int, prec: int,
                          layout: int, A_out, b_out=None, status=None, stream=None) -> int:
    """Enqueue the integration of n_elem elements of degree p with constant
    coefficients (one direct launch; see fem.h)."""
    return _check("fem_integrate_uniform", load().fem_integrate_uniform(
        t.handle, p, n_elem, _addr(coords), _addr(coeffs), coeff_stride, prec, layout,
        _addr(A_out), _addr(b_out), _addr(status), _stream(stream)))


def fem_sync_status(t: Tables, status, n_elem: int, stream=None):
    """(code, bits, n_flagged): waits for the stream and reduces status[]; code
    is FEM_OK, FEM_EELEMENT or FEM_ETIMEOUT (returned, not raised); other
    codes raise FemError."""
    bits = ctypes.c_int32()
    nflag = ctypes.c_int64()
    code = load().fem_sync_status(t.handle, _addr(status), n_elem, ctypes.byref(bits),
                                  ctypes.byref(nflag), _stream(stream))
    if code not in (FEM_OK, FEM_EELEMENT, FEM_ETIMEOUT):
        raise FemError("fem_sync_status", code, last_error())
    return code, bits.value, nflag.value


def fem_apply(t: Tables, p: int, n_elem: int, coords, coeffs, coeff_stride: int, prec: int, x, y,
              status=None, stream=None) -> int:
    """Enqueue y_e = A_e x_e for n_elem elements without forming A_e (see fem.h)."""
    return _check("fem_apply", load().fem_apply(
        t.handle, p, n_elem, _addr(coords), _addr(coeffs), coeff_stride, prec, _addr(x), _addr(y),
        _addr(status), _stream(stream)))


def fem_error_flag(t: Tables, clear: bool = True) -> int:
    """FEM_ETIMEOUT if a bounded device wait expired since the last clear,
    FEM_ECHECKED if a kernel index check of the checked build failed, else
    FEM_OK (synchronises)."""
    return load().fem_error_flag(t.handle, 1 if clear else 0)


def fem_output_offsets(elem: int, p_host, layout: int):
    """(offA [n], offb [n], total_A, total_b) for a mixed-degree mesh (int8 degrees)."""
    p_host = np.ascontiguousarray(p_host, dtype=np.int8)
    n = p_host.shape[0]
    offA = np.zeros(n, dtype=np.int64)
    offb = np.zeros(n, dtype=np.int64)
    tot = np.zeros(2, dtype=np.int64)
    _check("fem_output_offsets", load().fem_output_offsets(elem, p_host.ctypes.data, n, layout,
                                                           offA.ctypes.data, offb.ctypes.data,
                                                           tot.ctypes.data))
    return offA, offb, int(tot[0]), int(tot[1])


class Plan:
    """Owning wrapper of a fem_plan handle (mixed-degree prism mesh)."""

    def __init__(self, t: Tables, p_host, prec: int, layout: int = FEM_OUT_FULL, flags: int = 0,
                 tune_cache: str | None = None):
        p_host = np.ascontiguousarray(p_host, dtype=np.int8)
        self.n = p_host.shape[0]
        self.tables = t
        h = ctypes.c_void_p()
        _check("fem_plan_create", load().fem_plan_create(
            t.handle, self.n, p_host.ctypes.data, prec, layout, flags,
            tune_cache.encode() if tune_cache else None, ctypes.byref(h)))
        self.handle = h

    def variant(self, p: int):
        ms = np.zeros(4)
        v = load().fem_plan_variant(self.handle, p, ms.ctypes.data)
        return v, ms

    def close(self):
        if self.handle:
            load().fem_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fem_plan_create(t: Tables, p_host, prec: int, layout: int = FEM_OUT_FULL, flags: int = 0,
                    tune_cache: str | None = None) -> Plan:
    return Plan(t, p_host, prec, layout, flags, tune_cache)


def fem_plan_execute(plan: Plan, coords, coeffs, coeff_stride: int, A_out, b_out=None, status=None,
                     stream=None) -> int:
    return _check("fem_plan_execute", load().fem_plan_execute(
        plan.handle, _addr(coords), _addr(coeffs), coeff_stride, _addr(A_out), _addr(b_out),
        _addr(status), _stream(stream)))


def fem_plan_variant(plan: Plan, p: int):
    return plan.variant(p)


def fem_plan_destroy(plan: Plan) -> None:
    plan.close()


def fem_integrate_mixed_noalloc(t: Tables, p_host, coords, coeffs, coeff_stride: int, prec: int,
                                layout: int, A_out, b_out=None, status=None, stream=None) -> int:
    """Mixed-degree integration with no device allocation (fixed static scratch,
    at most 16384 elements); outputs laid out as fem_output_offsets describes."""
    p_host = np.ascontiguousarray(p_host, dtype=np.int8)
    return _check("fem_integrate_mixed_noalloc", load().fem_integrate_mixed_noalloc(
        t.handle, p_host.shape[0], p_host.ctypes.data, _addr(coords), _addr(coeffs), coeff_stride,
        prec, layout, _addr(A_out), _addr(b_out), _addr(status), _stream(stream)))


# ---------------------------------------------------------------- law and surrogate

def _f64arr(x):
    return np.ascontiguousarray(x, dtype=np.float64)


class Mlp:
    """Owning wrapper of a fem_mlp handle (2 -> 64 -> 64 -> 1 tanh surrogate)."""

    def __init__(self, box=None, seed: int = 42, handle=None):
        if handle is not None:
            self.handle = handle
            return
        b = _f64arr(box)
        h = ctypes.c_void_p()
        _check("fem_mlp_create", load().fem_mlp_create(b.ctypes.data, seed, ctypes.byref(h)))
        self.handle = h

    @staticmethod
    def nparams() -> int:
        return load().fem_mlp_nparams()

    def params(self):
        """(master FP32 [P], compute BF16-rounded [P], box [4]) as numpy arrays."""
        P = self.nparams()
        a = np.zeros(P, dtype=np.float32)
        c = np.zeros(P, dtype=np.float32)
        box = np.zeros(4)
        _check("fem_mlp_get", load().fem_mlp_get(self.handle, a.ctypes.data, c.ctypes.data, box.ctypes.data))
        return a, c, box

    def set_params(self, master):
        m = np.ascontiguousarray(master, dtype=np.float32)
        _check("fem_mlp_set", load().fem_mlp_set(self.handle, m.ctypes.data))

    def close(self):
        if self.handle:
            load().fem_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fem_mlp_create(box, seed: int = 42) -> Mlp:
    return Mlp(box, seed)


def fem_mlp_destroy(m: Mlp) -> None:
    m.close()


def fem_mlp_nparams() -> int:
    return Mlp.nparams()


def fem_mlp_forward(m: Mlp, n: int, us, y, stream=None) -> int:
    return _check("fem_mlp_forward", load().fem_mlp_forward(m.handle, n, _addr(us), _addr(y), _stream(stream)))


def fem_mlp_loss_grad(m: Mlp, n: int, us, t, grad, loss, stream=None) -> int:
    return _check("fem_mlp_loss_grad", load().fem_mlp_loss_grad(
        m.handle, n, _addr(us), _addr(t), _addr(grad), _addr(loss), _stream(stream)))


def fem_mlp_train(m: Mlp, n: int, us, t, steps: int, batch: int, lr: float, seed: int,
                  losses: bool = True, stream=None):
    """Run `steps` Adam steps; returns the per-step minibatch losses (numpy) or None."""
    out = np.zeros(max(steps, 1), dtype=np.float32) if losses else None
    _check("fem_mlp_train", load().fem_mlp_train(
        m.handle, n, _addr(us), _addr(t), steps, batch, float(lr), seed,
        out.ctypes.data if out is not None else None, _stream(stream)))
    return out[:steps] if out is not None else None


def fem_mlp_get(m: Mlp):
    return m.params()


def fem_mlp_set(m: Mlp, master) -> None:
    m.set_params(master)


def fem_mlp_save(m: Mlp, path: str) -> int:
    return _check("fem_mlp_save", load().fem_mlp_save(m.handle, path.encode()))


def fem_mlp_load(path: str) -> Mlp:
    h = ctypes.c_void_p()
    _check("fem_mlp_load", load().fem_mlp_load(path.encode(), ctypes.byref(h)))
    return Mlp(handle=h)


def fem_law_samples(n: int, box, seed: int, us, k, stream=None) -> int:
    b = _f64arr(box)
    return _check("fem_law_samples", load().fem_law_samples(n, b.ctypes.data, seed, _addr(us), _addr(k),
                                                            _stream(stream)))


def fem_field_samples(t: Tables, p: int, n: int, coords, ucoef, us, stream=None) -> int:
    return _check("fem_field_samples", load().fem_field_samples(
        t.handle, p, n, _addr(coords), _addr(ucoef), _addr(us), _stream(stream)))


def fem_box_from_samples(us_host, lo_pct: float = 0.1, hi_pct: float = 99.9):
    a = np.ascontiguousarray(us_host, dtype=np.float32).reshape(-1, 2)
    box = np.zeros(4)
    _check("fem_box_from_samples", load().fem_box_from_samples(a.shape[0], a.ctypes.data, lo_pct, hi_pct,
                                                               box.ctypes.data))
    return box


def fem_integrate_law(t: Tables, p: int, n_elem: int, coords, coeffs, coeff_stride: int, ucoef,
                      law: int, mlp, prec: int, layout: int, A_out, b_out=None, status=None,
                      stream=None) -> int:
    return _check("fem_integrate_law", load().fem_integrate_law(
        t.handle, p, n_elem, _addr(coords), _addr(coeffs), coeff_stride, _addr(ucoef), law,
        mlp.handle if mlp is not None else None, prec, layout, _addr(A_out), _addr(b_out),
        _addr(status), _stream(stream)))


def fem_integrate_host(t: Tables, p: int, n_elem: int, coords, coeffs, coeff_stride: int, prec: int,
                       layout: int, A_out, b_out=None, status=None, chunk: int = 0) -> int:
    """Integration with host buffers (pinned for overlap); synchronous."""
    return _check("fem_integrate_host", load().fem_integrate_host(
        t.handle, p, n_elem, _addr(coords), _addr(coeffs), coeff_stride, prec, layout, _addr(A_out),
        _addr(b_out), _addr(status), chunk))


def fem_integrate_elastic(t: Tables, p: int, n_elem: int, coords, coeffs, coeff_stride: int, prec: int,
                          A_out, b_out=None, status=None, stream=None) -> int:
    """Linear elastostatics: A_out [n][3][3][NS][NS], b_out [n][3][NS] (see fem.h)."""
    return _check("fem_integrate_elastic", load().fem_integrate_elastic(
        t.handle, p, n_elem, _addr(coords), _addr(coeffs), coeff_stride, prec, _addr(A_out),
        _addr(b_out), _addr(status), _stream(stream)))


def fem_jacobian_terms(t: Tables, p: int, n_elem: int, coords, terms, status=None, stream=None) -> int:
    """Split geometry pass: terms [n][NQ][10] = det J, J^{-1} per point (see fem.h)."""
    return _check("fem_jacobian_terms", load().fem_jacobian_terms(
        t.handle, p, n_elem, _addr(coords), _addr(terms), _addr(status), _stream(stream)))


def fem_integrate_terms(t: Tables, p: int, n_elem: int, terms, coeffs, coeff_stride: int, prec: int,
                        layout: int, A_out, b_out=None, status=None, stream=None) -> int:
    """Integration from stored Jacobian terms (NOJAC); outputs as fem_integrate."""
    return _check("fem_integrate_terms", load().fem_integrate_terms(
        t.handle, p, n_elem, _addr(terms), _addr(coeffs), coeff_stride, prec, layout,
        _addr(A_out), _addr(b_out), _addr(status), _stream(stream)))


def fem_integrate_elastic_terms(t: Tables, p: int, n_elem: int, terms, coeffs, coeff_stride: int,
                                prec: int, A_out, b_out=None, status=None, stream=None) -> int:
    """Linear elastostatics from stored Jacobian terms; outputs as fem_integrate_elastic."""
    return _check("fem_integrate_elastic_terms", load().fem_integrate_elastic_terms(
        t.handle, p, n_elem, _addr(terms), _addr(coeffs), coeff_stride, prec, _addr(A_out),
        _addr(b_out), _addr(status), _stream(stream)))


def fem_debug_shrink_bound(plan) -> int:
    """Checked-build test hook: the plan's next execution takes A_out as one
    value shorter, so the last block fails its offset check (see fem.h)."""
    return _check("fem_debug_shrink_bound", load().fem_debug_shrink_bound(plan.handle))


def fem_debug_stall_next(t: Tables) -> int:
    """Test hook: the next tensor-core launch withholds its operand copies (bounded waits expire)."""
    return _check("fem_debug_stall_next", load().fem_debug_stall_next(t.handle))

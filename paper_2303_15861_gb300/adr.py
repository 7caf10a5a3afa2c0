"""Thin ctypes binding of libadr (include/adr.h): argument marshalling only.

Every function has the name of the C entry point it calls. Device arrays are torch
tensors (their data pointers are passed), host coefficient arrays are numpy arrays,
streams are torch.cuda.Stream objects (their cudaStream_t is passed). All compute
runs in libadr's CUDA kernels; there is no fallback: loading fails loudly when the
library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libadr.so")

ADR_OK = 0
STATUS = {0: "ADR_OK", 1: "ADR_ERR_ARG", 2: "ADR_ERR_ALLOC", 3: "ADR_ERR_CUDA",
          4: "ADR_ERR_ILL_CONDITIONED", 5: "ADR_ERR_COMPLEX_SPECTRUM", 6: "ADR_ERR_TIMEOUT",
          7: "ADR_ERR_STATE", 8: "ADR_ERR_UNSUPPORTED"}
PRECISION = {"fp64": 0, "fp32": 1, "tf32x3": 2, "bf16x3": 3}
PHI_ROUTE = {"auto": 0, "eigen": 1, "doubling": 2, "fourier": 3}
BC = {"dirichlet": 0, "mixed": 1}          # faces x_mu = 1: Dirichlet, or Neumann ("mixed")
FORM = {"flux": 0, "adelta": 1}
SCHEME = {"lawson_euler": 0, "etd2rk": 1, "lawson4": 2, "exponential_euler": 3, "erk2p1": 4,
          "stabilized_lawson_euler": 5, "lawson2a": 6, "lawson2b": 7, "stabilized_lawson2": 8}


class AdrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class adr_params(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("lambda_", C.c_double),
                ("abar_override", C.c_double), ("tau", C.c_double), ("scheme", C.c_int),
                ("precision", C.c_int), ("kappa_tol", C.c_double), ("batch", C.c_int),
                ("n_batch", C.POINTER(C.c_int)), ("batch_tile", C.c_int), ("phi_route", C.c_int),
                ("bc_hi", C.c_int), ("form", C.c_int), ("periodic", C.c_int), ("length", C.c_double)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libadr.so (built by build_lib.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libadr.so not found at {path}: run paper_2303_15861_gb300.build_lib.build() "
                           "(the CUDA library is required; there is no CPU fallback)")
    lib = C.CDLL(path)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
    sig = {
        "adr_create": (ip, [C.POINTER(adr_params), vp, C.POINTER(vp)]),
        "adr_set_coeffs": (ip, [vp, ip, dp, dp, dp]),
        "adr_set_coeffs_periodic": (ip, [vp, dp, dp, dp]),
        "adr_step": (ip, [vp, vp, C.c_double]),
        "adr_integrate": (ip, [vp, vp, C.c_double, C.c_double, ip]),
        "adr_integrate_host": (ip, [vp, vp, C.c_double, C.c_double, ip]),
        "adr_eval_rhs": (ip, [vp, vp, vp, vp]),
        "adr_apply_exp": (ip, [vp, C.c_double, vp, vp]),
        "adr_apply_phi": (ip, [vp, ip, vp, vp]),
        "adr_synchronize": (ip, [vp]),
        "adr_test_bounded_wait": (ip, [vp, C.c_double]),
        "adr_profile_step": (ip, [vp, vp, ip, C.POINTER(C.c_float), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "adr_get_info": (ip, [vp, dp, dp, dp]),
        "adr_get_instance_info": (ip, [vp, ip, dp, dp, dp]),
        "adr_get_batch_plan": (ip, [vp, ip, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "adr_mumode_apply_static": (ip, [ip, C.POINTER(C.c_int), C.POINTER(vp), vp, vp, vp]),
        "adr_kernels_per_step": (ip, [vp]),
        "adr_tc_factor_slices": (ip, [vp, C.POINTER(C.c_int)]),
        "adr_phi_route_used": (ip, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "adr_stability_bound": (ip, [ip, dp]),
        "adr_measure_peak": (ip, [ip, ip, dp]),
        "adr_lambda_scan": (ip, [C.POINTER(adr_params), dp, dp, dp, dp, ip, ip, dp, ip, ip, vp, dp, dp]),
        "adr_lambda_scan_periodic": (ip, [C.POINTER(adr_params), dp, dp, dp, dp, ip, ip, dp, ip, ip, vp, dp, dp]),
        "adr_last_error": (C.c_char_p, [vp]),
        "adr_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status, ctx=None):
    if status != ADR_OK:
        msg = _lib.adr_last_error(ctx).decode()
        raise AdrError(status, msg)


def _ptr(t):
    """Data pointer of a device tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device arrays must be contiguous CUDA tensors")
    return C.c_void_p(t.data_ptr())


def _dbl(a, count=None):
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if count is not None and arr.size != count:
        raise ValueError(f"expected {count} values, got {arr.size}")
    return arr, arr.ctypes.data_as(C.POINTER(C.c_double))


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(int(stream.cuda_stream))


# ------------------------------------------------------------------- C entry points
def adr_create(dims, tau, scheme="lawson4", precision="fp64", lam=1.0, abar_override=0.0,
               kappa_tol=0.0, stream=None, batch_dims=None, batch_tile=0, phi_route="auto", bc="dirichlet",
               form="flux", periodic=False, length=0.0):
    """dims: grid of a single-grid context; batch_dims: [(n1, n2), ...] of a batched 2-D
    context (dims is then ignored); periodic=True with the box side `length`: a periodic
    Fourier pseudospectral context (coefficients through adr_set_coeffs_periodic)."""
    lib = load_library()
    p = adr_params()
    nb = None
    if batch_dims is not None:
        flat = [int(v) for d in batch_dims for v in d]
        nb = (C.c_int * len(flat))(*flat)
        p.dim = 2
        p.batch = len(batch_dims)
        p.n_batch = C.cast(nb, C.POINTER(C.c_int))
        p.batch_tile = int(batch_tile)
        dims = ()
    else:
        p.dim = len(dims)
    for i, n in enumerate(dims):
        p.n[i] = int(n)
    p.lambda_ = float(lam)
    p.abar_override = float(abar_override)
    p.tau = float(tau)
    p.scheme = SCHEME[scheme] if isinstance(scheme, str) else int(scheme)
    p.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    p.kappa_tol = float(kappa_tol)
    p.phi_route = PHI_ROUTE[phi_route] if isinstance(phi_route, str) else int(phi_route)
    p.bc_hi = BC[bc] if isinstance(bc, str) else int(bc)
    p.form = FORM[form] if isinstance(form, str) else int(form)
    p.periodic = 1 if periodic else 0
    p.length = float(length)
    ctx = C.c_void_p()
    _check(lib.adr_create(C.byref(p), _stream_handle(stream), C.byref(ctx)))
    return ctx


def adr_set_coeffs(ctx, instance, a_nodes, b, r_poly):
    a, ap = _dbl(a_nodes)
    bb, bp = _dbl(list(b) + [0.0] * (3 - len(b)), 3)
    rr, rp = _dbl(r_poly, 4)
    _check(_lib.adr_set_coeffs(ctx, int(instance), ap, bp, rp), ctx)


def adr_set_coeffs_periodic(ctx, a_diag, b_field, r_poly):
    """a_diag, b_field: d nodal arrays each (a_11, a_22[, a_33]; b_1, b_2[, b_3]), x1 fastest."""
    a, ap = _dbl(np.stack([np.ravel(np.asarray(x, dtype=np.float64)) for x in a_diag]))
    b, bp = _dbl(np.stack([np.ravel(np.asarray(x, dtype=np.float64)) for x in b_field]))
    if a.shape != b.shape:
        raise ValueError("a_diag and b_field must hold the same number of nodal arrays")
    rr, rp = _dbl(r_poly, 4)
    _check(_lib.adr_set_coeffs_periodic(ctx, ap, bp, rp), ctx)


PEAK_KIND = {"fp64_fma": 0, "fp32_fma": 1}


def adr_measure_peak(kind="fp64_fma", iters=2048):
    """Measured FMA peak of the current device in TFLOP/s (see adr.h)."""
    out = C.c_double()
    _check(load_library().adr_measure_peak(PEAK_KIND[kind] if isinstance(kind, str) else int(kind), int(iters),
                                           C.byref(out)))
    return out.value


def adr_step(ctx, u, t=0.0):
    _check(_lib.adr_step(ctx, _ptr(u), float(t)), ctx)


def adr_integrate(ctx, u, t0, T, m):
    _check(_lib.adr_integrate(ctx, _ptr(u), float(t0), float(T), int(m)), ctx)


def adr_integrate_host(ctx, u_host, t0, T, m):
    """u_host: contiguous CPU torch tensor or numpy array of the state dtype (in/out)."""
    if hasattr(u_host, "data_ptr"):
        if u_host.is_cuda or not u_host.is_contiguous():
            raise ValueError("u_host must be a contiguous CPU tensor")
        ptr = C.c_void_p(u_host.data_ptr())
    else:
        if not u_host.flags["C_CONTIGUOUS"]:
            raise ValueError("u_host must be C-contiguous")
        ptr = C.c_void_p(u_host.ctypes.data)
    _check(_lib.adr_integrate_host(ctx, ptr, float(t0), float(T), int(m)), ctx)


def adr_eval_rhs(ctx, u, F_out=None, g_out=None):
    _check(_lib.adr_eval_rhs(ctx, _ptr(u), _ptr(F_out), _ptr(g_out)), ctx)


def adr_apply_exp(ctx, c, v, y):
    _check(_lib.adr_apply_exp(ctx, float(c), _ptr(v), _ptr(y)), ctx)


def adr_apply_phi(ctx, k, v, y):
    _check(_lib.adr_apply_phi(ctx, int(k), _ptr(v), _ptr(y)), ctx)


def adr_test_bounded_wait(ctx, limit_ms=1.0):
    """Enqueue a wait that runs out after limit_ms (see adr.h); the next synchronize raises
    AdrError(ADR_ERR_TIMEOUT)."""
    _check(_lib.adr_test_bounded_wait(ctx, float(limit_ms)), ctx)


def adr_synchronize(ctx):
    """Wait for the context stream; raises AdrError(ADR_ERR_TIMEOUT) if a bounded device
    wait gave up."""
    _check(_lib.adr_synchronize(ctx), ctx)


def adr_profile_step(ctx, u, max_ops=256):
    """One step with per-operation CUDA-event timing; returns [(kind, ms), ...]."""
    ms = (C.c_float * max_ops)()
    kind = (C.c_int * max_ops)()
    n = C.c_int()
    _check(_lib.adr_profile_step(ctx, _ptr(u), int(max_ops), ms, kind, C.byref(n)), ctx)
    return [(int(kind[i]), float(ms[i])) for i in range(n.value)]


def adr_mumode_apply_static(factors, v, y, stream=None):
    """y = v x_1 M_1 x_2 M_2 (x_3 M_3) in FP64 without any device allocation (see adr.h).
    factors: list of contiguous CUDA float64 tensors (n_mu x n_mu); v, y: CUDA float64
    tensors of numpy shape (n3, n2, n1) or (n2, n1)."""
    load_library()
    dims = tuple(int(f.shape[0]) for f in factors)
    n = (C.c_int * 3)(*(list(dims) + [1] * (3 - len(dims))))
    fp = (C.c_void_p * 3)(*([f.data_ptr() for f in factors] + [None] * (3 - len(factors))))
    st = _lib.adr_mumode_apply_static(len(dims), n, fp, _ptr(v), _ptr(y), _stream_handle(stream))
    if st != ADR_OK:
        raise AdrError(st, "adr_mumode_apply_static failed")


def adr_get_info(ctx):
    kappa = (C.c_double * 3)()
    abar = C.c_double()
    beta = (C.c_double * 3)()
    _check(_lib.adr_get_info(ctx, kappa, C.byref(abar), beta), ctx)
    return {"kappa": list(kappa), "abar": abar.value, "beta": list(beta)}


def adr_get_instance_info(ctx, instance):
    kappa = (C.c_double * 3)()
    abar = C.c_double()
    beta = (C.c_double * 3)()
    _check(_lib.adr_get_instance_info(ctx, int(instance), kappa, C.byref(abar), beta), ctx)
    return {"kappa": list(kappa), "abar": abar.value, "beta": list(beta)}


def adr_get_batch_plan(ctx, mode, batch):
    edges = (C.c_int * int(batch))()
    grid = C.c_int()
    _check(_lib.adr_get_batch_plan(ctx, int(mode), edges, C.byref(grid)), ctx)
    return list(edges), grid.value


def adr_phi_route_used(ctx):
    """(route name or None, halvings, Taylor terms) of a context after adr_set_coeffs."""
    s, p = C.c_int(), C.c_int()
    r = int(_lib.adr_phi_route_used(ctx, C.byref(s), C.byref(p)))
    return ({0: None, 1: "eigen", 2: "doubling", 3: "fourier"}[r], s.value, p.value)


def adr_stability_bound(scheme):
    """Smallest lambda of unconditional stability on the model problem (Table 1)."""
    lib = load_library()
    out = C.c_double()
    _check(lib.adr_stability_bound(SCHEME[scheme] if isinstance(scheme, str) else int(scheme), C.byref(out)))
    return out.value


NORM = {"l2": 0, "max": 1}


def adr_lambda_scan(dims, tau, scheme, precision, a_nodes, b, r_poly, u0, m, lambdas=None, n_lambdas=8,
                    ref_substeps=8, abar_override=0.0, stream=None, norm="l2", bc="dirichlet", form="flux"):
    """Section 3's lambda scan on a small problem: returns (best lambda, [(lambda, error)])."""
    bb, bp = _dbl(list(b) + [0.0] * (3 - len(b)), 3)
    a, ap = _dbl(a_nodes)
    extra = {"bc_hi": BC[bc] if isinstance(bc, str) else int(bc), "form": FORM[form] if isinstance(form, str) else int(form)}
    return _scan("adr_lambda_scan", dims, tau, scheme, precision, (ap, bp), r_poly, u0, m, lambdas, n_lambdas,
                 ref_substeps, abar_override, stream, norm, extra, (a, bb))


def adr_lambda_scan_periodic(dims, length, tau, scheme, precision, a_diag, b_field, r_poly, u0, m, lambdas=None,
                             n_lambdas=8, ref_substeps=8, stream=None, norm="l2"):
    """The lambda scan of a periodic Fourier problem: returns (best lambda, [(lambda, error)])."""
    a, ap = _dbl(np.stack([np.ravel(np.asarray(x, dtype=np.float64)) for x in a_diag]))
    b, bp = _dbl(np.stack([np.ravel(np.asarray(x, dtype=np.float64)) for x in b_field]))
    return _scan("adr_lambda_scan_periodic", dims, tau, scheme, precision, (ap, bp), r_poly, u0, m, lambdas,
                 n_lambdas, ref_substeps, 0.0, stream, norm, {"periodic": 1, "length": float(length)}, (a, b))


def _scan(name, dims, tau, scheme, precision, coef_ptrs, r_poly, u0, m, lambdas, n_lambdas, ref_substeps,
          abar_override, stream, norm, extra, keep):
    lib = load_library()
    p = adr_params()
    p.dim = len(dims)
    for i, n in enumerate(dims):
        p.n[i] = int(n)
    p.abar_override = float(abar_override)
    p.tau = float(tau)
    p.scheme = SCHEME[scheme] if isinstance(scheme, str) else int(scheme)
    p.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    for k, v in extra.items():
        setattr(p, k, v)
    ap, bp = coef_ptrs
    rr, rp = _dbl(r_poly, 4)
    uu, up = _dbl(u0)
    if lambdas is not None:
        lam_arr, lamp = _dbl(lambdas)
        n_lambdas = lam_arr.size
        lam_list = [float(x) for x in lam_arr]
    else:
        lamp = None
        lo = adr_stability_bound(scheme)
        lam_list = [1.0] if n_lambdas == 1 else [lo + (1.0 - lo) * i / (n_lambdas - 1) for i in range(n_lambdas)]
    errs = (C.c_double * int(n_lambdas))()
    best = C.c_double()
    _check(getattr(lib, name)(C.byref(p), ap, bp, rp, up, int(m), int(n_lambdas), lamp, int(ref_substeps),
                              NORM[norm] if isinstance(norm, str) else int(norm), _stream_handle(stream), errs,
                              C.byref(best)))
    del keep
    return best.value, list(zip(lam_list, list(errs)))


def adr_kernels_per_step(ctx):
    return int(_lib.adr_kernels_per_step(ctx))


def adr_tc_factor_slices(ctx):
    n = C.c_int()
    _check(_lib.adr_tc_factor_slices(ctx, C.byref(n)), ctx)
    return n.value


def adr_last_error(ctx=None):
    return _lib.adr_last_error(ctx).decode()


def adr_destroy(ctx):
    if ctx is not None and ctx.value:
        _lib.adr_destroy(ctx)


# ------------------------------------------------------------------- convenience wrapper
class Context:
    """Owns one adr_ctx; methods forward to the C entry points above."""

    def __init__(self, dims, tau, scheme="lawson4", precision="fp64", stream=None, **kw):
        self.batch_dims = [tuple(int(v) for v in d) for d in kw["batch_dims"]] if kw.get("batch_dims") else None
        self.dims = tuple(int(n) for n in dims) if dims is not None else ()
        self.precision = precision
        self.ctx = adr_create(self.dims, tau, scheme, precision, stream=stream, **kw)

    def set_coeffs(self, a_nodes, b, r_poly, instance=0):
        adr_set_coeffs(self.ctx, instance, a_nodes, b, r_poly)
        return self

    def set_coeffs_periodic(self, a_diag, b_field, r_poly):
        adr_set_coeffs_periodic(self.ctx, a_diag, b_field, r_poly)
        return self

    def offsets(self):
        """Element offsets of the instances in a packed batched state (plus the total)."""
        out = [0]
        for n1, n2 in self.batch_dims:
            out.append(out[-1] + n1 * n2)
        return out

    def instance_info(self, i):
        return adr_get_instance_info(self.ctx, i)

    def batch_plan(self, mode):
        return adr_get_batch_plan(self.ctx, mode, len(self.batch_dims))

    def step(self, u, t=0.0):
        adr_step(self.ctx, u, t)

    def integrate(self, u, t0, T, m):
        adr_integrate(self.ctx, u, t0, T, m)

    def integrate_host(self, u_host, t0, T, m):
        adr_integrate_host(self.ctx, u_host, t0, T, m)

    def eval_rhs(self, u, F_out=None, g_out=None):
        adr_eval_rhs(self.ctx, u, F_out, g_out)

    def apply_exp(self, c, v, y):
        adr_apply_exp(self.ctx, c, v, y)

    def apply_phi(self, k, v, y):
        adr_apply_phi(self.ctx, k, v, y)

    def info(self):
        return adr_get_info(self.ctx)

    def synchronize(self):
        adr_synchronize(self.ctx)

    def profile_step(self, u):
        return adr_profile_step(self.ctx, u)

    def kernels_per_step(self):
        return adr_kernels_per_step(self.ctx)

    def tc_factor_slices(self):
        return adr_tc_factor_slices(self.ctx)

    def phi_route(self):
        return adr_phi_route_used(self.ctx)

    def close(self):
        adr_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            if self.ctx is not None:
                self.close()
        except Exception:
            pass

    @property
    def torch_dtype(self):
        import torch
        return torch.float64 if self.precision == "fp64" else torch.float32

"""Thin ctypes binding of liblqcd (include/lqcd.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Arrays are
torch tensors (complex128 fields, device tensors unless the C call accepts
host memory); each is passed as its data pointer, with the current CUDA
stream of the tensor's device.  No computation happens in Python, and there is
no fallback: if the library is not built, loading raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblqcd.so")

LQCD_OK = 0
LQCD_ERR_INVALID = -1
LQCD_ERR_CUDA = -2
LQCD_ERR_NOT_CONVERGED = -3
LQCD_ERR_BREAKDOWN = -4
LQCD_ERR_NONFINITE = -5
LQCD_ERR_TIMEOUT = -6
LQCD_ERR_NO_GAUGE = -7
LQCD_ERR_NOT_SU3 = -8
LQCD_ERR_OOM = -9
STATUS_NAMES = {0: "OK", -1: "INVALID", -2: "CUDA", -3: "NOT_CONVERGED", -4: "BREAKDOWN", -5: "NONFINITE",
                -6: "TIMEOUT", -7: "NO_GAUGE", -8: "NOT_SU3", -9: "OOM"}

LQCD_PREC_FP64 = 0
LQCD_PREC_MIXED_FP16 = 1
LQCD_PREC_MIXED_BF16 = 2
LQCD_SOLVER_BICGSTAB = 0
LQCD_SOLVER_CG = 1
LQCD_DILUTE_NONE = 0
LQCD_DILUTE_T = 1
LQCD_DILUTE_TS = 2
LQCD_DILUTE_TSC = 3
LQCD_DILUTE_EO = 4    # spatial even-odd partition, OR-ed onto a scheme above
LQCD_DILUTE_CUBE = 8  # spatial cubic (2^3 vertices) partition, OR-ed likewise
LQCD_STREAM_LP = 0
LQCD_STREAM_HP = 1


class LqcdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class lqcd_solver_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("precision", ctypes.c_int),
                ("solver", ctypes.c_int), ("delta", ctypes.c_double), ("rhs_block", ctypes.c_int),
                ("timeout_ms", ctypes.c_double)]


class lqcd_solve_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("status", ctypes.c_int), ("true_rel_residual", ctypes.c_double),
                ("reliable_updates", ctypes.c_int), ("restarts", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lqcd_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("hop_launches", ctypes.c_longlong), ("hop_ms", ctypes.c_double),
                ("hop_site_rhs", ctypes.c_double), ("hop_bytes", ctypes.c_double), ("hop_flops", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lqcd_stochastic_params(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("first_noise", ctypes.c_uint64), ("dilution", ctypes.c_int),
                ("n_lp", ctypes.c_int), ("n_hp", ctypes.c_int), ("tol_lp", ctypes.c_double),
                ("tol_hp", ctypes.c_double), ("chunk", ctypes.c_int)]


def stochastic_params(seed, n_lp, n_hp=0, tol_lp=1e-10, tol_hp=1e-10, dilution=LQCD_DILUTE_TSC, first_noise=0,
                      chunk=0):
    return lqcd_stochastic_params(seed, first_noise, dilution, n_lp, n_hp, tol_lp, tol_hp, chunk)


def solver_params(tol=1e-10, max_iter=20000, precision=LQCD_PREC_FP64, solver=LQCD_SOLVER_BICGSTAB, delta=0.05,
                  rhs_block=0, timeout_ms=0.0):
    return lqcd_solver_params(tol, max_iter, precision, solver, delta, rhs_block, timeout_ms)


_lib = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_u64 = ctypes.c_uint64
_SIGS = {
    "lqcd_create": (_i, [ctypes.POINTER(_vp), ctypes.POINTER(_i), _i]),
    "lqcd_destroy": (_i, [_vp]),
    "lqcd_last_error": (ctypes.c_char_p, [_vp]),
    "lqcd_set_gauge": (_i, [_vp, _vp, _vp]),
    "lqcd_set_gauge_general": (_i, [_vp, _vp, _vp]),
    "lqcd_set_kappa": (_i, [_vp, _d]),
    "lqcd_plaquette": (_i, [_vp, ctypes.POINTER(_d), _vp]),
    "lqcd_apply_dirac": (_i, [_vp, _vp, _vp, _i, _i, _vp]),
    "lqcd_solve_batch": (_i, [_vp, _vp, _vp, _i, ctypes.POINTER(lqcd_solver_params),
                              ctypes.POINTER(lqcd_solve_stats), _vp]),
    "lqcd_point_sources": (_i, [_vp, ctypes.POINTER(ctypes.c_int64), _i, _vp, _vp]),
    "lqcd_noise_generate": (_i, [_u64, _u64, _u64, ctypes.POINTER(_i), _i, _i, _i, _vp, _vp]),
    "lqcd_loops_batch": (_i, [_vp, _vp, _vp, _i, _d, _vp, _vp, _vp]),
    "lqcd_batch_create": (_i, [ctypes.POINTER(_vp)]),
    "lqcd_batch_add": (_i, [_vp, _vp, _vp, _vp, _i]),
    "lqcd_batch_run": (_i, [_vp, ctypes.POINTER(lqcd_solver_params), ctypes.POINTER(lqcd_solve_stats), _i, _vp]),
    "lqcd_batch_rhs": (_i, [_vp, ctypes.POINTER(_i)]),
    "lqcd_batch_destroy": (_i, [_vp]),
    "lqcd_autotune": (_i, [_vp, _i, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "lqcd_tuned_choice": (_i, [_vp, _i, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "lqcd_loops_stochastic": (_i, [_vp, ctypes.POINTER(lqcd_stochastic_params), ctypes.POINTER(lqcd_solver_params),
                                   _vp, _vp, ctypes.POINTER(lqcd_solve_stats), _vp]),
    "lqcd_gradient": (_i, [_vp, _vp, _vp, _i, _vp, _d, ctypes.POINTER(lqcd_solver_params), ctypes.POINTER(_d), _vp,
                           ctypes.POINTER(lqcd_solve_stats), _vp]),
    "lqcd_loops_batch_noalloc": (_i, [ctypes.POINTER(_i), _vp, _vp, _i, _d, _vp, _vp, _vp]),
    "lqcd_profile_begin": (_i, [_vp]),
    "lqcd_profile_end": (_i, [_vp, ctypes.POINTER(lqcd_profile)]),
    "lqcd_launch_count": (ctypes.c_longlong, []),
    "lqcd_dilution_pieces": (_i, [ctypes.POINTER(_i), _i]),
    "lqcd_loops_momentum": (_i, [_vp, _vp, _i, ctypes.POINTER(_i), _vp, _vp]),
    "lqcd_disconnected_correlator": (_i, [_vp, _vp, _i, _i, _i, _i, _vp, _vp]),
    "lqcd_smear_ape": (_i, [_vp, _d, _i, _vp, _vp]),
    "lqcd_smear_gaussian": (_i, [_vp, _vp, _vp, _i, _d, _i, _i, _i, _vp]),
}
OPTIONAL_SIGS = {}


def load():
    """Load liblqcd.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise OSError(f"liblqcd.so not built at {LIB_PATH}; run paper_1108_2473_gb300.build_lib.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in list(_SIGS.items()) + list(OPTIONAL_SIGS.items()):
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def declared_symbols():
    return sorted(list(_SIGS) + list(OPTIONAL_SIGS))


def _err(h):
    msg = load().lqcd_last_error(h)
    return msg.decode() if msg else ""


def _check(rc, h=None):
    if rc != LQCD_OK:
        raise LqcdError(rc, _err(h))
    return rc


def _ptr(t):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(t=None):
    if t is not None and t.is_cuda:
        return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)
    if torch.cuda.is_available():
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return None


def _dims(dims):
    arr = (ctypes.c_int * 4)(*[int(d) for d in dims])
    return arr


# lattice dims and device of every live context (recorded by lqcd_create), so
# that array arguments can be checked against them before the C call
_CTX = {}


def _ctx_info(h):
    info = _CTX.get(getattr(h, "value", h))
    if info is None:
        raise ValueError("unknown or destroyed lqcd context")
    return info


def _volume(dims):
    v = 1
    for d in dims:
        v *= int(d)
    return v


def _fields(device, *specs):
    """Check array arguments before a C call.  Each spec is (tensor or None,
    complex element count, name[, host_ok]).  Every tensor's dtype
    (complex128), contiguity and size are checked first, then that each is on
    CUDA device `device` (any device when None) unless host memory is allowed."""
    specs = [sp for sp in specs if sp[0] is not None]
    for sp in specs:
        t, count, name = sp[:3]
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name}: a torch tensor is required")
        if t.dtype != torch.complex128:
            raise ValueError(f"{name}: complex128 required, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name}: tensor must be contiguous")
        if t.numel() != count:
            raise ValueError(f"{name}: {t.numel()} complex elements, expected {count}")
    for sp in specs:
        t, name, host_ok = sp[0], sp[2], (sp[3] if len(sp) > 3 else False)
        if t.is_cuda:
            if device is not None and t.device.index != device:
                raise ValueError(f"{name}: on cuda:{t.device.index}, the lattice is on cuda:{device}")
        elif not host_ok:
            raise ValueError(f"{name}: must be a CUDA tensor")


# --------------------------------------------------------------------- calls
def lqcd_create(dims, device=0):
    h = ctypes.c_void_p()
    rc = load().lqcd_create(ctypes.byref(h), _dims(dims), int(device))
    _check(rc, None)
    _CTX[h.value] = (tuple(int(d) for d in dims), int(device))
    return h


def lqcd_destroy(h):
    _CTX.pop(getattr(h, "value", h), None)
    return load().lqcd_destroy(h)


def lqcd_last_error(h=None):
    return _err(h)


def lqcd_set_gauge(h, U):
    """U: complex128 [V][4][3][3] (any shape with that element count), device or host."""
    dims, dev = _ctx_info(h)
    _fields(dev, (U, _volume(dims) * 36, "U", True))
    return _check(load().lqcd_set_gauge(h, _ptr(U), _stream(U)), h)


def lqcd_set_gauge_general(h, U):
    """Arbitrary complex links (no SU(3) check; FP64 solves only)."""
    dims, dev = _ctx_info(h)
    _fields(dev, (U, _volume(dims) * 36, "U", True))
    return _check(load().lqcd_set_gauge_general(h, _ptr(U), _stream(U)), h)


def lqcd_set_kappa(h, kappa):
    return _check(load().lqcd_set_kappa(h, float(kappa)), h)


def lqcd_plaquette(h):
    out = ctypes.c_double()
    _check(load().lqcd_plaquette(h, ctypes.byref(out), _stream()), h)
    return out.value


def lqcd_apply_dirac(h, inp, out, dagger=False):
    nrhs = inp.shape[0]
    dims, dev = _ctx_info(h)
    _fields(dev, (inp, nrhs * _volume(dims) * 12, "in"), (out, nrhs * _volume(dims) * 12, "out"))
    return _check(load().lqcd_apply_dirac(h, _ptr(inp), _ptr(out), nrhs, int(bool(dagger)), _stream(inp)), h)


def lqcd_solve_batch(h, b, x, params):
    """Solve D x = b for the leading dimension of b, x.  Returns (status, [stats dicts]).

    Non-convergence is reported in the status and stats, not raised; argument
    and CUDA errors raise LqcdError.
    """
    nrhs = b.shape[0]
    dims, dev = _ctx_info(h)
    _fields(dev, (b, nrhs * _volume(dims) * 12, "b", True), (x, nrhs * _volume(dims) * 12, "x", True))
    stats = (lqcd_solve_stats * max(nrhs, 1))()
    rc = load().lqcd_solve_batch(h, _ptr(b), _ptr(x), nrhs, ctypes.byref(params), stats, _stream(b))
    if rc in (LQCD_ERR_INVALID, LQCD_ERR_CUDA, LQCD_ERR_NO_GAUGE, LQCD_ERR_OOM):
        raise LqcdError(rc, _err(h))
    return rc, [stats[k].as_dict() for k in range(nrhs)]


def lqcd_point_sources(h, sites, out):
    dims, dev = _ctx_info(h)
    _fields(dev, (out, 12 * len(sites) * _volume(dims) * 12, "out"))
    arr = (ctypes.c_int64 * len(sites))(*[int(s) for s in sites])
    return _check(load().lqcd_point_sources(h, arr, len(sites), _ptr(out), _stream(out)), h)


def lqcd_noise_generate(seed, noise_stream, noise_index, dims, dilution, first_piece, n_pieces, out):
    _fields(None, (out, int(n_pieces) * _volume(dims) * 12, "out"))
    rc = load().lqcd_noise_generate(int(seed), int(noise_stream), int(noise_index), _dims(dims), int(dilution),
                                    int(first_piece), int(n_pieces), _ptr(out), _stream(out))
    return _check(rc, None)


def lqcd_dilution_pieces(dims, dilution):
    n = load().lqcd_dilution_pieces(_dims(dims), int(dilution))
    if n < 0:
        raise LqcdError(LQCD_ERR_INVALID, f"unknown dilution scheme {dilution} or bad dims {tuple(dims)}")
    return n


def lqcd_loops_momentum(h, per_site, moms, out):
    """out[m, t, g] = sum_{x in t} exp(+i p_m.x) per_site[x, g]; moms: integer triples (n_x, n_y, n_z)."""
    dims, dev = _ctx_info(h)
    _fields(dev, (per_site, _volume(dims) * 6, "per_site"), (out, len(moms) * dims[3] * 6, "out"))
    flat = [int(v) for m in moms for v in m]
    arr = (_i * len(flat))(*flat)
    return _check(load().lqcd_loops_momentum(h, _ptr(per_site), len(moms), arr, _ptr(out), _stream(out)), h)


def lqcd_disconnected_correlator(loops_p, loops_mp, l3, out, unbiased=True):
    """D[t, A, B] from [n_vec, Lt, 6] loops at momenta p and -p (device tensors)."""
    n, lt = loops_p.shape[0], loops_p.shape[1]
    _fields(loops_p.device.index,
            (loops_p, n * lt * 6, "loops_p"),
            (loops_mp, n * lt * 6, "loops_mp"),
            (out, lt * 36, "out"))
    rc = load().lqcd_disconnected_correlator(_ptr(loops_p), _ptr(loops_mp), n, lt, int(l3), int(bool(unbiased)),
                                             _ptr(out), _stream(out))
    return _check(rc, None)


def lqcd_smear_ape(h, alpha, n_iter, out=None, stream=None):
    """APE-smear the context's spatial links (kept for lqcd_smear_gaussian); optional copy to out."""
    dims, dev = _ctx_info(h)
    _fields(dev, (out, _volume(dims) * 36, "out"))
    st = stream if (out is None and stream is not None) else _stream(out)
    return _check(load().lqcd_smear_ape(h, float(alpha), int(n_iter), _ptr(out), st), h)


def lqcd_smear_gaussian(h, src, out, alpha=4.0, n_iter=50, ape_links=False, normalise=False):
    """out = (1 + alpha H)^n_iter src on each time slice (device tensors [n, V, 4, 3])."""
    dims, dev = _ctx_info(h)
    _fields(dev, (src, src.shape[0] * _volume(dims) * 12, "src"), (out, src.shape[0] * _volume(dims) * 12, "out"))
    rc = load().lqcd_smear_gaussian(h, _ptr(src), _ptr(out), src.shape[0], float(alpha), int(n_iter),
                                    int(bool(ape_links)), int(bool(normalise)), _stream(out))
    return _check(rc, h)


def lqcd_loops_batch(h, src, sol, weight=1.0, per_site=None, per_t=None):
    nrhs = src.shape[0]
    dims, dev = _ctx_info(h)
    V = _volume(dims)
    _fields(dev,
            (src, nrhs * V * 12, "src"),
            (sol, nrhs * V * 12, "sol"),
            (per_site, V * 6, "per_site"),
            (per_t, dims[3] * 6, "per_t", True))
    st = _stream(src)
    return _check(load().lqcd_loops_batch(h, _ptr(src), _ptr(sol), nrhs, float(weight), _ptr(per_site),
                                          _ptr(per_t), st), h)


def lqcd_profile_begin(h):
    return _check(load().lqcd_profile_begin(h), h)


def lqcd_profile_end(h):
    out = lqcd_profile()
    _check(load().lqcd_profile_end(h, ctypes.byref(out)), h)
    return out.as_dict()


def lqcd_launch_count():
    return int(load().lqcd_launch_count())


def lqcd_loops_batch_noalloc(dims, src, sol, weight=1.0, per_site=None, per_t=None):
    """Loop contraction that allocates no device memory (see include/lqcd.h).

    For callers that cannot allocate: it needs no context and uses a fixed
    device array inside the library for its partial sums.  All tensors must be
    on the current CUDA device.
    """
    nrhs = src.shape[0]
    V = _volume(dims)
    dev = src.device.index if src.is_cuda else None
    _fields(dev,
            (src, nrhs * V * 12, "src"),
            (sol, nrhs * V * 12, "sol"),
            (per_site, V * 6, "per_site"),
            (per_t, dims[3] * 6, "per_t"))
    rc = load().lqcd_loops_batch_noalloc(_dims(dims), _ptr(src), _ptr(sol), nrhs, float(weight), _ptr(per_site),
                                         _ptr(per_t), _stream(src))
    return _check(rc, None)


def lqcd_gradient(h, src, sol, coef, params, weight=1.0, dU=None):
    """Adjoint-solve gradient of a real loss of the per-time-slice loops.

    coef: complex128 host tensor/array [Lt, 6] (d loss / d Re L + i d loss / d Im L).
    Returns (d loss / d kappa, status, stats); d loss / d U is accumulated into dU.
    """
    import numpy as np
    c = np.ascontiguousarray(np.asarray(coef.cpu() if hasattr(coef, "cpu") else coef, dtype=np.complex128))
    nrhs = src.shape[0]
    dims, dev = _ctx_info(h)
    V = _volume(dims)
    if c.size != dims[3] * 6:
        raise ValueError(f"coef: {c.size} elements, expected Lt * 6 = {dims[3] * 6}")
    _fields(dev, (src, nrhs * V * 12, "src"), (sol, nrhs * V * 12, "sol"), (dU, V * 36, "dU"))
    stats = (lqcd_solve_stats * max(nrhs, 1))()
    dk = ctypes.c_double(0.0)
    rc = load().lqcd_gradient(h, _ptr(src), _ptr(sol), nrhs, c.ctypes.data_as(ctypes.c_void_p), float(weight),
                              ctypes.byref(params), ctypes.byref(dk), _ptr(dU), stats, _stream(src))
    if rc in (LQCD_ERR_INVALID, LQCD_ERR_CUDA, LQCD_ERR_NO_GAUGE, LQCD_ERR_OOM):
        raise LqcdError(rc, _err(h))
    return dk.value, rc, [stats[k].as_dict() for k in range(nrhs)]


def lqcd_loops_stochastic(h, sparams, solver, per_site=None, per_t=None):
    """Plain diluted or truncated-solver-method loops, accumulated into per_site / per_t.

    Returns (status, [LP summary, HP summary]); argument and CUDA errors raise.
    """
    dims, dev = _ctx_info(h)
    _fields(dev, (per_site, _volume(dims) * 6, "per_site"), (per_t, dims[3] * 6, "per_t", True))
    summ = (lqcd_solve_stats * 2)()
    st = _stream(per_site) if per_site is not None else _stream(per_t)
    rc = load().lqcd_loops_stochastic(h, ctypes.byref(sparams), ctypes.byref(solver), _ptr(per_site), _ptr(per_t),
                                      summ, st)
    if rc in (LQCD_ERR_INVALID, LQCD_ERR_CUDA, LQCD_ERR_NO_GAUGE, LQCD_ERR_OOM):
        raise LqcdError(rc, _err(h))
    return rc, [summ[0].as_dict(), summ[1].as_dict()]


def lqcd_batch_create():
    h = ctypes.c_void_p()
    _check(load().lqcd_batch_create(ctypes.byref(h)), None)
    return h


def lqcd_batch_add(batch, ctx, b, x):
    dims, dev = _ctx_info(ctx)
    _fields(dev, (b, b.shape[0] * _volume(dims) * 12, "b"), (x, b.shape[0] * _volume(dims) * 12, "x"))
    return _check(load().lqcd_batch_add(batch, ctx, _ptr(b), _ptr(x), b.shape[0]), None)


def lqcd_batch_rhs(batch):
    """Total right-hand sides registered in the batch."""
    n = ctypes.c_int(0)
    _check(load().lqcd_batch_rhs(batch, ctypes.byref(n)), None)
    return n.value


def lqcd_batch_run(batch, params, total_rhs=None, stream=None):
    """Solve every registered entry; returns (status, [stats dicts in add order]).

    total_rhs sizes the stats array (default: the batch's own count); the
    library rejects a value below the batch's RHS total."""
    if total_rhs is None:
        total_rhs = lqcd_batch_rhs(batch)
    stats = (lqcd_solve_stats * max(total_rhs, 1))()
    st = ctypes.c_void_p(stream.cuda_stream) if stream is not None else _stream()
    rc = load().lqcd_batch_run(batch, ctypes.byref(params), stats, int(total_rhs), st)
    if rc in (LQCD_ERR_INVALID, LQCD_ERR_CUDA, LQCD_ERR_NO_GAUGE, LQCD_ERR_OOM):
        raise LqcdError(rc, _err(None))
    return rc, [stats[k].as_dict() for k in range(total_rhs)]


def lqcd_batch_destroy(batch):
    return load().lqcd_batch_destroy(batch)


def lqcd_tuned_choice(h, nrhs, precision):
    """The launch choice later solves of (nrhs, precision) use: (blocks per SM, hop variant)."""
    best = ctypes.c_int(0)
    var = ctypes.c_int(0)
    _check(load().lqcd_tuned_choice(h, int(nrhs), int(precision), ctypes.byref(best), ctypes.byref(var)), h)
    return best.value, var.value


def lqcd_autotune(h, nrhs, precision, with_variant=False):
    """Tune the hop kernel; returns blocks per SM (and the hop variant if with_variant)."""
    best = ctypes.c_int(0)
    var = ctypes.c_int(0)
    _check(load().lqcd_autotune(h, int(nrhs), int(precision), ctypes.byref(best), ctypes.byref(var)), h)
    return (best.value, var.value) if with_variant else best.value

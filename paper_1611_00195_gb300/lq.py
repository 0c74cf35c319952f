"""ctypes binding of liblq.so: argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this module converts
torch tensors / numpy arrays to pointers, sizes and streams, allocates caller-owned output
buffers, and maps error codes to exceptions.  There is no fallback: if liblq.so cannot be
loaded, every call raises.

Field conventions (see include/lq.h): spinor batches are complex128 [nsrc][V][4][3]; gauge
fields complex128 [4][V][3][3]; su(3) directions float64 [4][V][8]; U(1) directions
float64 [4][V].  Inputs may live on the host (numpy or CPU tensors) or on the context's GPU
(CUDA tensors); outputs are created on the same side as the input.
"""
import ctypes
import os

import numpy as np

try:
    import torch
except Exception:  # the binding also works with numpy-only callers
    torch = None

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblq.so")

LQ_OK = 0
LQ_ERR_ARG, LQ_ERR_LAYOUT, LQ_ERR_BREAKDOWN, LQ_ERR_NEWTON, LQ_ERR_NONFINITE = -1, -2, -5, -6, -9
# Revision tag of the stencil kernel; stored ncu traffic figures are only valid for this one.
KERNEL_REV = "hop-v7"
ERRORS = {-1: "LQ_ERR_ARG", -2: "LQ_ERR_LAYOUT", -3: "LQ_ERR_OOM", -4: "LQ_ERR_CUDA", -5: "LQ_ERR_BREAKDOWN",
          -6: "LQ_ERR_NEWTON", -7: "LQ_ERR_TIMEOUT", -8: "LQ_ERR_NOT_READY", -9: "LQ_ERR_NONFINITE",
          -10: "LQ_ERR_NOT_CONVERGED"}
LQ_FP64, LQ_MIXED, LQ_MIXED_BF16, LQ_FLOAT_FLOAT = 0, 1, 2, 3
LQ_DIR_MU, LQ_DIR_SU3, LQ_DIR_U1 = 0, 1, 2
LQ_PROJ_AUTO, LQ_PROJ_NEWTON, LQ_PROJ_QUAD, LQ_PROJ_NESTED = 0, 1, 2, 3
LQ_EIG_SHIFT_INVERT, LQ_EIG_CHEBYSHEV = 0, 1
LQ_RESERVE_BLOCK, LQ_RESERVE_ADJOINT, LQ_RESERVE_TWO_PASS, LQ_RESERVE_SOLVE, LQ_RESERVE_REBIORTH = 1, 2, 4, 8, 16

EXPORTED = ["lq_default_opts", "lq_create", "lq_destroy", "lq_last_error", "lq_upload_gauge", "lq_set_mu",
            "lq_reserve", "lq_apply_H", "lq_set_direction", "lq_apply_block", "lq_sign_apply",
            "lq_sign_derivative_apply", "lq_tsl_coefficients", "lq_newton_sign", "lq_profile_enable",
            "lq_profile_read", "lq_newton_sign_noalloc", "lq_nested_sign", "lq_error_estimate",
            "lq_upload_deflation", "lq_deflation_derivatives", "lq_sign_bilinear_grad",
            "lq_dense_eig", "lq_compute_deflation", "lq_eig_stats_read", "lq_overlap_apply", "lq_batch_apply", "lq_overlap_solve",
            "lq_axial_current"]


class LatticeDesc(ctypes.Structure):
    _fields_ = [("nt", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("m_w", ctypes.c_double), ("r", ctypes.c_double), ("mu", ctypes.c_double),
                ("t_antiperiodic", ctypes.c_int), ("precision", ctypes.c_int)]


class Opts(ctypes.Structure):
    _fields_ = [("kmax", ctypes.c_int), ("breakdown_tol", ctypes.c_double), ("newton_max_iter", ctypes.c_int),
                ("newton_tol", ctypes.c_double), ("deflate", ctypes.c_int), ("projected", ctypes.c_int),
                ("quad_nodes", ctypes.c_int), ("proj_tol", ctypes.c_double), ("hop_variant", ctypes.c_int),
                ("defl_kmax", ctypes.c_int), ("defl_nderiv", ctypes.c_int), ("two_pass", ctypes.c_int),
                ("graph", ctypes.c_int), ("split", ctypes.c_int), ("nested_m", ctypes.c_int),
                ("update_variant", ctypes.c_int), ("rebiorth", ctypes.c_int)]


class Report(ctypes.Structure):
    _fields_ = [("k_eff", ctypes.c_int), ("newton_iters", ctypes.c_int), ("status", ctypes.c_int),
                ("projected", ctypes.c_int), ("newton_change", ctypes.c_double), ("x_norm", ctypes.c_double),
                ("proj_check", ctypes.c_double), ("hop_variant", ctypes.c_int), ("reserved", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class Profile(ctypes.Structure):
    _fields_ = [("enabled", ctypes.c_int), ("reserved", ctypes.c_int), ("launches", ctypes.c_longlong),
                ("hop_ms", ctypes.c_double), ("hop_launches", ctypes.c_longlong),
                ("update_ms", ctypes.c_double), ("update_launches", ctypes.c_longlong),
                ("newton_ms", ctypes.c_double), ("newton_iterations", ctypes.c_longlong),
                ("other_ms", ctypes.c_double), ("other_launches", ctypes.c_longlong)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class EigOpts(ctypes.Structure):
    _fields_ = [("nev", ctypes.c_int), ("nsub", ctypes.c_int), ("degree", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("tol", ctypes.c_double), ("method", ctypes.c_int), ("inner_max", ctypes.c_int)]


class EigStats(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("restarts", ctypes.c_int), ("solves", ctypes.c_longlong),
                ("inner_iterations", ctypes.c_longlong), ("refinements", ctypes.c_longlong),
                ("norm_estimate", ctypes.c_double), ("max_residual", ctypes.c_double),
                ("pair_mismatch", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Direction(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("field", ctypes.c_void_p)]


_lib = None


class SolveReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("status", ctypes.c_int), ("residual", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class BatchItem(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("dir", ctypes.POINTER(Direction)), ("x", ctypes.c_void_p),
                ("y_sign", ctypes.c_void_p), ("y_deriv", ctypes.c_void_p), ("nsrc", ctypes.c_int),
                ("opts", ctypes.POINTER(Opts)), ("report", ctypes.POINTER(Report))]


def lib():
    """Load liblq.so (built in-tree by paper_1611_00195_gb300.build); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("liblq.so is not built (%s); run paper_1611_00195_gb300.build.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.lq_default_opts.argtypes = [ctypes.POINTER(Opts)]
        L.lq_default_opts.restype = None
        L.lq_create.argtypes = [ctypes.POINTER(LatticeDesc), ctypes.POINTER(P)]
        L.lq_destroy.argtypes = [P]
        L.lq_destroy.restype = None
        L.lq_last_error.argtypes = [P]
        L.lq_last_error.restype = ctypes.c_char_p
        L.lq_upload_gauge.argtypes = [P, P, P]
        L.lq_set_mu.argtypes = [P, D]
        L.lq_reserve.argtypes = [P, I, I, I]
        L.lq_apply_H.argtypes = [P, P, P, I, I, P]
        L.lq_set_direction.argtypes = [P, ctypes.POINTER(Direction), P]
        L.lq_apply_block.argtypes = [P, P, P, P, P, I, I, P]
        L.lq_sign_apply.argtypes = [P, P, P, I, ctypes.POINTER(Opts), ctypes.POINTER(Report), P]
        L.lq_sign_derivative_apply.argtypes = [P, ctypes.POINTER(Direction), P, P, P, I, ctypes.POINTER(Opts),
                                               ctypes.POINTER(Report), P]
        L.lq_overlap_apply.argtypes = [P, ctypes.POINTER(Direction), P, P, P, I, ctypes.POINTER(Opts),
                                       ctypes.POINTER(Report), P]
        L.lq_tsl_coefficients.argtypes = [P, I, I, P, P, P]
        L.lq_profile_enable.argtypes = [P, I]
        L.lq_profile_read.argtypes = [P, ctypes.POINTER(Profile)]
        L.lq_newton_sign.argtypes = [P, P, P, I, I, I, D, ctypes.POINTER(I), P]
        L.lq_nested_sign.argtypes = [P, P, P, P, P, I, I, I, P, P, P]
        L.lq_error_estimate.argtypes = [P, ctypes.POINTER(Direction), P, I, ctypes.POINTER(Opts), P, P]
        L.lq_upload_deflation.argtypes = [P, I, P, P, P, P]
        L.lq_deflation_derivatives.argtypes = [P, ctypes.POINTER(Direction), ctypes.POINTER(Opts), P, P, P, P]
        L.lq_sign_bilinear_grad.argtypes = [P, P, P, ctypes.POINTER(Opts), P, P, P, P]
        L.lq_dense_eig.argtypes = [I, P, P, P]
        L.lq_compute_deflation.argtypes = [P, ctypes.POINTER(EigOpts), P, P, P, P]
        L.lq_eig_stats_read.argtypes = [P, ctypes.POINTER(EigStats)]
        L.lq_newton_sign_noalloc.argtypes = [P, P, I, I, I, D, ctypes.POINTER(I), P]
        L.lq_batch_apply.argtypes = [ctypes.POINTER(BatchItem), I, P]
        L.lq_overlap_solve.argtypes = [P, P, P, I, D, D, I, ctypes.POINTER(Opts), ctypes.POINTER(SolveReport), P]
        L.lq_axial_current.argtypes = [P, ctypes.POINTER(Direction), P, I, D, D, I, ctypes.POINTER(Opts), P,
                                       ctypes.POINTER(SolveReport), P]
        for name in EXPORTED:
            if name not in ("lq_default_opts", "lq_destroy", "lq_last_error"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


class LQError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "LQ_ERR"), code, msg))
        self.code = code


# ---- marshalling helpers -------------------------------------------------------------------

def _is_tensor(x):
    return torch is not None and isinstance(x, torch.Tensor)


def _ptr(x):
    if x is None:
        return None
    if _is_tensor(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError("expected a torch.Tensor or numpy.ndarray, got %r" % type(x))


def _as_c128(x):
    if _is_tensor(x):
        return x.to(torch.complex128).contiguous()
    return np.ascontiguousarray(x, dtype=np.complex128)


def _as_f64(x):
    if _is_tensor(x):
        return x.to(torch.float64).contiguous()
    return np.ascontiguousarray(x, dtype=np.float64)


def _empty_like(x, shape=None):
    shape = tuple(x.shape) if shape is None else tuple(shape)
    if _is_tensor(x):
        return torch.empty(shape, dtype=x.dtype, device=x.device)
    return np.empty(shape, dtype=x.dtype)


def _stream(x=None):
    if torch is not None and torch.cuda.is_available():
        dev = x.device if (_is_tensor(x) and x.is_cuda) else None
        return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    return ctypes.c_void_p(0)


class SignBilinearForce(torch.autograd.Function if torch is not None else object):
    """S = Re <y| sgn(H(mu)) |x> as a function of the link tangent coordinates omega [4][V][8]
    (U_nu(s) -> exp(i omega^a lambda_a/2) U_nu(s)) and of mu, evaluated at omega = 0 (the
    uploaded links) and at the context's mu.  backward returns the fermionic force dS/domega and
    dS/dmu from the library's adjoint (lq_sign_bilinear_grad); x, y and the context are not
    differentiated.  Usage: S = SignBilinearForce.apply(omega, mu, ctx, x, y, k)."""

    @staticmethod
    def forward(fctx, omega, mu, lqctx, x, y, k):
        if torch.count_nonzero(omega).item() != 0:
            raise ValueError("the force is evaluated at the uploaded links: omega must be zero")
        if abs(float(mu) - lqctx.mu) > 0.0:
            raise ValueError("mu must equal the context's mu")
        S, F, dmu = lqctx.bilinear_grad(x, y, k)
        F = F if _is_tensor(F) else torch.from_numpy(F)
        fctx.save_for_backward(F.to(omega.device, torch.float64), torch.tensor(dmu, dtype=torch.float64))
        return torch.tensor(S, dtype=torch.float64, device=omega.device)

    @staticmethod
    def backward(fctx, gS):
        F, dmu = fctx.saved_tensors
        return gS * F, (gS.cpu() * dmu).to(gS.device), None, None, None, None


def newton_sign_noalloc(X, max_iter=50, tol=1e-13):
    """Batched dense sign of complex k x k matrices X [nb][k][k] (CUDA tensor, k <= 128, nb <= 8)
    through the allocation-free entry point: no context and no device allocation by the library
    (the output tensor is allocated here, by the caller's allocator).  The call runs on X's
    device and current stream."""
    if not (_is_tensor(X) and X.is_cuda):
        raise TypeError("newton_sign_noalloc takes a CUDA tensor (the entry point reads device memory only)")
    X = _as_c128(X)
    nb, k = X.shape[0], X.shape[1]
    with torch.cuda.device(X.device):
        S = _empty_like(X)
        iters = (ctypes.c_int * nb)()
        code = lib().lq_newton_sign_noalloc(_ptr(X), _ptr(S), int(k), int(nb), int(max_iter), float(tol), iters,
                                            _stream(X))
    if code != LQ_OK:
        raise LQError(code, "lq_newton_sign_noalloc (k <= 128, nb <= 8)")
    return S, list(iters)


def batch_apply(members):
    """Ragged batch through lq_batch_apply: the Krylov loops of all members in one CUDA graph
    launch.  `members` is a list of dicts with keys ctx (a Context, each at most once), x
    ([nsrc][V][4][3]), k, and optionally kind / field (a derivative along that direction, as in
    Context.sign_derivative_apply; kind=None for the sign alone) and any option of Context.opts.
    Returns one (y_sign, y_deriv or None, reports) per member."""
    n = len(members)
    items = (BatchItem * n)()
    keep, outs = [], []
    for i, m in enumerate(members):
        c = m["ctx"]
        x = _as_c128(m["x"])
        nsrc = x.shape[0]
        kind = m.get("kind", LQ_DIR_MU)
        ys = _empty_like(x)
        yd = _empty_like(x) if kind is not None else None
        o = Context.opts(m["k"], **{key: v for key, v in m.items() if key not in ("ctx", "x", "k", "kind", "field")})
        rep = (Report * nsrc)()
        d, f = c._direction(kind, m.get("field")) if kind is not None else (None, None)
        keep += [x, o, rep, d, f]
        items[i] = BatchItem(c._h, ctypes.pointer(d) if d is not None else None, _ptr(x), _ptr(ys), _ptr(yd),
                             int(nsrc), ctypes.pointer(o), rep)
        outs.append((ys, yd, rep))
    code = lib().lq_batch_apply(items, n, _stream(keep[0]))
    if code != LQ_OK:
        msg = ""   # from the first member context that holds one
        for m in members:
            e = lib().lq_last_error(m["ctx"]._h)
            if e:
                msg = e.decode()
                break
        raise LQError(code, msg)
    del keep
    return [(ys, yd, [r.as_dict() for r in rep]) for ys, yd, rep in outs]


class Context:
    """One lattice, gauge field, Wilson parameters and workspace on the current CUDA device.

    dims = (nt, nx, ny, nz); precision = LQ_FP64 or LQ_MIXED (include/lq.h)."""

    def __init__(self, dims, m_w=-2.0, mu=0.0, precision=LQ_FP64, antiperiodic_t=True, r=1.0):
        self._L = lib()
        nt, nx, ny, nz = (int(d) for d in dims)
        self.dims = (nt, nx, ny, nz)
        self.V = nt * nx * ny * nz
        self.precision = precision
        d = LatticeDesc(nt, nx, ny, nz, float(m_w), float(r), float(mu), int(bool(antiperiodic_t)), int(precision))
        h = ctypes.c_void_p()
        self._check(self._L.lq_create(ctypes.byref(d), ctypes.byref(h)), None)
        self._h = h
        self.mu = float(mu)

    def close(self):
        if getattr(self, "_h", None):
            self._L.lq_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, code, h="self"):
        if code != LQ_OK:
            msg = ""
            handle = self._h if h == "self" else h
            if handle:
                m = self._L.lq_last_error(handle)
                msg = m.decode() if m else ""
            raise LQError(code, msg)

    # --- set-up -----------------------------------------------------------------------
    def upload_gauge(self, U):
        U = _as_c128(U)
        self._U = U
        self._check(self._L.lq_upload_gauge(self._h, _ptr(U), _stream(U)))

    def set_mu(self, mu):
        self._check(self._L.lq_set_mu(self._h, float(mu)))
        self.mu = float(mu)

    def reserve(self, kmax, nsrc, block=True, adjoint=False, two_pass=False, solve=False, rebiorth=False):
        flags = ((LQ_RESERVE_BLOCK if block else 0) | (LQ_RESERVE_ADJOINT if adjoint else 0)
                 | (LQ_RESERVE_TWO_PASS if two_pass else 0) | (LQ_RESERVE_SOLVE if solve else 0)
                 | (LQ_RESERVE_REBIORTH if rebiorth else 0))
        self._check(self._L.lq_reserve(self._h, int(kmax), int(nsrc), int(flags)))

    def _direction(self, kind, field):
        if kind == LQ_DIR_MU:
            return Direction(LQ_DIR_MU, None), None
        f = _as_f64(field)
        return Direction(kind, _ptr(f)), f

    def set_direction(self, kind, field=None):
        d, keep = self._direction(kind, field)
        self._check(self._L.lq_set_direction(self._h, ctypes.byref(d), _stream(keep)))
        self._dir_keep = keep

    # --- operators ----------------------------------------------------------------------
    def apply_H(self, x, dagger=False):
        """H(mu) x (or H(mu)^dag x) for x of shape [nsrc][V][4][3]."""
        x = _as_c128(x)
        nsrc = x.shape[0]
        y = _empty_like(x)
        self._check(self._L.lq_apply_H(self._h, _ptr(x), _ptr(y), int(nsrc), int(bool(dagger)), _stream(x)))
        return y

    def apply_block(self, top, bottom, dagger=False):
        """B (top, bottom) = (A top + dA bottom, A bottom), or B^dag, along the current direction."""
        top, bottom = _as_c128(top), _as_c128(bottom)
        yt, yb = _empty_like(top), _empty_like(bottom)
        self._check(self._L.lq_apply_block(self._h, _ptr(top), _ptr(bottom), _ptr(yt), _ptr(yb), int(top.shape[0]),
                                           int(bool(dagger)), _stream(top)))
        return yt, yb

    @staticmethod
    def opts(k, breakdown_tol=1e-14, newton_max_iter=50, newton_tol=1e-13, projected=LQ_PROJ_AUTO, quad_nodes=64,
             proj_tol=1e-11, hop_variant=-1, deflate=0, defl_kmax=0, defl_nderiv=0, two_pass=0, graph=-1, split=-1,
             nested_m=100, update_variant=-1, rebiorth=0):
        o = Opts()
        lib().lq_default_opts(ctypes.byref(o))
        o.kmax = int(k)
        o.breakdown_tol = float(breakdown_tol)
        o.newton_max_iter = int(newton_max_iter)
        o.newton_tol = float(newton_tol)
        o.projected = int(projected)
        o.quad_nodes = int(quad_nodes)
        o.proj_tol = float(proj_tol)
        o.hop_variant = int(hop_variant)
        o.deflate = int(deflate)
        o.defl_kmax = int(defl_kmax)
        o.defl_nderiv = int(defl_nderiv)
        o.two_pass = int(two_pass)
        o.graph = int(graph)
        o.split = int(split)
        o.nested_m = int(nested_m)
        o.update_variant = int(update_variant)
        o.rebiorth = int(rebiorth)
        return o

    def sign_apply(self, x, k, out=None, **kw):
        """sgn(H(mu)) x by k steps of two-sided Lanczos; returns (y, reports)."""
        x = _as_c128(x)
        nsrc = x.shape[0]
        y = _empty_like(x) if out is None else out
        o = self.opts(k, **kw)
        rep = (Report * nsrc)()
        self._check(self._L.lq_sign_apply(self._h, _ptr(x), _ptr(y), int(nsrc), ctypes.byref(o), rep, _stream(x)))
        return y, [r.as_dict() for r in rep]

    def sign_derivative_apply(self, x, k, kind=LQ_DIR_MU, field=None, out=None, **kw):
        """Eq. (2.6): returns (sgn(H) x, d_t sgn(H) x, reports) along the direction (kind, field).
        out = (y_sign, y_deriv) lets the caller supply the output buffers (host or device)."""
        x = _as_c128(x)
        nsrc = x.shape[0]
        ys, yd = (_empty_like(x), _empty_like(x)) if out is None else out
        d, keep = self._direction(kind, field)
        o = self.opts(k, **kw)
        rep = (Report * nsrc)()
        self._check(self._L.lq_sign_derivative_apply(self._h, ctypes.byref(d), _ptr(x), _ptr(ys), _ptr(yd), int(nsrc),
                                                     ctypes.byref(o), rep, _stream(x)))
        del keep
        return ys, yd, [r.as_dict() for r in rep]

    def overlap_apply(self, x, k, kind=LQ_DIR_MU, field=None, derivative=True, out=None, **kw):
        """Eq. (1.1): returns (D_ov x, d_t D_ov x or None, reports), D_ov = 1 + gamma5 sgn(H(mu)),
        the derivative along the direction (kind, field) when `derivative`."""
        x = _as_c128(x)
        nsrc = x.shape[0]
        y, dy = (_empty_like(x), _empty_like(x) if derivative else None) if out is None else out
        d, keep = self._direction(kind, field) if derivative else (None, None)
        o = self.opts(k, **kw)
        rep = (Report * nsrc)()
        self._check(self._L.lq_overlap_apply(self._h, ctypes.byref(d) if d is not None else None, _ptr(x), _ptr(y),
                                             _ptr(dy), int(nsrc), ctypes.byref(o), rep, _stream(x)))
        del keep
        return y, dy, [r.as_dict() for r in rep]

    def overlap_solve(self, b, k, mass=0.0, tol=1e-10, max_iter=100, **kw):
        """z = D(m)^{-1} b, D(m) = (1 - m/2) D_ov + m (include/lq.h: lq_overlap_solve); returns
        (z, per-source solve reports)."""
        b = _as_c128(b)
        nsrc = b.shape[0]
        z = _empty_like(b)
        o = self.opts(k, **kw)
        rep = (SolveReport * nsrc)()
        self._check(self._L.lq_overlap_solve(self._h, _ptr(b), _ptr(z), int(nsrc), float(mass), float(tol), int(max_iter),
                                             ctypes.byref(o), rep, _stream(b)))
        return z, [r.as_dict() for r in rep]

    def axial_current(self, eta, k, kind=LQ_DIR_U1, field=None, mass=0.0, tol=1e-10, max_iter=100, **kw):
        """Per noise vector eta_s: eta_s^dag D(m)^{-1} dD(m) gamma5 eta_s along the direction (kind,
        field) (include/lq.h: lq_axial_current); returns (complex array [nsrc], solve reports)."""
        eta = _as_c128(eta)
        nsrc = eta.shape[0]
        d, keep = self._direction(kind, field)
        o = self.opts(k, **kw)
        out = np.zeros(2 * nsrc, np.float64)
        rep = (SolveReport * nsrc)()
        self._check(self._L.lq_axial_current(self._h, ctypes.byref(d), _ptr(eta), int(nsrc), float(mass), float(tol),
                                             int(max_iter), ctypes.byref(o), _ptr(out), rep, _stream(eta)))
        del keep
        return out[0::2] + 1j * out[1::2], [r.as_dict() for r in rep]

    def profile_enable(self, enable=True):
        """Reset the kernel-time totals and launch count; enable CUDA-event timing."""
        self._check(self._L.lq_profile_enable(self._h, int(bool(enable))))

    def profile(self):
        p = Profile()
        self._check(self._L.lq_profile_read(self._h, ctypes.byref(p)))
        return p.as_dict()

    def tsl_coefficients(self, src, k):
        """(alpha, beta, delta) of the projected tridiagonal T_k from the last solve."""
        a = np.zeros(k, np.complex128)
        b = np.zeros(k, np.complex128)
        d = np.zeros(k, np.float64)
        self._check(self._L.lq_tsl_coefficients(self._h, int(src), int(k), _ptr(a), _ptr(b), _ptr(d)))
        return a, b[:k - 1], d[:k - 1]

    def upload_deflation(self, lam, R, L):
        """Eigenpairs for the deflation of Sec. 3: lam [l] complex, R [l][V][4][3] right
        eigenvectors, L [l][V][4][3] left eigenvectors as kets (<L_i|R_j> = delta_ij)."""
        lam = np.ascontiguousarray(np.asarray(lam, dtype=np.complex128))
        R, L = _as_c128(R), _as_c128(L)
        self._defl_keep = (lam, R, L)
        self._check(self._L.lq_upload_deflation(self._h, int(lam.shape[0]), _ptr(lam), _ptr(R), _ptr(L), _stream(R)))

    def compute_deflation(self, nev, X0, nsub=0, degree=0, max_iter=0, tol=0.0, method=LQ_EIG_SHIFT_INVERT, inner_max=0):
        """Install the nev eigenpairs of H(mu) closest to zero as the deflation space, from the
        library's eigensolver (method LQ_EIG_SHIFT_INVERT: start fields X0[0] (right) and X0[1]
        (left), basis size nsub; LQ_EIG_CHEBYSHEV: subspace X0 [nsub][V][4][3]); returns
        (lambda [nev], residuals [nev]).  eig_stats() gives the run's statistics."""
        X0 = _as_c128(X0)
        if method == LQ_EIG_CHEBYSHEV and not nsub:
            nsub = X0.shape[0]
        eo = EigOpts(int(nev), int(nsub), int(degree), int(max_iter), float(tol), int(method), int(inner_max))
        lam = np.zeros(nev, np.complex128)
        res = np.zeros(nev, np.float64)
        self._check(self._L.lq_compute_deflation(self._h, ctypes.byref(eo), _ptr(X0), _ptr(lam), _ptr(res), _stream(X0)))
        self._defl_keep = (lam,)
        return lam, res

    def eig_stats(self):
        """Statistics of the last compute_deflation (restarts, solves, inner iterations, seconds ...)."""
        s = EigStats()
        self._check(self._L.lq_eig_stats_read(self._h, ctypes.byref(s)))
        return s.as_dict()

    def deflation_derivatives(self, k, kind=LQ_DIR_MU, field=None, **kw):
        """(dlambda [l], dR [l][V][4][3], dL kets [l][V][4][3]) along the direction (host arrays)."""
        l = self._defl_keep[0].shape[0]
        dlam = np.zeros(l, np.complex128)
        dR = np.zeros((l, self.V, 4, 3), np.complex128)
        dL = np.zeros((l, self.V, 4, 3), np.complex128)
        d, keep = self._direction(kind, field)
        o = self.opts(k, **kw)
        self._check(self._L.lq_deflation_derivatives(self._h, ctypes.byref(d), ctypes.byref(o), _ptr(dlam), _ptr(dR),
                                                     _ptr(dL), _stream(None)))
        return dlam, dR, dL

    def bilinear_grad(self, x, y, k, **kw):
        """(S, force [4][V][8], dS/dmu) for S = Re <y| sgn(H) |x>; x, y single fields [V][4][3]."""
        x, y = _as_c128(x), _as_c128(y)
        S = ctypes.c_double()
        dmu = ctypes.c_double()
        if _is_tensor(x):
            force = torch.empty((4, self.V, 8), dtype=torch.float64, device=x.device)
        else:
            force = np.empty((4, self.V, 8), dtype=np.float64)
        o = self.opts(k, **kw)
        self._check(self._L.lq_sign_bilinear_grad(self._h, _ptr(x), _ptr(y), ctypes.byref(o), ctypes.byref(S), _ptr(force),
                                                  ctypes.byref(dmu), _stream(x)))
        return S.value, force, dmu.value

    def error_estimate(self, x, k, kind=None, field=None, **kw):
        """eps_A of Sec. 4 per source: the sign (kind None) or the derivative version (kind = LQ_DIR_*)."""
        x = _as_c128(x)
        nsrc = x.shape[0]
        eps = np.zeros(nsrc, np.float64)
        o = self.opts(k, **kw)
        if kind is None:
            code = self._L.lq_error_estimate(self._h, None, _ptr(x), int(nsrc), ctypes.byref(o), _ptr(eps), _stream(x))
        else:
            d, keep = self._direction(kind, field)
            code = self._L.lq_error_estimate(self._h, ctypes.byref(d), _ptr(x), int(nsrc), ctypes.byref(o), _ptr(eps),
                                             _stream(x))
        self._check(code)
        return eps

    def nested_sign(self, alpha, beta, delta, m, scale=None):
        """sgn(T) e_1 of tridiagonal T (alpha [nb][k] diagonal, beta [nb][k-1] super, delta
        [nb][k-1] real sub-diagonal) by the nested two-sided Lanczos process (inner size m, scale c
        per matrix or the library's estimate); returns (s [nb][k], involution residual [nb])."""
        alpha, beta = _as_c128(alpha), _as_c128(beta)
        delta = _as_f64(delta)
        nb, k = alpha.shape[0], alpha.shape[1]
        out = _empty_like(alpha)
        chk = np.zeros(nb, np.float64)
        sc = None if scale is None else _as_f64(scale)
        self._check(self._L.lq_nested_sign(self._h, _ptr(alpha), _ptr(beta), _ptr(delta), _ptr(sc), int(k), int(nb), int(m),
                                           _ptr(out), _ptr(chk), _stream(alpha)))
        return out, chk

    def newton_sign(self, X, max_iter=50, tol=1e-13):
        """Batched dense sign of complex k x k matrices X [nb][k][k] (CUDA tensor)."""
        X = _as_c128(X)
        nb, k = X.shape[0], X.shape[1]
        S = _empty_like(X)
        iters = (ctypes.c_int * nb)()
        self._check(self._L.lq_newton_sign(self._h, _ptr(X), _ptr(S), int(k), int(nb), int(max_iter), float(tol),
                                           iters, _stream(X)))
        return S, list(iters)

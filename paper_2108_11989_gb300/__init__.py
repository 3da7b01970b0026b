"""Python binding of libqstar (include/qstar.h): argument marshalling only.

Every function here forwards to the C-ABI entry point of the same name (without
the ``qs_`` prefix); device buffers are torch tensors (their data pointers are
passed through), host inputs are numpy arrays.  There is no fallback: if the
CUDA library is not built or not loadable, importing this package raises.
"""
import ctypes
import os

import numpy as np

from .build import LIB

__all__ = ["QStarError", "Lattice", "create_lattice", "load_gauge", "apply_Dw", "apply_Q",
           "lowmodes_at_mass", "pfaffian_sign", "eig_default_opts", "sign_default_opts",
           "set_profiling", "get_profile", "apply_Q_batch", "MLP",
           "strerror", "QS_F64", "QS_F32", "QS_F16", "QS_BF16", "lib"]

QS_F64, QS_F32, QS_F16, QS_BF16 = 0, 1, 2, 3
QS_LAYOUT_TILED = 16
Q16_BYTES_PER_SITE = 52     # 16-bit storage: 24 16-bit reals + one FP32 scale per site


class QStarError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = _lib.qs_strerror(code).decode()
        cu = _lib.qs_last_cuda_error().decode()
        super().__init__(f"{where}: {msg} ({code})" + (f" [{cu}]" if code == -3 and cu else ""))


class _Geom(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("T", ctypes.c_int), ("cstar_mask", ctypes.c_int),
                ("t_antiperiodic", ctypes.c_int), ("device", ctypes.c_int)]


class BatchItem(ctypes.Structure):
    _fields_ = [("lat", ctypes.c_void_p), ("inp", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("nrhs", ctypes.c_int), ("m0", ctypes.POINTER(ctypes.c_double))]


class EigOpts(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("nwant", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("cheb_degree", ctypes.c_int), ("warm_start", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("precision", ctypes.c_int), ("pairing", ctypes.c_int)]


class EigStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("filter_passes", ctypes.c_int), ("refine_passes", ctypes.c_int),
                ("dslash_f32", ctypes.c_int64), ("dslash_f64", ctypes.c_int64),
                ("cg_iterations", ctypes.c_int64), ("seconds", ctypes.c_double)]


QS_TRACE_MAX = 1024


QS_WINDOW = 24


class SignOpts(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double), ("m0_max", ctypes.c_double), ("max_steps", ctypes.c_int),
                ("eig", EigOpts), ("step_model", ctypes.c_void_p),
                ("window_trace", ctypes.POINTER(ctypes.c_double)), ("retreat", ctypes.c_int),
                ("log_path", ctypes.c_char_p), ("checkpoint_path", ctypes.c_char_p), ("resume", ctypes.c_int)]


class SignReport(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("mass", ctypes.c_double * QS_TRACE_MAX),
                ("lambda_bar", ctypes.c_double * QS_TRACE_MAX), ("resid", ctypes.c_double * QS_TRACE_MAX),
                ("phase", ctypes.c_char * QS_TRACE_MAX), ("crossings", ctypes.c_int),
                ("steps_a", ctypes.c_int), ("steps_b", ctypes.c_int),
                ("dslash_f32", ctypes.c_int64), ("dslash_f64", ctypes.c_int64),
                ("cg_iterations", ctypes.c_int64), ("seconds", ctypes.c_double),
                ("learned_accepted", ctypes.c_int), ("learned_rejected", ctypes.c_int),
                ("fail_reason", ctypes.c_int), ("checkpoint_errors", ctypes.c_int),
                ("resumed_from", ctypes.c_double)]

    def as_dict(self):
        n = min(self.n, QS_TRACE_MAX)
        return {"n": self.n, "mass": list(self.mass[:n]), "lambda_bar": list(self.lambda_bar[:n]),
                "resid": list(self.resid[:n]), "phase": self.phase[:n].decode(),
                "crossings": self.crossings, "steps_a": self.steps_a, "steps_b": self.steps_b,
                "dslash_f32": self.dslash_f32, "dslash_f64": self.dslash_f64,
                "cg_iterations": self.cg_iterations, "seconds": self.seconds,
                "learned_accepted": self.learned_accepted, "learned_rejected": self.learned_rejected,
                "fail_reason": self.fail_reason, "checkpoint_errors": self.checkpoint_errors,
                "resumed_from": self.resumed_from}


class KernelProf(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ms", ctypes.c_double), ("bytes", ctypes.c_double)]


class Profile(ctypes.Structure):
    _fields_ = [("dslash", KernelProf * 4)]


def _load():
    if not os.path.exists(LIB):
        raise ImportError(f"libqstar.so is not built ({LIB}); run __graft_entry__.build() "
                          "or python -m paper_2108_11989_gb300.build")
    lib = ctypes.CDLL(LIB)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "qs_create_lattice": (I, [ctypes.POINTER(_Geom), P, ctypes.POINTER(P)]),
        "qs_destroy_lattice": (I, [P]),
        "qs_n_sites": (ctypes.c_int64, [P]),
        "qs_load_gauge": (I, [P, P, P, D, D]),
        "qs_apply_Dw": (I, [P, D, P, P, I, I]),
        "qs_apply_Q": (I, [P, D, P, P, I, I]),
        "qs_eig_default_opts": (None, [ctypes.POINTER(EigOpts)]),
        "qs_lowmodes_at_mass": (I, [P, D, ctypes.POINTER(EigOpts), P, P, P, ctypes.POINTER(EigStats)]),
        "qs_sign_default_opts": (None, [ctypes.POINTER(SignOpts)]),
        "qs_pfaffian_sign": (I, [P, D, ctypes.POINTER(SignOpts), ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(SignReport)]),
        "qs_pfaffian_sign_batch": (I, [P, I, P, ctypes.POINTER(SignOpts), P, P, P]),
        "qs_set_profiling": (I, [P, I]),
        "qs_get_profile": (I, [P, ctypes.POINTER(Profile)]),
        "qs_kernel_launches": (ctypes.c_int64, []),
        "qs_mlp_create": (I, [I, I, I, I, P, ctypes.POINTER(P)]),
        "qs_mlp_destroy": (I, [P]),
        "qs_mlp_n_params": (ctypes.c_int64, [P]),
        "qs_mlp_set_params": (I, [P, P]),
        "qs_mlp_get_params": (I, [P, P]),
        "qs_mlp_get_grads": (I, [P, P]),
        "qs_mlp_forward": (I, [P, P, I, P]),
        "qs_mlp_train_step": (I, [P, P, P, I, ctypes.c_float, ctypes.POINTER(ctypes.c_float)]),
        "qs_apply_Q_batch": (I, [ctypes.POINTER(BatchItem), I, I, P]),
        "qs_convert_spinors": (I, [P, P, I, P, I, I]),
        "qs_log_det_oo": (I, [P, I, P, P]),
        "qs_cstar_partner": (I, [P, P, P, I, I]),
        "qs_w_eo": (I, [P, D, D, P, P]),
        "qs_apply_Dhat": (I, [P, D, P, P, I, I]),
        "qs_block_bounds": (I, [P, P, I, I, P, P]),
        "qs_ratapprox": (I, [I, D, D, P, P, P, P]),
        "qs_solve_D": (I, [P, D, P, P, I, I, D, I, P]),
        "qs_w_mass": (I, [P, D, D, I, P, P, P, I, D, I, P, P, P]),
        "qs_apply_Q_norm2_noalloc": (I, [P, D, P, P, I, I, P]),
        "qs_strerror": (ctypes.c_char_p, [I]),
        "qs_last_cuda_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    return lib


_lib = _load()
lib = _lib


def _check(code, where):
    if code != 0:
        raise QStarError(code, where)


def strerror(code):
    return _lib.qs_strerror(code).decode()


def _prec_of(t):
    import torch
    if t.dtype == torch.float64:
        return QS_F64
    if t.dtype == torch.float32:
        return QS_F32
    raise TypeError(f"unsupported spinor dtype {t.dtype}")


def _stream_ptr(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def create_lattice(L, T, cstar_mask=0b111, t_antiperiodic=False, device=0, stream=None):
    """qs_create_lattice; returns the opaque handle (ctypes.c_void_p)."""
    g = _Geom(L, T, cstar_mask, int(bool(t_antiperiodic)), device)
    h = ctypes.c_void_p()
    _check(_lib.qs_create_lattice(ctypes.byref(g), _stream_ptr(stream), ctypes.byref(h)), "create_lattice")
    return h


def load_gauge(h, su3, theta, csw_su3, csw_u1):
    """qs_load_gauge from host numpy arrays su3[T,L,L,L,4,3,3] complex128, theta[T,L,L,L,4] or None."""
    su3 = np.ascontiguousarray(su3, dtype=np.complex128)
    th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float64)
    _check(_lib.qs_load_gauge(h, su3.ctypes.data, None if th is None else th.ctypes.data,
                              float(csw_su3), float(csw_u1)), "load_gauge")


def _nrhs(h, t, prec=None):
    ns = _lib.qs_n_sites(h)
    if prec in (QS_F16, QS_BF16):
        nb = t.numel() * t.element_size()
        n = nb // (ns * Q16_BYTES_PER_SITE)
        if n * ns * Q16_BYTES_PER_SITE != nb:
            raise ValueError("16-bit spinor buffer is not a multiple of N_s * 52 bytes")
        return n
    n = t.numel() // (ns * 24)
    if n * ns * 24 != t.numel():
        raise ValueError("spinor size is not a multiple of N_s * 24 reals")
    return n


def _op_prec(t, prec, tiled):
    p = _prec_of(t) if prec is None else prec
    if p in (QS_F16, QS_BF16) and not tiled:
        raise ValueError("16-bit storage exists in the tiled layout only")
    return p


def apply_Dw(h, m0, inp, out, tiled=False, prec=None):
    """qs_apply_Dw on device tensors: float64 or float32 (canonical layout, or the
    site-tiled one with tiled=True), or prec=QS_F16 / QS_BF16 with byte buffers in
    the tiled 16-bit format (see include/qstar.h)."""
    p = _op_prec(inp, prec, tiled)
    _check(_lib.qs_apply_Dw(h, float(m0), inp.data_ptr(), out.data_ptr(), _nrhs(h, inp, p),
                            p | (QS_LAYOUT_TILED if tiled else 0)), "apply_Dw")


def apply_Q(h, m0, inp, out, tiled=False, prec=None):
    p = _op_prec(inp, prec, tiled)
    _check(_lib.qs_apply_Q(h, float(m0), inp.data_ptr(), out.data_ptr(), _nrhs(h, inp, p),
                           p | (QS_LAYOUT_TILED if tiled else 0)), "apply_Q")


def to_tiled(x, n_sites):
    """Canonical [rhs][site][12][2] -> tiled [rhs][site/16][12][site%16][2] (torch, any device)."""
    n = x.numel() // (n_sites * 24)
    return x.reshape(n, n_sites // 16, 16, 12, 2).permute(0, 1, 3, 2, 4).contiguous().reshape(-1)


def from_tiled(x, n_sites):
    n = x.numel() // (n_sites * 24)
    return x.reshape(n, n_sites // 16, 12, 16, 2).permute(0, 1, 3, 2, 4).contiguous().reshape(-1)


def eig_default_opts(**kw):
    o = EigOpts()
    _lib.qs_eig_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def sign_default_opts(eig=None, **kw):
    o = SignOpts()
    _lib.qs_sign_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k in ("log_path", "checkpoint_path") and isinstance(v, (str, os.PathLike)):
            v = os.fsencode(v)
        setattr(o, k, v)
    if eig is not None:
        for k, v in (eig.items() if isinstance(eig, dict) else []):
            setattr(o.eig, k, v)
    return o


def lowmodes_at_mass(h, m0, opts=None, evecs=None, allow_noconv=False):
    """qs_lowmodes_at_mass: returns (evals, resid, stats dict); evecs: optional device tensor."""
    o = opts if opts is not None else eig_default_opts()
    ev = np.zeros(o.k)
    rs = np.zeros(o.k)
    st = EigStats()
    code = _lib.qs_lowmodes_at_mass(h, float(m0), ctypes.byref(o), ev.ctypes.data, rs.ctypes.data,
                                    None if evecs is None else evecs.data_ptr(), ctypes.byref(st))
    if not (code == 0 or (allow_noconv and code == -4)):
        _check(code, "lowmodes_at_mass")
    stats = {f: getattr(st, f) for f, _ in EigStats._fields_}
    stats["status"] = code
    return ev, rs, stats


def pfaffian_sign(h, m0_target, opts=None, step_model=None, trace=False):
    """qs_pfaffian_sign: returns (sign, report dict).  step_model: an MLP (learned
    step); trace=True adds report["windows"] (masses visited x QS_WINDOW)."""
    o = opts if opts is not None else sign_default_opts()
    o.step_model = None if step_model is None else step_model.h
    buf = None
    if trace:
        buf = np.zeros(o.max_steps * QS_WINDOW)
        o.window_trace = buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    else:
        o.window_trace = None
    sg = ctypes.c_int(0)
    rep = SignReport()
    code = _lib.qs_pfaffian_sign(h, float(m0_target), ctypes.byref(o), ctypes.byref(sg), ctypes.byref(rep))
    if code != 0:
        err = QStarError(code, "pfaffian_sign")
        err.report = rep.as_dict()
        raise err
    out = rep.as_dict()
    if trace:
        out["windows"] = buf[:min(rep.n, o.max_steps) * QS_WINDOW].reshape(-1, QS_WINDOW).copy()
    return sg.value, out


def cstar_partner(h, inp, out, tiled=False):
    """qs_cstar_partner: out = C T gamma_5 conj(in) for float64 device spinors."""
    _check(_lib.qs_cstar_partner(h, inp.data_ptr(), out.data_ptr(), _nrhs(h, inp),
                                 QS_F64 | (QS_LAYOUT_TILED if tiled else 0)), "cstar_partner")


def log_det_oo(h, masses):
    """qs_log_det_oo: log|det D^oo(m0)| for each bare mass (numpy array)."""
    m = np.ascontiguousarray(masses, dtype=np.float64)
    out = np.zeros(len(m))
    _check(_lib.qs_log_det_oo(h, len(m), m.ctypes.data, out.ctypes.data), "log_det_oo")
    return out


def block_bounds(theta, res, nwant):
    """qs_block_bounds: (lambda_bar, lo) step A takes from a block of Ritz pairs."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    rs = np.ascontiguousarray(res, dtype=np.float64)
    if th.shape != rs.shape or th.ndim != 1:
        raise ValueError("theta and res must be 1-D arrays of one length")
    lb, lo = ctypes.c_double(), ctypes.c_double()
    _check(_lib.qs_block_bounds(th.ctypes.data, rs.ctypes.data, th.size, int(nwant), ctypes.byref(lb),
                                ctypes.byref(lo)), "block_bounds")
    return lb.value, lo.value


def solve_D(h, m0, b, x, even_odd=True, tol=1e-10, max_iter=20000):
    """qs_solve_D: x = D(m0)^-1 b (float64 device spinors); returns the CG iterations."""
    import torch
    if b.dtype != torch.float64 or x.dtype != torch.float64 or b.shape != x.shape:
        raise TypeError("solve_D takes two float64 spinor tensors of one shape")
    it = ctypes.c_int()
    _check(_lib.qs_solve_D(h, float(m0), b.data_ptr(), x.data_ptr(), _nrhs(h, b), int(bool(even_odd)), float(tol),
                           int(max_iter), ctypes.byref(it)), "solve_D")
    return it.value


def ratapprox(n, ra, rb):
    """qs_ratapprox: (A, nu, mu, delta) of the optimal (n, n) relative approximation of
    y^-1/4 on [ra^2, rb^2] (host computation)."""
    A, d = ctypes.c_double(), ctypes.c_double()
    nu, mu = np.zeros(max(n, 1)), np.zeros(max(n, 1))
    _check(_lib.qs_ratapprox(int(n), float(ra), float(rb), ctypes.byref(A), nu.ctypes.data, mu.ctypes.data,
                             ctypes.byref(d)), "ratapprox")
    return A.value, nu[:n].copy(), mu[:n].copy(), d.value


def w_mass(h, m, mp, nu, mu, eta, tol=1e-10, max_iter=20000):
    """qs_w_mass: (q [n][nsrc], log W_mass estimate, CG iterations); eta a float64 device
    tensor of nsrc spinors."""
    import torch
    if eta.dtype != torch.float64 or not eta.is_cuda or not eta.is_contiguous():
        raise TypeError("eta must be a contiguous float64 CUDA tensor")
    nuv = np.ascontiguousarray(nu, dtype=np.float64)
    muv = np.ascontiguousarray(mu, dtype=np.float64)
    if nuv.shape != muv.shape or nuv.ndim != 1:
        raise ValueError("nu and mu must be 1-D arrays of one length")
    nsrc = _nrhs(h, eta)
    q = np.zeros(nuv.size * nsrc)
    lw, it = ctypes.c_double(), ctypes.c_int()
    _check(_lib.qs_w_mass(h, float(m), float(mp), nuv.size, nuv.ctypes.data, muv.ctypes.data, eta.data_ptr(),
                          nsrc, float(tol), int(max_iter), q.ctypes.data, ctypes.byref(lw), ctypes.byref(it)),
           "w_mass")
    return q.reshape(nuv.size, nsrc), lw.value, it.value


def apply_Dhat(h, m0, inp, out, gamma5=False):
    """qs_apply_Dhat: even-odd preconditioned D_hat (or Q_hat) on float64 device spinors."""
    import torch
    if inp.dtype != torch.float64 or out.dtype != torch.float64 or inp.shape != out.shape:
        raise TypeError("apply_Dhat takes two float64 spinor tensors of one shape")
    _check(_lib.qs_apply_Dhat(h, float(m0), inp.data_ptr(), out.data_ptr(), _nrhs(h, inp), int(bool(gamma5))),
           "apply_Dhat")


def w_eo(h, m, mp):
    """qs_w_eo: (W_eo(m -> m'), log W_eo)."""
    w, lw = ctypes.c_double(0), ctypes.c_double(0)
    _check(_lib.qs_w_eo(h, float(m), float(mp), ctypes.byref(w), ctypes.byref(lw)), "w_eo")
    return w.value, lw.value


def convert_spinors(h, inp, in_prec, out, out_prec, nrhs):
    """qs_convert_spinors: tiled spinors from one precision to another (device buffers)."""
    _check(_lib.qs_convert_spinors(h, inp.data_ptr(), in_prec, out.data_ptr(), out_prec, nrhs), "convert_spinors")


def pfaffian_sign_batch(lattices, m0_targets, opts=None):
    """qs_pfaffian_sign_batch: [(sign, status, report dict)] for several lattices at once."""
    n = len(lattices)
    hs = (ctypes.c_void_p * n)(*[(l.h if hasattr(l, "h") else l).value for l in lattices])
    m = np.ascontiguousarray(m0_targets, dtype=np.float64)
    o = opts if opts is not None else sign_default_opts()
    o.step_model = None
    o.window_trace = None
    signs = np.zeros(n, dtype=np.int32)
    status = np.zeros(n, dtype=np.int32)
    reps = (SignReport * n)()
    code = _lib.qs_pfaffian_sign_batch(hs, n, m.ctypes.data, ctypes.byref(o), signs.ctypes.data,
                                       status.ctypes.data, reps)
    if code not in (0,) and not np.any(status != 0):
        _check(code, "pfaffian_sign_batch")
    return [(int(signs[i]), int(status[i]), reps[i].as_dict()) for i in range(n)]


def apply_Q_norm2_noalloc(h, m0, inp, out, norm2):
    """qs_apply_Q_norm2_noalloc: out = Q in and norm2[r] = |out_r|^2 (device tensors),
    with no device allocation by the library."""
    _check(_lib.qs_apply_Q_norm2_noalloc(h, float(m0), inp.data_ptr(), out.data_ptr(), _nrhs(h, inp),
                                         _prec_of(inp), norm2.data_ptr()), "apply_Q_norm2_noalloc")


def apply_Q_batch(entries, tiled=False, stream=None, prec=None):
    """qs_apply_Q_batch: one launch over [(lattice, in, out, masses), ...]; masses has one
    bare mass per right-hand side of that lattice's in/out tensors (prec as for apply_Q)."""
    n = len(entries)
    arr = (BatchItem * n)()
    keep = []
    common = None
    for i, (lat, inp, out, masses) in enumerate(entries):
        h = lat.h if hasattr(lat, "h") else lat
        m = (ctypes.c_double * len(masses))(*[float(x) for x in masses])
        keep.append(m)
        p = _op_prec(inp, prec, tiled)
        nr = _nrhs(h, inp, p)
        if nr != len(masses):
            raise ValueError("one mass per right-hand side")
        arr[i] = BatchItem(h, inp.data_ptr(), out.data_ptr(), nr, m)
        if common is not None and p != common:
            raise TypeError("all items of a batch share one precision")
        common = p
    _check(_lib.qs_apply_Q_batch(arr, n, common | (QS_LAYOUT_TILED if tiled else 0), _stream_ptr(stream)),
           "apply_Q_batch")


class MLP:
    """Owning wrapper around qs_mlp (the step-proposal network)."""

    def __init__(self, n_in, n_hidden, n_out, max_batch, stream=None):
        self.shape = (n_in, n_hidden, n_out)
        self.h = ctypes.c_void_p()
        _check(_lib.qs_mlp_create(n_in, n_hidden, n_out, max_batch, _stream_ptr(stream), ctypes.byref(self.h)),
               "mlp_create")
        self.n_params = _lib.qs_mlp_n_params(self.h)

    def set_params(self, tensors):
        flat = np.concatenate([np.asarray(t, dtype=np.float32).ravel() for t in tensors])
        assert flat.size == self.n_params
        _check(_lib.qs_mlp_set_params(self.h, flat.ctypes.data), "mlp_set_params")

    def _split(self, flat):
        ni, nh, no = self.shape
        shapes = [(nh, ni), (nh,), (nh, nh), (nh,), (no, nh), (no,)]
        out, o = [], 0
        for sh in shapes:
            n = int(np.prod(sh))
            out.append(flat[o:o + n].reshape(sh))
            o += n
        return out

    def get_params(self):
        flat = np.empty(self.n_params, dtype=np.float32)
        _check(_lib.qs_mlp_get_params(self.h, flat.ctypes.data), "mlp_get_params")
        return self._split(flat)

    def get_grads(self):
        flat = np.empty(self.n_params, dtype=np.float32)
        _check(_lib.qs_mlp_get_grads(self.h, flat.ctypes.data), "mlp_get_grads")
        return self._split(flat)

    def _rows(self, t, width, name):
        import torch
        if t.dtype != torch.float32 or t.dim() != 2 or t.shape[1] != width or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float32 tensor [B][{width}], got "
                             f"{t.dtype} {tuple(t.shape)}")
        return t.shape[0]

    def forward(self, X):
        """X: float32 device tensor [B][in] -> device tensor [B][out]."""
        import torch
        self._rows(X, self.shape[0], "X")
        Y = torch.empty((X.shape[0], self.shape[2]), dtype=torch.float32, device=X.device)
        _check(_lib.qs_mlp_forward(self.h, X.data_ptr(), X.shape[0], Y.data_ptr()), "mlp_forward")
        return Y

    def train_step(self, X, T, lr):
        """One Adam step on X [B][in], T [B][out] (float32 device tensors)."""
        b = self._rows(X, self.shape[0], "X")
        if self._rows(T, self.shape[2], "T") != b:
            raise ValueError("X and T must have the same number of rows")
        loss = ctypes.c_float(0)
        _check(_lib.qs_mlp_train_step(self.h, X.data_ptr(), T.data_ptr(), X.shape[0], float(lr),
                                      ctypes.byref(loss)), "mlp_train_step")
        return loss.value

    def close(self):
        if self.h is not None:
            _lib.qs_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_launches():
    """qs_kernel_launches: kernels launched by the library so far in this process."""
    return _lib.qs_kernel_launches()


def set_profiling(h, on):
    _check(_lib.qs_set_profiling(h, int(bool(on))), "set_profiling")


def get_profile(h):
    """{"f64": {...}, "f32": {...}, "f16": {...}, "bf16": {...}} with launches, ms and
    algorithmic bytes of the operator kernels, by spinor precision."""
    p = Profile()
    _check(_lib.qs_get_profile(h, ctypes.byref(p)), "get_profile")
    out = {}
    for name, i in (("f64", QS_F64), ("f32", QS_F32), ("f16", QS_F16), ("bf16", QS_BF16)):
        k = p.dslash[i]
        out[name] = {"launches": k.launches, "ms": k.ms, "bytes": k.bytes}
    return out


class Lattice:
    """Owning wrapper around a qs_lattice handle."""

    def __init__(self, L, T, cstar_mask=0b111, t_antiperiodic=False, device=0, stream=None):
        self.L, self.T = L, T
        self.h = create_lattice(L, T, cstar_mask, t_antiperiodic, device, stream)
        self.n_sites = _lib.qs_n_sites(self.h)

    def load_gauge(self, su3, theta, csw_su3, csw_u1):
        load_gauge(self.h, su3, theta, csw_su3, csw_u1)

    def apply_Dw(self, m0, inp, out, tiled=False, prec=None):
        apply_Dw(self.h, m0, inp, out, tiled, prec)

    def apply_Q(self, m0, inp, out, tiled=False, prec=None):
        apply_Q(self.h, m0, inp, out, tiled, prec)

    def apply_Dhat(self, m0, inp, out, gamma5=False):
        apply_Dhat(self.h, m0, inp, out, gamma5)

    def solve_D(self, m0, b, x, even_odd=True, tol=1e-10, max_iter=20000):
        return solve_D(self.h, m0, b, x, even_odd, tol, max_iter)

    def w_mass(self, m, mp, nu, mu, eta, tol=1e-10, max_iter=20000):
        return w_mass(self.h, m, mp, nu, mu, eta, tol, max_iter)

    def lowmodes_at_mass(self, m0, opts=None, evecs=None, allow_noconv=False):
        return lowmodes_at_mass(self.h, m0, opts, evecs, allow_noconv)

    def pfaffian_sign(self, m0_target, opts=None, step_model=None, trace=False):
        return pfaffian_sign(self.h, m0_target, opts, step_model, trace)

    def set_profiling(self, on):
        set_profiling(self.h, on)

    def get_profile(self):
        return get_profile(self.h)

    def close(self):
        if self.h is not None:
            _lib.qs_destroy_lattice(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

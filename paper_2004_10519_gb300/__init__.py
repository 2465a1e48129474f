"""waveprop: TTI, elastic (3D and 2D) and isotropic acoustic wave propagators on one GB300 (sm_103a).

Thin ctypes binding of ``libwaveprop.so`` (C ABI in ``include/waveprop.h``).
Every step of the propagators runs in the library's CUDA kernels; this module
only marshals arguments.  PyTorch is used for device memory and streams when
tensors are passed.  If the library is missing the import of ``lib()`` fails
loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwaveprop.so")

PROP_OK, PROP_EINVAL, PROP_ENOMEM, PROP_ECUDA, PROP_EUNSTABLE, PROP_ETIMEOUT, PROP_ESTATE = \
    0, -1, -2, -3, -4, -5, -6
PROP_TTI, PROP_ELASTIC, PROP_ACOUSTIC, PROP_ELASTIC2D = 1, 2, 3, 4
SNAP_FULL_FP32, SNAP_CKPT_FP32, SNAP_CKPT_BF16, SNAP_CKPT_FP16 = 0, 1, 2, 3
ERR_NAMES = {0: "PROP_OK", -1: "PROP_EINVAL", -2: "PROP_ENOMEM", -3: "PROP_ECUDA",
             -4: "PROP_EUNSTABLE", -5: "PROP_ETIMEOUT", -6: "PROP_ESTATE"}

# exported symbols declared in include/waveprop.h
ABI_SYMBOLS = ("prop_create", "prop_forward", "prop_adjoint", "prop_gradient",
               "prop_forward_saved", "prop_backward", "prop_grid_dims", "prop_set_state",
               "prop_get_state", "prop_step", "prop_dt", "prop_destroy",
               "prop_last_error", "prop_forward_noalloc", "prop_tile_planes", "prop_tile_rows",
               "prop_gradient_batch", "prop_gradient_bytes", "prop_plan_waves",
               "prop_gradient_aniso", "prop_stack_image", "prop_trim", "prop_forward_batch")
# measurement and self-test hooks declared in include/waveprop_diag.h
DIAG_SYMBOLS = ("prop_profile", "prop_kernel_stats", "prop_kernel_time", "prop_last_launches",
                "prop_batch_stats", "prop_fp32_peak", "prop_selftest_wait")


class PropDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("nbl", C.c_int), ("h", C.c_float), ("space_order", C.c_int), ("nt", C.c_int),
                ("dt", C.c_float), ("vdamp", C.c_float), ("snap_mode", C.c_int),
                ("ckpt_interval", C.c_int), ("check_nan", C.c_int), ("tti_operator", C.c_int)]


class PropError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load libwaveprop.so (built by ``__graft_entry__.build()``).  With
    WAVEPROP_CHECK=1 in the environment, the bounds-checking build
    libwaveprop_check.so instead (compiled on first use)."""
    global _lib
    if _lib is None:
        path = LIB_PATH
        if os.environ.get("WAVEPROP_CHECK") == "1":
            from . import _build
            path = _build.build(check=True)
        if not os.path.exists(path):
            raise RuntimeError(f"waveprop CUDA library not built ({path} missing); "
                               "run __graft_entry__.build() -- there is no CPU fallback")
        L = C.CDLL(path)
        vp = C.c_void_p
        fpp = C.POINTER(C.c_void_p)
        L.prop_create.argtypes = [C.POINTER(PropDesc), fpp, vp, C.POINTER(vp)]
        L.prop_forward.argtypes = [vp, vp, vp, C.c_int, vp, C.c_int, vp]
        L.prop_forward_saved.argtypes = [vp, vp, vp, C.c_int, vp, C.c_int, vp]
        L.prop_adjoint.argtypes = [vp, vp, vp, C.c_int, vp, C.c_int, vp]
        L.prop_gradient.argtypes = [vp, vp, vp, C.c_int, vp, C.c_int, vp, vp, C.POINTER(C.c_double)]
        L.prop_backward.argtypes = [vp, vp, vp, vp]
        L.prop_gradient_aniso.argtypes = [vp, vp, vp, C.c_int, vp, C.c_int, vp, vp, C.POINTER(C.c_double)]
        L.prop_grid_dims.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.prop_set_state.argtypes = [vp, fpp]
        L.prop_get_state.argtypes = [vp, fpp]
        L.prop_step.argtypes = [vp, C.c_int, C.c_int]
        L.prop_dt.restype = C.c_float
        L.prop_dt.argtypes = [vp]
        L.prop_kernel_time.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
        L.prop_tile_planes.argtypes = [vp]
        L.prop_tile_rows.argtypes = [vp]
        L.prop_gradient_batch.argtypes = [fpp, C.c_int, fpp, fpp, C.POINTER(C.c_int), fpp,
                                          C.POINTER(C.c_int), fpp, fpp, C.POINTER(C.c_double),
                                          C.c_size_t]
        L.prop_forward_batch.argtypes = [fpp, C.c_int, fpp, fpp, C.POINTER(C.c_int), fpp,
                                         C.POINTER(C.c_int), fpp]
        L.prop_gradient_bytes.restype = C.c_size_t
        L.prop_gradient_bytes.argtypes = [vp, C.c_int]
        L.prop_plan_waves.argtypes = [C.POINTER(C.c_size_t), C.c_int, C.c_size_t, C.POINTER(C.c_int)]
        L.prop_stack_image.argtypes = [vp, vp, vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_float]
        L.prop_trim.argtypes = [vp]
        L.prop_selftest_wait.argtypes = [vp, C.c_float]
        L.prop_destroy.argtypes = [vp]
        L.prop_last_error.restype = C.c_char_p
        L.prop_last_error.argtypes = [vp]
        L.prop_profile.argtypes = [vp, C.c_int]
        L.prop_kernel_stats.argtypes = [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
        L.prop_fp32_peak.argtypes = [C.POINTER(C.c_double)]
        L.prop_batch_stats.argtypes = [C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
        L.prop_last_launches.restype = C.c_longlong
        L.prop_last_launches.argtypes = [vp]
        _lib = L
    return _lib


def _is_torch(x):
    return type(x).__module__.startswith("torch")


class _Arg:
    """Pointer to a caller buffer: numpy (host) or torch (host/device), float32
    contiguous.  Keeps the converted object alive."""

    def __init__(self, x, n=None, writable=False):
        if _is_torch(x):
            import torch
            if x.dtype != torch.float32 or not x.is_contiguous():
                if writable:
                    raise ValueError("output tensor must be contiguous float32")
                x = x.contiguous().to(torch.float32)
            self.obj = x
            self.ptr = C.c_void_p(x.data_ptr())
            size = x.numel()
        else:
            a = np.asarray(x)
            if a.dtype != np.float32 or not a.flags.c_contiguous:
                if writable:
                    raise ValueError("output array must be C-contiguous float32")
                a = np.ascontiguousarray(a, dtype=np.float32)
            self.obj = a
            self.ptr = C.c_void_p(a.ctypes.data)
            size = a.size
        if n is not None and size < n:
            raise ValueError(f"buffer has {size} elements, need {n}")


def _npts(a):
    n = a.obj.numel() if _is_torch(a.obj) else a.obj.size
    if n % 3:
        raise ValueError("coordinates must be [n][3]")
    return n // 3


def _stream_of(*xs):
    for x in xs:
        if _is_torch(x) and x.is_cuda:
            import torch
            return C.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
    return C.c_void_p(0)


class Propagator:
    """Handle on one propagator (``prop_t``).

    kind: PROP_TTI, PROP_ELASTIC, PROP_ACOUSTIC or PROP_ELASTIC2D (x-z plane,
    shape (nx, 1, nz)); model: list of physical-grid float32 arrays (TTI: vp,
    eps, delta, theta, phi; elastic and 2D elastic: vp, vs, rho; acoustic:
    vp) as numpy arrays or torch tensors (host or device)."""

    def __init__(self, kind, shape, nbl, h, space_order, nt, model, dt=0.0, vdamp=0.0,
                 snap_mode=SNAP_FULL_FP32, ckpt_interval=0, check_nan=0, stream=None, tti_operator=0):
        L = lib()
        nx, ny, nz = shape
        self.desc = PropDesc(kind, nx, ny, nz, nbl, float(h), space_order, nt, float(dt),
                             float(vdamp), snap_mode, ckpt_interval, check_nan, tti_operator)
        args = [_Arg(m, nx * ny * nz) for m in model]
        arr = (C.c_void_p * len(args))(*[a.ptr for a in args])
        if stream is None:
            stream = _stream_of(*model)
        elif not isinstance(stream, C.c_void_p):
            stream = C.c_void_p(int(stream))
        self.stream = stream
        h_ = C.c_void_p()
        rc = L.prop_create(C.byref(self.desc), arr, stream, C.byref(h_))
        if rc:
            raise PropError(rc, L.prop_last_error(None).decode())
        self.h = h_
        self.kind, self.nt = kind, nt
        self.shape = (nx, ny, nz)
        d = (C.c_int * 3)()
        nf = C.c_int()
        L.prop_grid_dims(self.h, d, C.byref(nf))
        self.grid = (d[0], d[1], d[2])
        self.nfields = nf.value

    @classmethod
    def from_problem(cls, prob, model=None, **kw):
        keys = {PROP_TTI: ("vp", "eps", "delta", "theta", "phi"), PROP_ELASTIC: ("vp", "vs", "rho"),
                PROP_ACOUSTIC: ("vp",), PROP_ELASTIC2D: ("vp", "vs", "rho")}[prob.kind]
        ml = model if model is not None else [prob.model[k] for k in keys]
        kw.setdefault("dt", prob.dt)
        kw.setdefault("vdamp", getattr(prob, "vdamp", 0.0) or 0.0)
        kw.setdefault("tti_operator", getattr(prob, "tti_op", 0) or 0)
        return cls(prob.kind, (prob.nx, prob.ny, prob.nz), prob.nbl, prob.h, prob.so, prob.nt, ml, **kw)

    def close(self):
        if getattr(self, "h", None):
            lib().prop_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc:
            raise PropError(rc, lib().prop_last_error(self.h).decode())

    @property
    def dt(self):
        return lib().prop_dt(self.h)

    @property
    def tile_planes(self):
        """x-planes per CTA chosen by the autotuner at creation."""
        return lib().prop_tile_planes(self.h)

    @property
    def tile_rows(self):
        """y-rows per tile (8, 16 or 32) chosen by the autotuner at creation."""
        return lib().prop_tile_rows(self.h)

    def _out(self, like, shape):
        if _is_torch(like):
            import torch
            return torch.empty(shape, dtype=torch.float32, device=like.device)
        return np.empty(shape, np.float32)

    def forward(self, wavelet, src, rec, out=None, save=False):
        src_a, rec_a = _Arg(src), _Arg(rec)
        nsrc, nrec = _npts(src_a), _npts(rec_a)
        w = _Arg(wavelet, nsrc * self.nt)
        if out is None:
            out = self._out(wavelet, (nrec, self.nt))
        o = _Arg(out, nrec * self.nt, writable=True)
        f = lib().prop_forward_saved if save else lib().prop_forward
        self._check(f(self.h, w.ptr, src_a.ptr, nsrc, rec_a.ptr, nrec, o.ptr))
        return out

    def adjoint(self, traces, src, rec, out=None):
        src_a, rec_a = _Arg(src), _Arg(rec)
        nsrc, nrec = _npts(src_a), _npts(rec_a)
        t = _Arg(traces, nrec * self.nt)
        if out is None:
            out = self._out(traces, (nsrc, self.nt))
        o = _Arg(out, nsrc * self.nt, writable=True)
        self._check(lib().prop_adjoint(self.h, t.ptr, rec_a.ptr, nrec, src_a.ptr, nsrc, o.ptr))
        return out

    def _gshape(self):
        nx, ny, nz = self.shape
        return (3, nx, ny, nz) if self.kind == PROP_ELASTIC else (nx, ny, nz)

    def gradient(self, wavelet, src, rec, d_obs, out=None):
        src_a, rec_a = _Arg(src), _Arg(rec)
        nsrc, nrec = _npts(src_a), _npts(rec_a)
        w = _Arg(wavelet, nsrc * self.nt)
        d = _Arg(d_obs, nrec * self.nt)
        if out is None:
            out = self._out(d_obs, self._gshape())
        o = _Arg(out, int(np.prod(self._gshape())), writable=True)
        J = C.c_double()
        self._check(lib().prop_gradient(self.h, w.ptr, src_a.ptr, nsrc, rec_a.ptr, nrec, d.ptr,
                                        o.ptr, C.byref(J)))
        return out, J.value

    def gradient_aniso(self, wavelet, src, rec, d_obs, out=None):
        """TTI: gradient w.r.t. (m, epsilon, delta, theta, phi), shape
        [5][nx][ny][nz], and the misfit (``prop_gradient_aniso``)."""
        src_a, rec_a = _Arg(src), _Arg(rec)
        nsrc, nrec = _npts(src_a), _npts(rec_a)
        w = _Arg(wavelet, nsrc * self.nt)
        d = _Arg(d_obs, nrec * self.nt)
        shape = (5,) + self.shape
        if out is None:
            out = self._out(d_obs, shape)
        o = _Arg(out, int(np.prod(shape)), writable=True)
        J = C.c_double()
        self._check(lib().prop_gradient_aniso(self.h, w.ptr, src_a.ptr, nsrc, rec_a.ptr, nrec, d.ptr,
                                              o.ptr, C.byref(J)))
        return out, J.value

    def selftest_wait(self, seconds=0.2):
        """Failure-path self-test (``prop_selftest_wait``,
        include/waveprop_diag.h): a device wait that nothing completes;
        raises PropError PROP_ETIMEOUT after ``seconds``."""
        self._check(lib().prop_selftest_wait(self.h, float(seconds)))

    def trim(self):
        """Release the work arrays and keep the model (``prop_trim``)."""
        self._check(lib().prop_trim(self.h))

    def stack_image(self, image, stack, offset, weight=1.0):
        """Add ``weight * image`` (this handle's physical grid) into the device
        array ``stack`` with the window's first point at ``offset``
        (``prop_stack_image``)."""
        im = _Arg(image, int(np.prod(self.shape)))
        st = _Arg(stack, writable=True)
        dims = (C.c_int * 3)(*[int(v) for v in stack.shape])
        off = (C.c_int * 3)(*[int(v) for v in offset])
        self._check(lib().prop_stack_image(self.h, im.ptr, st.ptr, dims, off, float(weight)))
        return stack

    def backward(self, resid, grad_out=True, src_grad_out=True, nsrc=None):
        r = _Arg(resid)
        g = self._out(resid, self._gshape()) if grad_out is True else grad_out
        sg = None
        if src_grad_out is True:
            sg = self._out(resid, (nsrc, self.nt))
        elif src_grad_out is not None and src_grad_out is not False:
            sg = src_grad_out
        ga = _Arg(g, writable=True) if g is not None and g is not False else None
        sa = _Arg(sg, writable=True) if sg is not None else None
        self._check(lib().prop_backward(self.h, r.ptr, ga.ptr if ga else None,
                                        sa.ptr if sa else None))
        return (g if ga else None), (sg if sa else None)

    # ---- state -----------------------------------------------------------
    def set_state(self, fields):
        args = [_Arg(f, int(np.prod(self.grid))) for f in fields]
        arr = (C.c_void_p * len(args))(*[a.ptr for a in args])
        self._check(lib().prop_set_state(self.h, arr))

    def get_state(self, like=None):
        outs = [self._out(like if like is not None else np.zeros(1), self.grid)
                for _ in range(self.nfields)]
        args = [_Arg(o, writable=True) for o in outs]
        arr = (C.c_void_p * len(args))(*[a.ptr for a in args])
        self._check(lib().prop_get_state(self.h, arr))
        return outs

    def step(self, nsteps=1, adjoint=False):
        self._check(lib().prop_step(self.h, nsteps, int(adjoint)))

    # ---- measurement -------------------------------------------------------
    def profile(self, on=True):
        self._check(lib().prop_profile(self.h, int(on)))

    def kernel_stats(self, kid):
        ms = C.c_double()
        n = C.c_longlong()
        self._check(lib().prop_kernel_stats(self.h, kid, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def last_launches(self):
        return lib().prop_last_launches(self.h)

    def gradient_bytes(self, nrec):
        """Device bytes a gradient call with nrec receivers would allocate."""
        return lib().prop_gradient_bytes(self.h, int(nrec))


# kernel groups of Propagator.kernel_stats (PROP_K_* of include/waveprop_diag.h)
K_TTI_FWD, K_TTI_ADJ, K_EL_FWD, K_EL_ADJ, K_EL_ADJ_GRAD, K_EL_ADJ_U, K_AC_STEP, K_AC_IMG = 0, 1, 2, 3, 4, 5, 6, 7


def fp32_peak():
    """Measured FP32 FMA throughput of the current device [TFLOP/s]."""
    t = C.c_double()
    rc = lib().prop_fp32_peak(C.byref(t))
    if rc:
        raise PropError(rc, "prop_fp32_peak")
    return t.value


def plan_waves(nbytes, budget):
    """Wave index of each shot under ``prop_plan_waves`` (first fit in order)."""
    n = len(nbytes)
    b = (C.c_size_t * max(n, 1))(*[int(x) for x in nbytes])
    w = (C.c_int * max(n, 1))()
    rc = lib().prop_plan_waves(b, n, int(budget), w)
    if rc < 0:
        raise PropError(rc, "prop_plan_waves")
    return [w[i] for i in range(n)], rc


def gradient_batch(props, wavelets, srcs, recs, d_obs, outs=None, budget_bytes=0):
    """Gradients of independent shots (``prop_gradient_batch``); shot i uses
    ``props[i]`` and the i-th entry of every list.  Returns (grads, misfits)."""
    n = len(props)
    keep, W, S, R, D, G = [], [], [], [], [], []
    ns, nr = (C.c_int * max(n, 1))(), (C.c_int * max(n, 1))()
    grads = []
    for i, p in enumerate(props):
        sa, ra = _Arg(srcs[i]), _Arg(recs[i])
        ns[i], nr[i] = _npts(sa), _npts(ra)
        w = _Arg(wavelets[i], ns[i] * p.nt)
        d = _Arg(d_obs[i], nr[i] * p.nt)
        out = outs[i] if outs is not None else p._out(d_obs[i], p._gshape())
        o = _Arg(out, int(np.prod(p._gshape())), writable=True)
        grads.append(out)
        keep += [sa, ra, w, d, o]
        W.append(w.ptr); S.append(sa.ptr); R.append(ra.ptr); D.append(d.ptr); G.append(o.ptr)
    arr = lambda xs: (C.c_void_p * max(n, 1))(*xs)
    J = (C.c_double * max(n, 1))()
    rc = lib().prop_gradient_batch(arr([p.h for p in props]), n, arr(W), arr(S), ns, arr(R), nr,
                                   arr(D), arr(G), J, int(budget_bytes))
    if rc:
        raise PropError(rc, lib().prop_last_error(None).decode())
    return grads, [J[i] for i in range(n)]


def forward_batch(props, wavelets, srcs, recs, outs=None):
    """Forward modelling of independent shots in lockstep
    (``prop_forward_batch``); shot i uses ``props[i]`` and the i-th entry
    of every list.  Returns the list of traces [nrec_i][nt]."""
    n = len(props)
    keep, W, S, R, T = [], [], [], [], []
    ns, nr = (C.c_int * max(n, 1))(), (C.c_int * max(n, 1))()
    trs = []
    for i, p in enumerate(props):
        sa, ra = _Arg(srcs[i]), _Arg(recs[i])
        ns[i], nr[i] = _npts(sa), _npts(ra)
        w = _Arg(wavelets[i], ns[i] * p.nt)
        out = outs[i] if outs is not None else p._out(wavelets[i], (nr[i], p.nt))
        o = _Arg(out, nr[i] * p.nt, writable=True)
        trs.append(out)
        keep += [sa, ra, w, o]
        W.append(w.ptr); S.append(sa.ptr); R.append(ra.ptr); T.append(o.ptr)
    arr = lambda xs: (C.c_void_p * max(n, 1))(*xs)
    rc = lib().prop_forward_batch(arr([p.h for p in props]), n, arr(W), arr(S), ns, arr(R), nr, arr(T))
    if rc:
        raise PropError(rc, lib().prop_last_error(None).decode())
    return trs


def batch_stats():
    """Rounds of TTI steps of the last ``gradient_batch`` call that shared one
    launch per pass across the shots of a wave, and rounds launched shot by
    shot (measurement hook ``prop_batch_stats``, not in the public header)."""
    a, b = C.c_longlong(), C.c_longlong()
    lib().prop_batch_stats(C.byref(a), C.byref(b))
    return a.value, b.value

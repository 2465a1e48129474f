"""FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline
leg may import this package.  It wraps ``oracle.c`` (plain C, double
precision, OpenMP over independent lines) through ctypes.  It shares no code
with the CUDA library; the only thing both sides use is the seeded input
generator module ``synth``.

``build()`` compiles ``liboracle.so`` next to this file with gcc.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (FP64, no fast-math,
    no FMA contraction so that x86 and Arm hosts round alike)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class _Desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("nbl", C.c_int), ("so", C.c_int), ("nt", C.c_int),
                ("h", C.c_double), ("dt", C.c_double), ("vdamp", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            P = C.c_void_p
            dp = C.POINTER(C.c_double)
            fp = C.POINTER(C.c_float)
            lp = C.POINTER(C.c_long)
            L.or_create.restype = P
            L.or_create.argtypes = [C.POINTER(_Desc), C.POINTER(fp)]
            L.or_destroy.argtypes = [P]
            L.or_npoints.restype = C.c_long
            L.or_npoints.argtypes = [P]
            L.or_dims.argtypes = [P, C.POINTER(C.c_int)]
            L.or_param.restype = dp
            L.or_param.argtypes = [P, C.c_int]
            for f in ("or_tti_forward", "or_el_forward", "or_ac_forward"):
                getattr(L, f).argtypes = [P, C.c_int, fp, fp, C.c_int, fp, dp, C.c_int]
            for f in ("or_tti_adjoint", "or_el_adjoint", "or_ac_adjoint"):
                getattr(L, f).argtypes = [P, C.c_int, fp, dp, C.c_int, fp, dp]
            for f in ("or_tti_gradient", "or_el_gradient", "or_ac_gradient"):
                getattr(L, f).argtypes = [P, C.c_int, fp, fp, C.c_int, fp, dp, dp, dp, dp]
            L.or_tti_backward.argtypes = [P, C.c_int, fp, fp, C.c_int, fp, dp, dp, dp]
            L.or_ac_backward.argtypes = [P, C.c_int, fp, fp, C.c_int, fp, dp, dp, dp]
            L.or_ac_step_state_d.argtypes = [P, dp, dp, C.c_int]
            L.or_ac_step_points.argtypes = [C.POINTER(_Desc), fp, fp, fp, C.c_int, lp, dp]
            L.or_weights_d2.argtypes = [C.c_int, dp]
            L.or_tti_set_operator.argtypes = [P, C.c_int]
            L.or_el2_forward.argtypes = [P, C.c_int, fp, fp, C.c_int, fp, dp]
            L.or_el2_adjoint.argtypes = [P, C.c_int, fp, dp, C.c_int, fp, dp]
            L.or_el2_step_state_d.argtypes = [P, dp, C.c_int, C.c_int]
            L.or_tti_gradient_aniso.argtypes = [P, C.c_int, fp, fp, C.c_int, fp, dp, dp, dp, dp]
            L.or_tti_apply_L.argtypes = [P, dp, dp, dp, dp]
            L.or_tti_step_state.argtypes = [P, fp, fp, fp, fp, dp, dp, C.c_int]
            L.or_tti_step_state_d.argtypes = [P, dp, dp, dp, dp, C.c_int]
            L.or_el_step_state.argtypes = [P, fp, dp, C.c_int, C.c_int]
            L.or_el_step_state_d.argtypes = [P, dp, C.c_int, C.c_int]
            L.or_tti_step_points.argtypes = [C.POINTER(_Desc), C.POINTER(fp), fp, fp, fp, fp,
                                             C.c_int, lp, dp, C.c_int]
            L.or_tti_step_points_op.argtypes = [C.POINTER(_Desc), C.POINTER(fp), fp, fp, fp, fp,
                                                C.c_int, lp, dp, C.c_int, C.c_int]
            L.or_el_step_points.argtypes = [C.POINTER(_Desc), C.POINTER(fp), C.POINTER(fp),
                                            C.c_int, lp, dp]
            L.or_weights_centred.argtypes = [C.c_int, dp]
            L.or_weights_staggered.argtypes = [C.c_int, dp]
            L.or_fornberg.argtypes = [C.c_int, C.c_double, dp, C.c_int, dp]
            L.or_line_op.argtypes = [C.c_int, C.c_int, C.c_double, dp, dp, C.c_int]
            L.or_sparse_weights.argtypes = [P, fp, lp, dp]
            L.or_fold_grad.argtypes = [P, dp, dp]
            L.or_tti_sigma_at.restype = C.c_double
            L.or_tti_sigma_at.argtypes = [P, C.c_long]
            L.or_cerjan_at.restype = C.c_double
            L.or_cerjan_at.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int]
            _lib = L
    return _lib


def _f(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _lp(a):
    return a.ctypes.data_as(C.POINTER(C.c_long))


# ---------------------------------------------------------------------------
def weights_centred(so):
    w = np.zeros(so // 2)
    if lib().or_weights_centred(so, _dp(w)):
        raise ValueError(so)
    return w


def weights_staggered(so):
    w = np.zeros(so // 2)
    if lib().or_weights_staggered(so, _dp(w)):
        raise ValueError(so)
    return w


def fornberg(order, z, x):
    x = _d(x)
    w = np.zeros(x.size)
    if lib().or_fornberg(order, float(z), _dp(x), x.size, _dp(w)):
        raise ValueError((order, z))
    return w


LINE_OPS = {"D": 0, "DT": 1, "Dp": 2, "Dm": 3, "DpT": 4, "DmT": 5}


def line_op(name, so, h, f):
    f = _d(f)
    out = np.zeros_like(f)
    if lib().or_line_op(LINE_OPS[name], so, float(h), _dp(f), _dp(out), f.size):
        raise ValueError(name)
    return out


def desc_of(prob, nt=None, dt=None):
    return _Desc(prob.kind, prob.nx, prob.ny, prob.nz, prob.nbl, prob.so,
                 prob.nt if nt is None else nt, float(prob.h),
                 float(prob.dt if dt is None else dt),
                 float(getattr(prob, "vdamp", 0.0) or 0.0))


class Problem:
    """Oracle instance for one synthetic problem (``synth.Problem``)."""

    def __init__(self, prob, model=None):
        self.prob = prob
        self.desc = desc_of(prob)
        ml = prob.model_list() if model is None else [_f(a) for a in model]
        self._keep = ml
        arr = (C.POINTER(C.c_float) * len(ml))(*[_fp(a) for a in ml])
        self.h = lib().or_create(C.byref(self.desc), arr)
        if not self.h:
            raise ValueError("oracle: invalid problem")
        if getattr(prob, "tti_op", 0):
            lib().or_tti_set_operator(self.h, int(prob.tti_op))
        d = (C.c_int * 3)()
        lib().or_dims(self.h, d)
        self.shape = (d[0], d[1], d[2])
        self.N = lib().or_npoints(self.h)

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().or_destroy(self.h)
                self.h = None
        except Exception:
            pass

    @property
    def nt(self):
        return self.desc.nt

    def param(self, which):
        ptr = lib().or_param(self.h, which)
        if not ptr:
            raise ValueError(which)
        return np.ctypeslib.as_array(ptr, shape=(self.N,)).reshape(self.shape).copy()

    def _geom(self, src, rec, wav):
        p = self.prob
        src = _f(p.src if src is None else src)
        rec = _f(p.rec if rec is None else rec)
        wav = _f(p.wavelet if wav is None else wav)
        return src, rec, wav

    def forward(self, wavelet=None, src=None, rec=None, store=False):
        src, rec, wav = self._geom(src, rec, wavelet)
        tr = np.zeros((rec.shape[0], self.nt))
        if self.prob.kind == 4:
            rc = lib().or_el2_forward(self.h, src.shape[0], _fp(src), _fp(wav), rec.shape[0], _fp(rec), _dp(tr))
        else:
            f = {1: lib().or_tti_forward, 2: lib().or_el_forward, 3: lib().or_ac_forward}[self.prob.kind]
            rc = f(self.h, src.shape[0], _fp(src), _fp(wav), rec.shape[0], _fp(rec), _dp(tr), int(store))
        if rc:
            raise ValueError(f"oracle forward rc={rc}")
        return tr

    def adjoint(self, traces, src=None, rec=None):
        src, rec, _ = self._geom(src, rec, None)
        traces = _d(traces)
        q = np.zeros((src.shape[0], self.nt))
        f = {1: lib().or_tti_adjoint, 2: lib().or_el_adjoint, 3: lib().or_ac_adjoint,
             4: lib().or_el2_adjoint}[self.prob.kind]
        rc = f(self.h, rec.shape[0], _fp(rec), _dp(traces), src.shape[0], _fp(src), _dp(q))
        if rc:
            raise ValueError(f"oracle adjoint rc={rc}")
        return q

    def gradient(self, d_obs, wavelet=None, src=None, rec=None, comp=False):
        src, rec, wav = self._geom(src, rec, wavelet)
        d_obs = _d(d_obs)
        p = self.prob
        nf = 3 if p.kind == 2 else 1
        g = np.zeros((nf, p.nx, p.ny, p.nz))
        gc = np.zeros((nf,) + self.shape) if comp else None
        J = C.c_double(0.0)
        f = {1: lib().or_tti_gradient, 2: lib().or_el_gradient, 3: lib().or_ac_gradient}[p.kind]
        rc = f(self.h, src.shape[0], _fp(src), _fp(wav), rec.shape[0], _fp(rec), _dp(d_obs),
               _dp(g), C.byref(J), _dp(gc) if comp else None)
        if rc:
            raise ValueError(f"oracle gradient rc={rc}")
        g = g[0] if nf == 1 else g
        if comp:
            return g, J.value, (gc[0] if nf == 1 else gc)
        return g, J.value

    def gradient_aniso(self, d_obs, wavelet=None, src=None, rec=None, magnitudes=False):
        """TTI only: gradient w.r.t. (m, epsilon, delta, theta, phi) on the
        physical grid, shape [5][nx][ny][nz], and the misfit; with
        ``magnitudes`` also the theta and phi sums over the magnitudes of
        their terms, shape [2][nx][ny][nz]."""
        src, rec, wav = self._geom(src, rec, wavelet)
        p = self.prob
        g = np.zeros((5, p.nx, p.ny, p.nz))
        a = np.zeros((2, p.nx, p.ny, p.nz)) if magnitudes else None
        J = C.c_double(0.0)
        rc = lib().or_tti_gradient_aniso(self.h, src.shape[0], _fp(src), _fp(wav), rec.shape[0],
                                         _fp(rec), _dp(_d(d_obs)), _dp(g), C.byref(J),
                                         _dp(a) if magnitudes else None)
        if rc:
            raise ValueError(f"oracle gradient rc={rc}")
        return (g, J.value, a) if magnitudes else (g, J.value)

    def backward(self, resid, wavelet=None, src=None, rec=None):
        """TTI and acoustic: (dJ/dm physical, dJ/dwavelet) for a given trace
        residual."""
        src, rec, wav = self._geom(src, rec, wavelet)
        p = self.prob
        g = np.zeros((p.nx, p.ny, p.nz))
        q = np.zeros((src.shape[0], self.nt))
        f = lib().or_ac_backward if p.kind == 3 else lib().or_tti_backward
        rc = f(self.h, src.shape[0], _fp(src), _fp(wav), rec.shape[0],
               _fp(rec), _dp(_d(resid)), _dp(g), _dp(q))
        if rc:
            raise ValueError(rc)
        return g, q

    # ---- single steps -------------------------------------------------
    def tti_step(self, p0, p1, r0, r1, adjoint=False):
        a = [_f(x).reshape(-1) for x in (p0, p1, r0, r1)]
        p2 = np.zeros(self.N)
        r2 = np.zeros(self.N)
        lib().or_tti_step_state(self.h, *[_fp(x) for x in a], _dp(p2), _dp(r2), int(adjoint))
        return p2.reshape(self.shape), r2.reshape(self.shape)

    def tti_run_d(self, p0, p1, r0, r1, nsteps):
        a = [_d(x).reshape(-1).copy() for x in (p0, p1, r0, r1)]
        lib().or_tti_step_state_d(self.h, *[_dp(x) for x in a], nsteps)
        return [x.reshape(self.shape) for x in a]

    def ac_run_d(self, u0, u1, nsteps):
        """Acoustic: nsteps source-free steps of (u^{n-1}, u^n); returns the
        last two levels (older first)."""
        a = [_d(x).reshape(-1).copy() for x in (u0, u1)]
        lib().or_ac_step_state_d(self.h, _dp(a[0]), _dp(a[1]), nsteps)
        return [x.reshape(self.shape) for x in a]

    def el_step(self, state, adjoint=False, nsteps=1):
        s = _f(state).reshape(9, -1)
        out = np.zeros((9, self.N))
        lib().or_el_step_state(self.h, _fp(s), _dp(out), int(adjoint), nsteps)
        return out.reshape((9,) + self.shape)

    def el2_run_d(self, state, nsteps, adjoint=False):
        """2D elastic: nsteps source-free (transposed) steps of a state
        [9][NX][1][NZ] in the 3D slot order (VX, VZ, TXX, TZZ, TXZ used)."""
        s = _d(state).reshape(9, -1).copy()
        lib().or_el2_step_state_d(self.h, _dp(s), int(adjoint), nsteps)
        return s.reshape((9,) + self.shape)

    def el_run_d(self, state, nsteps, adjoint=False):
        s = _d(state).reshape(9, -1).copy()
        lib().or_el_step_state_d(self.h, _dp(s), int(adjoint), nsteps)
        return s.reshape((9,) + self.shape)

    def tti_apply_L(self, p, r):
        p = _d(p).reshape(-1)
        r = _d(r).reshape(-1)
        Lp = np.zeros(self.N)
        Lr = np.zeros(self.N)
        lib().or_tti_apply_L(self.h, _dp(p), _dp(r), _dp(Lp), _dp(Lr))
        return Lp.reshape(self.shape), Lr.reshape(self.shape)

    def sparse_weights(self, xyz):
        idx = np.zeros(8, np.int64)
        w = np.zeros(8)
        n = lib().or_sparse_weights(self.h, _fp(_f(xyz).reshape(3)), _lp(idx), _dp(w))
        if n < 0:
            raise ValueError("point outside grid")
        return idx[:n], w[:n]

    def fold(self, comp):
        p = self.prob
        out = np.zeros((p.nx, p.ny, p.nz))
        lib().or_fold_grad(self.h, _dp(_d(comp).reshape(-1)), _dp(out))
        return out


def tti_step_points(prob, state, idx, adjoint=False):
    """One TTI step evaluated only at linear indices ``idx`` (computational
    grid), with the problem's operator form (``prob.tti_op``: 0 centred, 1
    staggered pair).  state = (p0, p1, r0, r1) float32 computational-grid
    arrays."""
    d = desc_of(prob)
    ml = prob.model_list()
    arr = (C.POINTER(C.c_float) * 5)(*[_fp(a) for a in ml])
    st = [_f(s).reshape(-1) for s in state]
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros((idx.size, 2))
    rc = lib().or_tti_step_points_op(C.byref(d), arr, *[_fp(s) for s in st], idx.size, _lp(idx),
                                     _dp(out), int(adjoint), int(getattr(prob, "tti_op", 0)))
    if rc:
        raise ValueError(rc)
    return out


def weights_d2(so):
    w = np.zeros(so // 2 + 1)
    if lib().or_weights_d2(so, _dp(w)):
        raise ValueError(so)
    return w


def ac_step_points(prob, state, idx):
    """One acoustic step evaluated only at ``idx``; state = (u0, u1) float32
    computational-grid arrays."""
    d = desc_of(prob)
    vp = _f(prob.model["vp"])
    st = [_f(s).reshape(-1) for s in state]
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros(idx.size)
    rc = lib().or_ac_step_points(C.byref(d), _fp(vp), _fp(st[0]), _fp(st[1]), idx.size, _lp(idx),
                                 _dp(out))
    if rc:
        raise ValueError(rc)
    return out


def el_step_points(prob, state, idx):
    """One elastic step evaluated only at ``idx``; state = 9 float32 arrays."""
    d = desc_of(prob)
    ml = prob.model_list()
    arr = (C.POINTER(C.c_float) * 3)(*[_fp(a) for a in ml])
    st = [_f(s).reshape(-1) for s in state]
    sarr = (C.POINTER(C.c_float) * 9)(*[_fp(s) for s in st])
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros((idx.size, 9))
    rc = lib().or_el_step_points(C.byref(d), arr, sarr, idx.size, _lp(idx), _dp(out))
    if rc:
        raise ValueError(rc)
    return out

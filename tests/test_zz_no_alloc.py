"""prop_forward_noalloc: forward modelling for callers that cannot allocate
device memory (an application whose own allocator already owns the GPU's
memory, or a service that forbids cudaMalloc after start-up).  It must give
the same traces as prop_create + prop_forward, on consecutive calls that
share its static device array.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def wp():
    import paper_2004_10519_gb300 as wp
    L = wp.lib()
    vp = C.c_void_p
    L.prop_forward_noalloc.argtypes = [C.POINTER(wp.PropDesc), C.POINTER(vp), vp, vp, C.c_int,
                                       vp, C.c_int, vp, vp]
    return wp


def _desc(wp, p):
    return wp.PropDesc(p.kind, p.nx, p.ny, p.nz, p.nbl, float(p.h), p.so, p.nt, float(p.dt),
                       float(p.vdamp or 0.0), wp.SNAP_FULL_FP32, 0, 1)


def _noalloc(wp, p):
    keys = ("vp", "eps", "delta", "theta", "phi") if p.kind == synth.TTI else ("vp", "vs", "rho")
    model = [np.ascontiguousarray(p.model[k], np.float32) for k in keys]
    arr = (C.c_void_p * len(model))(*[m.ctypes.data for m in model])
    wav = np.ascontiguousarray(p.wavelet, np.float32)
    src = np.ascontiguousarray(p.src, np.float32)
    rec = np.ascontiguousarray(p.rec, np.float32)
    out = np.empty((rec.shape[0], p.nt), np.float32)
    d = _desc(wp, p)
    rc = wp.lib().prop_forward_noalloc(C.byref(d), arr, wav.ctypes.data, src.ctypes.data,
                                       src.shape[0], rec.ctypes.data, rec.shape[0],
                                       out.ctypes.data, None)
    assert rc == 0, wp.lib().prop_last_error(None).decode()
    return out


def _rel(a, b):
    return float(np.linalg.norm(a.astype(np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("kind", ["tti", "elastic"])
def test_noalloc_matches_prop_forward(wp, kind):
    if kind == "tti":
        p = synth.tti_two_layer(n=40, nbl=8, so=8, nt=120)
    else:
        p = synth.elastic_random(n=36, nbl=8, so=8, nt=120, corr_len=80.0)
        p.rec = synth.line_receivers(10.0, 30.0, 12, 180.0, 5.0)
    prop = wp.Propagator.from_problem(p, check_nan=1)
    ref = prop.forward(p.wavelet, p.src, p.rec).astype(np.float64)
    prop.close()
    assert np.max(np.abs(ref)) > 0
    first = _noalloc(wp, p)
    second = _noalloc(wp, p)            # the static array keeps the first call's contents
    assert _rel(first, ref) <= TOL
    assert _rel(second, ref) <= TOL


def test_noalloc_rejects_oversized_problem(wp):
    p = synth.tti_two_layer(n=96, nbl=10, so=8, nt=10)        # 116^3 points need > 48 MiB
    model = [np.ascontiguousarray(p.model[k], np.float32)
             for k in ("vp", "eps", "delta", "theta", "phi")]
    arr = (C.c_void_p * 5)(*[m.ctypes.data for m in model])
    out = np.empty((p.rec.shape[0], p.nt), np.float32)
    d = _desc(wp, p)
    rc = wp.lib().prop_forward_noalloc(C.byref(d), arr, p.wavelet.ctypes.data, p.src.ctypes.data,
                                       1, p.rec.ctypes.data, p.rec.shape[0], out.ctypes.data, None)
    assert rc == wp.PROP_EINVAL
    assert "MiB" in wp.lib().prop_last_error(None).decode()

"""The bounds-checking build (WAVEPROP_CHECK=1 loads libwaveprop_check.so,
compiled with WP_CHECK): every shared-memory read of the TMA-fed passes
must lie in the CTA's dynamic shared memory, every float2 access of a field
below the grid size, every TMA copy must start on a 16-byte boundary.  A
failed check skips the access and makes the call return PROP_ECUDA.

A child process runs, on the checked library, the TMA-fed passes of every
family on grids ragged in y and z: elastic and centred TTI at all three
tile heights (forward, adjoint, gradient; TTI also the (m, eps, delta,
theta, phi) gradient), the staggered-pair operators (forward and the
five-parameter gradient), acoustic forward, batched gradients with shared
launches (TTI and elastic), lockstep gradients and lockstep forward
modelling.  No check may
fire, and every result must be bitwise that of the normal build."""
import os
import subprocess
import sys

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _tti(nx=30, ny=25, nz=34, so=12, nt=30, h=10.0, op=0, seed=0):
    m = synth.layered_tti(nx, ny, nz, 4 + seed, noise_sigma=3.0, smooth_sigma=1.5)
    dt = synth.cfl_dt(h, float(np.max(m["vp"] * np.sqrt(1 + 2 * m["eps"]))))
    src = np.array([[nx * h / 2 + 0.3, ny * h / 2 - 0.8, 3.1 * h]], np.float32)
    rec = synth.carpet_receivers(4.0, 5.0, 3.3 * h, 7, 6, 2.2 * h)
    p = synth.Problem(synth.TTI, nx, ny, nz, 7, h, so, nt, dt, m, src, synth.ricker(22.0, dt, nt)[None], rec)
    p.tti_op = op
    return p


def _elastic(nx=26, ny=22, nz=30, nt=30, h=10.0, seed=0):
    m = synth.random_elastic(nx, ny, nz, 8 + seed, 3.0)
    dt = synth.cfl_dt(h, float(m["vp"].max()))
    src = np.array([[nx * h / 2 + 0.4, ny * h / 2, nz * h / 2 - 0.6]], np.float32)
    rec = synth.carpet_receivers(3.3, 4.4, 3.3 * h, 6, 5, 0.0)
    return synth.Problem(synth.ELASTIC, nx, ny, nz, 7, h, 8, nt, dt, m, src,
                         synth.ricker(20.0, dt, nt)[None], rec)


def _data(p, seed):
    return np.random.default_rng(seed).standard_normal((p.rec.shape[0], p.nt)).astype(np.float32)


def run_cases(wp):
    """Results of every case, keyed by name (numpy arrays)."""
    out = {}
    for kind, mk in (("tti", _tti), ("elastic", _elastic)):
        p = mk()
        assert (p.ny + 2 * p.nbl) % 8 != 0 and (p.nz + 2 * p.nbl) % 4 == 0
        d = _data(p, 1)
        for ty in (8, 16, 32):
            os.environ["WAVEPROP_TILE_Y"] = str(ty)
            prop = wp.Propagator.from_problem(p)
            assert prop.tile_rows == ty
            out[f"{kind}{ty}_fwd"] = prop.forward(p.wavelet, p.src, p.rec)
            out[f"{kind}{ty}_adj"] = prop.adjoint(d, p.src, p.rec)
            g, J = prop.gradient(p.wavelet, p.src, p.rec, d)
            out[f"{kind}{ty}_grad"], out[f"{kind}{ty}_J"] = g, np.array([J])
            if kind == "tti":
                g, J = prop.gradient_aniso(p.wavelet, p.src, p.rec, d)
                out[f"{kind}{ty}_aniso"], out[f"{kind}{ty}_Janiso"] = g, np.array([J])
            prop.close()
        os.environ.pop("WAVEPROP_TILE_Y", None)
    p = _tti(op=1)
    d = _data(p, 2)
    prop = wp.Propagator.from_problem(p)
    out["sp_fwd"] = prop.forward(p.wavelet, p.src, p.rec)
    out["sp_aniso"] = prop.gradient_aniso(p.wavelet, p.src, p.rec, d)[0]
    prop.close()
    p = synth.acoustic_small(shape=(30, 26, 34), nbl=7, so=12, nt=30)
    prop = wp.Propagator.from_problem(p)
    out["ac_fwd"] = prop.forward(p.wavelet, p.src, p.rec)
    prop.close()
    # batched gradients (shared launches) and lockstep forward modelling
    for kind, mk in (("tti", _tti), ("elastic", _elastic)):
        ps = [mk(nx=26 + 4 * i, ny=22 + 2 * i, seed=i) for i in range(2)]
        props = [wp.Propagator.from_problem(p) for p in ps]
        gs, Js = wp.gradient_batch(props, [p.wavelet for p in ps], [p.src for p in ps], [p.rec for p in ps],
                                   [_data(p, 3 + i) for i, p in enumerate(ps)])
        for i in range(2):
            out[f"batch_{kind}{i}"], out[f"batch_{kind}{i}_J"] = gs[i], np.array([Js[i]])
        if kind == "tti":
            trs = wp.forward_batch(props, [p.wavelet for p in ps], [p.src for p in ps], [p.rec for p in ps])
            for i in range(2):
                out[f"fwdbatch{i}"] = trs[i]
        for q in props:
            q.close()
    # lockstep gradients (BF16 checkpoints: graph-replayed segments)
    ps = [_tti(nx=26 + 4 * i, ny=22 + 2 * i, seed=i) for i in range(2)]
    props = [wp.Propagator.from_problem(p, snap_mode=wp.SNAP_CKPT_BF16, ckpt_interval=7) for p in ps]
    gs, Js = wp.gradient_batch(props, [p.wavelet for p in ps], [p.src for p in ps], [p.rec for p in ps],
                               [_data(p, 5 + i) for i, p in enumerate(ps)])
    for i in range(2):
        out[f"lockstep{i}"], out[f"lockstep{i}_J"] = gs[i], np.array([Js[i]])
    for q in props:
        q.close()
    return out


def _child(path):
    import paper_2004_10519_gb300 as wp
    np.savez(path, **run_cases(wp))


def test_checked_build_passes_and_matches(tmp_path):
    import paper_2004_10519_gb300 as wp
    wp.lib()
    path = str(tmp_path / "checked.npz")
    env = dict(os.environ, WAVEPROP_CHECK="1")
    env.pop("WAVEPROP_TILE_Y", None)
    code = ("import sys; sys.path[:0] = [%r, %r]; import test_gpu_check as t; t._child(%r)"
            % (ROOT, os.path.join(ROOT, "tests"), path))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert os.path.exists(os.path.join(ROOT, "paper_2004_10519_gb300", "libwaveprop_check.so"))
    checked = np.load(path)
    plain = run_cases(wp)
    assert sorted(checked.files) == sorted(plain)
    for k in plain:
        np.testing.assert_array_equal(checked[k], plain[k], err_msg=k)

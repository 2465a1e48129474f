"""The TMA-fed stencil passes (used when the computational NZ is a multiple
of 4) and the pipelined or direct passes (any NZ; forced with
WAVEPROP_NO_TMA=1) compute the same discrete operators: their traces agree
to FP32 rounding."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def tti_problem(shape=(36, 30, 44), nbl=6, so=12, nt=60, h=10.0):
    nx, ny, nz = shape
    m = synth.layered_tti(nx, ny, nz, 5, noise_sigma=3.0, smooth_sigma=1.5)
    dt = synth.cfl_dt(h, float(np.max(m["vp"] * np.sqrt(1 + 2 * m["eps"]))))
    src = np.array([[nx * h / 2 + 0.3, ny * h / 2 - 0.8, 3.1 * h]], np.float32)
    rec = synth.carpet_receivers(5.0, 6.0, 3.3 * h, 9, 8, 2.2 * h)
    return synth.Problem(synth.TTI, nx, ny, nz, nbl, h, so, nt, dt, m, src,
                         synth.ricker(22.0, dt, nt)[None], rec)


def ac_problem(shape=(36, 30, 44), nbl=6, so=12, nt=60):
    return synth.acoustic_small(shape=shape, nbl=nbl, so=so, nt=nt)


def el_problem(shape=(34, 30, 44), nbl=6, so=8, nt=60, h=10.0):
    nx, ny, nz = shape
    m = synth.random_elastic(nx, ny, nz, 8, 4.0)
    dt = synth.cfl_dt(h, float(m["vp"].max()))
    src = np.array([[nx * h / 2 + 0.3, ny * h / 2 - 0.8, nz * h / 2]], np.float32)
    rec = synth.carpet_receivers(5.0, 6.0, 3.3 * h, 9, 8, 0.0)
    return synth.Problem(synth.ELASTIC, nx, ny, nz, nbl, h, so, nt, dt, m, src,
                         synth.ricker(20.0, dt, nt)[None], rec)


@pytest.mark.parametrize("kind", ["tti", "tti_sp", "elastic", "acoustic"])
def test_tma_and_pipelined_paths_agree(kind, monkeypatch):
    import paper_2004_10519_gb300 as wp
    wp.lib()
    p = {"tti": tti_problem, "tti_sp": tti_problem, "elastic": el_problem, "acoustic": ac_problem}[kind]()
    if kind == "tti_sp":
        p.tti_op = 1                      # staggered-pair operators
    assert (p.nz + 2 * p.nbl) % 4 == 0
    d = np.random.default_rng(3).standard_normal((p.rec.shape[0], p.nt)).astype(np.float32)
    out = {}
    for tag, env in (("tma", None), ("pipelined", "1")):
        if env:
            monkeypatch.setenv("WAVEPROP_NO_TMA", env)
        else:
            monkeypatch.delenv("WAVEPROP_NO_TMA", raising=False)
        prop = wp.Propagator.from_problem(p)
        out[tag] = (prop.forward(p.wavelet, p.src, p.rec).astype(np.float64),
                    prop.adjoint(d, p.src, p.rec).astype(np.float64))
        prop.close()
    # each path is within 2e-6 of the FP64 oracle; the staggered-pair
    # adjoint of random traces reaches that on both paths (rounding order of
    # the twelve fluxes), so their difference may reach twice it
    tol = 5e-6 if kind == "tti_sp" else 2e-6
    for i in range(2):
        a, b = out["tma"][i], out["pipelined"][i]
        assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b), (kind, i)


@pytest.mark.parametrize("kind", ["tti", "elastic", "acoustic"])
def test_tile_planes_do_not_change_results(kind, monkeypatch):
    """The autotuned x-extent of the stencil tiles only moves CTA boundaries:
    traces are bitwise identical to the occupancy heuristic's."""
    import paper_2004_10519_gb300 as wp
    wp.lib()
    p = {"tti": tti_problem, "elastic": el_problem, "acoustic": ac_problem}[kind](nt=40)
    out, planes = {}, {}
    for tag, env in (("tuned", None), ("heuristic", "0")):
        if env:
            monkeypatch.setenv("WAVEPROP_AUTOTUNE", env)
        else:
            monkeypatch.delenv("WAVEPROP_AUTOTUNE", raising=False)
        prop = wp.Propagator.from_problem(p)
        planes[tag] = prop.tile_planes
        out[tag] = prop.forward(p.wavelet, p.src, p.rec)
        prop.close()
    assert planes["tuned"] >= 8 and planes["heuristic"] >= 8
    np.testing.assert_array_equal(out["tuned"], out["heuristic"])


@pytest.mark.parametrize("kind", ["tti", "elastic"])
def test_tile_heights_give_the_same_bits(kind, monkeypatch):
    """The tile height of the TMA-fed passes (8, 16 or 32 rows of y, each a
    separately compiled set of kernels that the autotuner chooses between)
    only moves CTA boundaries: forward traces, adjoint source-side traces
    and gradients (TTI also w.r.t. eps, delta, theta, phi) are bitwise the
    same at every height, on a grid whose NY (42) is ragged for all three."""
    import paper_2004_10519_gb300 as wp
    wp.lib()
    p = {"tti": tti_problem, "elastic": el_problem}[kind](nt=40)
    assert (p.ny + 2 * p.nbl) % 8 != 0
    d = np.random.default_rng(5).standard_normal((p.rec.shape[0], p.nt)).astype(np.float32)
    out = {}
    for ty in (16, 8, 32):
        monkeypatch.setenv("WAVEPROP_TILE_Y", str(ty))
        prop = wp.Propagator.from_problem(p)
        assert prop.tile_rows == ty
        res = [prop.forward(p.wavelet, p.src, p.rec), prop.adjoint(d, p.src, p.rec)]
        g, J = prop.gradient(p.wavelet, p.src, p.rec, d)
        res += [g, np.array([J])]
        if kind == "tti":
            ga, Ja = prop.gradient_aniso(p.wavelet, p.src, p.rec, d)
            res += [ga, np.array([Ja])]
        prop.close()
        out[ty] = res
    for ty in (8, 32):
        for a, b in zip(out[ty], out[16]):
            np.testing.assert_array_equal(a, b)


def test_autotuner_reports_a_tile_shape(monkeypatch):
    """The autotuner's choice is one of the compiled heights and an x-extent
    of at least 8 planes; WAVEPROP_AUTOTUNE=0 keeps 16 rows."""
    import paper_2004_10519_gb300 as wp
    wp.lib()
    p = el_problem(nt=10)
    monkeypatch.delenv("WAVEPROP_TILE_Y", raising=False)
    monkeypatch.delenv("WAVEPROP_AUTOTUNE", raising=False)
    prop = wp.Propagator.from_problem(p)
    assert prop.tile_rows in (8, 16, 32) and prop.tile_planes >= 8
    prop.close()
    monkeypatch.setenv("WAVEPROP_AUTOTUNE", "0")
    prop = wp.Propagator.from_problem(p)
    assert prop.tile_rows == 16
    prop.close()

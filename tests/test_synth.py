"""The seeded synthetic inputs follow their stated recipes (they stand in
for the paper's unavailable models at the paper's scales): ranges,
structure, seeds, and the constraints the propagators need (eps >= delta,
vs <= vp / sqrt(2), sources and receivers inside the physical grid)."""
import math

import numpy as np
import pytest

import synth


def test_ricker_peak_and_zero_crossings():
    """q(t) = (1 - 2 pi^2 f^2 (t - t0)^2) exp(-pi^2 f^2 (t - t0)^2), t0 = 1/f:
    peak 1 at t0, zeros at t0 +- 1/(pi f sqrt 2)."""
    f, dt = 10.0, 1e-4
    q = synth.ricker(f, dt, 4000).astype(np.float64)
    i0 = int(round(1.0 / f / dt))
    assert np.argmax(q) == i0 and abs(q[i0] - 1.0) < 1e-6
    iz = int(round((1.0 / f + 1.0 / (math.pi * f * math.sqrt(2.0))) / dt))
    assert abs(q[iz]) < 1e-3


def test_cfl_dt_rule():
    assert synth.cfl_dt(12.5, 4.5) == np.float32(0.4 * 12.5 / 4500.0)


def test_layered_tti_recipe():
    m = synth.layered_tti(40, 36, 50, 20043)
    vp, eps, dl, th, ph = (m[k].astype(np.float64) for k in ("vp", "eps", "delta", "theta", "phi"))
    assert vp.min() >= 1.5 - 1e-6 and vp.max() <= 4.5 + 1e-6
    assert vp[:, :, -5:].mean() > vp[:, :, :5].mean() + 1.0          # increases with depth
    assert eps.min() >= 0.0 and eps.max() <= 0.3 + 1e-6
    np.testing.assert_allclose(dl, eps / 2, rtol=1e-6)
    assert np.all(eps >= dl)
    assert th.min() >= 0.0 and th.max() <= 40 * synth.DEG + 1e-6
    assert ph.min() >= 0.0 and ph.max() <= 90 * synth.DEG + 1e-6
    again = synth.layered_tti(40, 36, 50, 20043)
    assert all(np.array_equal(m[k], again[k]) for k in m)            # seeded
    other = synth.layered_tti(40, 36, 50, 20044)
    assert not np.array_equal(m["vp"], other["vp"])


def test_random_elastic_recipe():
    m = synth.random_elastic(30, 30, 30, 20042, 4.0)
    vp, vs, rho = (m[k].astype(np.float64) for k in ("vp", "vs", "rho"))
    assert vp.min() == pytest.approx(1.5, abs=1e-5) and vp.max() == pytest.approx(4.5, abs=1e-5)
    assert rho.min() == pytest.approx(1.0, abs=1e-5) and rho.max() == pytest.approx(2.5, abs=1e-5)
    np.testing.assert_allclose(vs, vp / 1.73, rtol=1e-6)
    assert np.all(vp * vp >= 2 * vs * vs)                              # lambda >= 0


def test_tti_two_layer_config():
    p = synth.tti_two_layer()
    assert (p.nx, p.ny, p.nz, p.nbl, p.so, p.nt) == (64, 64, 64, 10, 8, 150)
    top = p.model["vp"][:, :, 0]
    bottom = p.model["vp"][:, :, -1]
    assert np.all(top == 1.5) and np.all(bottom == 2.5)
    assert np.all(p.model["theta"][:, :, -1] == np.float32(30 * synth.DEG))
    assert p.rec.shape == (64, 3)


def test_batch_windows_recipe():
    shots = synth.tti_batch_shots(nshots=3, nt=20, size_range=(20, 60), nz=30, global_cells=(100, 100, 50))
    for true, start in shots:
        assert 20 <= true.nx <= 60 and 20 <= true.ny <= 60 and true.nz == 30
        assert np.all(true.model["eps"] >= true.model["delta"])
        # source at the window centre, 25 m deep; receivers inside the window
        assert true.src[0, 2] == 25.0
        assert true.rec[:, 0].max() <= (true.nx - 1) * true.h and true.rec[:, 1].max() <= (true.ny - 1) * true.h
        # starting model: vp linear in depth, other parameters true
        v = start.model["vp"][0, 0, :].astype(np.float64)
        assert np.allclose(np.diff(v, 2), 0.0, atol=1e-5)
        assert np.array_equal(start.model["eps"], true.model["eps"])


def test_marine_2d_recipe():
    p = synth.marine_elastic_2d(nx=101, nz=81, h=5.0, nbl=10, nt=20, water_depth=100.0, rec_dx=20.0)
    vp, vs, rho = (p.model[k][:, 0, :].astype(np.float64) for k in ("vp", "vs", "rho"))
    water = np.arange(81) * 5.0 < 100.0
    assert np.all(vp[:, water] == 1.5) and np.all(vs[:, water] == 0.0)
    assert np.allclose(rho[:, water], 1.02)
    assert vp[:, ~water].min() >= 1.6 - 1e-6 and vp[:, ~water].max() <= 4.5 + 1e-6
    np.testing.assert_allclose(vs[:, ~water], vp[:, ~water] / 1.9, rtol=1e-6)
    np.testing.assert_allclose(rho[:, ~water], 0.31 * (1000 * vp[:, ~water]) ** 0.25, rtol=1e-6)
    assert np.all(p.rec[:, 2] == 5.0) and p.src[0, 2] == 10.0


def test_random_state_seeded_and_smooth():
    a = synth.random_state(2, (20, 20, 20), 5)
    b = synth.random_state(2, (20, 20, 20), 5)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    # smoothed: neighbouring values correlate
    x = a[0].astype(np.float64)
    c = np.corrcoef(x[:-1].ravel(), x[1:].ravel())[0, 1]
    assert c > 0.3

"""Pins of the FP64 oracle's sparse-point weights and absorbing layers.

Sparse points (Sec. II-A, ``inject`` / ``interpolate``): the oracle places a
source or receiver off the grid with trilinear weights.  Trilinear
interpolation reproduces every function in span{1, x, y, z, xy, xz, yz, xyz}
exactly and its weights sum to one; a swapped weight (f <-> 1 - f) or a
wrong corner order breaks that at any fraction other than 0 and 1/2.  The
time loop must then inject and record with those weights: after one step
the recorded value is dt^2 q^0 / m summed over the products of the source's
and the receiver's weights.

Absorbing layers: a wave that enters a layer whose damping varies slowly on
the scale of a wavelength keeps its shape and loses amplitude at the local
rate of the damping (WKB).  Measured as the ratio of the first arrival at a
receiver inside the +x layer to the same receiver on a grid extended in +x
(where that point is interior and undamped), the attenuation must equal
  TTI (m u_tt + m sigma u_t = ...):   exp(-int_0^d sigma(s) ds / (2 c)),
  sigma(s) = sigma0 (s/L)^2, sigma0 = 3 v / (2 L) ln(1/R0), R0 = 1e-3,
  elastic (Cerjan taper g = exp(-(0.015 d)^2) applied once per step):
  exp(-sum over the steps the wave spends in the layer of (0.015 d)^2)
  = exp(-(0.015)^2 d^3 / 3 * h / (c dt)).
A wrong exponent, a depth in metres instead of cells, or a damping term that
is not m*sigma in one of the two time levels fails these bounds.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _homogeneous(kind, shape, h, nbl, so, nt, dt, vp=2.0):
    if kind == synth.TTI:
        model = {"vp": np.full(shape, vp, np.float32), "eps": np.zeros(shape, np.float32),
                 "delta": np.zeros(shape, np.float32), "theta": np.full(shape, 0.3, np.float32),
                 "phi": np.full(shape, 0.2, np.float32)}
    else:
        model = {"vp": np.full(shape, vp, np.float32), "vs": np.full(shape, vp / 1.73, np.float32),
                 "rho": np.full(shape, 1.0, np.float32)}
    src = np.zeros((1, 3), np.float32)
    return synth.Problem(kind, shape[0], shape[1], shape[2], nbl, h, so, nt, dt, model, src,
                         np.zeros((1, nt), np.float32), src.copy())


# --------------------------------------------------------------------------
# trilinear weights
# --------------------------------------------------------------------------
def _corner_xyz(o, idx):
    """Computational linear index -> physical coordinates in metres."""
    p = o.prob
    NX, NY, NZ = o.shape
    ix, rem = np.divmod(idx, NY * NZ)
    iy, iz = np.divmod(rem, NZ)
    return np.stack([(ix - p.nbl) * p.h, (iy - p.nbl) * p.h, (iz - p.nbl) * p.h], -1)


@pytest.mark.parametrize("kind", [synth.TTI, synth.ELASTIC])
def test_trilinear_weights_reproduce_trilinear_functions(kind):
    p = _homogeneous(kind, (9, 7, 8), 12.5, 3, 4, 4, 1e-3)
    o = oracle.Problem(p)
    rng = np.random.default_rng(11)
    coef = rng.standard_normal(8)

    def f(x, y, z):
        a, b, c, d, e, g, k, m = coef
        return a + b * x + c * y + d * z + e * x * y + g * x * z + k * y * z + m * x * y * z

    lo = -p.nbl * p.h
    hi = np.array([(n - 1 - p.nbl) * p.h for n in o.shape])
    pts = lo + rng.uniform(0.0, 1.0, (60, 3)) * (hi - lo)
    # fractions away from 0 and 1/2 in every axis (where a swapped weight
    # would go unnoticed)
    frac = (pts / p.h) % 1.0
    keep = np.all((np.abs(frac - 0.5) > 0.05) & (frac > 0.05) & (frac < 0.95), axis=1)
    pts = pts[keep]
    assert len(pts) >= 20
    for xyz in pts:
        idx, w = o.sparse_weights(xyz.astype(np.float32))
        assert len(idx) == 8
        assert np.all(w > 0)
        assert abs(w.sum() - 1.0) < 1e-14
        cxyz = _corner_xyz(o, idx)
        # the corners are the 8 nodes of the cell holding the point
        span = cxyz.max(0) - cxyz.min(0)
        np.testing.assert_allclose(span, p.h, rtol=0, atol=1e-9)
        x32 = xyz.astype(np.float32).astype(np.float64)
        val = np.dot(w, f(cxyz[:, 0], cxyz[:, 1], cxyz[:, 2]))
        assert abs(val - f(*x32)) < 1e-9 * (1 + abs(f(*x32))), xyz


def test_trilinear_weights_on_nodes_and_faces():
    """A point on a node has the single weight 1; on a cell face, zero
    weights are dropped and the rest still reproduce linear functions."""
    p = _homogeneous(synth.TTI, (6, 6, 6), 10.0, 2, 4, 4, 1e-3)
    o = oracle.Problem(p)
    idx, w = o.sparse_weights(np.array([20.0, 30.0, 10.0], np.float32))
    assert len(idx) == 1 and w[0] == 1.0
    np.testing.assert_allclose(_corner_xyz(o, idx)[0], [20.0, 30.0, 10.0])
    xyz = np.array([20.0, 33.0, 17.5], np.float32)
    idx, w = o.sparse_weights(xyz)
    assert len(idx) == 4
    c = _corner_xyz(o, idx)
    np.testing.assert_allclose(np.dot(w, c), xyz, atol=1e-9)
    with pytest.raises(ValueError):
        o.sparse_weights(np.array([-30.0, 0.0, 0.0], np.float32))      # beyond the layer


@pytest.mark.parametrize("kind", [synth.TTI, synth.ELASTIC])
def test_injection_and_recording_use_the_weights(kind):
    """Step 0 records u^0 = 0 and injects q^0 into u^1; step 1 records u^1.
    TTI: d^1 = dt^2 q^0 / m * sum_c w_s(c) w_r(c) (receivers sample p);
    elastic: d^1 = 3 dt q^0 * sum_c w_s(c) w_r(c) (tau_xx + tau_yy + tau_zz,
    each receiving dt q^0 w_s)."""
    nt = 4
    dt = 1e-3
    p = _homogeneous(kind, (10, 9, 11), 10.0, 3, 4, nt, dt)
    p.src = np.array([[41.3, 37.7, 52.6]], np.float32)
    p.rec = np.array([[41.3, 37.7, 52.6], [44.9, 33.1, 58.2], [36.2, 42.0, 47.9],
                      [70.4, 10.6, 20.3]], np.float32)
    p.wavelet = np.array([[1.0, 0.0, 0.0, 0.0]], np.float32)
    o = oracle.Problem(p)
    tr = o.forward()
    s_idx, s_w = o.sparse_weights(p.src[0])
    sw = dict(zip(s_idx.tolist(), s_w))
    m = 1.0 / (1000.0 * 2.0) ** 2
    for j, r in enumerate(p.rec):
        r_idx, r_w = o.sparse_weights(r)
        overlap = sum(wr * sw.get(i, 0.0) for i, wr in zip(r_idx.tolist(), r_w))
        want = dt * dt / m * overlap if kind == synth.TTI else 3.0 * dt * overlap
        assert tr[j, 0] == 0.0
        assert abs(tr[j, 1] - want) <= 1e-12 * max(abs(want), 1e-30) + 1e-300, (j, tr[j, 1], want)
    assert tr[3, 1] == 0.0             # no shared cell with the source
    assert tr[0, 1] > 0 and tr[1, 1] > 0


# --------------------------------------------------------------------------
# absorbing layers
# --------------------------------------------------------------------------
H, NBL, SO, F0, C = 10.0, 20, 8, 15.0, 2000.0
DEPTHS = (5, 10, 15)       # receiver depths into the +x layer, cells


def _layer_runs(kind):
    """Traces at receivers DEPTHS cells into the +x layer of a homogeneous
    grid (40 x 20 x 20 physical cells, 20-cell layer) and at the same points
    of a grid extended by 45 cells in +x.  A 4x4x4 binomial source (no
    energy at the Nyquist wavenumber) 24 cells before the physical edge."""
    dt = 0.4 * H / C
    nyz, xs, nxa = 20, 5, 30
    nxb = nxa + max(DEPTHS) + 30
    rmax = nxa - 1 + max(DEPTHS) - xs
    nt = int((rmax * H / C + 1.0 / F0 + 0.6 / F0) / dt)
    bw = np.array([1.0, 3.0, 3.0, 1.0]) / 8.0
    offs = np.array([[(a - 1.5) * H, (b - 1.5) * H, (d - 1.5) * H]
                     for a in range(4) for b in range(4) for d in range(4)])
    wts = np.array([bw[a] * bw[b] * bw[d] for a in range(4) for b in range(4) for d in range(4)])
    yc = nyz // 2 * H + 0.5 * H
    out = []
    for nx in (nxa, nxb):
        p = _homogeneous(kind, (nx, nyz, nyz), H, NBL, SO, nt, dt, vp=C / 1000.0)
        p.src = (np.array([[xs * H, yc, yc]]) + offs).astype(np.float32)
        p.rec = np.array([[(nxa - 1 + d) * H, yc, yc] for d in DEPTHS], np.float32)
        p.wavelet = (wts[:, None] * synth.ricker(F0, dt, nt)[None]).astype(np.float32)
        out.append(oracle.Problem(p).forward())
    return out[0], out[1], dt, xs, nxa


def _first_arrival_ratios(A, B, dt, xs, nxa):
    ratios = []
    for i, d in enumerate(DEPTHS):
        r = (nxa - 1 + d - xs) * H
        ia, w = int(round((r / C + 1.0 / F0) / dt)), int(round(0.35 / F0 / dt))
        sl = slice(ia - w, ia + w + 1)
        ratios.append(np.max(np.abs(A[i, sl])) / np.max(np.abs(B[i, sl])))
    return np.array(ratios)


def test_tti_damping_layer_attenuates_as_its_profile_implies():
    A, B, dt, xs, nxa = _layer_runs(synth.TTI)
    got = _first_arrival_ratios(A, B, dt, xs, nxa)
    L = NBL * H
    sig0 = 3.0 * C / (2.0 * L) * math.log(1.0 / 1e-3)        # vp = v_max, eps = 0
    want = np.array([math.exp(-sig0 * L * (d / NBL) ** 3 / 3.0 / (2.0 * C)) for d in DEPTHS])
    np.testing.assert_allclose(got, want, rtol=0.03)
    # the layer is where the damping is: the interior trace is untouched
    # until the arrival reflected by the layer could come back
    assert np.all(got < 1.0) and got[-1] < 0.55


def test_elastic_cerjan_taper_attenuates_as_its_profile_implies():
    A, B, dt, xs, nxa = _layer_runs(synth.ELASTIC)
    got = _first_arrival_ratios(A, B, dt, xs, nxa)
    steps_per_cell = H / (C * dt)           # P waves at vp
    want = np.array([math.exp(-(0.015 ** 2) * d ** 3 / 3.0 * steps_per_cell) for d in DEPTHS])
    np.testing.assert_allclose(got, want, rtol=0.03)
    assert got[-1] < 0.6

"""Pins of the FP64 oracle's 2D elastic system (the Sec. IV-A velocity-stress
equations in the x-z plane, the 2D example of Sec. IV-B):

- a y-invariant state of the 3D elastic oracle (itself pinned by energy
  conservation, the acoustic limit and Green's function tests) evolves on
  its central y plane exactly like the 2D state, forward and transposed,
  until the y faces' influence arrives;
- exact adjoint (dot test) of forward modelling with the Cerjan layer;
- mu = 0: the two normal stresses stay equal and txz stays zero (water).
"""
import numpy as np
import pytest

import oracle
import synth

E2 = (0, 2, 3, 5, 7)       # VX, VZ, TXX, TZZ, TXZ in the 3D slot order


@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("so", [4, 8])
def test_matches_y_invariant_3d(so, adjoint):
    nx, nz, nbl, h, nsteps = 14, 12, 3, 10.0, 4
    M = so // 2
    ny = 2 * (2 * M * nsteps + 2) + 1          # y faces farther than the stencils reach
    p2 = synth.elastic2d_small(shape=(nx, nz), nbl=nbl, h=h, so=so, nt=10)
    m3 = {k: np.ascontiguousarray(np.repeat(v, ny, axis=1)) for k, v in p2.model.items()}
    p3 = synth.Problem(synth.ELASTIC, nx, ny, nz, nbl, h, so, 10, p2.dt, m3, p2.src, p2.wavelet, p2.rec)
    o2, o3 = oracle.Problem(p2), oracle.Problem(p3)
    rs = synth.random_state(5, (o2.shape[0], 1, o2.shape[2]), seed=17)
    s2 = np.zeros((9,) + o2.shape)
    for c, a in zip(E2, rs):
        s2[c] = a
    s3 = np.repeat(s2, o3.shape[1], axis=2)
    out2 = o2.el2_run_d(s2, nsteps, adjoint=adjoint)
    out3 = o3.el_run_d(s3, nsteps, adjoint=adjoint)
    yc = o3.shape[1] // 2
    for c in E2:
        ref = out3[c][:, yc:yc + 1, :]
        np.testing.assert_allclose(out2[c], ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    # the unused slots stay zero in 2D
    for c in (1, 4, 6, 8):
        assert np.all(out2[c] == 0.0)


@pytest.mark.parametrize("so", [4, 8])
def test_dot_product(so):
    p = synth.elastic2d_small(shape=(24, 20), nbl=4, so=so, nt=50)
    o = oracle.Problem(p)
    rng = np.random.default_rng(3)
    q = rng.standard_normal((2, p.nt)).astype(np.float32)
    d = rng.standard_normal((p.rec.shape[0], p.nt))
    a = np.sum(o.forward(wavelet=q) * d)
    b = np.sum(q.astype(np.float64) * o.adjoint(d))
    assert abs(a - b) <= 1e-12 * abs(a), (a, b)


def test_water_acoustic_limit():
    """mu = 0 everywhere and equal initial normal stresses: txx = tzz at every
    step (an isotropic stress stays isotropic) and txz stays exactly 0."""
    p = synth.elastic2d_small(shape=(24, 20), nbl=3, so=8, nt=10)
    p.model["vs"] = np.zeros_like(p.model["vs"])
    o = oracle.Problem(p)
    rs = synth.random_state(3, (o.shape[0], 1, o.shape[2]), seed=6)
    s = np.zeros((9,) + o.shape)
    s[0], s[2], s[3] = rs
    s[5] = s[3]
    out = o.el2_run_d(s, 12)
    np.testing.assert_array_equal(out[3], out[5])
    assert np.all(out[7] == 0.0)
    assert np.abs(out[3]).max() > 0

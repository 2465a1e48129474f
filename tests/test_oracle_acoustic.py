"""Pins of the FP64 oracle's isotropic acoustic propagator (Sec. II-A,
Eq. (acou): m u_tt - laplace(u) + damp u_t = q, the wave-equation listing's
second-order leapfrog, injection s*dt**2/m and interpolation):

- second-derivative weights against textbook values and the moment
  conditions;
- the point-source Green's function of the 3D wave equation, with
  second-order convergence of the leapfrog under refinement;
- exact conservation of the discrete leapfrog energy without damping
  (a symmetric Laplacian and the right update);
- exactness of the adjoint: dot test and the assembled one-step matrix;
- Taylor test of the zero-lag cross-correlation gradient.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("so", [4, 8, 12, 16])
def test_d2_moment_conditions(so):
    """sum_k w_|k| k^j = 2 delta_{j2} for j = 0..so (exact for polynomials of
    degree so + 1: the odd moments vanish by symmetry)."""
    w = oracle.weights_d2(so)
    M = so // 2
    for j in range(0, so + 1, 2):
        mom = (w[0] if j == 0 else 0.0) + sum(2.0 * w[k] * k ** j for k in range(1, M + 1))
        assert abs(mom - (2.0 if j == 2 else 0.0)) < 1e-9 * max(1.0, M ** j), (j, mom)


def test_d2_textbook_values():
    exp4 = [Fraction(-5, 2), Fraction(4, 3), Fraction(-1, 12)]
    exp8 = [Fraction(-205, 72), Fraction(8, 5), Fraction(-1, 5), Fraction(8, 315), Fraction(-1, 560)]
    for so, exp in ((4, exp4), (8, exp8)):
        np.testing.assert_allclose(oracle.weights_d2(so), [float(f) for f in exp], rtol=1e-13)


def _point_problem(h, n, so, c, f0, nt, dt, s, rec):
    vp = np.full((n, n, n), c / 1000.0, np.float32)
    wav = synth.ricker(f0, dt, nt)[None]
    return synth.Problem(synth.ACOUSTIC, n, n, n, 0, h, so, nt, dt, {"vp": vp},
                         np.asarray([s], np.float32), wav, np.asarray([rec], np.float32))


def test_greens_function_convergence():
    """Homogeneous medium, one-node source: u(r, t) ~ h^3 q(t - r/c) / (4 pi r)
    (the Kronecker injection carries no 1/h^3).  The misfit is the leapfrog's
    O(dt^2) dispersion (dt = 0.1 h / c): halving h divides it by about 4."""
    c, f0, so, L = 1500.0, 20.0, 8, 360.0
    t0 = 1.0 / f0
    errs = []
    for h in (10.0, 5.0):
        n = int(L / h)
        s = np.array([n // 2, n // 2, n // 2]) * h
        rec = s + np.array([60.0, 50.0, 40.0])
        r = float(np.linalg.norm(rec - s))
        dt = float(np.float32(0.1 * h / c))
        nt = int((r / c + t0 + 0.8 / f0) / dt) + 1
        tr = oracle.Problem(_point_problem(h, n, so, c, f0, nt, dt, s, rec)).forward()[0]
        tau = np.arange(nt) * dt - r / c - t0
        q = (1 - 2 * (math.pi * f0 * tau) ** 2) * np.exp(-(math.pi * f0 * tau) ** 2)
        ana = h ** 3 * q / (4 * math.pi * r)
        errs.append(np.linalg.norm(tr - ana) / np.linalg.norm(ana))
    assert errs[1] < 0.02, errs
    assert 3.0 < errs[0] / errs[1] < 5.0, errs


def test_energy_conservation_undamped():
    """No layer, no source: E = sum m ((u^{n+1} - u^n)/dt)^2 - <L u^{n+1}, u^n>
    is constant for the leapfrog with a symmetric L (to rounding)."""
    n, h, so = 16, 10.0, 8
    rng = np.random.default_rng(8)
    vp = (1.5 + rng.random((n, n, n))).astype(np.float32)
    dt = synth.cfl_dt(h, 2.5)
    p = synth.Problem(synth.ACOUSTIC, n, n, n, 0, h, so, 10, dt, {"vp": vp},
                      np.zeros((1, 3), np.float32), np.zeros((1, 10), np.float32),
                      np.zeros((1, 3), np.float32))
    o = oracle.Problem(p)
    m = 1.0 / (1000.0 * vp.astype(np.float64)) ** 2
    u0, u1 = synth.random_state(2, (n, n, n), 4)
    u0, u1 = u0.astype(np.float64), u1.astype(np.float64)

    def lap(u):
        w = oracle.weights_d2(so)
        up = np.pad(u, so // 2)
        M = so // 2
        out = 3 * w[0] * u
        for ax in range(3):
            for k in range(1, M + 1):
                for sgn in (1, -1):
                    sl = [slice(M, M + n)] * 3
                    sl[ax] = slice(M + sgn * k, M + sgn * k + n)
                    out = out + w[k] * up[tuple(sl)]
        return out / h ** 2

    def energy(a, b):      # a = u^n, b = u^{n+1}
        return float(np.sum(m * ((b - a) / dt) ** 2) - np.sum(lap(b) * a))

    E = [energy(u0, u1)]
    for _ in range(6):
        u0, u1 = o.ac_run_d(u0, u1, 5)
        E.append(energy(u0, u1))
    scale = float(np.sum(m * (u1 / dt) ** 2))
    assert max(abs(e - E[0]) for e in E) <= 1e-11 * scale, (E, scale)


def _small(so=4, nt=40, nbl=4, n=12):
    p = synth.acoustic_small(shape=(n, n + 1, n + 2), nbl=nbl, so=so, nt=nt)
    p.src = np.array([[55.3, 57.1, 31.7], [20.0, 80.4, 60.2]], np.float32)
    p.rec = synth.line_receivers(3.1, 9.7, 10, 52.2, 22.9)
    return p


@pytest.mark.parametrize("so", [4, 8])
def test_dot_product(so):
    p = _small(so=so)
    o = oracle.Problem(p)
    rng = np.random.default_rng(12)
    q = rng.standard_normal((2, p.nt)).astype(np.float32)
    d = rng.standard_normal((p.rec.shape[0], p.nt))
    a = np.sum(o.forward(wavelet=q) * d)
    b = np.sum(q.astype(np.float64) * o.adjoint(d))
    assert abs(a - b) <= 1e-12 * abs(a), (a, b)


def test_one_step_matrix_symmetry():
    """Brute force on a 5x6x7 grid (with layer): assemble the step
    u^{n+1} = S1 u^n + S2 u^{n-1} from unit vectors; A S1 = dt^2 L + 2m and
    A S2 = -B must be symmetric and diagonal (A, B of the damped leapfrog)."""
    p = synth.acoustic_small(shape=(3, 4, 5), nbl=1, so=4, nt=5)
    o = oracle.Problem(p)
    N = o.N
    z = np.zeros(N)
    S1 = np.zeros((N, N))
    S2 = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        S1[:, j] = o.ac_run_d(z.reshape(o.shape), e.reshape(o.shape), 1)[1].reshape(-1)
        S2[:, j] = o.ac_run_d(e.reshape(o.shape), z.reshape(o.shape), 1)[1].reshape(-1)
    sig = np.array([lib_sigma(o, q) for q in range(N)])
    m = 1.0 / (1000.0 * np.pad(p.model["vp"].astype(np.float64), 1, mode="edge")) ** 2
    A = m.reshape(-1) * (1 + 0.5 * sig * p.dt)
    AS1 = A[:, None] * S1
    np.testing.assert_allclose(AS1, AS1.T, rtol=0, atol=1e-12 * np.abs(AS1).max())
    AS2 = A[:, None] * S2
    np.testing.assert_allclose(AS2, np.diag(np.diag(AS2)), rtol=0, atol=1e-15 * np.abs(AS2).max())


def lib_sigma(o, q):
    return oracle.lib().or_tti_sigma_at(o.h, q)


def test_taylor_gradient():
    """J(m + h d) - J(m) - h <g, d> = O(h^2) along a smooth direction d; the
    model is given as vp [km/s], the gradient is w.r.t. m = 1/vp^2 [s^2/m^2]."""
    p = _small(so=4, nt=60)
    p.vdamp = 4500.0
    dobs = oracle.Problem(p).forward()
    vp0 = synth.smooth_model(p.model, 2.0)["vp"].astype(np.float32)
    m0 = 1.0 / (1000.0 * vp0.astype(np.float64)) ** 2

    def J_of(m):
        vp = (1.0 / (1000.0 * np.sqrt(m))).astype(np.float32)
        return 0.5 * np.sum((oracle.Problem(p, model=[vp]).forward() - dobs) ** 2)

    J0 = J_of(m0)
    g, J = oracle.Problem(p, model=[vp0]).gradient(dobs)
    assert abs(J - J0) <= 1e-12 * J0
    d = 0.02 * m0 * synth.perturbation(m0.shape, 2, 21).astype(np.float64)
    lin = float(np.sum(g * d))
    assert abs(lin) > 0
    e2 = []
    for hh in (1.0, 0.5, 0.25, 0.125):
        e2.append(abs(J_of(m0 + hh * d) - J0 - hh * lin))
    slopes = [math.log(e2[i] / e2[i + 1], 2) for i in range(len(e2) - 1)]
    assert all(abs(s - 2.0) < 0.2 for s in slopes), (slopes, e2)

"""Pins of the FP64 elastic oracle (Sec. IV, Eq. elas1, elastic listing).

- exact adjoint (dot test) of forward modelling with the Cerjan layer;
- discrete energy of the undamped staggered scheme is conserved exactly
  (summation by parts with (D+)^T = -D-);
- mu = 0: shear stresses stay exactly zero (water layer, Sec. IV-B), and the
  three normal stresses coincide (acoustic limit);
- acoustic limit vs the analytic point-source solution;
- Taylor tests of the (lambda, mu, buoyancy) gradient.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def el_problem(n=12, nbl=3, so=4, nt=40, h=10.0, seed=5, model=None):
    p = synth.elastic_random(n=n, h=h, nbl=nbl, so=so, nt=nt, corr_len=3 * h, seed=seed)
    if model is not None:
        p.model = model
    p.src = np.array([[n * h * 0.45 + 0.3, n * h * 0.5 + 1.7, n * h * 0.4 + 2.1],
                      [n * h * 0.3 + 0.1, n * h * 0.6 - 0.7, n * h * 0.55]], np.float32)
    p.wavelet = np.vstack([p.wavelet[0], 0.7 * np.roll(p.wavelet[0], 3)]).astype(np.float32)
    p.rec = synth.line_receivers(1.3, (n - 2) * h / 9, 10, n * h * 0.5 - 2.2, 3.3)
    return p


@pytest.mark.parametrize("so", [4, 8])
def test_dot_product(so):
    p = el_problem(so=so)
    o = oracle.Problem(p)
    rng = np.random.default_rng(2)
    q = rng.standard_normal((2, p.nt)).astype(np.float32)
    d = rng.standard_normal((p.rec.shape[0], p.nt))
    a = np.sum(o.forward(wavelet=q) * d)
    b = np.sum(q.astype(np.float64) * o.adjoint(d))
    assert abs(a - b) <= 1e-12 * abs(a), (a, b)


def _node_params(o):
    return o.param(10), o.param(11), o.param(12)


def _energy(o, s_prev, s_next):
    """E^n = 1/2 <v^{n+1}, M v^n> + 1/2 <tau^n, K tau^n>, M = 1/b at the
    velocity points, K = C^{-1} (3x3 block at nodes, 1/mu on edges)."""
    lam, mu, b = _node_params(o)

    def shift_mean(a, axes):
        acc = np.zeros_like(a)
        cnt = 0
        for s in range(2 ** len(axes)):
            sl = [slice(None)] * 3
            aa = a
            for j, ax in enumerate(axes):
                if (s >> j) & 1:
                    idx = np.minimum(np.arange(a.shape[ax]) + 1, a.shape[ax] - 1)
                    aa = np.take(aa, idx, axis=ax)
            acc += aa
            cnt += 1
        return acc / cnt

    E = 0.0
    for c in range(3):
        bc = shift_mean(b, [c])
        E += 0.5 * np.sum(s_next[c] * s_prev[c] / bc)
    t = s_prev[3:6]
    tr = t[0] + t[1] + t[2]
    # C^{-1} t = (t - lam/(3 lam + 2 mu) tr) / (2 mu)
    for c in range(3):
        E += 0.5 * np.sum(t[c] * (t[c] - lam / (3 * lam + 2 * mu) * tr) / (2 * mu))
    for c, axes in enumerate(([0, 1], [0, 2], [1, 2])):
        E += 0.5 * np.sum(s_prev[6 + c] ** 2 / shift_mean(mu, axes))
    return E


def test_energy_conservation():
    p = el_problem(n=16, nbl=0, so=8, nt=10)
    o = oracle.Problem(p)
    state = np.stack(synth.random_state(9, o.shape, seed=31, sigma_cells=1.2)).astype(np.float64)
    # scale stresses to the model's impedance so both energy terms matter
    lam, mu, b = _node_params(o)
    state[3:] *= float(np.sqrt(np.mean(lam + 2 * mu) * np.mean(1 / b)))
    dt = p.dt
    E = []
    s = state
    for _ in range(300):
        s1 = o.el_run_d(s, 1)
        E.append(_energy(o, s, s1))
        s = s1
    E = np.array(E)
    assert np.max(np.abs(E - E[0])) <= 1e-12 * abs(E[0]), (E.min(), E.max(), dt)


def test_mu_zero_invariants():
    n, h = 16, 10.0
    p = el_problem(n=n, nbl=2, so=8, nt=60, h=h)
    vs = p.model["vs"].copy()
    water = 6                                # top 6 physical cells have mu = 0
    vs[:, :, :water] = 0.0
    p.model["vs"] = vs
    p.src = np.array([[80.3, 77.7, 22.4]], np.float32)
    p.wavelet = p.wavelet[:1]
    o = oracle.Problem(p)
    assert np.max(np.abs(o.forward())) > 0
    # propagate a random state whose shear stresses start at 0: with mu = 0
    # in the water, edge stresses inside the water stay exactly 0
    st = np.stack(synth.random_state(9, o.shape, seed=3)).astype(np.float32)
    kw = p.nbl + water - 1                   # last computational z with mu = 0
    st[6:, :, :, :] = 0.0
    out = o.el_step(st, nsteps=20)
    assert np.all(out[6][:, :, :kw + 1] == 0.0)          # txy: nodes in one z plane
    assert np.all(out[7][:, :, :kw] == 0.0)              # txz: planes k, k+1
    assert np.all(out[8][:, :, :kw] == 0.0)              # tyz


def test_acoustic_limit_normal_stresses_equal():
    n, h = 14, 10.0
    p = el_problem(n=n, nbl=2, so=8, nt=30, h=h)
    p.model["vs"] = np.zeros_like(p.model["vs"])
    o = oracle.Problem(p)
    st = np.stack(synth.random_state(9, o.shape, seed=8)).astype(np.float32)
    st[4] = st[3]
    st[5] = st[3]
    st[6:] = 0.0
    out = o.el_step(st, nsteps=10)
    np.testing.assert_array_equal(out[3], out[4])
    np.testing.assert_array_equal(out[3], out[5])
    assert np.all(out[6:] == 0.0)


def test_acoustic_limit_greens_function():
    """mu = 0, constant lambda, rho: tau_p = h^3 q'(t - r/c - dt/2) / (4 pi c^2 r)
    (the explosive source adds dt q^n over [t_n, t_{n+1}], centred dt/2 late);
    the receiver records tau_xx + tau_yy + tau_zz = 3 tau_p."""
    n, h, so = 64, 10.0, 8
    c = 1500.0
    f0 = 10.0
    dt = float(np.float32(0.2 * h / c))
    r_vec = np.array([110.0, 80.0, 60.0])
    t0 = 1.0 / f0
    r0 = float(np.linalg.norm(r_vec))
    nt = int((r0 / c + t0 + 1.2 / f0) / dt) + 1
    m = {"vp": np.full((n, n, n), c / 1000.0, np.float32),
         "vs": np.zeros((n, n, n), np.float32), "rho": np.full((n, n, n), 1.0, np.float32)}
    s = np.array([290.0, 280.0, 270.0])
    bw = np.array([1.0, 3.0, 3.0, 1.0]) / 8.0
    offs, wts = [], []
    for a in range(4):
        for b in range(4):
            for d in range(4):
                offs.append([a * h, b * h, d * h])
                wts.append(bw[a] * bw[b] * bw[d])
    offs = np.array(offs)
    rec = s + 1.5 * h + r_vec
    q0 = synth.ricker(f0, dt, nt)
    p = synth.Problem(synth.ELASTIC, n, n, n, 0, h, so, nt, dt, m,
                      (s[None] + offs).astype(np.float32),
                      (np.array(wts)[:, None] * q0[None]).astype(np.float32),
                      rec[None].astype(np.float32))
    tr = oracle.Problem(p).forward()[0]
    t = np.arange(nt) * dt
    ana = np.zeros(nt)
    for o_, w_ in zip(offs, wts):
        rr = float(np.linalg.norm(rec - s - o_))
        tau = t - rr / c - t0 - 0.5 * dt
        a_ = (math.pi * f0 * tau) ** 2
        dq = 2 * math.pi ** 2 * f0 ** 2 * tau * (2 * a_ - 3) * np.exp(-a_)
        ana += 3.0 * w_ * h ** 3 * dq / (4 * math.pi * c * c * rr)
    # misfit 4% at h = 10 m, 2.3% at h = 6 m: dispersion of the high-frequency
    # tail of q' (order-independent); a wrong scale, speed or centring fails
    err = np.linalg.norm(tr - ana) / np.linalg.norm(ana)
    assert err < 0.05, err


@pytest.mark.parametrize("which", [0, 1, 2])
def test_taylor_gradient(which):
    """J(theta + h dtheta) for theta in (lambda, mu, b): slope 2 of the
    first-order Taylor remainder."""
    p = el_problem(n=10, nbl=2, so=4, nt=50)
    dobs = oracle.Problem(p).forward()
    base = synth.random_elastic(p.nx, p.ny, p.nz, 99, 2.0)
    o0 = oracle.Problem(p, model=[base["vp"], base["vs"], base["rho"]])
    vp = base["vp"].astype(np.float64) * 1000
    vs = base["vs"].astype(np.float64) * 1000
    rho = base["rho"].astype(np.float64) * 1000
    lam, mu, b = rho * (vp ** 2 - 2 * vs ** 2), rho * vs ** 2, 1 / rho
    theta = [lam, mu, b]

    def J_of(th):
        l_, m_, b_ = th
        r_ = 1 / b_
        model = [np.sqrt((l_ + 2 * m_) * b_) / 1000, np.sqrt(m_ * b_) / 1000, r_ / 1000]
        o = oracle.Problem(p, model=[a.astype(np.float32) for a in model])
        return 0.5 * np.sum((o.forward() - dobs) ** 2)

    J0 = J_of(theta)
    g, J = o0.gradient(dobs)
    assert abs(J - J0) <= 1e-6 * J0
    d = synth.perturbation(lam.shape, 1, 40 + which).astype(np.float64) * theta[which] * 0.05
    lin = float(np.sum(g[which] * d))
    e2 = []
    for hh in (1.0, 0.5, 0.25, 0.125):
        th = list(theta)
        th[which] = theta[which] + hh * d
        e2.append(abs(J_of(th) - J0 - hh * lin))
    slopes = [math.log(e2[i] / e2[i + 1], 2) for i in range(len(e2) - 1)]
    assert all(abs(s - 2.0) < 0.15 for s in slopes), (slopes, e2)

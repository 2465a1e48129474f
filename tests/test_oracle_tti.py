"""Pins of the FP64 TTI oracle against what the paper and mathematics fix.

- plane-wave symbol of the rotated operator vs the published pseudo-acoustic
  TTI dispersion relation (Alkhalifah 2000; the self-adjoint form of Zhang et
  al. 2011 / Duveneck & Bakker 2011 cited in Sec. III-A), with the expected
  convergence order in kh;
- eps = delta = 0 collapse to the isotropic acoustic leapfrog of Sec. II-A,
  Eq. (acou), for any tilt and azimuth;
- point-source Green's function of the 3D wave equation;
- exactness of the adjoint (Sec. III-A: "exactness being a mandatory
  requirement"): dot test and assembled one-step matrices;
- Taylor test of the zero-lag cross-correlation gradient.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def homogeneous_tti(n, h, so, vp, eps, delta, theta, phi, nbl=0, nt=10, dt=1e-3):
    m = {k: np.full((n, n, n), v, np.float32) for k, v in
         zip(("vp", "eps", "delta", "theta", "phi"), (vp, eps, delta, theta, phi))}
    src = np.zeros((1, 3), np.float32)
    rec = np.zeros((1, 3), np.float32)
    return synth.Problem(synth.TTI, n, n, n, nbl, h, so, nt, dt, m, src,
                         np.zeros((1, nt), np.float32), rec)


def pseudo_acoustic_v2(eps, delta, vartheta):
    """Published pseudo-acoustic dispersion: squared phase velocities / v0^2
    for propagation at angle vartheta from the symmetry axis."""
    s2, c2 = math.sin(vartheta) ** 2, math.cos(vartheta) ** 2
    a = 1 + 2 * eps * s2
    disc = math.sqrt(max(a * a - 8 * (eps - delta) * s2 * c2, 0.0))
    return 0.5 * (a + disc), 0.5 * (a - disc)


def symbol(o, k, x0):
    n = o.shape[0]
    h = o.prob.h
    ax = np.arange(n) * h
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    phase = k[0] * (X - x0[0]) + k[1] * (Y - x0[1]) + k[2] * (Z - x0[2])
    u = np.cos(phase)
    z = np.zeros_like(u)
    i0 = tuple(int(round(c / h)) for c in x0)
    S = np.zeros((2, 2))
    Lp, Lr = o.tti_apply_L(u, z)
    S[0, 0], S[1, 0] = Lp[i0], Lr[i0]
    Lp, Lr = o.tti_apply_L(z, u)
    S[0, 1], S[1, 1] = Lp[i0], Lr[i0]
    return S


@pytest.mark.parametrize("theta,phi", [(0.0, 0.0), (0.5, 0.3), (0.9, 2.1), (1.3, -0.7)])
def test_plane_wave_dispersion(theta, phi):
    # the model is float32: evaluate the analytic relation at the same values
    f32 = lambda v: float(np.float32(v))
    eps, delta, theta, phi = f32(0.25), f32(0.1), f32(theta), f32(phi)
    n, h = 25, 10.0
    x0 = (12 * h, 12 * h, 12 * h)
    nvec = np.array([math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi),
                     math.cos(theta)])
    rng = np.random.default_rng(3)
    kdir = rng.standard_normal(3)
    kdir /= np.linalg.norm(kdir)
    vartheta = math.acos(abs(float(kdir @ nvec)))
    fast, slow = pseudo_acoustic_v2(eps, delta, vartheta)
    errs = {}
    for so in (2, 4, 8):
        o = oracle.Problem(homogeneous_tti(n, h, so, 2.0, eps, delta, theta, phi))
        e = []
        for kh in (0.2, 0.1):
            k = kdir * kh / h
            S = symbol(o, k, x0)
            ev = np.sort(np.linalg.eigvals(-S).real)[::-1] / (kh / h) ** 2
            e.append(max(abs(ev[0] - fast), abs(ev[1] - slow)))
        errs[so] = e
        # observed order of accuracy in kh
        order = math.log(e[0] / e[1], 2) if e[1] > 1e-14 else so
        assert order > so - 0.3, (so, e)
    assert errs[8][1] < 1e-8


def test_collapse_to_isotropic_acoustic():
    """eps = delta = 0: for any tilt/azimuth the TTI oracle reproduces an
    isotropic leapfrog m u_tt = sum_i D_i D_i u (written here with numpy)."""
    n, h, so, nt = 20, 10.0, 8, 60
    rng = np.random.default_rng(5)
    vp = (1.5 + rng.random((n, n, n))).astype(np.float32)
    th = rng.uniform(0, np.pi, (n, n, n)).astype(np.float32)
    ph = rng.uniform(-np.pi, np.pi, (n, n, n)).astype(np.float32)
    zero = np.zeros((n, n, n), np.float32)
    dt = synth.cfl_dt(h, 2.5)
    wav = synth.ricker(20.0, dt, nt)[None]
    src = np.array([[100.0, 90.0, 80.0]], np.float32)        # on grid nodes
    rec = np.array([[30.0, 50.0, 150.0], [180.0, 20.0, 10.0]], np.float32)
    traces = []
    for angles in ((th, ph), (zero, zero)):
        m = {"vp": vp, "eps": zero, "delta": zero, "theta": angles[0], "phi": angles[1]}
        p = synth.Problem(synth.TTI, n, n, n, 0, h, so, nt, dt, m, src, wav, rec)
        traces.append(oracle.Problem(p).forward())

    # independent isotropic leapfrog (no absorbing layer)
    c = oracle.weights_centred(so)
    M = so // 2

    def D(u, ax):
        up = np.pad(u, [(M, M) if a == ax else (0, 0) for a in range(3)])
        out = np.zeros_like(u)
        L = u.shape[ax]
        for k in range(1, M + 1):
            sp = [slice(None)] * 3
            sm = [slice(None)] * 3
            sp[ax] = slice(M + k, M + k + L)
            sm[ax] = slice(M - k, M - k + L)
            out += c[k - 1] * (up[tuple(sp)] - up[tuple(sm)])
        return out / h

    m2 = 1.0 / (vp.astype(np.float64) * 1000.0) ** 2
    u0 = np.zeros((n, n, n))
    u1 = np.zeros((n, n, n))
    tr = np.zeros((2, nt))
    si = tuple(int(v / h) for v in src[0])
    ri = [tuple(int(v / h) for v in r) for r in rec]
    for it in range(nt):
        for j, r in enumerate(ri):
            tr[j, it] = u1[r]
        lap = sum(D(D(u1, a), a) for a in range(3))
        u2 = 2 * u1 - u0 + dt * dt / m2 * lap
        u2[si] += dt * dt / m2[si] * wav[0, it]
        u0, u1 = u1, u2
    scale = np.max(np.abs(tr))
    assert scale > 0
    np.testing.assert_allclose(traces[0], tr, atol=1e-10 * scale)
    np.testing.assert_allclose(traces[1], tr, atol=1e-10 * scale)


def test_greens_function():
    """Homogeneous medium: u(r,t) ~ h^3 q(t - r/c) / (4 pi r) (Eq. acou with the
    Kronecker injection s*dt**2/m of the Sec. II-A listing)."""
    n, h, so = 72, 10.0, 8
    c = 1500.0
    f0 = 10.0
    dt = float(np.float32(0.1 * h / c))
    r_vec = np.array([120.0, 90.0, 60.0])
    r = float(np.linalg.norm(r_vec))
    t0 = 1.0 / f0
    t_end = r / c + t0 + 1.2 / f0
    nt = int(t_end / dt) + 1
    p = homogeneous_tti(n, h, so, c / 1000.0, 0.0, 0.0, 0.3, 0.2, nbl=0, nt=nt, dt=dt)
    s = np.array([340.0, 330.0, 320.0])
    # The centred first derivative applied twice has a parasitic mode at the
    # Nyquist wavenumber (u -> (-1)^i u) that a one-node source excites and
    # that travels sum_j 2 j c_j (-1)^(j+1) times faster (2.66x at so 8).
    # A 4x4x4 binomial source ([1,3,3,1]/8 per axis) has a triple zero at
    # Nyquist; the analytic field is the superposition of its 64 point
    # sources.
    bw = np.array([1.0, 3.0, 3.0, 1.0]) / 8.0
    offs, wts = [], []
    for a in range(4):
        for b in range(4):
            for d in range(4):
                offs.append([a * h, b * h, d * h])
                wts.append(bw[a] * bw[b] * bw[d])
    offs = np.array(offs)
    p.src = (s[None] + offs).astype(np.float32)
    rec = s + 1.5 * h + r_vec
    p.rec = rec[None].astype(np.float32)
    q0 = synth.ricker(f0, dt, nt)
    p.wavelet = (np.array(wts)[:, None] * q0[None]).astype(np.float32)
    tr = oracle.Problem(p).forward()[0]
    t = np.arange(nt) * dt
    ana = np.zeros(nt)
    for o_, w_ in zip(offs, wts):
        rr = float(np.linalg.norm(rec - s - o_))
        tau = t - rr / c - t0
        q = (1 - 2 * (math.pi * f0 * tau) ** 2) * np.exp(-(math.pi * f0 * tau) ** 2)
        ana += w_ * h ** 3 * q / (4 * math.pi * rr)
    # Reflections from the grid faces arrive after t_end.  The remaining
    # misfit (3% at h = 10 m) is the numerical dispersion of the wavelet's
    # high-frequency tail (kh > 1.5) and shrinks with h, not with the order.
    err = np.linalg.norm(tr - ana) / np.linalg.norm(ana)
    assert err < 0.05, err


def _greens_2d_error(so, h, dt, c=1500.0, f0=10.0, D=360.0):
    """Relative L2 error of the oracle against the analytic Green's function
    of the 2D wave equation.  With ny = 1 and no layer the zero extension
    makes D_y vanish, so the TTI oracle (eps = delta = 0, any tilt and
    azimuth) solves m u_tt = (D_x D_x + D_z D_z) u + q: a Kronecker source of
    amplitude q in a cell of area h^2 radiates
        u(r, t) = (h^2 / (2 pi)) int_0^inf q(t - (r/c) cosh s) ds.
    Source: 4 x 4 binomial weights on nodes (no energy at the Nyquist
    wavenumber, where the centred D D has its parasitic modes); receivers
    on nodes of every grid (multiples of 20 m); each trace compared within
    +-0.6/f0 of its main arrival (before any faster parasitic or reflected
    energy can arrive)."""
    t0 = 1.0 / f0
    n = int(round(2 * D / h)) + 1
    rel = np.array([[180.0, 140.0], [-200.0, 100.0], [-120.0, -180.0], [220.0, -40.0], [60.0, 220.0]])
    rmax = max(np.linalg.norm(rel, axis=1))
    nt = int((rmax / c + t0 + 0.7 / f0) / dt) + 1
    sh = (n, 1, n)
    p = homogeneous_tti(1, h, so, c / 1000.0, 0.0, 0.0, 0.4, 0.7, nbl=0, nt=nt, dt=dt)
    p.nx, p.ny, p.nz = sh
    p.model = {k: np.full(sh, float(v.flat[0]), np.float32) for k, v in p.model.items()}
    s = np.array([D, 0.0, D])
    bw = np.array([1.0, 3.0, 3.0, 1.0]) / 8.0
    offs = np.array([[a * h, 0.0, d * h] for a in range(4) for d in range(4)])
    wts = np.array([bw[a] * bw[d] for a in range(4) for d in range(4)])
    rec = np.stack([s[0] + rel[:, 0], np.zeros(len(rel)), s[2] + rel[:, 1]], 1)
    p.src = (s[None] + offs).astype(np.float32)
    p.rec = rec.astype(np.float32)
    p.wavelet = (wts[:, None] * synth.ricker(f0, dt, nt)[None]).astype(np.float32)
    tr = oracle.Problem(p).forward()
    t = np.arange(nt) * dt
    # in the windows (r/c) cosh s beyond s = 3 lies > 8/f0 before the
    # wavelet's centre, where the Ricker is below 1e-200
    sq = np.linspace(0.0, 3.0, 3001)
    wq = np.full(sq.size, sq[1] - sq[0])
    wq[0] = wq[-1] = 0.5 * (sq[1] - sq[0])
    num = den = 0.0
    for j in range(len(rel)):
        rj = float(np.linalg.norm(rec[j] - s - 1.5 * h * np.array([1.0, 0.0, 1.0])))
        win = (t >= rj / c + t0 - 0.6 / f0) & (t <= rj / c + t0 + 0.6 / f0)
        tw = t[win]
        ana = np.zeros(tw.size)
        for o_, w_ in zip(offs, wts):
            rr = float(np.linalg.norm(rec[j] - s - o_))
            tau = tw[:, None] - (rr / c) * np.cosh(sq)[None, :] - t0
            a2 = (math.pi * f0 * tau) ** 2
            ana += w_ * h * h / (2 * math.pi) * (((1 - 2 * a2) * np.exp(-a2)) @ wq)
        num += np.sum((tr[j, win] - ana) ** 2)
        den += np.sum(ana ** 2)
    return math.sqrt(num / den)


@pytest.mark.parametrize("so,dt,floor", [(2, 4e-4, 0.12), (4, 2e-4, 4e-3)])
def test_greens_function_spatial_convergence(so, dt, floor):
    """Spatial order of the TTI oracle against the analytic 2D Green's
    function at a time step small enough that the leapfrog error is far
    below the spatial one: halving h (10 -> 5 m, 15 -> 30 points per
    wavelength at f0) divides the error by 2^so (slope 2.0 and 3.8
    measured), and the fine-grid error is small in absolute terms (a wrong
    injection scale or a time shift would leave a constant error)."""
    e10 = _greens_2d_error(so, 10.0, dt)
    e5 = _greens_2d_error(so, 5.0, dt)
    slope = math.log2(e10 / e5)
    assert so - 0.5 <= slope <= so + 0.5, (e10, e5, slope)
    assert e5 < floor, e5


def _small_problem(so=4, nt=40, nbl=4, n=12):
    p = synth.tti_two_layer(n=n, nbl=nbl, so=so, nt=nt)
    p.src = np.array([[55.3, 57.1, 31.7], [20.0, 80.4, 60.2]], np.float32)
    p.wavelet = np.vstack([p.wavelet[0], 0.5 * np.roll(p.wavelet[0], 5)]).astype(np.float32)
    p.rec = synth.line_receivers(3.1, 9.7, 10, 52.2, 22.9)
    return p


@pytest.mark.parametrize("so", [4, 8])
def test_dot_product(so):
    p = _small_problem(so=so)
    o = oracle.Problem(p)
    rng = np.random.default_rng(11)
    q = rng.standard_normal((2, p.nt)).astype(np.float32)
    d = rng.standard_normal((p.rec.shape[0], p.nt))
    a = np.sum(o.forward(wavelet=q) * d)
    b = np.sum(q.astype(np.float64) * o.adjoint(d))
    assert abs(a - b) <= 1e-12 * abs(a), (a, b)


def test_one_step_matrices_transpose():
    """Brute force on a 6^3 grid: assemble the forward step blocks
    u^{n+1} = S1 u^n + S2 u^{n-1} and the adjoint step blocks
    lam^k = T1 lam^{k+1} + T2 lam^{k+2}; lam = A^{-1} mu implies
    T_j = A^{-1} S_j^T A."""
    p = synth.tti_two_layer(n=4, nbl=1, so=4, nt=5, h=10.0)
    p.model["theta"][:] = 0.4
    p.model["phi"][:] = 1.1
    p.model["eps"][:] = 0.3
    p.model["delta"][:] = 0.1
    o = oracle.Problem(p)
    N = o.N
    z = np.zeros(N, np.float32)

    def blocks(adj):
        S1 = np.zeros((2 * N, 2 * N))
        S2 = np.zeros((2 * N, 2 * N))
        for j in range(2 * N):
            e = np.zeros(2 * N, np.float32)
            e[j] = 1.0
            ep, er = e[:N], e[N:]
            p2, r2 = o.tti_step(z, ep, z, er, adjoint=adj)       # from u^n / lam^{k+1}
            S1[:, j] = np.concatenate([p2.ravel(), r2.ravel()])
            p2, r2 = o.tti_step(ep, z, er, z, adjoint=adj)       # from u^{n-1} / lam^{k+2}
            S2[:, j] = np.concatenate([p2.ravel(), r2.ravel()])
        return S1, S2

    S1, S2 = blocks(False)
    T1, T2 = blocks(True)
    m = o.param(0).ravel()
    sig = o.param(5).ravel()
    A = np.tile(m * (1 + 0.5 * sig * p.dt), 2)
    for S, T in ((S1, T1), (S2, T2)):
        ref = (S.T * A[None, :]) / A[:, None]
        np.testing.assert_allclose(T, ref, atol=1e-13 * np.abs(ref).max())


def test_taylor_gradient():
    p = _small_problem(so=4, nt=60)
    p.vdamp = 2500.0 * math.sqrt(1.4)       # damping held fixed under perturbation
    keys = ("vp", "eps", "delta", "theta", "phi")
    dobs = oracle.Problem(p).forward()
    vp0 = (p.model["vp"].astype(np.float64) * 0.97)

    def J_and(vp):
        mm = dict(p.model)
        mm["vp"] = vp.astype(np.float32)
        o = oracle.Problem(p, model=[mm[k] for k in keys])
        return 0.5 * np.sum((o.forward() - dobs) ** 2), o, mm

    J0, o0, mm0 = J_and(vp0)
    vp0 = mm0["vp"].astype(np.float64)
    g, J = o0.gradient(dobs)
    assert abs(J - J0) <= 1e-12 * J0
    m = 1.0 / (vp0 * 1000.0) ** 2
    dm = synth.perturbation(vp0.shape, 2, 7).astype(np.float64) * m * 0.05
    lin = float(np.sum(g * dm))
    e2 = []
    for hh in (1.0, 0.5, 0.25, 0.125, 0.0625):
        Jh, _, _ = J_and(1.0 / np.sqrt(m + hh * dm) / 1000.0)
        e2.append(abs(Jh - J0 - hh * lin))
    slopes = [math.log(e2[i] / e2[i + 1], 2) for i in range(len(e2) - 1)]
    assert all(abs(s - 2.0) < 0.1 for s in slopes), slopes


@pytest.mark.parametrize("op", [0, 1])
@pytest.mark.parametrize("which", ["eps", "delta"])
def test_taylor_gradient_anisotropy(which, op):
    """Gradient w.r.t. epsilon and delta: the step depends on them only
    through the coupling C of Sec. III-A (dC/deps = [[2, 0], [0, 0]],
    dC/ddelta = [[0, s'], [s', 0]], s' = 1/sqrt(1 + 2 delta)).  Pinned by the
    Taylor test (second-order remainder) along a smooth direction that keeps
    eps >= delta; its m component equals the m-only gradient."""
    p = _small_problem(so=4, nt=60)
    p.vdamp = 2500.0 * math.sqrt(1.4)       # damping held fixed under perturbation
    p.tti_op = op                           # centred or staggered-pair operators
    keys = ("vp", "eps", "delta", "theta", "phi")
    dobs = oracle.Problem(p).forward()
    base = dict(p.model)
    base["eps"] = (base["eps"].astype(np.float64) + 0.02).astype(np.float32)   # off the data model
    idx = {"eps": 1, "delta": 2}[which]
    sign = 1.0 if which == "eps" else -1.0    # raise eps / lower delta: eps >= delta holds

    def J_of(field):
        mm = dict(base)
        mm[which] = field.astype(np.float32)
        o = oracle.Problem(p, model=[mm[k] for k in keys])
        return 0.5 * np.sum((o.forward() - dobs) ** 2), o, mm

    J0, o0, mm0 = J_of(base[which].astype(np.float64))
    f0 = mm0[which].astype(np.float64)
    g3, J = o0.gradient_aniso(dobs)
    assert abs(J - J0) <= 1e-12 * J0
    g_m, _ = oracle.Problem(p, model=[mm0[k] for k in keys]).gradient(dobs)
    np.testing.assert_array_equal(g3[0], g_m)
    d = sign * 0.05 * np.abs(synth.perturbation(f0.shape, 2, 9).astype(np.float64))
    lin = float(np.sum(g3[idx] * d))
    assert abs(lin) > 0
    e2 = []
    # the staggered-pair delta direction is still visibly nonlinear at the
    # largest step (slopes 1.70, 1.85, 1.92, 1.96 from h = 1): start lower
    hs = (1.0, 0.5, 0.25, 0.125, 0.0625) if op == 0 else (0.25, 0.125, 0.0625, 0.03125, 0.015625)
    for hh in hs:
        Jh, _, _ = J_of(f0 + hh * d)
        e2.append(abs(Jh - J0 - hh * lin))
    slopes = [math.log(e2[i] / e2[i + 1], 2) for i in range(len(e2) - 1)]
    assert all(abs(s - 2.0) < 0.15 for s in slopes), slopes


@pytest.mark.parametrize("op", [0, 1])
@pytest.mark.parametrize("which", ["theta", "phi"])
def test_taylor_gradient_tilt_azimuth(which, op):
    """Gradient w.r.t. the tilt and azimuth of the symmetry axis (Eq. rot):
    the step depends on them only through the frame inside H0 and Hz (op 1:
    also through the half-point averages of the staggered-pair diagonal
    terms).  Pinned by the Taylor test (second-order remainder) along a
    smooth direction; the other components equal those of the (m, eps,
    delta) gradient computed without them."""
    p = _small_problem(so=4, nt=60)
    p.vdamp = 2500.0 * math.sqrt(1.4)
    p.tti_op = op
    keys = ("vp", "eps", "delta", "theta", "phi")
    dobs = oracle.Problem(p).forward()
    base = dict(p.model)
    base["theta"] = (base["theta"].astype(np.float64) + 0.15).astype(np.float32)   # off the data model
    idx = {"theta": 3, "phi": 4}[which]

    def J_of(field):
        mm = dict(base)
        mm[which] = field.astype(np.float32)
        o = oracle.Problem(p, model=[mm[k] for k in keys])
        return 0.5 * np.sum((o.forward() - dobs) ** 2), o, mm

    J0, o0, mm0 = J_of(base[which].astype(np.float64))
    f0 = mm0[which].astype(np.float64)
    g5, J, mag = o0.gradient_aniso(dobs, magnitudes=True)
    assert abs(J - J0) <= 1e-12 * J0
    g_m, _ = oracle.Problem(p, model=[mm0[k] for k in keys]).gradient(dobs)
    np.testing.assert_array_equal(g5[0], g_m)
    # the sum of the term magnitudes bounds the sum (triangle inequality)
    assert np.all(mag[idx - 3] >= np.abs(g5[idx]) * (1 - 1e-12))
    d = 0.2 * synth.perturbation(f0.shape, 2, 13).astype(np.float64)
    lin = float(np.sum(g5[idx] * d))
    assert abs(lin) > 0
    e2 = []
    for hh in (1.0, 0.5, 0.25, 0.125, 0.0625):
        Jh, _, _ = J_of(f0 + hh * d)
        e2.append(abs(Jh - J0 - hh * lin))
    slopes = [math.log(e2[i] / e2[i + 1], 2) for i in range(len(e2) - 1)]
    assert all(abs(s - 2.0) < 0.15 for s in slopes), slopes


@pytest.mark.parametrize("op", [0, 1])
def test_gradient_azimuth_vanishes_for_vertical_axis(op):
    """With theta = 0 everywhere the symmetry axis is vertical whatever phi
    is (the frame only spins about it, x-bar x-bar^T + y-bar y-bar^T is
    unchanged; so are the projector diagonals averaged by the staggered
    pair), so dJ/dphi is zero while dJ/dtheta is not."""
    p = _small_problem(so=4, nt=50)
    p.tti_op = op
    keys = ("vp", "eps", "delta", "theta", "phi")
    dobs = oracle.Problem(p).forward()
    mm = dict(p.model)
    mm["theta"] = np.zeros_like(mm["theta"])
    mm["phi"] = (2.0 * synth.perturbation(mm["phi"].shape, 2, 5)).astype(np.float32)
    g5, J = oracle.Problem(p, model=[mm[k] for k in keys]).gradient_aniso(dobs)
    assert J > 0
    gt, gf = np.abs(g5[3]).max(), np.abs(g5[4]).max()
    assert gt > 0
    assert gf <= 1e-12 * gt, (gf, gt)


# ---------------------------------------------------------------------------
# staggered-pair variant of the rotated operators (diagonal terms D+^T D+)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("theta,phi", [(0.5, 0.3), (1.3, -0.7)])
def test_plane_wave_dispersion_staggered_pair(theta, phi):
    """The staggered-pair operator approximates the same pseudo-acoustic
    dispersion relation with the same order in kh."""
    f32 = lambda v: float(np.float32(v))
    eps, delta, theta, phi = f32(0.25), f32(0.1), f32(theta), f32(phi)
    n, h = 25, 10.0
    x0 = (12 * h, 12 * h, 12 * h)
    nvec = np.array([math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi), math.cos(theta)])
    kdir = np.random.default_rng(4).standard_normal(3)
    kdir /= np.linalg.norm(kdir)
    fast, slow = pseudo_acoustic_v2(eps, delta, math.acos(abs(float(kdir @ nvec))))
    for so in (4, 8):
        p = homogeneous_tti(n, h, so, 2.0, eps, delta, theta, phi)
        p.tti_op = 1
        o = oracle.Problem(p)
        e = []
        for kh in (0.2, 0.1):
            S = symbol(o, kdir * kh / h, x0)
            ev = np.sort(np.linalg.eigvals(-S).real)[::-1] / (kh / h) ** 2
            e.append(max(abs(ev[0] - fast), abs(ev[1] - slow)))
        assert math.log(e[0] / e[1], 2) > so - 0.3, (so, e)


def test_staggered_pair_removes_checkerboard_null_mode():
    """u = (-1)^(x+y+z), eps = delta = 0: the composed centred operator
    annihilates it in the interior; the staggered pair gives exactly
    -3 s^2 / h^2 u with s = 2 sum_k b_k (-1)^(k+1) (each diagonal D+^T D+),
    whatever the tilt and azimuth (the cross terms cancel, P0 + Pz = I)."""
    n, h, so = 24, 10.0, 8
    rng = np.random.default_rng(2)
    p = homogeneous_tti(n, h, so, 2.0, 0.0, 0.0, 0.0, 0.0)
    p.model["theta"] = rng.uniform(0, np.pi, (n, n, n)).astype(np.float32)
    p.model["phi"] = rng.uniform(-np.pi, np.pi, (n, n, n)).astype(np.float32)
    ii = np.indices((n, n, n)).sum(0)
    u = np.where(ii % 2 == 0, 1.0, -1.0)
    inner = (slice(so, n - so),) * 3
    b = oracle.weights_staggered(so)
    s = 2.0 * sum(b[k - 1] * (-1) ** (k + 1) for k in range(1, so // 2 + 1))
    for op in (0, 1):
        p.tti_op = op
        Lp, _ = oracle.Problem(p).tti_apply_L(u, u)
        if op == 0:
            assert np.abs(Lp[inner]).max() <= 1e-9 * (s / h) ** 2
        else:
            np.testing.assert_allclose(Lp[inner], -3.0 * s * s / h ** 2 * u[inner], rtol=1e-10)


def test_staggered_pair_collapse_to_isotropic():
    """eps = delta = 0, any tilt/azimuth: the staggered-pair TTI oracle is an
    isotropic leapfrog with the compact Laplacian sum_i D-_i D+_i (numpy)."""
    n, h, so, nt = 18, 10.0, 8, 50
    rng = np.random.default_rng(6)
    vp = (1.5 + rng.random((n, n, n))).astype(np.float32)
    zero = np.zeros((n, n, n), np.float32)
    m = {"vp": vp, "eps": zero, "delta": zero,
         "theta": rng.uniform(0, np.pi, (n, n, n)).astype(np.float32),
         "phi": rng.uniform(-np.pi, np.pi, (n, n, n)).astype(np.float32)}
    dt = synth.cfl_dt(h, 2.5)
    wav = synth.ricker(20.0, dt, nt)[None]
    src = np.array([[90.0, 80.0, 70.0]], np.float32)
    rec = np.array([[30.0, 50.0, 150.0], [160.0, 20.0, 10.0]], np.float32)
    p = synth.Problem(synth.TTI, n, n, n, 0, h, so, nt, dt, m, src, wav, rec)
    p.tti_op = 1
    tr = oracle.Problem(p).forward()
    b = oracle.weights_staggered(so)
    M = so // 2

    def sh(u, ax, d):
        out = np.zeros_like(u)
        L = u.shape[ax]
        src_sl, dst_sl = [slice(None)] * 3, [slice(None)] * 3
        if d >= 0:
            src_sl[ax], dst_sl[ax] = slice(d, L), slice(0, L - d)
        else:
            src_sl[ax], dst_sl[ax] = slice(0, L + d), slice(-d, L)
        out[tuple(dst_sl)] = u[tuple(src_sl)]
        return out                           # out[i] = u[i + d], zero outside

    def lap(u):
        acc = np.zeros_like(u)
        for ax in range(3):
            dp = sum(b[k - 1] * (sh(u, ax, k) - sh(u, ax, 1 - k)) for k in range(1, M + 1)) / h
            acc += sum(b[k - 1] * (sh(dp, ax, k - 1) - sh(dp, ax, -k)) for k in range(1, M + 1)) / h
        return acc

    m2 = 1.0 / (vp.astype(np.float64) * 1000.0) ** 2
    u0, u1 = np.zeros((n, n, n)), np.zeros((n, n, n))
    ref = np.zeros((2, nt))
    si = tuple(int(v / h) for v in src[0])
    ri = [tuple(int(v / h) for v in r) for r in rec]
    for it in range(nt):
        for j, r in enumerate(ri):
            ref[j, it] = u1[r]
        u2 = 2 * u1 - u0 + dt * dt / m2 * lap(u1)
        u2[si] += dt * dt / m2[si] * wav[0, it]
        u0, u1 = u1, u2
    np.testing.assert_allclose(tr, ref, atol=1e-10 * np.max(np.abs(ref)))


@pytest.mark.parametrize("so", [4, 8])
def test_staggered_pair_dot_product(so):
    p = _small_problem(so=so)
    p.tti_op = 1
    o = oracle.Problem(p)
    rng = np.random.default_rng(11)
    q = rng.standard_normal((2, p.nt)).astype(np.float32)
    d = rng.standard_normal((p.rec.shape[0], p.nt))
    a = np.sum(o.forward(wavelet=q) * d)
    b = np.sum(q.astype(np.float64) * o.adjoint(d))
    assert abs(a - b) <= 1e-12 * abs(a), (a, b)


def test_staggered_pair_taylor_gradient():
    p = _small_problem(so=4, nt=60)
    p.tti_op = 1
    p.vdamp = 2500.0 * math.sqrt(1.4)
    keys = ("vp", "eps", "delta", "theta", "phi")
    dobs = oracle.Problem(p).forward()
    vp0 = synth.smooth_model(p.model, 2.0)["vp"].astype(np.float32)
    base = dict(p.model)

    def J_of(vp):
        mm = dict(base)
        mm["vp"] = vp.astype(np.float32)
        return 0.5 * np.sum((oracle.Problem(p, model=[mm[k] for k in keys]).forward() - dobs) ** 2)

    m0 = 1.0 / (1000.0 * vp0.astype(np.float64)) ** 2
    J0 = J_of(vp0)
    mm = dict(base)
    mm["vp"] = vp0
    g, J = oracle.Problem(p, model=[mm[k] for k in keys]).gradient(dobs)
    assert abs(J - J0) <= 1e-12 * J0
    d = 0.02 * m0 * synth.perturbation(m0.shape, 2, 23).astype(np.float64)
    lin = float(np.sum(g * d))
    e2 = []
    for hh in (1.0, 0.5, 0.25, 0.125):
        e2.append(abs(J_of(1.0 / (1000.0 * np.sqrt(m0 + hh * d))) - J0 - hh * lin))
    slopes = [math.log(e2[i] / e2[i + 1], 2) for i in range(len(e2) - 1)]
    assert all(abs(s - 2.0) < 0.2 for s in slopes), (slopes, e2)


@pytest.mark.parametrize("op", [0, 1])
def test_energy_conservation_undamped(op):
    """Undamped leapfrog m (u^{n+1} - 2u^n + u^{n-1}) = dt^2 C H u^n of the
    TTI system (Sec. III-A; u = (p, r), H = diag(H0, Hz) symmetric in both
    operator forms, C symmetric positive definite when eps > delta): with
    M = m C^{-1} pointwise,
      E^{n+1/2} = (u^{n+1} - u^n)^T M (u^{n+1} - u^n) - dt^2 (u^{n+1})^T H u^n
    is exactly constant (take the step against u^{n+1} - u^{n-1}).  H u^n is
    C^{-1} L u^n with the oracle's L = C H."""
    n, h, so = 14, 10.0, 8
    rng = np.random.default_rng(41)
    shp = (n, n, n)
    eps = rng.uniform(0.05, 0.3, shp)
    m = {"vp": rng.uniform(1.5, 3.0, shp).astype(np.float32), "eps": eps.astype(np.float32),
         "delta": (eps * rng.uniform(0.2, 0.6, shp)).astype(np.float32),
         "theta": rng.uniform(0.0, 0.7, shp).astype(np.float32),
         "phi": rng.uniform(-1.0, 1.0, shp).astype(np.float32)}
    dt = synth.cfl_dt(h, float(np.max(m["vp"] * np.sqrt(1 + 2 * m["eps"]))))
    z3 = np.zeros((1, 3), np.float32)
    p = synth.Problem(synth.TTI, n, n, n, 0, h, so, 10, dt, m, z3, np.zeros((1, 10), np.float32), z3)
    p.tti_op = op
    o = oracle.Problem(p)
    e = m["eps"].astype(np.float64)
    dl = m["delta"].astype(np.float64)
    a, s = 1 + 2 * e, np.sqrt(1 + 2 * dl)
    det = a - s * s                                   # 2 (eps - delta) > 0
    mm = 1.0 / (1000.0 * m["vp"].astype(np.float64)) ** 2
    st = [x.astype(np.float64) for x in synth.random_state(4, o.shape, seed=17, sigma_cells=1.2)]
    p0, p1, r0, r1 = st[0], st[1], st[2], st[3]

    def energy(p0, p1, r0, r1):
        dp, dr = p1 - p0, r1 - r0
        kin = np.sum(mm * (dp * dp - 2 * s * dp * dr + a * dr * dr) / det)   # du^T m C^{-1} du
        Lp, Lr = o.tti_apply_L(p0, r0)                                     # C H u^n
        Hp, Hr = (Lp - s * Lr) / det, (a * Lr - s * Lp) / det
        return kin - dt * dt * np.sum(p1 * Hp + r1 * Hr)

    E = []
    for _ in range(150):
        E.append(energy(p0, p1, r0, r1))
        p0, p1, r0, r1 = o.tti_run_d(p0, p1, r0, r1, 1)
    E = np.array(E)
    assert E[0] > 0
    assert np.max(np.abs(E - E[0])) <= 1e-11 * abs(E[0]), (E.min(), E.max())


@pytest.mark.parametrize("which", ["theta", "phi"])
def test_taylor_tilt_azimuth_staggered_pair_to_the_faces(which):
    """The staggered-pair tilt/azimuth gradient with a perturbation that
    reaches the physical faces, so the edge-replicated layer values change
    up to the last computational node, where the half-point average's
    partner is clamped (weight 1 instead of 1/2) and the first node has no
    half point below it: the Taylor remainder stays second order."""
    p = _small_problem(so=4, nt=60, nbl=0)           # the faces are the grid's ends
    p.vdamp = 2500.0 * math.sqrt(1.4)
    p.tti_op = 1
    keys = ("vp", "eps", "delta", "theta", "phi")
    dobs = oracle.Problem(p).forward()
    base = dict(p.model)
    base["theta"] = (base["theta"].astype(np.float64) + 0.15).astype(np.float32)
    idx = {"theta": 3, "phi": 4}[which]

    def J_of(field):
        mm = dict(base)
        mm[which] = field.astype(np.float32)
        o = oracle.Problem(p, model=[mm[k] for k in keys])
        return 0.5 * np.sum((o.forward() - dobs) ** 2), o

    J0, o0 = J_of(base[which].astype(np.float64))
    f0 = base[which].astype(np.float64)
    g5, _ = o0.gradient_aniso(dobs)
    # weight the faces: the perturbation is largest on the outermost cells
    n = f0.shape[0]
    edge = np.zeros(f0.shape)
    for ax in range(3):
        sl = [slice(None)] * 3
        sl[ax] = slice(0, 1)
        edge[tuple(sl)] = 1.0
        sl[ax] = slice(n - 1, n)
        edge[tuple(sl)] = 1.0
    d = 0.3 * edge * synth.perturbation(f0.shape, 0, 19).astype(np.float64)
    lin = float(np.sum(g5[idx] * d))
    assert abs(lin) > 0
    e2 = []
    for hh in (0.5, 0.25, 0.125, 0.0625, 0.03125):
        Jh, _ = J_of(f0 + hh * d)
        e2.append(abs(Jh - J0 - hh * lin))
    slopes = [math.log(e2[i] / e2[i + 1], 2) for i in range(len(e2) - 1)]
    assert all(abs(s - 2.0) < 0.15 for s in slopes), slopes

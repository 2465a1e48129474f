"""GPU parity of the TTI propagator (C ABI, FP32 CUDA kernels) against the
FP64 oracle.  Tolerance: relative L2 <= 1e-5 on traces (the stated target of
the method's FP32 implementation); gradients 1e-4 (FP32 accumulation of a
cross-correlation over all steps)."""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def wp():
    import paper_2004_10519_gb300 as wp
    wp.lib()
    return wp


def ragged_tti(so, nt=70, seed=3, shape=(37, 29, 45), nbl=7, h=10.0):
    """Small heterogeneous TTI problem with ragged tile tails."""
    nx, ny, nz = shape
    m = synth.layered_tti(nx, ny, nz, seed, noise_sigma=3.0, smooth_sigma=1.5)
    vmax = float(np.max(m["vp"] * np.sqrt(1 + 2 * m["eps"])))
    dt = synth.cfl_dt(h, vmax)
    src = np.array([[nx * h * 0.45 + 1.3, ny * h * 0.55 - 2.1, 3.3 * h],
                    [nx * h * 0.25, ny * h * 0.3 + 0.7, nz * h * 0.6]], np.float32)
    wav = np.vstack([synth.ricker(25.0, dt, nt), 0.6 * synth.ricker(18.0, dt, nt)])
    rec = synth.carpet_receivers(5.2, 7.1, 3.7 * h, 9, 7, 1.9 * h)
    return synth.Problem(synth.TTI, nx, ny, nz, nbl, h, so, nt, dt, m, src, wav, rec)


def test_forward_parity_two_layer_so8(wp):
    """84^3 computational grid (64^3 + 10-cell layer), space order 8, 150
    steps, two-layer model: the small TTI workload in full."""
    p = synth.tti_two_layer()
    tr = wp.Propagator.from_problem(p).forward(p.wavelet, p.src, p.rec)
    ref = oracle.Problem(p).forward()
    assert rel(tr, ref) <= TOL


# computational NZ % 4 != 0 runs the pipelined kernels, NZ % 4 == 0 the TMA-fed ones
SHAPES = [(37, 29, 45), (37, 29, 42)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("so", [4, 8, 12, 16])
def test_forward_parity_ragged(wp, so, shape):
    p = ragged_tti(so, shape=shape)
    tr = wp.Propagator.from_problem(p).forward(p.wavelet, p.src, p.rec)
    ref = oracle.Problem(p).forward()
    assert rel(tr, ref) <= TOL, so


@pytest.mark.parametrize("shape", SHAPES)
def test_any_tilt_and_azimuth(wp, shape):
    """Tilts beyond 90 degrees and azimuths of any sign: the kernels store the
    symmetry axis with n_z >= 0 (n and -n give the same operator, which is
    quadratic in n); the oracle uses theta and phi as given."""
    p = ragged_tti(8, nt=60, shape=shape)
    rng = np.random.default_rng(9)
    p.model["theta"] = rng.uniform(0.0, np.pi, p.model["theta"].shape).astype(np.float32)
    p.model["phi"] = rng.uniform(-np.pi, np.pi, p.model["phi"].shape).astype(np.float32)
    tr = wp.Propagator.from_problem(p).forward(p.wavelet, p.src, p.rec)
    ref = oracle.Problem(p).forward()
    assert rel(tr, ref) <= TOL


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("so", [8, 12])
def test_adjoint_parity_and_dot(wp, so, shape):
    p = ragged_tti(so, nt=60, shape=shape)
    prop = wp.Propagator.from_problem(p)
    rng = np.random.default_rng(4)
    d = rng.standard_normal((p.rec.shape[0], p.nt)).astype(np.float32)
    q = rng.standard_normal((2, p.nt)).astype(np.float32)
    qa = prop.adjoint(d, p.src, p.rec)
    ref = oracle.Problem(p).adjoint(d)
    assert rel(qa, ref) <= TOL
    Fq = prop.forward(q, p.src, p.rec)
    a = float(np.sum(Fq.astype(np.float64) * d))
    b = float(np.sum(q.astype(np.float64) * qa))
    assert abs(a - b) <= 1e-5 * abs(a), (a, b)


def grad_problem(so=8, nt=80, shape=(30, 26, 34)):
    p = ragged_tti(so, nt=nt, shape=shape, nbl=6)
    p.vdamp = float(np.max(p.model["vp"] * np.sqrt(1 + 2 * p.model["eps"]))) * 1000.0
    true = oracle.Problem(p)
    d_obs = true.forward()
    start = synth.smooth_model(p.model, 3.0)
    p0 = synth.Problem(**{**p.__dict__, "model": start})
    return p, p0, d_obs


@pytest.mark.parametrize("shape", [(30, 26, 34), (30, 26, 36)])
def test_gradient_parity_and_checkpoint_modes(wp, shape):
    p, p0, d_obs = grad_problem(shape=shape)
    g_ref, J_ref = oracle.Problem(p0).gradient(d_obs)
    d32 = d_obs.astype(np.float32)
    res = {}
    for mode in (wp.SNAP_FULL_FP32, wp.SNAP_CKPT_FP32, wp.SNAP_CKPT_BF16, wp.SNAP_CKPT_FP16):
        prop = wp.Propagator.from_problem(p0, snap_mode=mode, ckpt_interval=9)
        res[mode] = prop.gradient(p0.wavelet, p0.src, p0.rec, d32)
        prop.close()
    g, J = res[wp.SNAP_FULL_FP32]
    assert abs(J - J_ref) <= 1e-5 * J_ref
    assert rel(g, g_ref) <= 1e-4
    # FP32 checkpoints recompute bit-identical forward wavefields
    np.testing.assert_array_equal(res[wp.SNAP_CKPT_FP32][0], g)
    # 16-bit checkpoints: stated error bound of the storage
    assert rel(res[wp.SNAP_CKPT_BF16][0], g_ref) <= 2e-2
    assert rel(res[wp.SNAP_CKPT_FP16][0], g_ref) <= 2e-3


@pytest.mark.parametrize("op,shape", [(0, (30, 26, 36)), (1, (30, 26, 36)), (0, (30, 26, 34))],
                         ids=["centred-tma", "staggered-pair-tma", "centred-pipelined"])
def test_gradient_aniso_parity(wp, op, shape):
    """dJ/d(m, eps, delta, theta, phi) (prop_gradient_aniso) against the
    oracle, centred (op 0) and staggered-pair (op 1) operators, full storage
    and FP32 checkpoints (bitwise equal to each other); the m component
    equals prop_gradient's.  Computational nz 48 runs the TMA-fed passes,
    46 the pipelined ones.  The theta and phi sums cancel strongly (the p
    and r terms of their imaging nearly balance, and the cross-correlation
    oscillates): their error is bounded relative to the oracle's sum of the
    term magnitudes, 1e-5 of it (FP32 wavefields carry relative errors of
    about 1e-6), instead of relative to the result."""
    p, p0, d_obs = grad_problem(shape=shape)
    p.tti_op = p0.tti_op = op
    g_ref, J_ref, mag = oracle.Problem(p0).gradient_aniso(d_obs, magnitudes=True)
    d32 = d_obs.astype(np.float32)
    res = {}
    for mode in (wp.SNAP_FULL_FP32, wp.SNAP_CKPT_FP32):
        prop = wp.Propagator.from_problem(p0, snap_mode=mode, ckpt_interval=9)
        res[mode] = prop.gradient_aniso(p0.wavelet, p0.src, p0.rec, d32)
        g_m, _ = prop.gradient(p0.wavelet, p0.src, p0.rec, d32)
        np.testing.assert_array_equal(res[mode][0][0], g_m)
        prop.close()
    g, J = res[wp.SNAP_FULL_FP32]
    assert abs(J - J_ref) <= 1e-5 * J_ref
    assert g.shape == g_ref.shape == (5, p0.nx, p0.ny, p0.nz)
    for c in range(3):
        assert rel(g[c], g_ref[c]) <= 1e-4, (c, rel(g[c], g_ref[c]))
    for c in (3, 4):
        err = float(np.linalg.norm(g[c].astype(np.float64) - g_ref[c]))
        assert err <= 1e-5 * float(np.linalg.norm(mag[c - 3])), (c, err, rel(g[c], g_ref[c]))
        assert rel(g[c], g_ref[c]) <= 1e-3, c
    np.testing.assert_array_equal(res[wp.SNAP_CKPT_FP32][0], g)
    if op == 1:
        # the staggered-pair imaging runs on the TMA-fed passes only: a
        # computational nz that is not a multiple of 4 is rejected and the
        # handle stays usable
        q, q0, d2 = grad_problem(shape=(30, 26, 34))
        q0.tti_op = op
        prop = wp.Propagator.from_problem(q0)
        with pytest.raises(wp.PropError) as e:
            prop.gradient_aniso(q0.wavelet, q0.src, q0.rec, d2.astype(np.float32))
        assert e.value.code == wp.PROP_EINVAL
        prop.gradient(q0.wavelet, q0.src, q0.rec, d2.astype(np.float32))


def test_backward_matches_oracle(wp):
    """prop_forward_saved + prop_backward (autograd form): gradient w.r.t. m
    and w.r.t. the wavelet for an arbitrary trace cotangent."""
    p, p0, _ = grad_problem(nt=60)
    rng = np.random.default_rng(9)
    resid = rng.standard_normal((p0.rec.shape[0], p0.nt)).astype(np.float32)
    g_ref, q_ref = oracle.Problem(p0).backward(resid)
    prop = wp.Propagator.from_problem(p0)
    prop.forward(p0.wavelet, p0.src, p0.rec, save=True)
    g, q = prop.backward(resid, nsrc=p0.src.shape[0])
    assert rel(g, g_ref) <= 1e-4
    assert rel(q, q_ref) <= TOL


def test_determinism(wp):
    p = ragged_tti(8, nt=40)
    prop = wp.Propagator.from_problem(p)
    a = prop.forward(p.wavelet, p.src, p.rec)
    b = prop.forward(p.wavelet, p.src, p.rec)
    np.testing.assert_array_equal(a, b)


def test_eps_delta_collapse_gpu(wp):
    """eps = delta = 0: p and r stay identical on the GPU (same expressions)."""
    p = ragged_tti(8, nt=40)
    for k in ("eps", "delta"):
        p.model[k] = np.zeros_like(p.model[k])
    prop = wp.Propagator.from_problem(p)
    prop.forward(p.wavelet, p.src, p.rec)
    st = prop.get_state()
    np.testing.assert_array_equal(st[0], st[1])
    np.testing.assert_array_equal(st[2], st[3])


def random_tti_model(shape, seed):
    rng = np.random.default_rng(seed)
    f = lambda lo, hi: rng.uniform(lo, hi, shape).astype(np.float32)
    eps = f(0.0, 0.3)
    return {"vp": f(1.5, 4.5), "eps": eps, "delta": (eps * f(0.0, 0.5)).astype(np.float32),
            "theta": f(0.0, 40 * synth.DEG), "phi": f(0.0, 90 * synth.DEG)}


def assert_pointwise(got, ref, tag=""):
    """Per-point bound of a sampled comparison: where the reference is at
    least 1 % of its largest sampled magnitude, the relative error of every
    point is at most TOL; everywhere the absolute error is at most 0.1 TOL
    of that magnitude (FP32 rounding of the step's terms: measured on the
    full-size grids at most 3.8e-6 relative where it applies, 1.7e-7 of the
    magnitude in absolute terms)."""
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    m = float(np.max(np.abs(ref)))
    ae = np.abs(got - ref)
    big = np.abs(ref) >= 0.01 * m
    assert big.sum() >= ref.size // 2, tag
    rel_pt = float(np.max(ae[big] / np.abs(ref[big])))
    assert rel_pt <= TOL, (tag, rel_pt)
    assert float(np.max(ae)) <= 0.1 * TOL * m, (tag, float(np.max(ae)) / m)


def sample_points(shape, n, seed):
    """Sampled outputs: random interior points plus every corner / face / edge class."""
    NX, NY, NZ = shape
    rng = np.random.default_rng(seed)
    pts = [(rng.integers(NX), rng.integers(NY), rng.integers(NZ)) for _ in range(n)]
    for x in (0, 1, NX // 2, NX - 2, NX - 1):
        for y in (0, NY // 3, NY - 1):
            for z in (0, 5, NZ - 3, NZ - 1):
                pts.append((x, y, z))
    return np.array([(x * NY + y) * NZ + z for x, y, z in pts], np.int64)


@pytest.mark.parametrize("op", [0, 1])
@pytest.mark.parametrize("adjoint", [False, True])
def test_one_step_sampled_full_size(wp, adjoint, op):
    """Industry-scale TTI grid (800x800x400 + 40-cell layer = 880x880x480),
    space order 12, centred (op 0) and staggered-pair (op 1) operators: one
    step from a seeded random state; the oracle evaluates the step at
    sampled points (interior, faces, edges, corners)."""
    nx, ny, nz, nbl, h = 800, 800, 400, 40, 12.5
    model = random_tti_model((nx, ny, nz), 77)
    dt = synth.cfl_dt(h, float(np.max(model["vp"] * np.sqrt(1 + 2 * model["eps"]))))
    p = synth.Problem(synth.TTI, nx, ny, nz, nbl, h, 12, 10, dt, model,
                      np.zeros((1, 3), np.float32), np.zeros((1, 10), np.float32),
                      np.zeros((1, 3), np.float32))
    p.tti_op = op
    prop = wp.Propagator.from_problem(p)
    shape = prop.grid
    rng = np.random.default_rng(5)
    state = [rng.standard_normal(shape, dtype=np.float32) for _ in range(4)]
    prop.set_state(state)          # p^n, r^n, p^{n-1}, r^{n-1}
    prop.step(1, adjoint=adjoint)
    out = prop.get_state()
    prop.close()
    idx = sample_points(shape, 400, 6)
    ref = oracle.tti_step_points(p, (state[2], state[0], state[3], state[1]), idx, adjoint=adjoint)
    got = np.stack([out[0].reshape(-1)[idx], out[1].reshape(-1)[idx]], axis=1)
    for c in range(2):
        assert_pointwise(got[:, c], ref[:, c], ("p", "r")[c])


# ---------------------------------------------------------------------------
# staggered-pair operators (desc.tti_operator = 1)
# ---------------------------------------------------------------------------
def sp_problem(so, nt=70, shape=(37, 29, 45)):
    p = ragged_tti(so, nt=nt, shape=shape)
    p.tti_op = 1
    return p


@pytest.mark.parametrize("so", [4, 8, 12, 16])
@pytest.mark.parametrize("shape", SHAPES)
def test_staggered_pair_forward_adjoint_parity(wp, so, shape):
    p = sp_problem(so, nt=60, shape=shape)
    prop = wp.Propagator.from_problem(p)
    o = oracle.Problem(p)
    assert rel(prop.forward(p.wavelet, p.src, p.rec), o.forward()) <= TOL
    rng = np.random.default_rng(4)
    d = rng.standard_normal((p.rec.shape[0], p.nt)).astype(np.float32)
    q = rng.standard_normal((2, p.nt)).astype(np.float32)
    qa = prop.adjoint(d, p.src, p.rec)
    assert rel(qa, o.adjoint(d)) <= TOL
    Fq = prop.forward(q, p.src, p.rec).astype(np.float64)
    a = float(np.sum(Fq * d))
    b = float(np.sum(q.astype(np.float64) * qa))
    # with forward and adjoint each within TOL (relative L2) of the exact
    # transposes, Cauchy-Schwarz bounds the dot-test gap by
    # TOL (|Fq| |d| + |q| |F^T d|) (random d makes <Fq, d> itself small)
    bound = TOL * (np.linalg.norm(Fq) * np.linalg.norm(d) + np.linalg.norm(q) * np.linalg.norm(qa))
    assert abs(a - b) <= bound, (a, b, bound)
    # the centred operators give different traces on the same model
    p0 = ragged_tti(so, nt=60, shape=shape)
    assert rel(wp.Propagator.from_problem(p0).forward(p.wavelet, p.src, p.rec), o.forward()) > 10 * TOL


def test_staggered_pair_gradient_parity(wp):
    p, p0, d_obs = grad_problem(shape=(30, 26, 36))
    p.tti_op = p0.tti_op = 1
    d_obs = oracle.Problem(p).forward()
    g_ref, J_ref = oracle.Problem(p0).gradient(d_obs)
    d32 = d_obs.astype(np.float32)
    res = {}
    for mode in (wp.SNAP_FULL_FP32, wp.SNAP_CKPT_FP32):
        prop = wp.Propagator.from_problem(p0, snap_mode=mode, ckpt_interval=9)
        res[mode] = prop.gradient(p0.wavelet, p0.src, p0.rec, d32)
        prop.close()
    g, J = res[wp.SNAP_FULL_FP32]
    assert abs(J - J_ref) <= 1e-5 * J_ref
    assert rel(g, g_ref) <= 1e-4
    np.testing.assert_array_equal(res[wp.SNAP_CKPT_FP32][0], g)


@pytest.mark.parametrize("adjoint", [False, True])
def test_staggered_pair_state_steps(wp, adjoint):
    p = sp_problem(12)
    prop = wp.Propagator.from_problem(p)
    st = synth.random_state(4, prop.grid, 21)
    prop.set_state(st)             # p^n, r^n, p^{n-1}, r^{n-1}
    prop.step(1, adjoint=adjoint)
    out = prop.get_state()
    p2, r2 = oracle.Problem(p).tti_step(st[2], st[0], st[3], st[1], adjoint=adjoint)
    assert rel(out[0], p2) <= TOL and rel(out[1], r2) <= TOL


@pytest.mark.parametrize("kind", ["tti", "acoustic"])
def test_checkpoint_tail_is_bitwise(wp, monkeypatch, kind):
    """FP32 checkpoints keep the last levels of the run in full when device
    memory allows (the adjoint sweep then recomputes only the checkpointed
    part).  The gradient is bitwise that of full storage with no tail, a
    partial tail (WAVEPROP_CKPT_TAIL caps it) and every level in the tail."""
    if kind == "tti":
        _, p0, d_obs = grad_problem(shape=(30, 26, 36))
    else:
        p0 = synth.acoustic_small(shape=(30, 26, 36), nbl=6, so=8, nt=70)
        d_obs = 1.1 * oracle.Problem(p0).forward()
    d32 = d_obs.astype(np.float32)
    prop = wp.Propagator.from_problem(p0, snap_mode=wp.SNAP_FULL_FP32)
    ref, J_ref = prop.gradient(p0.wavelet, p0.src, p0.rec, d32)
    prop.close()
    for cap in ("0", "7", "100000"):
        monkeypatch.setenv("WAVEPROP_CKPT_TAIL", cap)
        prop = wp.Propagator.from_problem(p0, snap_mode=wp.SNAP_CKPT_FP32, ckpt_interval=0)
        g, J = prop.gradient(p0.wavelet, p0.src, p0.rec, d32)
        prop.close()
        np.testing.assert_array_equal(g, ref, err_msg=cap)
        assert J == J_ref


def test_industry_recipe_at_reduced_size(wp):
    """The industry-scale TTI workload's recipe (layered-plus-noise model
    with eps, delta, tilt and azimuth derived from it, so 12, 12.5 m, 40-cell
    layer, 12 Hz source 25 m deep, surface carpet of receivers every 40 m) at
    200 x 200 x 100 physical points (280 x 280 x 180 computational), 150
    steps: traces against the FP64 oracle's whole run."""
    p = synth.tti_layered(nx=200, ny=200, nz=100, nt=150)
    assert p.rec.shape[0] > 1000
    prop = wp.Propagator.from_problem(p)
    tr = prop.forward(p.wavelet, p.src, p.rec)
    prop.close()
    ref = oracle.Problem(p).forward()
    assert np.max(np.abs(ref)) > 0
    assert rel(tr, ref) <= TOL, rel(tr, ref)

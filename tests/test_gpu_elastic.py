"""GPU parity of the elastic propagator (C ABI, FP32 CUDA kernels) against the
FP64 oracle."""
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


def ragged_el(so, nt=70, shape=(31, 27, 37), nbl=6, h=10.0, seed=11):
    nx, ny, nz = shape
    m = synth.random_elastic(nx, ny, nz, seed, 4.0)
    dt = synth.cfl_dt(h, float(m["vp"].max()))
    src = np.array([[nx * h * 0.5 + 0.7, ny * h * 0.45 - 1.1, nz * h * 0.4 + 2.3],
                    [nx * h * 0.3, ny * h * 0.6, nz * h * 0.7]], np.float32)
    wav = np.vstack([synth.ricker(22.0, dt, nt), -0.8 * synth.ricker(15.0, dt, nt)])
    rec = synth.carpet_receivers(3.3, 4.4, 3.3 * h, 8, 7, 0.0)
    return synth.Problem(synth.ELASTIC, nx, ny, nz, nbl, h, so, nt, dt, m, src, wav, rec)


def test_forward_parity_reduced_random_model(wp):
    """The elastic workload's recipe (smooth random vp 1.5-4.5 km/s, vs =
    vp/1.73, rho 1.0-2.5 g/cc, explosive 10 Hz Ricker at the centre, carpet
    of receivers at the surface, 20-cell layer, so 8) at 48^3 + 20, 300 steps."""
    p = synth.elastic_random(n=48, nbl=20, so=8, nt=300, corr_len=200.0)
    tr = wp.Propagator.from_problem(p).forward(p.wavelet, p.src, p.rec)
    ref = oracle.Problem(p).forward()
    assert rel(tr, ref) <= TOL


# computational NZ % 4 != 0 runs the pipelined kernels, NZ % 4 == 0 the TMA-fed ones
SHAPES = [(31, 27, 37), (31, 27, 40)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("so", [4, 8, 12, 16])
def test_forward_parity_ragged(wp, so, shape):
    p = ragged_el(so, shape=shape)
    tr = wp.Propagator.from_problem(p).forward(p.wavelet, p.src, p.rec)
    ref = oracle.Problem(p).forward()
    assert rel(tr, ref) <= TOL, so


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("so", [8, 12])
def test_adjoint_parity_and_dot(wp, so, shape):
    p = ragged_el(so, nt=60, shape=shape)
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


# computational NZ 32: TMA-fed passes with pointwise face products;
# NZ 33: the direct-load transposed step
@pytest.mark.parametrize("shape", [(22, 20, 24), (22, 20, 25)])
def test_gradient_parity_and_checkpoint_modes(wp, shape):
    p = ragged_el(8, nt=60, shape=shape, nbl=4)
    d_obs = oracle.Problem(p).forward()
    start = synth.random_elastic(p.nx, p.ny, p.nz, 5, 3.0)
    start = {k: (0.5 * (start[k] + p.model[k])).astype(np.float32) for k in start}
    p0 = synth.Problem(**{**p.__dict__, "model": start})
    g_ref, J_ref = oracle.Problem(p0).gradient(d_obs)
    d32 = d_obs.astype(np.float32)
    res = {}
    for mode in (wp.SNAP_FULL_FP32, wp.SNAP_CKPT_FP32, wp.SNAP_CKPT_BF16):
        prop = wp.Propagator.from_problem(p0, snap_mode=mode, ckpt_interval=7)
        res[mode] = prop.gradient(p0.wavelet, p0.src, p0.rec, d32)
        prop.close()
    g, J = res[wp.SNAP_FULL_FP32]
    assert abs(J - J_ref) <= 1e-5 * J_ref
    for c in range(3):
        assert rel(g[c], g_ref[c]) <= 1e-4, c
    np.testing.assert_array_equal(res[wp.SNAP_CKPT_FP32][0], g)
    for c in range(3):
        assert rel(res[wp.SNAP_CKPT_BF16][0][c], g_ref[c]) <= 2e-2, c


def test_determinism(wp):
    p = ragged_el(8, nt=40)
    prop = wp.Propagator.from_problem(p)
    a = prop.forward(p.wavelet, p.src, p.rec)
    b = prop.forward(p.wavelet, p.src, p.rec)
    np.testing.assert_array_equal(a, b)


def test_water_layer_shear_stress_zero(wp):
    """mu = 0 in a water layer: shear stresses there stay exactly 0 (Sec. IV-B)."""
    p = ragged_el(8, nt=80)
    vs = p.model["vs"].copy()
    vs[:, :, :10] = 0.0
    p.model["vs"] = vs
    p.src = np.array([[150.0, 130.0, 40.0]], np.float32)
    p.wavelet = p.wavelet[:1]
    prop = wp.Propagator.from_problem(p)
    prop.forward(p.wavelet, p.src, p.rec)
    st = prop.get_state()
    kw = p.nbl + 10 - 1
    assert np.abs(st[3][:, :, :kw]).max() > 0
    assert np.all(st[6][:, :, :kw + 1] == 0.0)
    assert np.all(st[7][:, :, :kw] == 0.0)
    assert np.all(st[8][:, :, :kw] == 0.0)


def sample_points(shape, n, seed):
    NX, NY, NZ = shape
    rng = np.random.default_rng(seed)
    pts = [(rng.integers(NX), rng.integers(NY), rng.integers(NZ)) for _ in range(n)]
    for x in (0, 1, NX // 2, NX - 2, NX - 1):
        for y in (0, NY // 3, NY - 1):
            for z in (0, 5, NZ - 3, NZ - 1):
                pts.append((x, y, z))
    return np.array([(x * NY + y) * NZ + z for x, y, z in pts], np.int64)


def test_one_step_sampled_full_size(wp):
    """The benchmarked elastic grid (256^3 + 20-cell layer = 296^3, so 8) in
    the benchmark's launch configuration: one step from a seeded random state,
    oracle at sampled points of all nine fields."""
    n, nbl, h = 256, 20, 10.0
    rng = np.random.default_rng(21)
    vp = rng.uniform(1.5, 4.5, (n, n, n)).astype(np.float32)
    model = {"vp": vp, "vs": (vp / 1.73).astype(np.float32),
             "rho": rng.uniform(1.0, 2.5, (n, n, n)).astype(np.float32)}
    dt = synth.cfl_dt(h, float(vp.max()))
    p = synth.Problem(synth.ELASTIC, n, n, n, nbl, h, 8, 10, dt, model,
                      np.zeros((1, 3), np.float32), np.zeros((1, 10), np.float32),
                      np.zeros((1, 3), np.float32))
    prop = wp.Propagator.from_problem(p)
    shape = prop.grid
    state = [rng.standard_normal(shape, dtype=np.float32) for _ in range(3)]
    state += [1e7 * rng.standard_normal(shape, dtype=np.float32) for _ in range(6)]
    prop.set_state(state)
    prop.step(1)
    out = prop.get_state()
    prop.close()
    idx = sample_points(shape, 300, 8)
    ref = oracle.el_step_points(p, state, idx)
    from test_gpu_tti import assert_pointwise
    for c in range(9):
        assert_pointwise(out[c].reshape(-1)[idx], ref[:, c], c)


def test_full_size_whole_grid_multistep(wp):
    """The elastic workload at its own size (256^3 + 20-cell layer = 296^3,
    so 8, its smooth random model): all nine fields over the whole grid
    after 200 source-free steps from a seeded smooth state, against 200
    FP64 oracle steps.  Each field within 1e-5 of the oracle's norm."""
    p = synth.elastic_random(n=256, nbl=20, so=8, nt=10)
    prop = wp.Propagator.from_problem(p)
    st = synth.random_state(9, prop.grid, 21, sigma_cells=3.0)
    prop.set_state(st)
    prop.step(200)
    gpu = prop.get_state()
    prop.close()
    ref = oracle.Problem(p).el_run_d(np.stack(st), 200)
    for f in range(9):
        e = rel(gpu[f], ref[f])
        assert e <= TOL, (f, e)


def test_full_size_dot_product(wp):
    """Adjoint test at the workload's own size and length: <F q, d> =
    <q, F^T d> for a seeded random wavelet q and traces d (4096 surface
    receivers, 1000 steps: the wave from the centre reaches the surface),
    the FP32 products accumulated in FP64."""
    p = synth.elastic_random(n=256, nbl=20, so=8, nt=1000)
    prop = wp.Propagator.from_problem(p)
    rng = np.random.default_rng(9)
    q = rng.standard_normal(p.wavelet.shape).astype(np.float32)
    d = rng.standard_normal((p.rec.shape[0], p.nt)).astype(np.float32)
    Fq = prop.forward(q, p.src, p.rec).astype(np.float64)
    Ftd = prop.adjoint(d, p.src, p.rec).astype(np.float64)
    prop.close()
    lhs = float(np.sum(Fq * d))
    rhs = float(np.sum(q.astype(np.float64) * Ftd))
    assert np.max(np.abs(Fq)) > 0
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs)), (lhs, rhs)

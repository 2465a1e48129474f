"""GPU parity of the isotropic acoustic propagator (Sec. II-A, Eq. acou; C ABI,
FP32 CUDA kernels) against the FP64 oracle.  Tolerances as for TTI: relative
L2 <= 1e-5 on traces and adjoint outputs, 1e-4 on gradients."""
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


# computational NZ = nz + 14: 59 (direct kernel) and 56 (TMA-fed pass)
SHAPES = [(37, 29, 45), (37, 29, 42)]


@pytest.mark.parametrize("so", [4, 8, 12, 16])
@pytest.mark.parametrize("shape", SHAPES)
def test_forward_parity(wp, so, shape):
    p = synth.acoustic_small(shape=shape, so=so)
    tr = wp.Propagator.from_problem(p).forward(p.wavelet, p.src, p.rec)
    assert rel(tr, oracle.Problem(p).forward()) <= TOL


@pytest.mark.parametrize("so", [8, 12])
@pytest.mark.parametrize("shape", SHAPES)
def test_adjoint_parity_and_dot(wp, so, shape):
    p = synth.acoustic_small(shape=shape, so=so, nt=60)
    prop = wp.Propagator.from_problem(p)
    rng = np.random.default_rng(4)
    d = rng.standard_normal((p.rec.shape[0], p.nt)).astype(np.float32)
    q = rng.standard_normal((2, p.nt)).astype(np.float32)
    qa = prop.adjoint(d, p.src, p.rec)
    assert rel(qa, oracle.Problem(p).adjoint(d)) <= TOL
    Fq = prop.forward(q, p.src, p.rec)
    a = float(np.sum(Fq.astype(np.float64) * d))
    b = float(np.sum(q.astype(np.float64) * qa))
    assert abs(a - b) <= 1e-5 * abs(a), (a, b)


def grad_problem(shape, so=8, nt=80):
    p = synth.acoustic_small(shape=shape, so=so, nt=nt, nbl=6)
    p.vdamp = float(p.model["vp"].max()) * 1000.0
    d_obs = oracle.Problem(p).forward()
    p0 = synth.Problem(**{**p.__dict__, "model": synth.smooth_model(p.model, 3.0)})
    return p, p0, d_obs


@pytest.mark.parametrize("shape", [(30, 26, 34), (30, 26, 36)])
def test_gradient_parity_and_checkpoint_modes(wp, shape):
    _, p0, d_obs = grad_problem(shape)
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
    np.testing.assert_array_equal(res[wp.SNAP_CKPT_FP32][0], g)
    assert rel(res[wp.SNAP_CKPT_BF16][0], g_ref) <= 2e-2
    assert rel(res[wp.SNAP_CKPT_FP16][0], g_ref) <= 2e-3


def test_backward_matches_oracle(wp):
    """prop_forward_saved + prop_backward: dJ/dm and dJ/dwavelet for an
    arbitrary trace cotangent."""
    _, p0, _ = grad_problem((30, 26, 36), nt=60)
    resid = np.random.default_rng(9).standard_normal((p0.rec.shape[0], p0.nt)).astype(np.float32)
    g_ref, q_ref = oracle.Problem(p0).backward(resid)
    prop = wp.Propagator.from_problem(p0)
    prop.forward(p0.wavelet, p0.src, p0.rec, save=True)
    g, q = prop.backward(resid, nsrc=p0.src.shape[0])
    assert rel(g, g_ref) <= 1e-4
    assert rel(q, q_ref) <= TOL


@pytest.mark.parametrize("shape", SHAPES)
def test_state_steps_match_oracle(wp, shape):
    """prop_set_state + prop_step (forward and transposed: the same map for
    the symmetric Laplacian) against the oracle's source-free steps."""
    p = synth.acoustic_small(shape=shape, so=12)
    prop = wp.Propagator.from_problem(p)
    u0, u1 = synth.random_state(2, prop.grid, 11)
    ref0, ref1 = oracle.Problem(p).ac_run_d(u0, u1, 7)
    for adjoint in (False, True):
        prop.set_state([u1, u0])            # u^n, u^{n-1}
        prop.step(7, adjoint=adjoint)
        st = prop.get_state()
        assert rel(st[0], ref1) <= TOL and rel(st[1], ref0) <= TOL


def test_determinism(wp):
    p = synth.acoustic_small(shape=SHAPES[1], so=8, nt=40)
    prop = wp.Propagator.from_problem(p)
    np.testing.assert_array_equal(prop.forward(p.wavelet, p.src, p.rec), prop.forward(p.wavelet, p.src, p.rec))


def test_one_step_sampled_full_size(wp):
    """Industry-scale grid (800x800x400 + 40-cell layer = 880x880x480), space
    order 12, the launch configuration of the benchmark: one step from a
    seeded random state; the oracle evaluates it at sampled points
    (interior, faces, edges, corners)."""
    from test_gpu_tti import assert_pointwise, sample_points
    nx, ny, nz, nbl, h = 800, 800, 400, 40, 12.5
    vp = np.random.default_rng(78).uniform(1.5, 4.5, (nx, ny, nz)).astype(np.float32)
    dt = synth.cfl_dt(h, float(vp.max()))
    p = synth.Problem(synth.ACOUSTIC, nx, ny, nz, nbl, h, 12, 10, dt, {"vp": vp},
                      np.zeros((1, 3), np.float32), np.zeros((1, 10), np.float32),
                      np.zeros((1, 3), np.float32))
    prop = wp.Propagator.from_problem(p)
    shape = prop.grid
    rng = np.random.default_rng(6)
    state = [rng.standard_normal(shape, dtype=np.float32) for _ in range(2)]
    prop.set_state(state)                # u^n, u^{n-1}
    prop.step(1)
    out = prop.get_state()[0]
    prop.close()
    idx = sample_points(shape, 400, 7)
    ref = oracle.ac_step_points(p, (state[1], state[0]), idx)
    assert_pointwise(out.reshape(-1)[idx], ref, "u")


def test_rtm_stack_matches_oracle(wp):
    """RTM over several shots: per-shot dJ/dm from one batched call, stacked on
    the device into the global image at each window's offset; against the
    oracle's per-shot gradients added at the same offsets."""
    import torch
    shots = synth.acoustic_rtm_shots(nshots=3, nt=60, size_range=(20, 28), nz=24, h=12.5, nbl=6,
                                     so=8, f0=25.0, global_cells=(48, 40, 30))
    dev = torch.device("cuda", 0)
    stack = torch.zeros((48, 40, 24), dtype=torch.float32, device=dev)
    ref = np.zeros((48, 40, 24))
    props, dobs = [], []
    for true, p0, off in shots:
        d = oracle.Problem(true).forward()
        g, _ = oracle.Problem(p0).gradient(d)
        ox, oy, oz = off
        ref[ox:ox + p0.nx, oy:oy + p0.ny, oz:oz + p0.nz] += g
        props.append(wp.Propagator.from_problem(p0))
        dobs.append(d.astype(np.float32))
    outs = [torch.zeros((p.nx, p.ny, p.nz), dtype=torch.float32, device=dev) for _, p, _ in shots]
    grads, _ = wp.gradient_batch(props, [p.wavelet for _, p, _ in shots], [p.src for _, p, _ in shots],
                                 [p.rec for _, p, _ in shots], dobs, outs=outs)
    for prop, (_, _, off), g in zip(props, shots, grads):
        prop.stack_image(g, stack, off)
    assert rel(stack.cpu().numpy(), ref) <= 1e-4
    # a window that does not fit is rejected
    with pytest.raises(wp.PropError):
        props[0].stack_image(outs[0], stack, (47, 0, 0))

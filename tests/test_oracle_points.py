"""Pins of the oracle's point evaluators (one step at chosen grid points, the
references of the full-size sampled GPU tests) against its whole-grid step
on small random problems: every point of the computational grid, absorbing
layer, faces, edges and corners included.  The two evaluate the same
recursion (Sec. III-A for TTI in both operator forms, Sec. II-A Eq. (acou),
Sec. IV for elastic) along different code paths: per point with the
derivatives of the neighbours formed on the fly, and array-wide with the
first-derivative fields stored."""
import numpy as np
import pytest

import oracle
import synth


def random_state(shape, n, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return [(scale * rng.standard_normal(shape)).astype(np.float32) for _ in range(n)]


def tti_problem(so, op, shape=(9, 8, 10), nbl=3, h=10.0, seed=5):
    rng = np.random.default_rng(seed)
    f = lambda lo, hi: rng.uniform(lo, hi, shape).astype(np.float32)
    eps = f(0.0, 0.3)
    m = {"vp": f(1.5, 4.5), "eps": eps, "delta": (eps * f(0.0, 0.5)).astype(np.float32),
         "theta": f(0.0, 40 * synth.DEG), "phi": f(0.0, 90 * synth.DEG)}
    dt = synth.cfl_dt(h, float(np.max(m["vp"] * np.sqrt(1 + 2 * m["eps"]))))
    z3 = np.zeros((1, 3), np.float32)
    p = synth.Problem(synth.TTI, *shape, nbl, h, so, 10, dt, m, z3, np.zeros((1, 10), np.float32), z3)
    p.tti_op = op
    return p


@pytest.mark.parametrize("op", [0, 1])
@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("so", [4, 8])
def test_tti_points_equal_grid_step(so, op, adjoint):
    p = tti_problem(so, op)
    o = oracle.Problem(p)
    p0, p1, r0, r1 = random_state(o.shape, 4, 11 + so + op)
    p2, r2 = o.tti_step(p0, p1, r0, r1, adjoint=adjoint)
    idx = np.arange(p2.size, dtype=np.int64)
    got = oracle.tti_step_points(p, (p0, p1, r0, r1), idx, adjoint=adjoint)
    ref = np.stack([p2.reshape(-1), r2.reshape(-1)], axis=1)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_tti_point_forms_differ():
    """The operator flag reaches the point evaluator: the two forms give
    different steps on the same state (the staggered pair changes the
    diagonal terms)."""
    outs = []
    for op in (0, 1):
        p = tti_problem(8, op)
        st = random_state(oracle.Problem(p).shape, 4, 3)
        idx = np.arange(200, dtype=np.int64)
        outs.append(oracle.tti_step_points(p, st, idx))
    assert np.max(np.abs(outs[0] - outs[1])) > 1e-3 * np.max(np.abs(outs[0]))


@pytest.mark.parametrize("so", [4, 12])
def test_acoustic_points_equal_grid_step(so):
    shape, nbl, h = (10, 9, 11), 6, 10.0
    vp = np.random.default_rng(2).uniform(1.5, 4.5, shape).astype(np.float32)
    dt = synth.cfl_dt(h, float(vp.max()))
    z3 = np.zeros((1, 3), np.float32)
    p = synth.Problem(synth.ACOUSTIC, *shape, nbl, h, so, 10, dt, {"vp": vp}, z3,
                      np.zeros((1, 10), np.float32), z3)
    o = oracle.Problem(p)
    u0, u1 = random_state(o.shape, 2, 4)
    ref = o.ac_run_d(u0, u1, 1)[1].reshape(-1)
    got = oracle.ac_step_points(p, (u0, u1), np.arange(ref.size, dtype=np.int64))
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_elastic_points_equal_grid_step():
    shape, nbl, h = (9, 10, 8), 4, 10.0
    rng = np.random.default_rng(9)
    vp = rng.uniform(1.5, 4.5, shape).astype(np.float32)
    model = {"vp": vp, "vs": (vp / 1.73).astype(np.float32),
             "rho": rng.uniform(1.0, 2.5, shape).astype(np.float32)}
    dt = synth.cfl_dt(h, float(vp.max()))
    z3 = np.zeros((1, 3), np.float32)
    p = synth.Problem(synth.ELASTIC, *shape, nbl, h, 8, 10, dt, model, z3, np.zeros((1, 10), np.float32), z3)
    o = oracle.Problem(p)
    state = random_state(o.shape, 3, 5) + random_state(o.shape, 6, 6, scale=1e7)
    ref = o.el_step(np.stack(state)).reshape(9, -1).T
    got = oracle.el_step_points(p, state, np.arange(ref.shape[0], dtype=np.int64))
    for c in range(9):
        assert np.max(np.abs(got[:, c] - ref[:, c])) <= 1e-12 * np.max(np.abs(ref[:, c])), c

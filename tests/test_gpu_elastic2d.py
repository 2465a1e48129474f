"""GPU parity of the 2D elastic propagator (x-z plane; Sec. IV-A system, 2D
example of Sec. IV-B) against the FP64 oracle: relative L2 <= 1e-5 on
traces, adjoint outputs and stepped states."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5
E2 = (0, 2, 3, 5, 7)       # oracle slots of vx, vz, txx, tzz, txz


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def wp():
    import paper_2004_10519_gb300 as wp
    wp.lib()
    return wp


@pytest.mark.parametrize("so", [4, 8, 12, 16])
def test_forward_parity(wp, so):
    p = synth.elastic2d_small(so=so)
    tr = wp.Propagator.from_problem(p).forward(p.wavelet, p.src, p.rec)
    assert rel(tr, oracle.Problem(p).forward()) <= TOL


@pytest.mark.parametrize("so", [8, 12])
def test_adjoint_parity_and_dot(wp, so):
    p = synth.elastic2d_small(so=so, nt=60)
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


def test_state_steps_match_oracle(wp):
    p = synth.elastic2d_small(so=8)
    prop = wp.Propagator.from_problem(p)
    rs = synth.random_state(5, prop.grid, 13)
    prop.set_state(rs)
    prop.step(9)
    got = prop.get_state()
    o = oracle.Problem(p)
    s = np.zeros((9,) + o.shape)
    for c, a in zip(E2, rs):
        s[c] = a
    ref = o.el2_run_d(s, 9)
    for i, c in enumerate(E2):
        assert rel(got[i], ref[c]) <= TOL, i
    with pytest.raises(wp.PropError) as e:
        prop.step(1, adjoint=True)
    assert e.value.code == wp.PROP_EINVAL


def test_marine_water_layer(wp):
    """Water layer (mu = 0) over an elastic subsurface, the structure of the
    2D example: pressure traces at 5 m depth against the oracle."""
    p = synth.marine_elastic_2d(nx=161, nz=101, h=5.0, nbl=20, nt=300, water_depth=150.0, rec_dx=20.0)
    tr = wp.Propagator.from_problem(p).forward(p.wavelet, p.src, p.rec)
    assert rel(tr, oracle.Problem(p).forward()) <= TOL


def test_rejected_calls(wp):
    p = synth.elastic2d_small(so=8, nt=30)
    prop = wp.Propagator.from_problem(p)
    d = np.zeros((p.rec.shape[0], p.nt), np.float32)
    with pytest.raises(wp.PropError) as e:
        prop.gradient(p.wavelet, p.src, p.rec, d)
    assert e.value.code == wp.PROP_EINVAL
    rec = p.rec.copy()
    rec[0, 1] = 5.0                        # off the x-z plane
    with pytest.raises(wp.PropError) as e:
        prop.forward(p.wavelet, p.src, rec)
    assert e.value.code == wp.PROP_EINVAL
    tr = prop.forward(p.wavelet, p.src, p.rec)          # the handle stays usable
    assert np.isfinite(tr).all()


def test_state_steps_full_size(wp):
    """The 2D marine workload's full grid (1701 x 701 @ 5 m + 40-cell layer
    = 1781 x 781, so 8) in the launch configuration of its modelling run:
    three steps from a seeded random state against the oracle's whole-grid
    steps, every point of every field."""
    p = synth.marine_elastic_2d(nt=10)
    prop = wp.Propagator.from_problem(p)
    rng = np.random.default_rng(31)
    shape = prop.grid
    rs = [rng.standard_normal(shape).astype(np.float32) for _ in range(2)]
    rs += [(1e6 * rng.standard_normal(shape)).astype(np.float32) for _ in range(3)]
    prop.set_state(rs)
    prop.step(3)
    got = prop.get_state()
    prop.close()
    o = oracle.Problem(p)
    s = np.zeros((9,) + o.shape)
    for c, a in zip(E2, rs):
        s[c] = a
    ref = o.el2_run_d(s, 3)
    for i, c in enumerate(E2):
        assert rel(got[i], ref[c]) <= TOL, i

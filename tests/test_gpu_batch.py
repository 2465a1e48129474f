"""Batched gradients (prop_gradient_batch): shots on model windows of
different sizes, run concurrently in waves, give bitwise the gradients and
misfits of one prop_gradient call per shot; two shots are checked against
the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def wp():
    import paper_2004_10519_gb300 as wp
    wp.lib()
    return wp


def window_shots(nt=60, h=10.0, nbl=6):
    """TTI shots on windows (random offsets, different nx, ny) cut from one
    layered model, source at the window centre near the surface."""
    big = synth.layered_tti(52, 46, 36, 17, noise_sigma=3.0, smooth_sigma=1.5)
    vmax = float(np.max(big["vp"] * np.sqrt(1 + 2 * big["eps"])))
    dt = synth.cfl_dt(h, vmax)
    shots = []
    for (ox, oy, nx, ny) in [(0, 0, 30, 26), (14, 9, 36, 30), (20, 4, 28, 34)]:
        m = {k: np.ascontiguousarray(v[ox:ox + nx, oy:oy + ny]) for k, v in big.items()}
        src = np.array([[nx * h / 2 + 0.7, ny * h / 2 - 1.3, 3.2 * h]], np.float32)
        rec = synth.carpet_receivers(4.1, 5.3, 3.0 * h, 8, 6, 1.7 * h)
        p = synth.Problem(synth.TTI, nx, ny, 36, nbl, h, 8, nt, dt, m, src,
                          synth.ricker(22.0, dt, nt)[None], rec)
        p.vdamp = vmax * 1000.0
        d_obs = oracle.Problem(p).forward()
        p0 = synth.Problem(**{**p.__dict__, "model": synth.smooth_model(p.model, 3.0)})
        shots.append((p0, d_obs.astype(np.float32)))
    return shots


def elastic_shot(nt=50):
    nx, ny, nz, h = 22, 20, 24, 10.0
    m = synth.random_elastic(nx, ny, nz, 8, 3.0)
    dt = synth.cfl_dt(h, float(m["vp"].max()))
    src = np.array([[nx * h / 2 + 0.4, ny * h / 2, nz * h / 2 - 0.6]], np.float32)
    rec = synth.carpet_receivers(3.3, 4.4, 3.3 * h, 6, 5, 0.0)
    p = synth.Problem(synth.ELASTIC, nx, ny, nz, 4, h, 8, nt, dt, m, src,
                      synth.ricker(20.0, dt, nt)[None], rec)
    d_obs = oracle.Problem(p).forward()
    start = synth.random_elastic(nx, ny, nz, 5, 3.0)
    start = {k: (0.5 * (start[k] + m[k])).astype(np.float32) for k in start}
    return synth.Problem(**{**p.__dict__, "model": start}), d_obs.astype(np.float32)


@pytest.fixture(scope="module")
def shots():
    return window_shots() + [elastic_shot()]


@pytest.mark.parametrize("budget", [0, 1])
def test_batch_equals_one_call_per_shot(wp, shots, budget):
    """budget 0: one wave of four concurrent shots; budget 1: every shot its
    own wave."""
    ref = []
    for p, d in shots:
        prop = wp.Propagator.from_problem(p)
        ref.append(prop.gradient(p.wavelet, p.src, p.rec, d))
        prop.close()
    props = [wp.Propagator.from_problem(p) for p, _ in shots]
    grads, J = wp.gradient_batch(props, [p.wavelet for p, _ in shots], [p.src for p, _ in shots],
                                 [p.rec for p, _ in shots], [d for _, d in shots],
                                 budget_bytes=budget)
    for i, (g, j) in enumerate(zip(grads, J)):
        np.testing.assert_array_equal(g, ref[i][0], err_msg=f"shot {i}")
        assert j == ref[i][1], i
    shared, alone = wp.batch_stats()
    if budget == 0:     # the three TTI shots share one launch per pass and step
        assert shared > 0 and alone == 0, (shared, alone)
    else:               # one shot per wave: nothing to share
        assert shared == 0 and alone == 0, (shared, alone)
    # the handles stay usable after the batch
    p, d = shots[0]
    again = props[0].gradient(p.wavelet, p.src, p.rec, d)
    np.testing.assert_array_equal(again[0], ref[0][0])
    for pr in props:
        pr.close()


def test_batch_two_shots_against_oracle(wp, shots):
    sel = [shots[0], shots[2]]
    props = [wp.Propagator.from_problem(p) for p, _ in sel]
    grads, J = wp.gradient_batch(props, [p.wavelet for p, _ in sel], [p.src for p, _ in sel],
                                 [p.rec for p, _ in sel], [d for _, d in sel])
    for (p, d), g, j in zip(sel, grads, J):
        g_ref, J_ref = oracle.Problem(p).gradient(d.astype(np.float64))
        assert abs(j - J_ref) <= 1e-5 * J_ref
        assert rel(g, g_ref) <= 1e-4


def test_batch_reports_failing_shot(wp, shots):
    """A shot whose observed data has the wrong receiver count is rejected
    by the argument check of its own call; the error names the shot and the
    other shots still produce their gradients."""
    (p, d), (p2, d2) = shots[0], shots[1]
    props = [wp.Propagator.from_problem(p), wp.Propagator.from_problem(p2)]
    import paper_2004_10519_gb300 as m
    with pytest.raises(m.PropError) as e:
        m.gradient_batch(props, [p.wavelet, p2.wavelet], [p.src, p2.src], [p.rec, p2.rec[:0]],
                         [d, d2])
    assert "shot 1" in str(e.value)
    for pr in props:
        pr.close()


@pytest.mark.parametrize("snap", [0, 2])
def test_trim_releases_work_arrays_only(wp, shots, snap):
    """prop_trim keeps the model: a trimmed handle gives bitwise the traces
    and gradient of a fresh one, and its state restarts at zero."""
    p0, d = shots[1]
    prop = wp.Propagator.from_problem(p0, snap_mode=snap, ckpt_interval=7)
    tr = prop.forward(p0.wavelet, p0.src, p0.rec)
    g, J = prop.gradient(p0.wavelet, p0.src, p0.rec, d)
    prop.trim()
    assert all(np.all(f == 0) for f in prop.get_state())
    prop.trim()
    np.testing.assert_array_equal(prop.forward(p0.wavelet, p0.src, p0.rec), tr)
    prop.trim()
    g2, J2 = prop.gradient(p0.wavelet, p0.src, p0.rec, d)
    np.testing.assert_array_equal(g2, g)
    assert J2 == J


def test_shared_launch_with_different_step_sequences(wp, shots):
    """Shots whose sweeps differ (full storage against FP32 checkpoints: the
    adjoint sweep of the second recomputes forward steps between its adjoint
    steps) still meet at every step: rounds of one kind share a launch,
    mixed rounds are launched shot by shot, and every gradient is bitwise
    that of its own prop_gradient call."""
    sel = [shots[0], shots[1], shots[2]]
    modes = [wp.SNAP_FULL_FP32, wp.SNAP_CKPT_FP32, wp.SNAP_FULL_FP32]
    ref = []
    for (p, d), mode in zip(sel, modes):
        prop = wp.Propagator.from_problem(p, snap_mode=mode, ckpt_interval=7)
        ref.append(prop.gradient(p.wavelet, p.src, p.rec, d))
        prop.close()
    props = [wp.Propagator.from_problem(p, snap_mode=mode, ckpt_interval=7) for (p, _), mode in zip(sel, modes)]
    grads, J = wp.gradient_batch(props, [p.wavelet for p, _ in sel], [p.src for p, _ in sel],
                                 [p.rec for p, _ in sel], [d for _, d in sel])
    shared, alone = wp.batch_stats()
    assert shared > 0 and alone > 0, (shared, alone)
    for i, (g, j) in enumerate(zip(grads, J)):
        np.testing.assert_array_equal(g, ref[i][0], err_msg=f"shot {i}")
        assert j == ref[i][1], i
    for pr in props:
        pr.close()


def test_shared_launch_switch(wp, shots, monkeypatch):
    """WAVEPROP_BATCH_LAUNCH=0 keeps every shot on its own launches; the
    gradients are the same bits either way."""
    sel = shots[:3]
    out = {}
    for env in ("1", "0"):
        monkeypatch.setenv("WAVEPROP_BATCH_LAUNCH", env)
        props = [wp.Propagator.from_problem(p) for p, _ in sel]
        out[env] = wp.gradient_batch(props, [p.wavelet for p, _ in sel], [p.src for p, _ in sel],
                                     [p.rec for p, _ in sel], [d for _, d in sel])
        out[env + "stats"] = wp.batch_stats()
        for pr in props:
            pr.close()
    assert out["1stats"][0] > 0 and out["0stats"] == (0, 0)
    for a, b in zip(out["1"][0], out["0"][0]):
        np.testing.assert_array_equal(a, b)
    assert out["1"][1] == out["0"][1]


@pytest.mark.parametrize("nt", [60, 61])
@pytest.mark.parametrize("graphs", ["1", "0"])
def test_forward_batch_equals_one_call_per_shot(wp, monkeypatch, nt, graphs):
    """prop_forward_batch: TTI shots on windows of different sizes advance in
    lockstep (one launch of each pass per step over all shots, two steps
    replayed from a CUDA graph); traces and final states are bitwise those
    of one prop_forward per shot, for even and odd nt (odd: a last step
    outside the graph) and with the graph off."""
    monkeypatch.setenv("WAVEPROP_GRAPHS", graphs)
    sel = window_shots(nt=nt)
    ref, st_ref = [], []
    for p, _ in sel:
        prop = wp.Propagator.from_problem(p)
        ref.append(prop.forward(p.wavelet, p.src, p.rec))
        st_ref.append(prop.get_state())
        prop.close()
    props = [wp.Propagator.from_problem(p) for p, _ in sel]
    trs = wp.forward_batch(props, [p.wavelet for p, _ in sel], [p.src for p, _ in sel], [p.rec for p, _ in sel])
    for i, (t, r) in enumerate(zip(trs, ref)):
        assert np.max(np.abs(r)) > 0
        np.testing.assert_array_equal(t, r, err_msg=f"shot {i}")
        for a, b in zip(props[i].get_state(), st_ref[i]):
            np.testing.assert_array_equal(a, b)
    for pr in props:
        pr.close()


def test_forward_batch_mixed_shots_fall_back(wp, shots):
    """A shot set that cannot advance in lockstep (here a TTI and an elastic
    shot) runs one prop_forward after another, with the same results."""
    sel = [shots[0], shots[3]]
    ref = []
    for p, _ in sel:
        prop = wp.Propagator.from_problem(p)
        ref.append(prop.forward(p.wavelet, p.src, p.rec))
        prop.close()
    props = [wp.Propagator.from_problem(p) for p, _ in sel]
    trs = wp.forward_batch(props, [p.wavelet for p, _ in sel], [p.src for p, _ in sel], [p.rec for p, _ in sel])
    for t, r in zip(trs, ref):
        np.testing.assert_array_equal(t, r)
    for pr in props:
        pr.close()


def elastic_window_shots(nt=50, h=10.0, nbl=4):
    """Elastic shots on windows of different sizes cut from one random model
    (computational nz 32: the TMA-fed passes), starting model halfway to
    another random model."""
    big = synth.random_elastic(40, 36, 24, 8, 3.0)
    other = synth.random_elastic(40, 36, 24, 5, 3.0)
    dt = synth.cfl_dt(h, float(big["vp"].max()))
    out = []
    for (ox, oy, nx, ny) in [(0, 0, 22, 20), (10, 6, 28, 26), (14, 12, 24, 22)]:
        m = {k: np.ascontiguousarray(v[ox:ox + nx, oy:oy + ny]) for k, v in big.items()}
        src = np.array([[nx * h / 2 + 0.4, ny * h / 2, 24 * h / 2 - 0.6]], np.float32)
        rec = synth.carpet_receivers(3.3, 4.4, 3.3 * h, 6, 5, 0.0)
        p = synth.Problem(synth.ELASTIC, nx, ny, 24, nbl, h, 8, nt, dt, m, src, synth.ricker(20.0, dt, nt)[None], rec)
        d_obs = oracle.Problem(p).forward()
        start = {k: (0.5 * (other[k][ox:ox + nx, oy:oy + ny] + m[k])).astype(np.float32) for k in m}
        out.append((synth.Problem(**{**p.__dict__, "model": start}), d_obs.astype(np.float32)))
    return out


@pytest.mark.parametrize("snap", [0, 1])
def test_elastic_batch_shares_launches(wp, monkeypatch, snap):
    """Elastic shots of one wave share their steps' launches (forward steps:
    the velocity and stress passes over all shots; transposed steps with
    imaging: the three passes, with the pointwise kernels per shot); the
    gradients are bitwise those of one prop_gradient per shot, with full
    storage and with FP32 checkpoints (recomputed forward steps), here with
    one host thread per shot (WAVEPROP_LOCKSTEP=0)."""
    monkeypatch.setenv("WAVEPROP_LOCKSTEP", "0")
    sel = elastic_window_shots()
    ref = []
    for p, d in sel:
        prop = wp.Propagator.from_problem(p, snap_mode=snap, ckpt_interval=7)
        ref.append(prop.gradient(p.wavelet, p.src, p.rec, d))
        prop.close()
    props = [wp.Propagator.from_problem(p, snap_mode=snap, ckpt_interval=7) for p, _ in sel]
    grads, J = wp.gradient_batch(props, [p.wavelet for p, _ in sel], [p.src for p, _ in sel],
                                 [p.rec for p, _ in sel], [d for _, d in sel])
    shared, alone = wp.batch_stats()
    assert shared > 0 and alone == 0, (shared, alone)
    for i, (g, j) in enumerate(zip(grads, J)):
        assert np.max(np.abs(ref[i][0])) > 0
        np.testing.assert_array_equal(g, ref[i][0], err_msg=f"shot {i}")
        assert j == ref[i][1], i
    for pr in props:
        pr.close()


@pytest.mark.parametrize("snap,interval", [(1, 7), (2, 7), (2, 6), (3, 5)],
                         ids=["fp32ckpt-K7", "bf16-K7", "bf16-K6", "fp16-K5"])
@pytest.mark.parametrize("graphs", ["1", "0"])
def test_lockstep_gradient_batch_is_bitwise(wp, monkeypatch, snap, interval, graphs):
    """A wave of TTI shots with checkpoints and one sweep runs in lockstep
    from one host thread: per step one launch of each pass over all shots,
    full segments replayed from CUDA graphs (two arrangements of the state
    when K is odd; a partial first adjoint segment and, for K = 7, a
    partial last forward segment launched directly).  Gradients and misfits
    are bitwise those of one prop_gradient per shot and of the per-thread
    batch (WAVEPROP_LOCKSTEP=0), with graphs on and off."""
    monkeypatch.setenv("WAVEPROP_GRAPHS", graphs)
    sel = window_shots(nt=60)
    kw = dict(snap_mode=snap, ckpt_interval=interval)
    ref = []
    for p, d in sel:
        prop = wp.Propagator.from_problem(p, **kw)
        ref.append(prop.gradient(p.wavelet, p.src, p.rec, d))
        prop.close()
    out = {}
    for lock in ("1", "0"):
        monkeypatch.setenv("WAVEPROP_LOCKSTEP", lock)
        props = [wp.Propagator.from_problem(p, **kw) for p, _ in sel]
        out[lock] = wp.gradient_batch(props, [p.wavelet for p, _ in sel], [p.src for p, _ in sel],
                                      [p.rec for p, _ in sel], [d for _, d in sel])
        out[lock + "stats"] = wp.batch_stats()
        # the handles stay usable after the batch
        p, d = sel[0]
        np.testing.assert_array_equal(props[0].gradient(p.wavelet, p.src, p.rec, d)[0], ref[0][0])
        for pr in props:
            pr.close()
    assert out["1stats"][0] > 0 and out["1stats"][1] == 0, out["1stats"]
    for i in range(len(sel)):
        assert np.max(np.abs(ref[i][0])) > 0
        for lock in ("1", "0"):
            np.testing.assert_array_equal(out[lock][0][i], ref[i][0], err_msg=f"shot {i} lockstep {lock}")
            assert out[lock][1][i] == ref[i][1], (i, lock)


@pytest.mark.parametrize("nt", [50, 51])
@pytest.mark.parametrize("graphs", ["1", "0"])
def test_forward_batch_elastic_equals_one_call_per_shot(wp, monkeypatch, nt, graphs):
    """prop_forward_batch with elastic shots: one launch of the velocity and
    of the stress pass per step over all shots (the state updated in place),
    steps replayed from a CUDA graph; traces and final states bitwise those
    of one prop_forward per shot, for even and odd nt and with the graph off."""
    monkeypatch.setenv("WAVEPROP_GRAPHS", graphs)
    sel = elastic_window_shots(nt=nt)
    ref, st_ref = [], []
    for p, _ in sel:
        prop = wp.Propagator.from_problem(p)
        ref.append(prop.forward(p.wavelet, p.src, p.rec))
        st_ref.append(prop.get_state())
        prop.close()
    props = [wp.Propagator.from_problem(p) for p, _ in sel]
    trs = wp.forward_batch(props, [p.wavelet for p, _ in sel], [p.src for p, _ in sel], [p.rec for p, _ in sel])
    for i, (t, r) in enumerate(zip(trs, ref)):
        assert np.max(np.abs(r)) > 0
        np.testing.assert_array_equal(t, r, err_msg=f"shot {i}")
        for a, b in zip(props[i].get_state(), st_ref[i]):
            np.testing.assert_array_equal(a, b)
    for pr in props:
        pr.close()


@pytest.mark.parametrize("snap,interval", [(1, 7), (2, 6), (3, 5)], ids=["fp32ckpt-K7", "bf16-K6", "fp16-K5"])
@pytest.mark.parametrize("graphs", ["1", "0"])
def test_elastic_lockstep_gradient_batch_is_bitwise(wp, monkeypatch, snap, interval, graphs):
    """A wave of elastic shots with checkpoints runs in lockstep from one
    host thread (fixed tables of the forward step and of the transposed step
    at every segment position; full segments replayed from a CUDA graph, the
    partial first adjoint segment launched directly): gradients (lambda, mu,
    b) and misfits bitwise those of one prop_gradient per shot and of the
    per-thread batch, with graphs on and off."""
    monkeypatch.setenv("WAVEPROP_GRAPHS", graphs)
    sel = elastic_window_shots()
    kw = dict(snap_mode=snap, ckpt_interval=interval)
    ref = []
    for p, d in sel:
        prop = wp.Propagator.from_problem(p, **kw)
        ref.append(prop.gradient(p.wavelet, p.src, p.rec, d))
        prop.close()
    out = {}
    for lock in ("1", "0"):
        monkeypatch.setenv("WAVEPROP_LOCKSTEP", lock)
        props = [wp.Propagator.from_problem(p, **kw) for p, _ in sel]
        out[lock] = wp.gradient_batch(props, [p.wavelet for p, _ in sel], [p.src for p, _ in sel],
                                      [p.rec for p, _ in sel], [d for _, d in sel])
        out[lock + "stats"] = wp.batch_stats()
        for pr in props:
            pr.close()
    assert out["1stats"][0] > 0 and out["1stats"][1] == 0, out["1stats"]
    for i in range(len(sel)):
        assert np.max(np.abs(ref[i][0])) > 0
        for lock in ("1", "0"):
            np.testing.assert_array_equal(out[lock][0][i], ref[i][0], err_msg=f"shot {i} lockstep {lock}")
            assert out[lock][1][i] == ref[i][1], (i, lock)


@pytest.mark.parametrize("kind", ["tti", "elastic"])
def test_replayed_graphs_count_their_launches(wp, monkeypatch, kind):
    """prop_last_launches counts the launches a replayed CUDA graph holds:
    after a lockstep gradient wave and a lockstep forward batch every shot
    reports the same launch count with graphs as with direct launches."""
    monkeypatch.setenv("WAVEPROP_LOCKSTEP", "1")
    sel = window_shots(nt=60) if kind == "tti" else elastic_window_shots()
    kw = dict(snap_mode=wp.SNAP_CKPT_BF16, ckpt_interval=6)
    counts = {}
    for graphs in ("1", "0"):
        monkeypatch.setenv("WAVEPROP_GRAPHS", graphs)
        props = [wp.Propagator.from_problem(p, **kw) for p, _ in sel]
        wp.gradient_batch(props, [p.wavelet for p, _ in sel], [p.src for p, _ in sel],
                          [p.rec for p, _ in sel], [d for _, d in sel])
        assert wp.batch_stats()[0] > 0
        grad = [pr.last_launches() for pr in props]
        wp.forward_batch(props, [p.wavelet for p, _ in sel], [p.src for p, _ in sel], [p.rec for p, _ in sel])
        fwd = [pr.last_launches() for pr in props]
        counts[graphs] = (grad, fwd)
        for pr in props:
            pr.close()
    assert counts["1"] == counts["0"], counts
    # at least one stencil launch per step and shot
    nt = sel[0][0].nt
    assert min(counts["0"][0]) >= 2 * nt and min(counts["0"][1]) >= nt, counts

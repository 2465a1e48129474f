"""Failure detection without a GPU fault.  Every failure here is made on the
host: a bounded device wait that nothing completes, an allocation that the
library's fault hook fails, a time step above the stability bound, and a
NaN written into the state through the public API.  Each returns its status
code, and the CUDA context stays usable afterwards."""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_expired_wait_reports_timeout_and_context_survives():
    import paper_2004_10519_gb300 as wp
    wp.lib()
    p = synth.acoustic_small(shape=(30, 26, 36), nbl=6, so=8, nt=40)
    prop = wp.Propagator.from_problem(p)
    ref = prop.forward(p.wavelet, p.src, p.rec)
    t0 = time.perf_counter()
    with pytest.raises(wp.PropError) as e:
        prop.selftest_wait(0.2)
    assert e.value.code == wp.PROP_ETIMEOUT
    assert 0.15 <= time.perf_counter() - t0 < 10.0
    with pytest.raises(wp.PropError) as e:
        prop.forward(p.wavelet, p.src, p.rec)
    assert e.value.code == wp.PROP_ESTATE
    prop.close()
    fresh = wp.Propagator.from_problem(p)
    np.testing.assert_array_equal(fresh.forward(p.wavelet, p.src, p.rec), ref)


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("kind", ["tti", "elastic"])
def test_injected_allocation_failure_returns_enomem_without_leak(monkeypatch, kind):
    """WAVEPROP_FAULT=alloc fails every device allocation of the library.
    prop_create and the calls that allocate work arrays, sparse tables and
    staging buffers return PROP_ENOMEM, the handle stays usable, and device
    memory returns to its starting level once the handles are destroyed."""
    import paper_2004_10519_gb300 as wp
    wp.lib()
    if kind == "tti":
        p = synth.tti_two_layer(n=24, nbl=6, so=8, nt=40)
    else:
        p = synth.elastic_random(n=24, nbl=6, so=8, nt=40, corr_len=60.0, rec_dx=40.0)
        p.rec = synth.line_receivers(10.0, 20.0, 8, 95.0, 5.0)
    # warm-up cycle: CUDA loads each kernel's module (device memory for its
    # code) at the first launch, which must not count as a leak
    w = wp.Propagator.from_problem(p)
    tr = w.forward(p.wavelet, p.src, p.rec)
    w.gradient(p.wavelet, p.src, p.rec, 0.5 * tr)
    w.close()
    before = _free_bytes()
    monkeypatch.setenv("WAVEPROP_FAULT", "alloc")
    with pytest.raises(wp.PropError) as e:
        wp.Propagator.from_problem(p)
    assert e.value.code == wp.PROP_ENOMEM
    assert _free_bytes() == before
    monkeypatch.delenv("WAVEPROP_FAULT")
    prop = wp.Propagator.from_problem(p)
    ref = prop.forward(p.wavelet, p.src, p.rec)
    prop.trim()                                    # work arrays go; the next call must allocate
    monkeypatch.setenv("WAVEPROP_FAULT", "alloc")
    with pytest.raises(wp.PropError) as e:
        prop.forward(p.wavelet, p.src, p.rec)
    assert e.value.code == wp.PROP_ENOMEM
    d = np.zeros_like(ref)
    with pytest.raises(wp.PropError) as e:
        prop.gradient(p.wavelet, p.src, p.rec, d)
    assert e.value.code == wp.PROP_ENOMEM
    monkeypatch.delenv("WAVEPROP_FAULT")
    np.testing.assert_array_equal(prop.forward(p.wavelet, p.src, p.rec), ref)
    prop.close()
    assert _free_bytes() == before


@pytest.mark.parametrize("kind", ["tti", "elastic", "acoustic"])
def test_time_step_above_stability_bound_is_rejected(kind):
    """prop_create returns PROP_EUNSTABLE when dt exceeds the scheme's CFL
    bound (and accepts a dt just below the bound)."""
    import paper_2004_10519_gb300 as wp
    wp.lib()
    if kind == "tti":
        p = synth.tti_two_layer(n=20, nbl=4, so=8, nt=10)
    elif kind == "elastic":
        p = synth.elastic_random(n=20, nbl=4, so=8, nt=10, corr_len=60.0, rec_dx=40.0)
    else:
        p = synth.acoustic_small(shape=(20, 20, 20), nbl=4, so=8, nt=10)
    ok = wp.Propagator.from_problem(p, dt=0.0)        # the default CFL 0.4 time step
    dt0 = ok.dt
    ok.close()
    # CFL 0.4 is well inside every bound; 5x that is far outside all of them
    with pytest.raises(wp.PropError) as e:
        wp.Propagator.from_problem(p, dt=5.0 * dt0)
    assert e.value.code == wp.PROP_EUNSTABLE
    assert "stability bound" in str(e.value)
    wp.Propagator.from_problem(p, dt=1.05 * dt0).close()      # staggered elastic bound: CFL 0.449


@pytest.mark.parametrize("kind", ["tti", "acoustic"])
def test_nan_in_state_is_reported_when_checked(kind):
    """A NaN written into the state through prop_set_state is caught by the
    fused NaN/Inf flag of the update pass: prop_step returns PROP_EUNSTABLE
    with check_nan = 1 and PROP_OK without; the handle stays usable."""
    import paper_2004_10519_gb300 as wp
    wp.lib()
    if kind == "tti":
        p = synth.tti_two_layer(n=24, nbl=6, so=8, nt=20)
    else:
        p = synth.acoustic_small(shape=(28, 24, 36), nbl=6, so=8, nt=20)
    for check in (1, 0):
        prop = wp.Propagator.from_problem(p, check_nan=check)
        st = [np.zeros(prop.grid, np.float32) for _ in range(prop.nfields)]
        st[0][prop.grid[0] // 2, prop.grid[1] // 2, prop.grid[2] // 2] = np.nan
        prop.set_state(st)
        if check:
            with pytest.raises(wp.PropError) as e:
                prop.step(3)
            assert e.value.code == wp.PROP_EUNSTABLE
        else:
            prop.step(3)
        # usable afterwards: a clean forward run gives finite traces
        tr = prop.forward(p.wavelet, p.src, p.rec)
        assert np.all(np.isfinite(tr)) and np.max(np.abs(tr)) > 0
        prop.close()


@pytest.mark.parametrize("kind", ["tti", "elastic"])
def test_injected_allocation_failure_in_batches(monkeypatch, kind):
    """WAVEPROP_FAULT=alloc also fails the allocations of the batched calls
    (per-shot work arrays and the batches' device tables): prop_gradient_batch
    and prop_forward_batch, in lockstep and with one thread per shot, return
    PROP_ENOMEM, the handles stay usable and give the reference results
    afterwards, and device memory returns to its starting level."""
    import paper_2004_10519_gb300 as wp
    wp.lib()
    if kind == "tti":
        ps = [synth.tti_two_layer(n=24 + 4 * i, nbl=6, so=8, nt=40) for i in range(2)]
    else:
        ps = [synth.elastic_random(n=24 + 4 * i, nbl=6, so=8, nt=40, corr_len=60.0, rec_dx=40.0) for i in range(2)]
        for p in ps:
            p.rec = synth.line_receivers(10.0, 20.0, 8, 95.0, 5.0)
    kw = dict(snap_mode=wp.SNAP_CKPT_BF16, ckpt_interval=6)
    args = lambda: ([p.wavelet for p in ps], [p.src for p in ps], [p.rec for p in ps])

    def run(lock):
        monkeypatch.setenv("WAVEPROP_LOCKSTEP", lock)
        props = [wp.Propagator.from_problem(p, **kw) for p in ps]
        trs = wp.forward_batch(props, *args())
        g, J = wp.gradient_batch(props, *args(), [0.5 * t for t in trs])
        return props, trs, g

    # warm-up: loads the modules of every kernel involved
    for lock in ("1", "0"):
        props, trs, g = run(lock)
        for q in props:
            q.close()
    before = _free_bytes()
    for lock in ("1", "0"):
        monkeypatch.setenv("WAVEPROP_LOCKSTEP", lock)
        props = [wp.Propagator.from_problem(p, **kw) for p in ps]
        ref = wp.forward_batch(props, *args())
        gref, _ = wp.gradient_batch(props, *args(), [0.5 * t for t in ref])
        for q in props:
            q.trim()
        monkeypatch.setenv("WAVEPROP_FAULT", "alloc")
        with pytest.raises(wp.PropError) as e:
            wp.forward_batch(props, *args())
        assert e.value.code == wp.PROP_ENOMEM, lock
        with pytest.raises(wp.PropError) as e:
            wp.gradient_batch(props, *args(), [0.5 * t for t in ref])
        assert e.value.code == wp.PROP_ENOMEM, lock
        monkeypatch.delenv("WAVEPROP_FAULT")
        trs = wp.forward_batch(props, *args())
        g, _ = wp.gradient_batch(props, *args(), [0.5 * t for t in ref])
        for i in range(2):
            np.testing.assert_array_equal(trs[i], ref[i])
            np.testing.assert_array_equal(g[i], gref[i])
        for q in props:
            q.close()
        assert _free_bytes() == before, lock

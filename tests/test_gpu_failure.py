"""Failure detection without a GPU fault: a bounded device wait that nothing
completes gives up after its limit, the call returns PROP_ETIMEOUT, the
handle reports PROP_ESTATE afterwards, and the CUDA context stays usable
(a new handle computes the same traces as before)."""
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

"""prop_step replays pairs of steps from a CUDA graph captured once per
handle, state buffers, direction and tile size: bitwise the states of
direct launches (WAVEPROP_GRAPHS=0), for every propagator, an odd step
count, repeated calls and a handle trimmed in between."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def problems():
    from test_gpu_paths import el_problem, tti_problem
    return {"tti": tti_problem(nt=10), "tti_sp": tti_problem(nt=10), "elastic": el_problem(nt=10),
            "acoustic": synth.acoustic_small(shape=(30, 26, 36), nbl=6, so=12, nt=10),
            "elastic2d": synth.elastic2d_small(so=8, nt=10)}


@pytest.mark.parametrize("kind", ["tti", "tti_sp", "elastic", "acoustic", "elastic2d"])
def test_graph_steps_bitwise(kind, monkeypatch):
    import paper_2004_10519_gb300 as wp
    wp.lib()
    p = problems()[kind]
    if kind == "tti_sp":
        p.tti_op = 1
    dirs = [False] if kind == "elastic2d" else [False, True]
    for adjoint in dirs:
        out = {}
        for tag, env in (("graph", "1"), ("direct", "0")):
            monkeypatch.setenv("WAVEPROP_GRAPHS", env)      # 1: a failed capture raises
            prop = wp.Propagator.from_problem(p)
            st = synth.random_state(prop.nfields, prop.grid, 5)
            prop.set_state(st)
            prop.step(7, adjoint=adjoint)
            prop.step(6, adjoint=adjoint)
            if tag == "graph":
                prop.trim()
                prop.set_state(st)
                prop.step(13, adjoint=adjoint)
            out[tag] = [np.array(f) for f in prop.get_state()]
            prop.close()
        # graph path: 13 steps after trim = the direct path's 7 + 6 steps
        for a, b in zip(out["graph"], out["direct"]):
            np.testing.assert_array_equal(a, b)

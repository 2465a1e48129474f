"""C ABI checks that need no GPU: the library builds/loads, exports every
function declared in include/waveprop.h and include/waveprop_diag.h (and no
other prop_ symbol), and the binding's prop_desc layout matches the C
compiler's."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "waveprop.h")
DIAG_HEADER = os.path.join(ROOT, "include", "waveprop_diag.h")


def _declared(path=HEADER):
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(prop_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2004_10519_gb300 import _build
    return _build.build()


def test_header_declares_entry_points():
    names = _declared()
    for n in ("prop_create", "prop_forward", "prop_adjoint", "prop_gradient", "prop_destroy",
              "prop_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(\w+)", out))
    declared = _declared() + _declared(DIAG_HEADER)
    missing = [n for n in declared if n not in exported]
    assert not missing, missing
    # every exported prop_ function is declared in one of the two headers
    undeclared = sorted(n for n in exported if n.startswith("prop_") and n not in declared)
    assert not undeclared, undeclared
    # and the binding lists exactly the headers' functions
    import paper_2004_10519_gb300 as wp
    assert sorted(wp.ABI_SYMBOLS) == _declared()
    assert sorted(wp.DIAG_SYMBOLS) == _declared(DIAG_HEADER)
    assert not set(_declared()) & set(_declared(DIAG_HEADER))


def test_library_loads_without_gpu(libpath):
    L = C.CDLL(libpath)
    for n in _declared() + _declared(DIAG_HEADER):
        assert hasattr(L, n)
    # calls that touch no device: NULL-safe destroy and error queries
    L.prop_destroy(None)
    L.prop_last_error.restype = C.c_char_p
    L.prop_last_error.argtypes = [C.c_void_p]
    assert isinstance(L.prop_last_error(None), bytes)


def test_prop_desc_layout_matches_binding():
    import paper_2004_10519_gb300 as wp
    fields = [f[0] for f in wp.PropDesc._fields_]
    prog = '#include <stdio.h>\n#include <stddef.h>\n#include "waveprop.h"\nint main(void){\n'
    prog += 'printf("%zu\\n", sizeof(prop_desc));\n'
    for f in fields:
        prog += f'printf("%zu\\n", offsetof(prop_desc, {f}));\n'
    prog += "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(src, "w").write(prog)
        subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), src, "-o", exe])
        vals = [int(v) for v in subprocess.check_output([exe]).split()]
    assert vals[0] == C.sizeof(wp.PropDesc)
    for f, off in zip(fields, vals[1:]):
        assert getattr(wp.PropDesc, f).offset == off, f


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_2004_10519_gb300 as wp
    monkeypatch.setattr(wp, "_lib", None)
    monkeypatch.setattr(wp, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        wp.lib()


def test_wave_plan_first_fit_in_order(libpath):
    """Host-side wave planner of the batched gradients: shots keep their
    order, a wave never exceeds the budget unless one shot alone does."""
    import paper_2004_10519_gb300 as wp
    assert wp.plan_waves([5, 3, 4, 10, 1, 1], 8) == ([0, 0, 1, 2, 3, 3], 4)
    assert wp.plan_waves([], 8) == ([], 0)
    assert wp.plan_waves([9], 8) == ([0], 1)
    assert wp.plan_waves([1] * 5, 100) == ([0] * 5, 1)
    rng = __import__("numpy").random.default_rng(1)
    b = [int(x) for x in rng.integers(1, 50, 40)]
    waves, n = wp.plan_waves(b, 60)
    assert waves == sorted(waves) and n == waves[-1] + 1
    for w in range(n):
        tot = sum(x for x, k in zip(b, waves) if k == w)
        assert tot <= 60
    L = wp.lib()
    assert L.prop_plan_waves(None, -1, 10, None) == wp.PROP_EINVAL
    assert L.prop_gradient_bytes(None, 10) == 0
    assert L.prop_tile_planes(None) == 0
    assert L.prop_tile_rows(None) == 0


def test_batch_argument_checks_need_no_gpu(libpath):
    import paper_2004_10519_gb300 as wp
    L = wp.lib()
    n = None
    assert L.prop_gradient_batch(n, 0, n, n, n, n, n, n, n, n, 0) == wp.PROP_OK
    assert L.prop_gradient_batch(n, -1, n, n, n, n, n, n, n, n, 0) == wp.PROP_EINVAL
    assert L.prop_gradient_batch(n, 2, n, n, n, n, n, n, n, n, 0) == wp.PROP_EINVAL
    handles = (C.c_void_p * 2)(None, None)
    arr = (C.c_void_p * 2)()
    ints = (C.c_int * 2)(1, 1)
    rc = L.prop_gradient_batch(handles, 2, arr, arr, ints, arr, ints, arr, arr, None, 0)
    assert rc == wp.PROP_EINVAL
    assert b"shot handle 0 is NULL" in L.prop_last_error(None)


def test_create_rejects_bad_descriptors_without_gpu(libpath):
    """prop_create validates the descriptor before any device call: each
    bad field returns PROP_EINVAL with a message naming it, no handle."""
    import paper_2004_10519_gb300 as wp
    L = wp.lib()
    dummy = (C.c_float * 1)()
    models = (C.c_void_p * 5)(*[C.cast(dummy, C.c_void_p)] * 5)

    def desc(**kw):
        d = dict(kind=wp.PROP_TTI, nx=8, ny=8, nz=8, nbl=2, h=10.0, space_order=8, nt=10, dt=0.0, vdamp=0.0,
                 snap_mode=0, ckpt_interval=0, check_nan=0, tti_operator=0)
        d.update(kw)
        return wp.PropDesc(**d)

    cases = [(dict(kind=7), b"kind must be"),
             (dict(kind=wp.PROP_ELASTIC2D, ny=3), b"ny = 1"),
             (dict(tti_operator=2), b"tti_operator"),
             (dict(kind=wp.PROP_ELASTIC, tti_operator=1), b"tti_operator"),
             (dict(nx=0), b"grid sizes"),
             (dict(nbl=-1), b"nbl"),
             (dict(h=0.0), b"h must be"),
             (dict(h=float("nan")), b"h must be"),
             (dict(space_order=6), b"space_order"),
             (dict(nt=1), b"nt must be"),
             (dict(snap_mode=4), b"snap_mode"),
             (dict(ckpt_interval=-2), b"ckpt_interval"),
             (dict(nx=2048, ny=2048, nz=1024), b"2^32")]
    for kw, msg in cases:
        h = C.c_void_p()
        rc = L.prop_create(C.byref(desc(**kw)), models, None, C.byref(h))
        assert rc == wp.PROP_EINVAL, kw
        assert h.value is None, kw
        assert msg in L.prop_last_error(None), (kw, L.prop_last_error(None))
    h = C.c_void_p()
    assert L.prop_create(C.byref(desc()), None, None, C.byref(h)) == wp.PROP_EINVAL
    assert b"model is NULL" in L.prop_last_error(None)
    assert L.prop_create(None, models, None, C.byref(h)) == wp.PROP_EINVAL
    assert L.prop_create(C.byref(desc()), models, None, None) == wp.PROP_EINVAL


def test_noalloc_rejects_huge_grids_without_gpu(libpath):
    """prop_forward_noalloc checks every size before it multiplies them or
    touches the device: axes whose product would wrap, grids of 2^32 points
    or more, and grids whose fields exceed the static array all return
    PROP_EINVAL (no CUDA call is made, so this runs without a GPU)."""
    import paper_2004_10519_gb300 as wp
    L = wp.lib()
    vp = C.c_void_p
    L.prop_forward_noalloc.argtypes = [C.POINTER(wp.PropDesc), C.POINTER(vp), vp, vp, C.c_int,
                                       vp, C.c_int, vp, vp]
    buf = (C.c_float * 16)()
    p = C.cast(buf, vp)
    models = (vp * 5)(*[p] * 5)
    big = 2 ** 31 - 100
    cases = [((big, big, big, 40), b"grid axis too long"),
             ((2 ** 20, 2 ** 20, 8, 0), b"2^32"),
             ((65536, 65536, 2, 0), b"2^32"),
             ((2048, 2048, 1024, 0), b"2^32"),
             ((200, 200, 200, 10), b"MiB"),
             ((1000, 1000, 10, 0), b"MiB")]
    for kind in (wp.PROP_TTI, wp.PROP_ELASTIC):
        for (nx, ny, nz, nbl), msg in cases:
            d = wp.PropDesc(kind, nx, ny, nz, nbl, 10.0, 8, 10, 0.0, 0.0, 0, 0, 0, 0)
            rc = L.prop_forward_noalloc(C.byref(d), models, p, p, 1, p, 1, p, None)
            assert rc == wp.PROP_EINVAL, (kind, nx, ny, nz)
            assert msg in L.prop_last_error(None), (kind, nx, L.prop_last_error(None))


def test_diag_hooks_reject_null_without_gpu(libpath):
    """The measurement hooks of include/waveprop_diag.h check their arguments
    before touching a device."""
    import threading
    L = C.CDLL(libpath)
    vp = C.c_void_p
    L.prop_profile.argtypes = [vp, C.c_int]
    L.prop_kernel_stats.argtypes = [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
    L.prop_kernel_time.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
    L.prop_last_launches.restype = C.c_longlong
    L.prop_last_launches.argtypes = [vp]
    L.prop_fp32_peak.argtypes = [C.POINTER(C.c_double)]
    L.prop_selftest_wait.argtypes = [vp, C.c_float]
    L.prop_batch_stats.argtypes = [C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
    EINVAL = -1
    assert L.prop_profile(None, 1) == EINVAL
    assert L.prop_kernel_stats(None, 0, None, None) == EINVAL
    assert L.prop_kernel_time(None, None, None) == EINVAL
    assert L.prop_last_launches(None) == 0
    assert L.prop_fp32_peak(None) == EINVAL
    assert L.prop_selftest_wait(None, 0.1) == EINVAL
    # the batch counters belong to the calling thread: zero in a new one
    out = []

    def reader():
        a, b = C.c_longlong(-7), C.c_longlong(-7)
        out.append((L.prop_batch_stats(C.byref(a), C.byref(b)), a.value, b.value))
        out.append(L.prop_batch_stats(None, None))

    t = threading.Thread(target=reader)
    t.start()
    t.join()
    assert out == [(0, 0, 0), 0]


def test_headers_compile_as_c_and_cxx():
    """Both headers are self-contained C (and C++): a translation unit that
    includes only waveprop_diag.h takes the address of every declared
    function with the declared types."""
    names = _declared() + _declared(DIAG_HEADER)
    body = "".join(f"    p[{i}] = (void (*)(void)){n};\n" for i, n in enumerate(names))
    prog = ('#include "waveprop_diag.h"\nint main(void){\n'
            f"    void (*p[{len(names)}])(void);\n{body}"
            "    return PROP_K_GROUPS == 8 && p[0] != 0 ? 0 : 1;\n}\n")
    with tempfile.TemporaryDirectory() as d:
        for lang, cc, ext in (("c", "gcc", ".c"), ("c++", "g++", ".cpp")):
            src = os.path.join(d, "t" + ext)
            open(src, "w").write(prog)
            subprocess.check_call([cc, "-std=c11" if lang == "c" else "-std=c++17", "-Wall", "-Werror",
                                   "-fsyntax-only", "-I", os.path.dirname(HEADER), src])

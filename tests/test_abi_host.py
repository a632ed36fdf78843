"""Host-side checks of libsmre.so that need no GPU: the library loads, exports
every entry point include/smre.h declares, computes the Sec. 2.1 bounds on
the host like the oracle does, and rejects bad arguments before touching CUDA.
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def smre():
    from paper_1503_03492_gb300 import build as b
    b.build()
    import paper_1503_03492_gb300 as m
    return m


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"SMRE_API[^;(]*?\b(smre_\w+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(smre):
    declared = _declared()
    assert "smre_dykstra_create" in declared and "smre_dykstra_project_incomplete" in declared
    lib = ctypes.CDLL(smre.lib_path())
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(smre.EXPORTED) == declared


def test_version(smre):
    assert "sm_103a" in smre.smre_version()


@pytest.mark.parametrize("mode,omode", [(0, "perset"), (1, "chi2")])
def test_host_bounds_match_oracle(smre, oracle_mod, mode, omode):
    sides = list(range(1, 17))
    for alpha in (0.5, 0.9, 0.99):
        p = smre.make_params(64, 64, sides, alpha=alpha, cmode=mode)
        got = np.array(smre.smre_bounds(p))
        ref = oracle_mod.bounds(sides, alpha, omode)
        assert np.allclose(got, ref, rtol=1e-12, atol=0), (alpha, got - ref)


def test_host_bounds_explicit_and_order(smre):
    p = smre.make_params(32, 32, [4, 1, 2], cmode=smre.SMRE_C_EXPLICIT, c_explicit=[5.0, 1.5, 3.0])
    assert smre.smre_bounds(p) == [5.0, 1.5, 3.0]


def test_repeated_side_needs_the_same_bound(smre):
    """A side listed twice is ignored when it repeats its bound; with two
    different explicit bounds the call fails (no schedule could honour both)."""
    p = smre.make_params(32, 32, [2, 1, 2], cmode=smre.SMRE_C_EXPLICIT, c_explicit=[3.0, 1.5, 3.0])
    assert smre.smre_bounds(p) == [3.0, 1.5, 3.0]
    p = smre.make_params(32, 32, [2, 1, 2], cmode=smre.SMRE_C_EXPLICIT, c_explicit=[3.0, 1.5, 4.0])
    with pytest.raises(smre.SmreError) as ei:
        smre.smre_bounds(p)
    assert ei.value.status == smre.SMRE_EINVAL and "twice" in str(ei.value)


def test_batch_schedule_flags_and_flag_rows(smre):
    """Batch flags are validated on the host: SMRE_BF_PER_SIDE is accepted
    alone and with a spread, an unknown bit or both spreads at once are not
    (image_bytes answers 0 for invalid parameters), and no flag changes an
    image's footprint."""
    sides = [1, 2, 3, 8]
    ok = [0, smre.SMRE_BF_PER_SIDE, smre.SMRE_BF_PER_SIDE | smre.SMRE_BF_SPREAD4,
          smre.SMRE_BF_PER_SIDE | smre.SMRE_BF_AUTOTUNE]
    sizes = {f: smre.smre_batch_image_bytes(smre.make_batch_params(sides, flags=f), 300, 200) for f in ok}
    assert len(set(sizes.values())) == 1 and sizes[0] > 0        # flags do not change the layout
    for bad in (16, smre.SMRE_BF_SPREAD2 | smre.SMRE_BF_SPREAD4, 1 << 20):
        assert smre.smre_batch_image_bytes(smre.make_batch_params(sides, flags=bad), 300, 200) == 0, bad
    # every part of the footprint, the flag row included, starts 256-byte aligned
    assert sizes[0] % 256 == 0


@pytest.mark.parametrize("kw,msg", [
    (dict(H=0, W=8, sides=[1]), "out of range"),
    (dict(H=8, W=5000, sides=[1]), "width"),
    (dict(H=8, W=8, sides=[9]), "window side"),
    (dict(H=40, W=40, sides=[33]), "window side"),
    (dict(H=8, W=8, sides=[0]), "window side"),
    (dict(H=8, W=8, sides=[1], alpha=1.0), "alpha"),
    (dict(H=8, W=8, sides=[1], max_cycles=0), "max_cycles"),
    (dict(H=8, W=8, sides=[1], tol=float("nan")), "NaN"),
    (dict(H=8, W=8, sides=[1, 2], cmode=3, c_explicit=[1.0, -2.0]), "positive"),
])
def test_create_rejects_bad_arguments_without_cuda(smre, kw, msg):
    H, W, sides = kw.pop("H"), kw.pop("W"), kw.pop("sides")
    p = smre.make_params(H, W, sides, **kw)
    with pytest.raises(smre.SmreError) as ei:
        smre.smre_dykstra_create(p)
    assert ei.value.status == smre.SMRE_EINVAL
    assert msg in str(ei.value)


def test_null_handle_calls_fail_cleanly(smre):
    lib = smre.load()
    assert lib.smre_dykstra_project(None, None, None, None) == smre.SMRE_EINVAL
    assert lib.smre_dykstra_set_stopping(None, 1, 0.0, 0) == smre.SMRE_EINVAL
    assert lib.smre_dykstra_device_bytes(None) == 0
    lib.smre_dykstra_destroy(None)
    assert b"NULL" in lib.smre_last_error(None)


def test_product_package_does_not_reach_the_oracle():
    """The product package neither imports nor links the oracle."""
    pkg = os.path.join(ROOT, "paper_1503_03492_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, fn
                assert "smre_oracle" not in txt and "liboracle" not in txt, fn


def test_admm_rejects_bad_parameters(smre):
    # validation happens before any CUDA call
    p = smre.make_params(32, 32, [1, 2])
    for kw in ({"sigma": -1.0}, {"sigma": 1.0, "radius": 17}, {"sigma": 1.0, "rho1": 0.0},
               {"sigma": 1.0, "gamma": 1.0}, {"sigma": 1.0, "max_iters": 0},
               {"sigma": 1.0, "tv_iters": -1}):
        with pytest.raises(smre.SmreError) as ei:
            smre.smre_admm_create(p, smre.make_admm_params(**kw))
        assert ei.value.status == smre.SMRE_EINVAL


def test_missing_library_fails_loudly(tmp_path):
    # the binding has no fallback: without libsmre.so every call raises
    import subprocess
    import sys
    code = (
        "import paper_1503_03492_gb300 as m\n"
        f"m.lib_path = lambda: {str(tmp_path / 'libsmre.so')!r}\n"
        "try:\n"
        "    m.smre_version()\n"
        "except ImportError as e:\n"
        "    print('raised', e)\n"
    )
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("raised"), r.stdout + r.stderr

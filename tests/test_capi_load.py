"""The C-ABI library loads without a GPU and exports every function that
include/crgb.h declares; the parameter defaults agree with the oracle's."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "crgb.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(cr_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2310_17274_gb300 import build, crgb
    build.build_library()
    return crgb.lib()


def test_every_declared_symbol_is_exported(lib):
    from paper_2310_17274_gb300 import crgb
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), f"{n} declared in crgb.h but not exported"
        assert n in crgb.SIGNATURES, f"{n} has no binding"


def test_defaults_match_oracle(lib, oracle_mod):
    import numpy as np
    from paper_2310_17274_gb300 import crgb
    a = crgb.params_default()
    b = oracle_mod.params_default()
    for k, v in b.items():
        if k == "alpha":
            assert np.allclose(a[k], v)
        else:
            assert a[k] == pytest.approx(v, rel=1e-7), k


def test_version_and_error_string(lib):
    assert b"sm_103a" in lib.cr_version()
    assert isinstance(lib.cr_last_error(), bytes)


def test_bad_descriptions_are_rejected_without_gpu(lib):
    """Validation runs on the host before any device call."""
    import numpy as np
    from paper_2310_17274_gb300 import crgb, synth
    rb = synth.make_robot(synth.SPHERES_42)
    bad = synth.Robot(**{**rb.__dict__, "axis": np.array([0, 1, 2, 3, 0, 1, 2], np.int32)})
    with pytest.raises(crgb.CrError, match="axis"):
        crgb.Robot(bad)
    bad = synth.Robot(**{**rb.__dict__, "pairs": np.array([[0, 0]], np.int32)})
    with pytest.raises(crgb.CrError, match="pair"):
        crgb.Robot(bad)
    w = synth.World(pose=np.array([[0, 0, 0, 0, 0, 0, 0.0]]), half_ext=np.ones((1, 3)))
    with pytest.raises(crgb.CrError, match="quaternion"):
        crgb.World(w)
    w = synth.World(pose=np.array([[0, 0, 0, 1, 0, 0, 0.0]]), half_ext=np.array([[1, 0, 1.0]]))
    with pytest.raises(crgb.CrError, match="half extents"):
        crgb.World(w)

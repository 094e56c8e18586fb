"""Host-side checks of the C-ABI library that need no GPU: it loads, exports every
entry point declared in include/csgs.h, and its pure host calls behave."""
import ctypes
import os
import re

import pytest

import paper_2607_02721_b300 as csgs
from paper_2607_02721_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return csgs.lib()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "csgs.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(csgs_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(csgs.EXPORTS)


def test_build_targets_sm103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_default_opts_are_the_rasteriser_conventions(lib):
    o = csgs.default_opts()
    assert o.resolution == csgs.RES_PIXEL and o.variant == csgs.VAR_L1
    assert abs(o.alpha_min - 1 / 255) < 1e-9 and abs(o.rho_max - 0.99) < 1e-7
    assert abs(o.t_min - 1e-4) < 1e-10 and o.cut2 == 9.0 and abs(o.dilation - 0.3) < 1e-7
    assert list(o.obj_w) == [1.0, 1.0, 1.0]


def test_struct_layouts_match_header(lib):
    # csgs_camera is 80 bytes; csgs_scene_desc 56; csgs_score_opts 52; csgs_stats 184
    assert ctypes.sizeof(csgs.Camera) == 80
    assert ctypes.sizeof(csgs.SceneDesc) == 56
    assert ctypes.sizeof(csgs.ScoreOpts) == 52
    assert ctypes.sizeof(csgs.Stats) == 184


def test_null_arguments_are_rejected_without_a_device(lib):
    assert lib.csgs_create(None, 0, None) == csgs.CSGS_E_INVAL
    assert lib.csgs_score(None, 0, None, None, None) == csgs.CSGS_E_INVAL
    assert lib.csgs_sync(None) == csgs.CSGS_E_INVAL
    lib.csgs_destroy(None)


def test_theorem_helpers(lib):
    import math

    S, eps, delta, nq = 120.5, 0.2, 0.05, 131072
    assert csgs.theorem2_sample_size(S, eps, delta, nq) == math.ceil(3 * S / eps ** 2 * math.log(2 * nq / delta))
    assert csgs.theorem2_sample_size(0.0, eps, delta, nq) == 0.0
    g, e = 0.1, 0.05
    assert abs(csgs.theorem3_eps(g, e) - max(1 - math.exp(-g) * (1 - e), math.exp(g) * (1 + e) - 1)) < 1e-15
    assert csgs.theorem3_eps(0.0, e) == pytest.approx(e)

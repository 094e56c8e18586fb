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
    assert o.tile_shape == csgs.TILE_AUTO and o.view_batch == 0 and o.persist_ctas == 0 and o.accumulate == 0


def test_struct_layouts_match_header(lib, tmp_path):
    """Every field offset and struct size of the binding's ctypes structs equals the C
    compiler's layout of include/csgs.h (a small C program built with gcc prints them)."""
    import shutil
    import subprocess

    structs = {"csgs_camera": csgs.Camera, "csgs_scene_desc": csgs.SceneDesc,
               "csgs_score_opts": csgs.ScoreOpts, "csgs_stats": csgs.Stats, "csgs_tuning": csgs.Tuning}
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "csgs.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)
    assert ctypes.sizeof(csgs.ScoreOpts) == 64


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

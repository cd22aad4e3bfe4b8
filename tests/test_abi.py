"""The C ABI library builds, loads and exports every entry point of include/gs.h (no GPU)."""
import ctypes as C
import os
import re
import subprocess
import textwrap

import pytest

from paper_2504_02437_gb300 import _native as N
from paper_2504_02437_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gs.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^GS_API [^(]*?\b(gs_\w+)\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return N.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(N.SIGNATURES), "binding and header disagree"


def test_nothing_else_is_exported():
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert exported == set(_declared())


def test_struct_layouts_match_header(tmp_path):
    """Compile a C probe against gs.h and compare sizeof/offsetof with the ctypes mirrors."""
    src = tmp_path / "probe.c"
    fields_cam = [f[0] for f in N.gs_camera._fields_]
    fields_cfg = [f[0] for f in N.gs_config._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gs.h"', 'int main(void) {',
             'printf("cam %zu\\n", sizeof(gs_camera));', 'printf("cfg %zu\\n", sizeof(gs_config));']
    lines += [f'printf("cam.{f} %zu\\n", offsetof(gs_camera, {f}));' for f in fields_cam]
    lines += [f'printf("cfg.{f} %zu\\n", offsetof(gs_config, {f}));' for f in fields_cfg]
    lines += ["return 0; }"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(ln.split() for ln in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    assert int(got["cam"]) == C.sizeof(N.gs_camera)
    assert int(got["cfg"]) == C.sizeof(N.gs_config)
    for f in fields_cam:
        assert int(got[f"cam.{f}"]) == getattr(N.gs_camera, f).offset, f
    for f in fields_cfg:
        assert int(got[f"cfg.{f}"]) == getattr(N.gs_config, f).offset, f


def test_default_config_is_the_documented_reading(lib):
    cfg = N.gs_config()
    lib.gs_default_config(C.byref(cfg))
    assert cfg.reg_floor == pytest.approx(0.01)            # Eq. 10
    assert cfg.lambda_photo == 0.0                          # pure L1 unless the SSIM term is asked for
    assert cfg.alpha_min == pytest.approx(1 / 255)
    assert cfg.alpha_max == pytest.approx(0.99)
    assert cfg.T_min == pytest.approx(1e-4)
    assert cfg.dilation == pytest.approx(0.3)
    assert cfg.near_z == pytest.approx(0.2)
    assert cfg.insert_opacity == pytest.approx(0.99)
    assert cfg.split_thresh == pytest.approx(2e-4)


def test_create_rejects_bad_config_without_gpu(lib):
    """Argument checks run before any device call."""
    cfg = N.gs_config()
    lib.gs_default_config(C.byref(cfg))
    cfg.capacity = 0
    ctx = C.c_void_p()
    assert lib.gs_create(C.byref(cfg), 0, C.byref(ctx)) == N.GS_ERR_ARG
    cfg.capacity = 1000
    cfg.tile_size = 12
    assert lib.gs_create(C.byref(cfg), 0, C.byref(ctx)) == N.GS_ERR_ARG
    assert lib.gs_last_error(None) == b"null context"


def test_product_path_has_no_oracle_dependency():
    """The package never imports the oracle (it is test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_2504_02437_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in txt.replace("Oracle", "oracle").split("import")[0] or "import oracle" not in txt
                assert "from oracle" not in txt and "import oracle" not in txt, f

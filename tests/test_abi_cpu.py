"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every entry point declared in include/zpic.h, and validates
configurations before it touches the device."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2106_12485_gb300 import zpic as Z
from paper_2106_12485_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(Z.LIB_PATH):
        from paper_2106_12485_gb300 import build
        build.build()
    return Z.lib()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(zpic_\w+)\s*\(", text,
                             flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("zpic_create", "zpic_step", "zpic_get_fields_f32",
              "zpic_get_particles", "zpic_energy", "zpic_destroy",
              "zpic_batch_create", "zpic_batch_step"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", Z.LIB_PATH],
                         capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = declared_symbols() - exported
    assert not missing, missing
    for n in declared_symbols():
        assert hasattr(lib, n)


def test_version_and_strerror(lib):
    assert lib.zpic_version() == 1
    assert lib.zpic_strerror(Z.ECFL) == b"time step violates the Courant condition"
    assert lib.zpic_strerror(12345) == b"unknown error"


def create_code(cfg):
    h = C.c_void_p()
    return Z.lib().zpic_create(C.byref(cfg), C.byref(h))


def test_config_validation_before_device(lib):
    good = W.uniform_thermal()
    # CFL: dt >= 1/sqrt(1/dx^2+1/dy^2) = 0.0707 for dx=dy=0.1
    bad = W.uniform_thermal(dt=0.0708)
    assert create_code(bad) == Z.ECFL
    ok = W.uniform_thermal(dt=0.0707)
    assert create_code(ok) != Z.ECFL
    c = W.uniform_thermal()
    c.nx = 2
    assert create_code(c) == Z.EINVAL
    c = W.uniform_thermal()
    c.moving_window = 1          # needs an open x boundary
    assert create_code(c) == Z.EINVAL
    c = W.uniform_thermal()
    c.species[0].ppc_x = 0
    assert create_code(c) == Z.EINVAL
    c = W.uniform_thermal()
    c.tile_x = 65
    assert create_code(c) == Z.EINVAL
    c = W.uniform_thermal()
    c.precision = 7
    assert create_code(c) == Z.EINVAL
    c = W.uniform_thermal()
    c.species[0].q_over_m = 0.0
    assert create_code(c) == Z.EINVAL
    # LWFA workload passes its own CFL check (dt = 0.019 < 0.0199)
    assert create_code(W.lwfa()) != Z.ECFL
    assert good.dt == 0.07
    assert lib.zpic_create(None, None) == Z.EINVAL


def test_null_handles(lib):
    assert lib.zpic_step(None, 1) == Z.EINVAL
    assert lib.zpic_sync(None) == Z.EINVAL
    assert lib.zpic_destroy(None) == Z.EINVAL
    assert lib.zpic_batch_destroy(None) == Z.EINVAL
    assert lib.zpic_set_allocator(None, C.c_void_p(1), None) == Z.EINVAL


def test_no_cpu_fallback_without_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    assert create_code(W.uniform_thermal()) == Z.ECUDA
    assert b"CUDA" in lib.zpic_last_error()

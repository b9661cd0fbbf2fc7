"""The C-ABI boundary on the CPU: the library builds, loads and exports every entry point
include/sgp.h declares, and fails loudly without a GPU.  No compute call is made here."""

import ctypes
import os
import re
import subprocess

import pytest
import torch

from paper_2106_06695_gb300 import _lib, build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _lib.declared_functions()
    for required in ("sgp_lattice_build", "sgp_mvm", "sgp_cg_solve", "sgp_lattice_free",
                     "sgp_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (sgp_\w+)", out))
    missing = set(_lib.declared_functions()) - exported
    assert not missing, missing
    for name in _lib.declared_functions():
        assert hasattr(lib, name)


def test_version_and_defaults(lib):
    assert lib.sgp_version() == 1
    o = _lib.sgp_opts()
    lib.sgp_opts_init(ctypes.byref(o))
    assert (o.order_r, o.kernel, o.spacing_s, o.outputscale, o.value_dtype, o.check_every) == (
        1, 0, 0.0, 1.0, 0, 8)
    assert o.stream is None


def test_invalid_arguments_are_rejected_before_any_device_work(lib):
    h = ctypes.c_void_p()
    rc = lib.sgp_lattice_build(None, None, 10, 3, None, ctypes.byref(h))
    assert rc == 1 and not h.value
    assert b"lengthscales" in lib.sgp_last_error()
    assert lib.sgp_mvm(None, None, 1, None) == 1


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU failure path")
def test_no_gpu_fails_loudly(lib):
    h = ctypes.c_void_p()
    buf = (ctypes.c_float * 4)()
    rc = lib.sgp_lattice_build(ctypes.addressof(buf), ctypes.addressof(buf), 1, 3, None,
                               ctypes.byref(h))
    assert rc == 6
    assert b"no CUDA device" in lib.sgp_last_error()


def test_missing_library_raises(monkeypatch):
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", os.path.join(ROOT, "no_such_libsgp.so"))
    with pytest.raises(ImportError):
        _lib.load()


def test_product_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2106_06695_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", text, re.M), f
                assert "sgp_oracle" not in text and "liboracle" not in text, f


def test_request_bytes_bound_is_host_only_and_monotone(lib):
    b = lambda n, d, k=9, dt=0, l=0: lib.sgp_request_bytes_bound(n, d, 1, k, dt, l)  # noqa: E731
    assert b(0, 3) == 0 and b(10, 0) == 0 and b(10, 3, l=-1) == 0 and b(10, 3, l=129) == 0
    assert b(1000, 3) < b(2000, 3) < b(2000, 8)
    assert b(1000, 3, k=9) < b(1000, 3, k=20)
    assert b(100_000, 20, dt=1) < b(100_000, 20, dt=0)
    # the preconditioner adds at least its factor B (n x l fp32)
    assert b(100_000, 3, l=100) >= b(100_000, 3) + 100_000 * 100 * 4
    # at least the lattice arrays at m = n (d + 1): keys, ids, weights, neighbour table
    n, d = 50_000, 8
    D = d + 1
    m = n * D
    assert b(n, d) >= 2 * m * D + 8 * n * D + 8 * D * m + 2 * m * 12 * 4


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU failure path")
def test_server_without_gpu_fails_loudly(lib):
    o = _lib.sgp_server_opts()
    lib.sgp_server_opts_init(ctypes.byref(o))
    assert (o.max_active, o.probes, o.max_iter, o.check_every, o.hbm_budget) == (16, 8, 1000, 8, 0)
    assert (o.precond_rank, o.precond_min_kappa, o.lane_classes) == (100, 1e3, 1)
    h = ctypes.c_void_p()
    assert lib.sgp_server_create(ctypes.byref(o), ctypes.byref(h)) == 6
    assert not h.value
    o.max_active = 0
    assert lib.sgp_server_create(ctypes.byref(o), ctypes.byref(h)) == 1


def test_struct_layouts_match_the_headers(tmp_path):
    """Every struct the binding mirrors has the header's size and field offsets: a C
    program compiled against include/*.h prints them and they are compared with ctypes."""
    import shutil

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [_lib.sgp_opts, _lib.sgp_server_opts, _lib.sgp_request, _lib.sgp_request_stats]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sgp_serve.h"',
             "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in st._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {(a, b): int(c) for a, b, c in (ln.split() for ln in out.strip().splitlines())}
    for st in structs:
        name = st.__name__
        assert got[(name, "sizeof")] == ctypes.sizeof(st), name
        for f, _ in st._fields_:
            assert got[(name, f)] == getattr(st, f).offset, (name, f)

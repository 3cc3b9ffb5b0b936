"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every entry point that include/bpimd.h declares, and rejects invalid
configurations on the host before touching CUDA."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2305_18025_gb300 import bpimd, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bpimd.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bpimd_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return bpimd.load(build_if_missing=False)


def test_header_declares_the_documented_calls():
    names = declared_functions()
    for required in ("bpimd_create", "bpimd_exchange_energy_forces", "bpimd_step", "bpimd_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s+(bpimd_\w+)", out))
    for name in declared_functions():
        assert name in exported, f"{name} declared in bpimd.h but not exported"
        assert hasattr(lib, name)
    assert set(bpimd.EXPORTED) <= exported


def test_library_is_built_for_sm_103a_only():
    """The build compiles every translation unit for sm_103a and nothing else
    (one -gencode; no PTX for other targets)."""
    flags = build.FLAGS
    gencodes = [flags[i + 1] for i, f in enumerate(flags) if f == "-gencode"]
    assert gencodes == ["arch=compute_103a,code=sm_103a"]
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_config_struct_matches_header_layout():
    # N, P (2 x int32) then 3 doubles, 2 int32, 4 doubles, 2 int32, 4 doubles, uint64
    assert ctypes.sizeof(bpimd.bpimd_config) == 8 + 24 + 8 + 32 + 8 + 32 + 8
    assert bpimd.bpimd_config.dt.offset == 40
    assert bpimd.bpimd_config.seed.offset == ctypes.sizeof(bpimd.bpimd_config) - 8


@pytest.mark.parametrize("field,value", [
    ("N", 0), ("P", 1), ("m", 0.0), ("omega_P", -1.0), ("beta", float("nan")),
    ("beta", float("inf")), ("precision", 7), ("precision", 3), ("flags", 4), ("flags", 8), ("N", 16385),
    ("box_L", -1.0), ("box_L", float("nan")), ("box_L", float("inf")),
])
def test_create_rejects_invalid_config_without_gpu(lib, field, value):
    cfg = bpimd.make_config(8, 4, 1.0, 2.0, 1.0)
    setattr(cfg, field, value)
    h = ctypes.c_void_p(123)
    rc = lib.bpimd_create(ctypes.byref(h), ctypes.byref(cfg), None)
    assert rc == bpimd.BPIMD_ERR_ARG
    assert h.value is None


def test_create_rejects_a_bead_count_past_the_index_range_without_gpu(lib):
    """N P beads of 3 coordinates must index within a 32-bit signed range."""
    cfg = bpimd.make_config(6912, 110_000, 1.0, 2.0, 1.0)
    h = ctypes.c_void_p(123)
    assert lib.bpimd_create(ctypes.byref(h), ctypes.byref(cfg), None) == bpimd.BPIMD_ERR_ARG
    assert h.value is None


def test_null_handles_are_rejected(lib):
    assert lib.bpimd_create(None, None, None) == bpimd.BPIMD_ERR_ARG
    assert lib.bpimd_destroy(None) == bpimd.BPIMD_OK
    assert lib.bpimd_exchange_energy_forces(None, None, None, None) == bpimd.BPIMD_ERR_ARG
    assert lib.bpimd_sync(None) == bpimd.BPIMD_ERR_ARG
    assert lib.bpimd_step(None, None, None, 1, None) == bpimd.BPIMD_ERR_ARG


def test_status_strings(lib):
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert bpimd.bpimd_status_string(code) != "unknown status"
    assert "sm_103a" in bpimd.bpimd_version()


@pytest.mark.parametrize("case", ["R0", "N0", "Nbig", "P1", "beta0", "omega_nan", "prec"])
def test_create_batched_rejects_invalid_arguments_without_gpu(lib, case):
    import numpy as np
    N = np.array([16, 40, 7], dtype=np.int32)
    P = np.array([8, 4, 2], dtype=np.int32)
    w = np.array([2.0, 1.5, 3.0])
    b = np.array([1.0, 0.5, 2.0])
    R = 3
    cfg = bpimd.make_config(0, 0, 1.0, 1.0, 1.0)
    if case == "R0":
        R = 0
    elif case == "N0":
        N[1] = 0
    elif case == "Nbig":
        N[2] = bpimd.BPIMD_STORE_MAX_N + 1
    elif case == "P1":
        P[0] = 1
    elif case == "beta0":
        b[2] = 0.0
    elif case == "omega_nan":
        w[1] = float("nan")
    elif case == "prec":
        cfg.precision = 5
    h = ctypes.c_void_p(123)
    rc = lib.bpimd_create_batched(ctypes.byref(h), ctypes.byref(cfg), R, N.ctypes.data, P.ctypes.data,
                                  w.ctypes.data, b.ctypes.data, None)
    assert rc == bpimd.BPIMD_ERR_ARG
    assert h.value is None


def test_batch_calls_reject_null_context(lib):
    assert lib.bpimd_exchange_energy_forces_batched(None, None, None, None) == bpimd.BPIMD_ERR_ARG
    assert lib.bpimd_batch_info(None, None, None, None) == bpimd.BPIMD_ERR_ARG
    assert lib.bpimd_batch_set_tuning(None, 8, 8) == bpimd.BPIMD_ERR_ARG


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_config_struct_layout_matches_the_header(tmp_path):
    """The ctypes mirror of bpimd_config has the size and field offsets that a C
    compiler gives the struct declared in include/bpimd.h."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    names = [f[0] for f in bpimd.bpimd_config._fields_]
    prog = tmp_path / "layout.c"
    prog.write_text(
        '#include <stdio.h>\n#include "bpimd.h"\nint main(void) {\n'
        '  printf("size %zu\\n", sizeof(bpimd_config));\n'
        + "".join(f'  printf("{n} %zu\\n", offsetof(bpimd_config, {n}));\n' for n in names)
        + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(root, "include"), "-o", str(exe), str(prog)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    assert int(got["size"]) == ctypes.sizeof(bpimd.bpimd_config)
    for n in names:
        assert int(got[n]) == getattr(bpimd.bpimd_config, n).offset, n


def test_binding_argument_kinds_match_the_header_prototypes():
    """Every prototype in include/bpimd.h and the binding's ctypes argtypes for
    it agree in the number of parameters and, position by position, pointer
    against integer."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "include", "bpimd.h")).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    protos = re.findall(r"(?:^|\n)\s*(?:int|const char \*)\s*(bpimd_\w+)\s*\(([^)]*)\)\s*;", text)
    assert {name for name, _ in protos} == set(bpimd.EXPORTED)
    lib = bpimd.load()
    for name, params in protos:
        params = " ".join(params.split())
        plist = [] if params in ("", "void") else [p.strip() for p in params.split(",")]
        want = ["ptr" if "*" in p else "int" for p in plist]
        argtypes = getattr(lib, name).argtypes or []
        got = ["int" if t in (ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64) else "ptr"
               for t in argtypes]
        assert got == want, (name, plist, argtypes)


def test_header_constants_match_the_binding():
    """The storage limits and the recompute flag of bpimd.h, as the binding uses them."""
    text = open(HEADER).read()
    for name in ("BPIMD_MAX_N", "BPIMD_STORE_MAX_N", "BPIMD_FLAG_RECOMPUTE", "BPIMD_MIXED32",
                 "BPIMD_NOALLOC_MAX_N"):
        m = re.search(r"#define\s+" + name + r"\s+(\d+)", text)
        assert m, name
        assert int(m.group(1)) == getattr(bpimd, name), name

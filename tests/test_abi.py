"""The C-ABI library builds, loads and exports what include/twofluid.h declares.

CPU only: no call here reaches the GPU (only the host-side argument checks of
tf_workspace_bytes / tf_create run).
"""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2511_00445_gb300 import _binding as B
from paper_2511_00445_gb300 import build as Bld

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "twofluid.h")


@pytest.fixture(scope="module")
def lib():
    Bld.build()
    return B.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.findall(r"^[A-Za-z_][\w\s\*]*?\b(tf_\w+)\s*\(", text, flags=re.M)


def test_header_declarations_match_binding():
    decl = declared_functions()
    assert decl == B.EXPORTS


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_params_struct_layout_matches_header(tmp_path):
    names = [f[0] for f in B.TFParams._fields_]
    cnames = ["lambda" if n == "lambda_" else n for n in names]
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "twofluid.h"\nint main(void){\n'
        + f'printf("%zu\\n", sizeof(tf_params));\n'
        + "".join(f'printf("%zu\\n", offsetof(tf_params, {n}));\n' for n in cnames)
        + "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(B.TFParams)
    for n, off in zip(names, out[1:]):
        assert getattr(B.TFParams, n).offset == off, n


def _arr(*ps):
    return (B.TFParams * len(ps))(*[p.to_c() for p in ps])


def test_workspace_bytes_host_checks(lib):
    good = B.SolverParams(nx=64, ny=48)
    n = lib.tf_workspace_bytes(_arr(good), 1)
    assert n > 0 and n % 256 == 0
    n4 = lib.tf_workspace_bytes(_arr(good, good.with_(zeta=0.01), good, good), 4)
    assert n4 > n
    assert lib.tf_workspace_bytes(_arr(good.with_(nx=0)), 1) == 0
    assert lib.tf_workspace_bytes(_arr(good.with_(tau1=0.5)), 1) == 0
    assert lib.tf_workspace_bytes(_arr(good.with_(n_sub=0)), 1) == 0
    assert lib.tf_workspace_bytes(_arr(good.with_(storage=7)), 1) == 0
    assert lib.tf_workspace_bytes(_arr(good, good.with_(nx=32)), 2) == 0   # sizes must agree
    assert lib.tf_workspace_bytes(_arr(good.with_(zeta=float("nan"))), 1) == 0
    assert lib.tf_workspace_bytes(_arr(good), 0) == 0


def test_storage_modes_size_the_workspace(lib):
    """16-bit population storage halves the two population buffers; the
    storage constants agree with the header; instances must share a mode."""
    hdr = open(HEADER).read()
    consts = dict((k, int(v)) for k, v in re.findall(r"#define (TF_STORE_\w+)\s+(\d+)", hdr))
    assert consts == {"TF_STORE_F32": B.STORE_F32, "TF_STORE_F16": B.STORE_F16,
                      "TF_STORE_BF16": B.STORE_BF16}
    p = B.SolverParams(nx=64, ny=48)
    n32 = lib.tf_workspace_bytes(_arr(p), 1)
    n16 = lib.tf_workspace_bytes(_arr(p.with_(storage=B.STORE_F16)), 1)
    nb16 = lib.tf_workspace_bytes(_arr(p.with_(storage=B.STORE_BF16)), 1)
    assert n16 == nb16 > 0
    pops = 2 * 18 * 64 * 48 * 2          # two buffers, 18 planes, 2 bytes saved per element
    assert n32 - n16 == pops             # every population plane is a multiple of 256 bytes here
    assert lib.tf_workspace_bytes(_arr(p, p.with_(storage=B.STORE_F16)), 2) == 0


def test_create_rejects_bad_workspace_before_any_device_call(lib):
    good = B.SolverParams(nx=16, ny=16)
    arr = _arr(good)
    ctx = ctypes.c_void_p()
    need = lib.tf_workspace_bytes(arr, 1)
    assert lib.tf_create(arr, 1, None, need, None, ctypes.byref(ctx)) == B.TF_ERR_WORKSPACE
    assert lib.tf_create(arr, 1, ctypes.c_void_p(256 * 1000 + 8), need, None,
                         ctypes.byref(ctx)) == B.TF_ERR_WORKSPACE
    assert lib.tf_create(arr, 1, ctypes.c_void_p(256 * 1000), need - 256, None,
                         ctypes.byref(ctx)) == B.TF_ERR_WORKSPACE
    assert lib.tf_create(arr, 0, ctypes.c_void_p(256 * 1000), need, None,
                         ctypes.byref(ctx)) == B.TF_ERR_ARG
    assert ctx.value is None
    assert lib.tf_destroy(None) == B.TF_ERR_ARG
    assert lib.tf_last_error(None) == b"null context"


def test_surrogate_config_host_checks(lib):
    """tf_sur_workspace_bytes validates the configuration on the host."""
    def nbytes(**kw):
        c = dict(levels=3, base_channels=16, nx=64, ny=64, max_batch=2, max_pairs=4, horizon=10)
        c.update(kw)
        cfg = B.TFSurConfig(*[c[k] for k in ("levels", "base_channels", "nx", "ny", "max_batch",
                                              "max_pairs", "horizon")])
        return lib.tf_sur_workspace_bytes(ctypes.byref(cfg))
    base = nbytes()
    assert base > 0 and base % 256 == 0
    assert nbytes(max_pairs=8) > base                   # dataset grows with the pairs
    assert nbytes(levels=0) == 0 and nbytes(levels=6) == 0
    assert nbytes(base_channels=24) == 0                # 16, 32 or 64
    assert nbytes(nx=48) == 0                           # multiple of 8 * 2^(levels-1) = 32
    assert nbytes(max_batch=0) == 0 and nbytes(horizon=0) == 0
    assert lib.tf_sur_workspace_bytes(None) == 0


def test_ensemble_workspace_host_checks(lib):
    assert lib.tf_ensemble_workspace_bytes(0) == 0
    assert lib.tf_ensemble_workspace_bytes(65) == 0
    n1, n64 = lib.tf_ensemble_workspace_bytes(1), lib.tf_ensemble_workspace_bytes(64)
    assert 0 < n1 < n64 and n1 % 256 == 0

"""CPU-side checks of the boundary: the C-ABI library builds and loads, it
exports every function include/truss.h declares, the Python binding has the
same names, and the product package never reaches the oracle."""
import ast
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "truss.h")
PKG = os.path.join(ROOT, "paper_1205_6693_gb300")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(truss_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("truss_ctx_create", "truss_ctx_destroy", "truss_support", "truss_decompose",
                 "truss_decompose_batch", "truss_strerror", "truss_last_stats"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_1205_6693_gb300 import truss as T
    lib = ctypes.CDLL(T.load()._name)
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert missing == []


def test_binding_has_the_same_names():
    from paper_1205_6693_gb300 import truss as T
    for f in declared_functions():
        assert hasattr(T, f), f
    assert set(T.EXPORTS) <= set(declared_functions())


def test_strerror_without_gpu():
    from paper_1205_6693_gb300 import truss as T
    assert "timed out" in T.truss_strerror(T.TRUSS_ETIMEOUT)
    assert T.truss_strerror(0) == "ok"


def test_ctx_create_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1205_6693_gb300 import truss as T
    with pytest.raises(T.TrussError):
        T.truss_ctx_create(0)


def test_product_package_never_imports_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if not f.endswith(".py"):
                continue
            tree = ast.parse(open(os.path.join(dirpath, f)).read())
            for node in ast.walk(tree):
                if isinstance(node, ast.Import):
                    names = [a.name for a in node.names]
                elif isinstance(node, ast.ImportFrom):
                    names = [node.module or ""]
                else:
                    continue
                assert not any(n.split(".")[0] in ("oracle", "graphgen") for n in names), f


def test_cuda_sources_do_not_include_oracle_code():
    for f in os.listdir(os.path.join(PKG, "csrc")):
        text = open(os.path.join(PKG, "csrc", f)).read()
        assert "oracle" not in text.lower() or f.endswith(".md"), f


def test_generator_splitmix64_reference_value():
    import graphgen
    # SplitMix64 from state 0: first output (Steele, Lea & Flood 2014)
    assert graphgen.lib().gg_splitmix64(0) == 0xE220A8397B1DCDAF


def test_generator_is_deterministic():
    import numpy as np
    import graphgen
    a = graphgen.rmat_raw(10, 5000, seed=3)
    b = graphgen.rmat_raw(10, 5000, seed=3)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    n, s, d = graphgen.tiny()
    assert len(s) == 33942 and n == 4096


def test_chung_lu_sorted_selection_equals_hash_set_selection():
    import numpy as np
    import graphgen
    for n, m, cap, seed in [(5000, 40000, 500.0, 1), (30000, 300000, 3000.0, 2)]:
        a = graphgen.chung_lu(n, m, 20.0, cap, 2.1, seed=seed)
        b = graphgen.chung_lu(n, m, 20.0, cap, 2.1, seed=seed, sorted_dedup=True)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_header_is_plain_c_and_links(tmp_path):
    """include/truss.h compiles as C99 with warnings as errors, and a C client
    links against the library (no GPU needed: truss_ctx_create reports the
    missing device as an error code)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    from paper_1205_6693_gb300 import truss as T
    lib = T.load()._name
    src = tmp_path / "client.c"
    src.write_text(
        '#include "truss.h"\n#include <stdio.h>\n'
        "int main(void) {\n"
        "  truss_ctx *ctx = 0;\n"
        "  int rc = truss_ctx_create(&ctx, 0, 0);\n"
        '  printf("%d %s\\n", rc, truss_strerror(rc));\n'
        "  if (ctx) truss_ctx_destroy(ctx);\n"
        "  return 0;\n}\n")
    exe = tmp_path / "client"
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                           lib, "-Wl,-rpath," + os.path.dirname(lib)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0
    rc = int(out.stdout.split()[0])
    assert rc in (T.TRUSS_OK, T.TRUSS_ECUDA, T.TRUSS_EINVAL)


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the C header's size and the
    same name and offset for each field (a C program compiled against
    include/truss.h prints them)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    from paper_1205_6693_gb300 import truss as T
    structs = [T.truss_opts, T.truss_run_stats, T.truss_serve_opts, T.truss_req_stats,
               T.truss_serve_stats]
    lines = ['#include "truss.h"', "#include <stddef.h>", "#include <stdio.h>",
             "int main(void) {"]
    for S in structs:
        c = S.__name__
        lines.append(f'  printf("{c} size %zu\\n", sizeof({c}));')
        for f, _ in S._fields_:
            lines.append(f'  printf("{c} {f} %zu\\n", offsetof({c}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I",
                           os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60, check=True)
    got = {}
    for ln in out.stdout.splitlines():
        c, f, v = ln.split()
        got[(c, f)] = int(v)
    for S in structs:
        c = S.__name__
        assert got[(c, "size")] == ctypes.sizeof(S), c
        for f, _ in S._fields_:
            assert got[(c, f)] == getattr(S, f).offset, (c, f)


def test_binding_checks_buffer_lengths_before_any_call():
    """A per-row buffer shorter than src would be read or written past its
    end by the library: the binding refuses it before calling in."""
    import numpy as np
    from paper_1205_6693_gb300 import truss as T
    src = np.array([0, 1, 2], np.int32)
    dst = np.array([1, 2, 0], np.int32)
    short = np.zeros(2, np.int32)
    ok = np.zeros(3, np.int32)
    with pytest.raises(TypeError):
        T.truss_support_noalloc(3, src, dst, short)
    with pytest.raises(TypeError):
        T.truss_support_noalloc(3, src, short, ok)
    with pytest.raises(TypeError):
        T.truss_decompose(None, 3, src, dst, ok, short)
    with pytest.raises(TypeError):
        T.truss_support(None, 3, src, dst, short)
    with pytest.raises(TypeError):
        T.truss_core(None, 3, src, dst, short)
    with pytest.raises(TypeError):
        T.truss_decompose_batch(None, [3], [0, 3], src, dst, ok, short)
    with pytest.raises(TypeError):
        T.truss_decompose_batch(None, [3], [0, 2], src, dst, ok, ok)

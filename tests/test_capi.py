"""CPU checks of the C ABI boundary: the library builds, loads and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include"))) if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?(?:int|void|char\s*\*|const char\s*\*|int64_t)\s*\**\s*(hz\w+)\s*\(",
                            src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hz_op_create", "hz_solve", "hz_op_destroy", "hz_solve_batched", "hz_version"):
        assert required in names, names


def test_library_exports_every_declared_symbol():
    import paper_1811_03852_gb300 as hz

    lib = ctypes.CDLL(hz._build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_defaults_without_gpu():
    import paper_1811_03852_gb300 as hz

    assert hz.version() == 4
    p = hz.default_params()
    assert p.tol == 1e-8 and p.restart == 150 and p.mode == hz.HZ_MODE_MIXED_IR and p.fgmres_m == 30
    # tri-SOR defaults of Sec. 2: three sweeps, omega = 1.5; T^-1 stays the default preconditioner
    assert p.precond == hz.HZ_PRE_TRI and p.sor_sweeps == 3 and p.sor_omega == 1.5
    # tri-SOR variant tables: FP32 pass/matvec/first, FP64 the same; invalid pairs count 0
    assert [hz.sor_variant_count(hz.HZ_PREC_FP32, k) for k in range(4)] == [9, 8, 6, 0]
    assert [hz.sor_variant_count(hz.HZ_PREC_FP64, k) for k in range(4)] == [6, 5, 4, 0]
    assert hz.sor_variant_count(7, 0) == 0 and hz.sor_variant_count(hz.HZ_PREC_FP32, -1) == 0
    names = [hz.load().hz_kernel_name(k).decode() for k in range(hz.NUM_KERNELS)]
    assert names[7:] == ["k_sor_first", "k_sor_pass", "k_mv_rb", "k_rb_copy"] and hz.load().hz_kernel_name(
        hz.NUM_KERNELS).decode() == ""
    assert hz.load().hz_status_str(hz.HZ_ERR_NOT_CONVERGED).decode() == "not converged"


def test_invalid_arguments_rejected_on_host():
    import paper_1811_03852_gb300 as hz

    L = hz.load()
    h = ctypes.c_void_p()
    # sizes are validated before any CUDA call
    assert L.hz_op_create(0, 4, 4, ctypes.c_void_p(1), None, ctypes.byref(h)) == hz.HZ_ERR_INVALID
    assert L.hz_op_create(4, 4, hz_max_levels() + 1, ctypes.c_void_p(1), None, ctypes.byref(h)) == hz.HZ_ERR_INVALID
    assert L.hz_solve(None, None, None, None, None, None) == hz.HZ_ERR_INVALID
    assert L.hz_op_destroy(None) == hz.HZ_OK


def hz_max_levels():
    src = open(os.path.join(ROOT, "include", "hz.h")).read()
    return int(re.search(r"#define HZ_MAX_LEVELS (\d+)", src).group(1))


def test_product_does_not_reference_oracle():
    pkg = os.path.join(ROOT, "paper_1811_03852_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "hz_oracle" not in txt, f


def test_binding_structs_match_the_header_layout(tmp_path):
    # compile a probe against include/hz.h and compare every field offset and
    # the sizes of the two host structs with the ctypes binding
    import subprocess

    import paper_1811_03852_gb300 as hz

    structs = {"hz_solve_params": hz.hz_solve_params, "hz_solve_info": hz.hz_solve_info}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hz.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    inc = os.path.join(ROOT, "include")
    subprocess.run(["gcc", "-I", inc, "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln.strip():
            a, b, c = ln.split()
            got[(a, b)] = int(c)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)

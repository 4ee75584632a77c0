"""CPU checks of the boundary: the CUDA library builds for sm_103a, loads,
and exports every entry point include/cgdir.h declares; the binding's
struct layouts match the header.  No compute call is made (no GPU here)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1301_0970_gb300 as cg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cgdir.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cgdir_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cgdir_create", "cgdir_register", "cgdir_destroy", "cgdir_strerror"):
        assert required in names


def test_library_builds_loads_and_exports_every_declared_symbol():
    lib = cg.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(cg._SIGNATURES)


def test_strerror_and_defaults_without_gpu():
    lib = cg.load()
    assert lib.cgdir_strerror(cg.CGDIR_EINVAL) == b"invalid argument"
    p = cg.cgdir_params()
    lib.cgdir_default_params(ctypes.byref(p))
    import json
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_parameters.json")))
    assert p.levels == g["pyramid_levels"]["value"]
    assert p.sigma_fluid == p.sigma_diff == g["gaussian_sigma_voxels"]["value"]
    assert p.eps == g["stop_eps"]["value"]
    assert list(p.spacing_mm) == g["voxel_spacing_mm"]["value"]
    assert p.margin_mm == g["uroi_margin_mm"]["value"]
    assert p.contour_level_mask == 1 << (p.levels - 1)     # contour term at the finest level only


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """Compile a probe against include/cgdir.h with the host C compiler and
    compare every struct size and field offset with the ctypes mirror."""
    structs = {"cgdir_config": cg.cgdir_config, "cgdir_volume": cg.cgdir_volume,
               "cgdir_masks": cg.cgdir_masks, "cgdir_params": cg.cgdir_params,
               "cgdir_level_stats": cg.cgdir_level_stats, "cgdir_tuning": cg.cgdir_tuning,
               "cgdir_kernel_time": cg.cgdir_kernel_time}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "cgdir.h"', "int main(void){"]
    expect = []
    for name, cls in structs.items():
        lines.append(f'printf("%zu\\n", sizeof({name}));')
        expect.append(ctypes.sizeof(cls))
        for fname, _ in cls._fields_:
            cname = "lambda" if fname == "lambda_" else fname
            lines.append(f'printf("%zu\\n", offsetof({name}, {cname}));')
            expect.append(getattr(cls, fname).offset)
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got == expect


def test_null_context_is_rejected_without_touching_the_gpu():
    lib = cg.load()
    assert lib.cgdir_register(None, None, None, None, None, None, None, 0, None) == cg.CGDIR_EINVAL
    assert lib.cgdir_create(None, None) == cg.CGDIR_EINVAL
    assert lib.cgdir_tuning_load(None, None, 0) == cg.CGDIR_EINVAL
    assert lib.cgdir_smooth_compose(None, None, None, 0, 1.0, 1, 1, 1, None) == cg.CGDIR_EINVAL


def test_sources_target_sm103a_only():
    from paper_1301_0970_gb300 import build as b
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]

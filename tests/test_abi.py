"""Host-side checks of the C ABI: the library loads, exports every declared
symbol, and its pure size functions agree with the paper's printed integers.
No CUDA compute is issued here."""

import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fnr():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2103_10380_gb300 as fnr
    return fnr


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"FNR_API\s+[\w\s\*]*?\b(fnr_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol(fnr):
    import ctypes
    names = declared_symbols()
    assert len(names) >= 10
    L = ctypes.CDLL(fnr.LIB_PATH)
    for n in sorted(names):
        assert hasattr(L, n), f"{n} declared in include/ but not exported"
    # the binding knows every declared symbol, with its signature
    assert names <= set(fnr.SIGNATURES), names - set(fnr.SIGNATURES)


STRUCTS = ("fnr_cache_desc", "fnr_mlp", "fnr_cache_source", "fnr_cache_layout", "fnr_camera", "fnr_render_params",
           "fnr_ray_stats", "fnr_request", "fnr_result", "fnr_serve_config")


def test_struct_layouts_match_header(fnr, tmp_path):
    """The binding's ctypes structures have the C header's size and field offsets (gcc compiles the
    header alone: it needs no CUDA header)."""
    import ctypes
    import subprocess
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fnr.h"', 'int main(void) {']
    for name in STRUCTS:
        lines.append(f'    printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in getattr(fnr, name)._fields_:
            lines.append(f'    printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("    return 0;\n}")
    src = tmp_path / "sizes.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                 text=True).stdout.splitlines())
    for name in STRUCTS:
        S = getattr(fnr, name)
        assert int(got[name]) == ctypes.sizeof(S), name
        for fname, _ in S._fields_:
            assert int(got[f"{name}.{fname}"]) == getattr(S, fname).offset, f"{name}.{fname}"


def test_cache_bytes_paper_integers(fnr):
    """fnr_cache_bytes follows the supplementary cache-size formula (second version)."""
    with open(os.path.join(ROOT, "tests", "golden", "cache_sizes.json")) as f:
        cases = {c["formula"]: c for c in json.load(f)["cases"]}
    c = cases["fastnerf"]
    d = fnr.make_desc(c["k"], c["D"], c["l"], fnr.FNR_PREC_FP16, fnr.FNR_PREC_FP16)
    assert fnr.fnr_cache_bytes(d) == c["pos_bytes"] + c["dir_bytes"]
    # FP32 storage doubles every term; FP8 halves the position cache and adds 25 scales
    d32 = fnr.make_desc(1024, 8, 1024, fnr.FNR_PREC_FP32, fnr.FNR_PREC_FP32)
    assert fnr.fnr_cache_bytes(d32) == 2 * (c["pos_bytes"] + c["dir_bytes"])
    d8 = fnr.make_desc(1024, 8, 1024, fnr.FNR_PREC_FP8_E4M3, fnr.FNR_PREC_FP16)
    # E4M3 adds 25 binary32 scales and 24 binary16 offsets per offset brick (16 cells a side at k = 1024)
    assert fnr.fnr_cache_bytes(d8) == c["pos_bytes"] // 2 + c["dir_bytes"] + 25 * 4 + 64 ** 3 * 24 * 2


def test_cache_footprint_and_invalid_desc(fnr):
    d = fnr.make_desc(512, 8, 512, fnr.FNR_PREC_FP32, fnr.FNR_PREC_FP32)
    # 512^3 * (4 + 96) + tables: the 100-byte records already sit on 16-byte boundaries
    assert fnr.fnr_cache_footprint(d) >= 512 ** 3 * 100 + 512 * 512 * 8 * 4
    # beyond the paper's size formula: bin tables, scales, 32 KB of brick bits, 32 KB of jump distances
    assert fnr.fnr_cache_footprint(d) - fnr.fnr_cache_bytes(d) < 1 << 17
    d6 = fnr.make_desc(64, 6, 64, fnr.FNR_PREC_FP32, fnr.FNR_PREC_FP32)  # 72-byte triples padded to 80
    assert fnr.fnr_cache_footprint(d6) >= 64 ** 3 * (4 + 80)
    for bad in (fnr.make_desc(0, 8, 64), fnr.make_desc(64, 17, 64), fnr.make_desc(64, 8, 1),
                fnr.make_desc(64, 8, 64, 7), fnr.make_desc(64, 8, 64, bmin=(0, 0, 0), bmax=(1, 0, 1))):
        assert fnr.fnr_cache_bytes(bad) == 0 and fnr.fnr_cache_footprint(bad) == 0


def test_null_arguments_rejected_without_gpu(fnr):
    L = fnr.lib()
    assert L.fnr_context_create(0, 0, None) == fnr.FNR_ERR_INVALID_ARG
    assert b"NULL" in L.fnr_last_error()
    assert L.fnr_render(None, None, None, 0, None, None, None, None, None) == fnr.FNR_ERR_INVALID_ARG
    assert L.fnr_context_destroy(None) == fnr.FNR_OK


def test_binding_constants_match_header(fnr):
    """Every integer constant the header defines (status codes, precisions, layouts, render flags,
    limits) has the same value in the binding, and the binding defines no FNR_ constant the header
    lacks; the render flags are distinct bits."""
    src = open(os.path.join(ROOT, "include", "fnr.h")).read()
    header = {n: int(v) for n, v in re.findall(r"^#define\s+(FNR_\w+)\s+(\d+)u?\s*(?:/\*.*)?$", src, re.M)}
    assert len(header) >= 25
    binding = {n: getattr(fnr, n) for n in dir(fnr) if n.startswith("FNR_") and isinstance(getattr(fnr, n), int)}
    for n, v in binding.items():
        assert n in header, f"{n} is not in fnr.h"
        assert header[n] == v, f"{n}: header {header[n]}, binding {v}"
    flags = [v for n, v in header.items() if n.startswith("FNR_RENDER_")]
    assert all(f & (f - 1) == 0 for f in flags) and len(set(flags)) == len(flags)
    for n in ("FNR_RENDER_SKIP_EMPTY", "FNR_RENDER_DIR_BILINEAR", "FNR_RENDER_VOXELS", "FNR_ERR_IO",
              "FNR_LAYOUT_BRICKS"):
        assert n in binding, n


def test_testing_hooks_validate_arguments(fnr):
    """The test hooks (fnr_testing.h) check their arguments and arm / disarm without touching the device."""
    L = fnr.lib()
    assert L.fnr_testing_mlp_cta_pair(1) == fnr.FNR_OK
    assert L.fnr_testing_mlp_cta_pair(0) == fnr.FNR_OK  # back to the single-CTA form
    assert L.fnr_testing_fail_allocations(-1, 1) == fnr.FNR_ERR_INVALID_ARG
    assert L.fnr_testing_fail_allocations(0, -1) == fnr.FNR_ERR_INVALID_ARG
    assert L.fnr_testing_mlp_fault(0, 3) == fnr.FNR_ERR_INVALID_ARG
    assert L.fnr_testing_fail_allocations(2, 1) == fnr.FNR_OK
    assert L.fnr_testing_fail_allocations(0, 0) == fnr.FNR_OK  # disarmed

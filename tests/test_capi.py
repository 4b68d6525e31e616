"""The C ABI builds, loads on a machine without a GPU, exports every entry
point that include/gbstokes.h declares, and the Python structs match the C
layout (no compute calls: those need a GPU)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbstokes.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gb_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1309_5048_gb300 import build
    path = build.build()
    return C.CDLL(path), path


def test_every_declared_symbol_is_exported(lib):
    L, path = lib
    names = declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(gb_[a-z0-9_]+)\b", out))
    assert set(names) <= exported
    import paper_1309_5048_gb300 as gb
    assert set(names) == set(gb.EXPORTED)


def test_status_strings_without_gpu(lib):
    L, _ = lib
    L.gb_status_string.restype = C.c_char_p
    assert L.gb_status_string(0) == b"ok"
    assert L.gb_status_string(4) == b"IC(0) breakdown"
    # argument validation happens before any device work
    L.gb_setup_pattern.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    assert L.gb_setup_pattern(None, None, None) == 1


def test_struct_layouts_match_header(tmp_path):
    import paper_1309_5048_gb300 as gb
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "gbstokes.h"
int main(void) {
  printf("%zu %zu %zu\\n", sizeof(gb_problem), sizeof(gb_solve_opts), sizeof(gb_info));
  printf("%zu %zu %zu %zu %zu %zu %zu\\n", offsetof(gb_solve_opts, precision), offsetof(gb_solve_opts, use_graph),
         offsetof(gb_solve_opts, forced_inner_host), offsetof(gb_solve_opts, nforced),
         offsetof(gb_solve_opts, pressure_block), offsetof(gb_solve_opts, forced_q_host),
         offsetof(gb_solve_opts, nforced_q));
  printf("%zu %zu\\n", offsetof(gb_solve_opts, stop_rule), offsetof(gb_solve_opts, velocity_block));
  printf("%zu %zu %zu %zu %zu %zu\\n", offsetof(gb_info, inner_its_total), offsetof(gb_info, inner_its_max),
         offsetof(gb_info, relres_true), offsetof(gb_info, q_inner_its_total), offsetof(gb_info, q_inner_its_max),
         offsetof(gb_info, status));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    sizes = [int(v) for v in lines[0].split()]
    assert sizes == [C.sizeof(gb.gb_problem), C.sizeof(gb.gb_solve_opts), C.sizeof(gb.gb_info)]
    offs = [int(v) for v in lines[1].split()]
    assert offs == [gb.gb_solve_opts.precision.offset, gb.gb_solve_opts.use_graph.offset,
                    gb.gb_solve_opts.forced_inner_host.offset, gb.gb_solve_opts.nforced.offset,
                    gb.gb_solve_opts.pressure_block.offset, gb.gb_solve_opts.forced_q_host.offset,
                    gb.gb_solve_opts.nforced_q.offset]
    offs = [int(v) for v in lines[2].split()]
    assert offs == [gb.gb_solve_opts.stop_rule.offset, gb.gb_solve_opts.velocity_block.offset]
    offs = [int(v) for v in lines[3].split()]
    assert offs == [gb.gb_info.inner_its_total.offset, gb.gb_info.inner_its_max.offset,
                    gb.gb_info.relres_true.offset, gb.gb_info.q_inner_its_total.offset,
                    gb.gb_info.q_inner_its_max.offset, gb.gb_info.status.offset]


def test_every_entry_point_rejects_a_null_context(lib):
    """Every call returns GB_ERR_INVALID_ARG (1) with a message for a null
    context before any device work, so this runs without a GPU; gb_destroy
    accepts a null context."""
    import paper_1309_5048_gb300 as gb
    L = gb.load_library()
    for name in gb.EXPORTED:
        if name in ("gb_status_string", "gb_last_error", "gb_destroy"):
            continue
        f = getattr(L, name)
        args = [1.0 if t is C.c_double else (1 if t in (C.c_int, C.c_int64) else None) for t in f.argtypes]
        # the message is thread-local and sticky: first leave a different one
        # (gb_setup_pattern and gb_sizes say "null argument", gb_assemble
        # "null context"), so each call must write its own
        if name in ("gb_setup_pattern", "gb_sizes"):
            assert L.gb_assemble(None, 1.0, 1.0) == 1
        else:
            assert L.gb_setup_pattern(None, None, None) == 1
        before = L.gb_last_error()
        assert f(*args) == 1, name
        after = L.gb_last_error()
        assert b"null" in after and after != before, name
    L.gb_destroy(None)
    codes = [L.gb_status_string(k) for k in range(8)]
    assert len(set(codes)) == 8 and all(codes)

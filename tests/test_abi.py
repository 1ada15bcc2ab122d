"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares; the binding wraps each of them.  No GPU calls."""

import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(pw_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def built_lib():
    from paper_2512_05460_gb300 import build

    build.build()
    from paper_2512_05460_gb300 import probewalk

    return probewalk


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pw_graph_load", "pw_graph_load32", "pw_graph_free", "pw_budget", "pw_query",
                     "pw_query_batch", "pw_server_create", "pw_server_submit", "pw_server_poll",
                     "pw_server_destroy", "pw_debug_walk", "pw_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    import ctypes

    so = ctypes.CDLL(built_lib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert missing == []


def test_binding_wraps_every_declared_symbol(built_lib):
    assert set(built_lib.SIGNATURES) == declared_functions()
    built_lib.lib()  # sets argtypes for all of them


def test_pure_host_entry_points(built_lib):
    import oracle

    assert built_lib.pw_version().startswith("probewalk")
    # the default seed is host arithmetic: it must agree with the oracle's own
    for args in ((1, 3, 4, 0.1, 200), (2**63 + 7, 100, 9, 0.05, 1000), (0, 0, 1, 0.2, 0)):
        assert built_lib.pw_default_seed(*args) == oracle.default_seed(*args)


@pytest.mark.parametrize("struct", ["pw_params", "pw_profile_stats", "pw_tune_result", "pw_server_tune_result"])
def test_struct_layout(built_lib, tmp_path, struct):
    """The binding's structs match the header's layout (sizeof, offsetof)."""
    import ctypes
    import subprocess

    cls = getattr(built_lib, struct)
    fields = [f for f, _ in cls._fields_]
    src = tmp_path / "layout.c"
    body = "".join(f'  printf("%zu\\n", offsetof({struct}, {f}));\n' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "probewalk.h"\nint main(void) {\n'
                   f'  printf("%zu\\n", sizeof({struct}));\n' + body + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(cls)] + [getattr(cls, f).offset for f in fields]
    assert got == want


def test_level_seed_matches_oracle(built_lib):
    import oracle

    for seed, L in ((1, 1), (2**64 - 1, 256), (987654321, 37)):
        assert built_lib.pw_level_seed(seed, L) == oracle.level_seed(seed, L)

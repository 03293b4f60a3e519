"""The C-ABI library loads and exports every function include/*.h declares (no GPU)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2409_09228_gb300 import build as libbuild
from paper_2409_09228_gb300 import fit

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(fit_\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if not libbuild.up_to_date():
        libbuild.build()
    return ctypes.CDLL(libbuild.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("fit_init", "fit_propagate_update", "fit_sync", "fit_destroy", "fit_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_names_match_header():
    for name in declared_functions():
        assert hasattr(fit, name), f"binding lacks {name}"


def test_binding_constants_match_header():
    defines = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        for m in re.finditer(r"^#define (FIT_\w+) \(?(-?\d+)u?\)?", open(h).read(), re.M):
            defines[m.group(1)] = int(m.group(2))
    for name in ("FIT_START_CROSSING", "FIT_START_LINE", "FIT_LAYOUT_SOA", "FIT_LAYOUT_AOSOA32",
                 "FIT_OK", "FIT_ERR_ARG", "FIT_ST_NOT_CONVERGED"):
        assert name in defines, name
    for name, value in defines.items():
        if hasattr(fit, name):
            assert getattr(fit, name) == value, name


def test_argument_errors_without_gpu(lib):
    L = fit.load()
    h = ctypes.c_void_p()
    assert L.fit_init(None, None, None, 0) == fit.FIT_ERR_ARG
    assert b"NULL" in L.fit_last_error()
    assert L.fit_init(ctypes.byref(h), None, None, 0) == fit.FIT_ERR_ARG
    assert L.fit_propagate_update(None, None, None, None, 0, None, 20, None, None) == fit.FIT_ERR_ARG
    assert L.fit_sync(None, None, 0.0, None) == fit.FIT_ERR_ARG
    L.fit_destroy(None)  # a no-op on NULL


def test_struct_layouts_match_header():
    # field offsets as a C compiler lays out the structs of fit.h (LP64)
    assert ctypes.sizeof(fit.fit_config) == 32
    assert fit.fit_config.surf.offset == 8
    assert fit.fit_config.start.offset == 24
    assert ctypes.sizeof(fit.fit_tracks_in) == 32
    assert ctypes.sizeof(fit.fit_tracks_out) == 56
    assert ctypes.sizeof(fit.fit_hits) == 24
    assert ctypes.sizeof(fit.fit_status) == 48


def test_header_compiles_as_c_and_matches_the_binding(tmp_path):
    """include/fit.h is plain C (C99, -pedantic, no warnings), and a C
    compiler lays out its structs as the ctypes binding does."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"fit_config": ["B", "nlayer", "surf", "max_iter", "tol", "start"],
               "fit_launch_config": ["threads_per_block", "blocks_per_sm", "persistent",
                                     "tracks_per_thread", "layout"],
               "fit_plan_info": ["config", "tracks", "items", "tuned", "best_ms"],
               "fit_tracks_in": ["par", "cov", "q", "ld"],
               "fit_tracks_out": ["par", "cov", "q", "chi2", "chi2_layer", "status", "ld"],
               "fit_hits": ["pos", "cov", "ld"],
               "fit_status": ["tracks", "no_intersection", "not_converged", "nonfinite",
                              "charge_flip", "iterations"]}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "fit.h"', "int main(void) {"]
    for name, fields in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for fld in fields:
            lines.append(f'  printf("{name}.{fld} %zu\\n", offsetof({name}, {fld}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True,
                                                       text=True, check=True).stdout.split("\n")
               if line)
    for name, fields in structs.items():
        cls = getattr(fit, name)
        assert int(got[name]) == ctypes.sizeof(cls), name
        for fld in fields:
            assert int(got[f"{name}.{fld}"]) == getattr(cls, fld).offset, f"{name}.{fld}"


def test_plan_struct_layouts():
    assert ctypes.sizeof(fit.fit_launch_config) == 20
    assert fit.fit_plan_info.tracks.offset == 24
    assert ctypes.sizeof(fit.fit_plan_info) == 48
    assert ctypes.sizeof(fit.fit_candidates) == 32
    assert ctypes.sizeof(fit.fit_mlp_train_config) == 40

"""Host-side checks of the C ABI (no GPU needed).

The library must load, export every function that include/*.h declares,
agree with the Python binding on every struct layout, and reject invalid
descriptors before touching the device.
"""
import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2606_07759_b300 import abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(synim_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_function():
    L = abi.load()
    names = declared_functions()
    assert len(names) >= 8
    for n in names:
        assert hasattr(L, n), n
        assert n in abi.SIGNATURES, f"binding misses {n}"


def test_struct_layouts_match_the_header(tmp_path):
    probe = tmp_path / "probe.c"
    structs = {"synim_dm_desc": abi.synim_dm_desc, "synim_wfs_desc": abi.synim_wfs_desc,
               "synim_misreg": abi.synim_misreg, "synim_opts": abi.synim_opts,
               "synim_noise_desc": abi.synim_noise_desc}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "synim.h"', "int main(void){"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0;}")
    probe.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(probe), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.split() for line in out if line)
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(got[f"{name}.{fname}"]) == getattr(cls, fname).offset, (name, fname)


def test_status_strings_and_invalid_create():
    L = abi.load()
    assert L.synim_status_string(0) == b"ok"
    assert L.synim_status_string(5) == b"bounded device wait timed out"
    ctx = ctypes.c_void_p()
    # no DM at all: rejected before any device call
    st = L.synim_im_create(None, 0, None, 0, None, ctypes.byref(ctx))
    assert st == 1 and not ctx.value
    assert b"DM" in L.synim_last_error(None)
    # grid_m not a multiple of n_sub with k >= 2
    cube = np.zeros((1, 8, 8), np.float32)
    dm = abi.synim_dm_desc(1, 8, 0.1, 0.0, cube.ctypes.data, 0, None, 1e-9)
    w = abi.synim_wfs_desc()
    w.n_sub, w.grid_m, w.pupil_diam_m = 4, 10, 1.0
    w.mag[0] = w.mag[1] = 1.0
    w.slope_scale = 1.0
    st = L.synim_im_create(ctypes.byref(dm), 1, ctypes.byref(w), 1, None, ctypes.byref(ctx))
    assert st == 2 and not ctx.value
    w.grid_m = 4  # k = 1: no sub-pixel resolution
    st = L.synim_im_create(ctypes.byref(dm), 1, ctypes.byref(w), 1, None, ctypes.byref(ctx))
    assert st == 2
    # query on a NULL context
    r, c = ctypes.c_int64(), ctypes.c_int64()
    assert L.synim_im_query(None, 0, 0, ctypes.byref(r), ctypes.byref(c)) == 1

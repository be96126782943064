"""The bounds-checked build (libsynim_bounds.so, -DSYNIM_DEBUG_BOUNDS): every
global and shared-memory index of the IM kernels (k_im, k_tele) is tested
against its buffer; an index outside skips the access and makes the next
synim_im_check return SYNIM_ERR_BOUNDS (8).  No device assert or trap.

CPU: the release library answers 0 to synim_debug_bounds, the bounds build 1
(a host query).
GPU: a child process with SYNIM_DEBUG_BOUNDS=1 computes the IMs (numerical
and telescoping engines), the tangents and the adjoint on reduced SCAO, ELT
and MCAO geometries; every check passes (no index left its buffer), and
the results equal the release build's bit for bit (the tests only add
branches that are never taken).
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2606_07759_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import ctypes, sys
import numpy as np
import torch
from paper_2606_07759_b300 import abi, workloads as W
from paper_2606_07759_b300.synim import SynIM

def run():
    L = abi.load()
    out = {"flag": np.array([L.synim_debug_bounds()])}
    cases = {"scao": W.scao_small(), "elt": W.elt_single(seed=7, n_side=21, grid_n=120, n_sub=17),
             "mcao": W.mcao_batched(seed=8, scale=0.2)}
    for name, wl in cases.items():
        for eng in ("numerical", "telescoping"):
            s = SynIM(wl.dms, wl.wfss, slope_engine=eng)
            ims = s.compute(wl.misregs)
            s.check()
            for p, t in enumerate(ims):
                if t is not None:
                    out[f"{name}_{eng}_{p}"] = t.cpu().numpy()
            s.close()
    wl = cases["scao"]
    s = SynIM(wl.dms, wl.wfss)
    ims, tans = s.sensitivity(wl.misregs)
    s.check()
    for k in range(4):
        out[f"tan_{k}"] = tans[0][k].cpu().numpy()
    g = torch.from_numpy(np.random.default_rng(3).standard_normal(tuple(ims[0].shape)).astype(np.float32)).cuda()
    out["vjp"] = s.vjp(wl.misregs, [g])
    s.check()
    s.close()
    np.savez(sys.argv[1], **out)

run()
'''


def test_release_and_bounds_builds_identify_themselves():
    L = ctypes.CDLL(B.lib_path(False))
    assert L.synim_debug_bounds() == 0
    if B.stale(True):
        pytest.skip("the bounds-checked library is not built (python -m paper_2606_07759_b300.build --bounds)")
    Lb = ctypes.CDLL(B.lib_path(True))
    assert Lb.synim_debug_bounds() == 1


def _run_child(path, bounds):
    env = dict(os.environ, SYNIM_DEBUG_BOUNDS="1" if bounds else "0",
               PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD, str(path)], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return dict(np.load(path))


@pytest.mark.gpu
def test_bounds_build_finds_no_index_outside_and_matches_release(tmp_path):
    dbg = _run_child(tmp_path / "bounds.npz", True)
    rel = _run_child(tmp_path / "release.npz", False)
    assert dbg.pop("flag")[0] == 1 and rel.pop("flag")[0] == 0
    assert sorted(dbg) == sorted(rel) and len(dbg) > 20
    for k in dbg:
        np.testing.assert_array_equal(dbg[k], rel[k], err_msg=k)

"""Tomographic covariances and the MMSE reconstructor on the GPU (Sec. 2.4)
against the FP64 oracle (oracle/covariance.py).

Criteria (FP32 data, tensor-core contractions with FP32-level products, FP32
Cholesky solves):
  - C_atm: max |C_gpu - C_ref| <= 2e-3 max |C_ref| (the Gram solve of a
    basis of overlapping Gaussians amplifies FP32 rounding by its condition
    number), symmetric;
  - C_n: relative 1e-6 per entry (host FP64 values rounded to FP32), exactly
    block-diagonal (x-y couplings only within a subaperture);
  - R: max |R_gpu - R_ref| <= 2e-3 max |R_ref| on the same FP32 inputs.
Workloads: the SCAO geometry (80 px grid, bin 4, 80 modes, 152 slopes) and
the learned-estimator geometry (352 px grid, bin 4, 1369 modes, 2528 slopes;
the basis Gram matrix has condition number 66 there, 6e5 at bin 8, where FP32
cannot hold C_atm), an LGS noise model with elongation and an NGS one.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from oracle import covariance as CV
from paper_2606_07759_b300 import abi
from paper_2606_07759_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _workload(name):
    wl = getattr(W, name)()
    return wl[0] if isinstance(wl, tuple) else wl   # learned() also returns its probe commands


def _atm(s, d, n, bin_, r0, L0):
    out = torch.empty(n, n, device="cuda")
    st = s._L.synim_atm_covariance(s._ctx, d, bin_, r0, L0, out.data_ptr(), _stream())
    assert st == 0, s._L.synim_last_error(s._ctx)
    return out.double().cpu().numpy()


@pytest.mark.parametrize("name,bin_", [("scao_small", 4), ("learned", 4)])
def test_atm_covariance_matches_oracle(name, bin_):
    from paper_2606_07759_b300.synim import SynIM
    wl = _workload(name)
    dm = wl.dms[0]
    s = SynIM([dm], wl.wfss[:1])
    r0, L0 = 0.15, 25.0
    got = _atm(s, 0, dm.n_act, bin_, r0, L0)
    ref = CV.atm_cov(dm.ifs, dm.pixel_pitch_m, bin_, r0, L0)
    assert np.abs(got - got.T).max() == 0.0
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= 2e-3, err
    s.close()


def _noise(s, w, nd, nv):
    out = torch.full((2 * nv, 2 * nv), float("nan"), device="cuda")
    st = s._L.synim_noise_covariance(s._ctx, w, ctypes.byref(nd), out.data_ptr(), _stream())
    assert st == 0, s._L.synim_last_error(s._ctx)
    return out.double().cpu().numpy()


@pytest.mark.parametrize("lgs", [0, 1])
def test_noise_covariance_matches_oracle(lgs):
    from paper_2606_07759_b300.synim import SynIM
    wl = W.mcao_batched(seed=3, scale=0.3)
    w = 0 if lgs else 6
    wfs = wl.wfss[w]
    s = SynIM(wl.dms[:1], [wfs])
    nv = s.shapes[(0, 0)][0] // 2
    nd = abi.synim_noise_desc(n_photons=300.0, ron_e=2.0, pixel_scale_rad=0.8e-6, n_pix=10, lgs=lgs,
                              fwhm_rad=1.2e-6, wavelength_m=589e-9 if lgs else 700e-9)
    nd.llt_xy_m[0], nd.llt_xy_m[1] = 20.0, -4.0
    nd.na_altitude_m, nd.na_thickness_m, nd.zenith_rad = 90e3, 10e3, 0.3
    got = _noise(s, 0, nd, nv)
    ros, _, nv2 = oracle.valid_subaps(wfs.pupil_mask, wfs.n_sub)
    assert nv2 == nv
    cen = CV.subap_centres(wfs.n_sub, wfs.pupil_diam_m, ros)
    ref = CV.noise_cov(cen, wfs.pupil_diam_m / wfs.n_sub, 300.0, 2.0, 0.8e-6, 10, 1.2e-6, nd.wavelength_m,
                       wfs.slope_scale, lgs=(20.0, -4.0, 90e3, 10e3, 0.3) if lgs else None)
    nz = ref != 0
    assert np.array_equal(got != 0, nz)
    np.testing.assert_allclose(got[nz], ref[nz], rtol=1e-6)
    s.close()


@pytest.mark.parametrize("name", ["scao_small", "learned"])
def test_mmse_reconstructor_matches_oracle(name):
    from paper_2606_07759_b300.synim import SynIM
    wl = _workload(name)
    s = SynIM(wl.dms, wl.wfss)
    im = s.compute(wl.misregs)[0]
    nm, ns = im.shape
    rng = np.random.default_rng(1)
    A = rng.standard_normal((nm, nm)) / np.sqrt(nm)
    ca = (A @ A.T + 0.5 * np.eye(nm)).astype(np.float32)
    cn = (np.diag(rng.uniform(0.5, 1.5, ns)) * float(im.abs().max()) ** 2 * 1e-2).astype(np.float32)
    ca_d, cn_d = torch.from_numpy(ca).cuda(), torch.from_numpy(cn).cuda()
    R = torch.empty(nm, ns, device="cuda")
    st = s._L.synim_mmse_reconstructor(nm, ns, im.data_ptr(), ca_d.data_ptr(), cn_d.data_ptr(), R.data_ptr(),
                                       _stream())
    assert st == 0, s._L.synim_last_error(None)
    ref = CV.mmse(im.double().cpu().numpy(), ca.astype(np.float64), cn.astype(np.float64))
    err = np.abs(R.double().cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err <= 2e-3, err
    s.close()

"""Misregistration sensitivities on the GPU: tangents (forward mode), the
adjoint (VJP) and the autograd function, against the FP64 oracle.

The oracle's analytic tangents are themselves pinned to central finite
differences of the oracle forward (tests/test_oracle_pins.py).  Criterion:
for every pair and parameter k, max |T_gpu - T_ref| <= 1e-4 * max |T_ref|,
on the IM entries whose subaperture has no sample within 1e-4 px of a
bilinear cell line: there the derivative of the interpolant jumps, and the
FP32 kernel may pick the neighbouring cell (a floor-cell derivative either
way; the flagged fraction is checked to stay small).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_07759_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-4


def stencil_pixels(wfs):
    """Pixels whose phase enters a subaperture sum: the two pixel lines at every
    subaperture boundary and the pixels where the pupil changes inside one."""
    P = np.pad(wfs.pupil_mask.astype(np.int8), 1)
    M, k = wfs.grid_m, wfs.grid_m // wfs.n_sub
    ii, jj = np.mgrid[0:M, 0:M]
    xl = np.isin(jj % k, (0, k - 1)) | (P[1:-1, :-2] != P[1:-1, 2:])
    yl = np.isin(ii % k, (0, k - 1)) | (P[:-2, 1:-1] != P[2:, 1:-1])
    return xl | yl


def kink_rows(wl, d, w, plist, near=1e-4, extra=None):
    """IM rows that use a stencil pixel sampled near a bilinear cell line (at
    plist[0]), whose cell changes across the parameter sets in plist, or that
    depend on a pixel flagged in extra (e.g. a change of the core set)."""
    from scipy.ndimage import binary_dilation
    dm, wfs = wl.dms[d], wl.wfss[w]
    M, n = wfs.grid_m, wfs.n_sub
    k = M // n
    ii, jj = np.mgrid[0:M, 0:M].astype(np.float64)
    bad = np.zeros((M, M), bool)
    cells = []
    for q, p in enumerate(plist):
        A, b = oracle.composite(oracle.pair_geom(dm, wfs), p)
        xy = (A[0] * jj + A[1] * ii + b[0], A[2] * jj + A[3] * ii + b[1])
        cells.append([np.floor(c) for c in xy])
        if q == 0:
            for c in xy:
                f = c - np.floor(c)
                bad |= (f < near) | (f > 1 - near)
    for c in cells[1:]:
        bad |= (c[0] != cells[0][0]) | (c[1] != cells[0][1])
    if extra is not None:
        bad |= extra
    # ring pixels reach core pixels 2 away; stencil pixels feed the neighbouring subapertures
    bad = binary_dilation(binary_dilation(bad, iterations=2) & stencil_pixels(wfs), iterations=1)
    ros, _, nv = oracle.valid_subaps(wfs.pupil_mask, n)
    badsub = bad.reshape(n, k, n, k).any(axis=(1, 3))
    rows = np.zeros(2 * nv, bool)
    for si in range(n):
        for sj in range(n):
            r = ros[si, sj]
            if r >= 0 and badsub[si, sj]:
                rows[r] = rows[nv + r] = True
    return rows


def check_tangents(wl, cols_per_dm=None, seed=0):
    from paper_2606_07759_b300.synim import SynIM
    s = SynIM(wl.dms, wl.wfss)
    ims, tans = s.sensitivity(wl.misregs)
    fwd = s.compute(wl.misregs)
    s.check()
    rng = np.random.default_rng(seed)
    for d, dm in enumerate(wl.dms):
        cols = np.arange(dm.n_act) if cols_per_dm is None else np.sort(
            rng.choice(dm.n_act, min(cols_per_dm, dm.n_act), replace=False))
        for w in range(len(wl.wfss)):
            p = d * len(wl.wfss) + w
            mis = wl.misregs[p].as_tuple()
            ref = oracle.pair_tangent(wl, d, w, cols=cols, misreg=mis)
            # the IM written by the tangent pass equals the forward pass to FP32
            # rounding: the forward pass forms each boundary segment as a dot
            # product of precomputed bilinear weights, the tangent pass
            # resamples pixel by pixel, so their sums round differently; each
            # is held to the parity bar against the oracle elsewhere, so the
            # two agree within twice that bar per column
            a, b_ = ims[p].cpu().numpy(), fwd[p].cpu().numpy()
            cpk = np.maximum(np.abs(b_).max(axis=1), 1e-2 * max(np.abs(b_).max(), 1e-30))
            assert np.all(np.abs(a - b_).max(axis=1) <= 2e-5 * cpk)
            bad = kink_rows(wl, d, w, [mis])
            assert bad.mean() < (0.25 if wl.wfss[w].n_sub > 4 else 0.8)
            for k in range(4):
                got = tans[p][k].cpu().numpy()[cols][:, ~bad].astype(np.float64)
                r = ref[k][:, ~bad]
                scale = np.abs(ref[k]).max()
                if scale == 0:
                    continue
                err = np.abs(got - r).max()
                assert err <= TOL * scale, f"{wl.name} dm{d} wfs{w} p{k}: {err / scale:.2e}"
    s.close()


def test_tangents_scao_small_all_columns():
    check_tangents(W.scao_small())


def test_tangents_elt_reduced():
    check_tangents(W.elt_single(seed=4, n_side=21, grid_n=120, n_sub=17))


def test_tangents_mcao_reduced():
    check_tangents(W.mcao_batched(seed=9, scale=0.15), cols_per_dm=40)


def test_tangents_elt_single_full_size_sampled_columns():
    # the ELT-scale sensitivity workload (81 x 81 DM on 480 px, 68 x 68 SH) at
    # its full size, sampled columns against the oracle's analytic tangents
    check_tangents(W.elt_single(seed=4), cols_per_dm=16, seed=4)


def test_tangents_match_oracle_central_differences():
    # GPU tangents against central differences of the FP64 oracle forward,
    # steps (1e-3 px, 1e-3 px, 1e-3 deg, 1e-5), on kink-free rows
    from paper_2606_07759_b300.synim import SynIM
    wl = W.elt_single(seed=4, n_side=21, grid_n=120, n_sub=17)
    s = SynIM(wl.dms, wl.wfss)
    _, tans = s.sensitivity(wl.misregs)
    s.check()
    p0 = np.array(wl.misregs[0].as_tuple())
    steps = [1e-3, 1e-3, 1e-3, 1e-5]
    cols = list(range(0, wl.dms[0].n_act, 7))
    for k in range(4):
        e = np.zeros(4)
        e[k] = steps[k]
        fd = (oracle.pair_im(wl, 0, 0, cols=cols, misreg=tuple(p0 + e)) -
              oracle.pair_im(wl, 0, 0, cols=cols, misreg=tuple(p0 - e))) / (2 * steps[k])
        # the tangent holds the core set fixed: rows reached by a pixel whose
        # core status changes across the stencil are excluded like kinks
        g = oracle.pair_geom(wl.dms[0], wl.wfss[0])
        c1 = oracle.core(wl.dms[0].mask, wl.dms[0].grid_n, wl.wfss[0].grid_m, *oracle.composite(g, p0 - e))[0]
        c2 = oracle.core(wl.dms[0].mask, wl.dms[0].grid_n, wl.wfss[0].grid_m, *oracle.composite(g, p0 + e))[0]
        bad = kink_rows(wl, 0, 0, [tuple(p0), tuple(p0 - e), tuple(p0 + e)], extra=(c1 != c2))
        assert bad.mean() < 0.5
        got = tans[0][k].cpu().numpy()[cols][:, ~bad].astype(np.float64)
        scale = np.abs(fd).max()
        assert np.abs(got - fd[:, ~bad]).max() <= TOL * scale, k
    s.close()


def test_vjp_is_the_adjoint_of_the_tangents():
    from paper_2606_07759_b300.synim import SynIM
    wl = W.mcao_batched(seed=10, scale=0.15)
    s = SynIM(wl.dms, wl.wfss)
    ims, tans = s.sensitivity(wl.misregs)
    g = torch.Generator(device="cuda").manual_seed(0)
    grads = [torch.randn(t.shape, device="cuda", generator=g) for t in ims]
    grads[3] = None  # zero cotangent for one pair
    gp = s.vjp(wl.misregs, grads)
    s.check()
    # per-column partials summed in a fixed order: a second call is bit-identical
    gp2 = s.vjp(wl.misregs, grads)
    assert np.array_equal(gp, gp2)
    for p in range(len(ims)):
        for k in range(4):
            if grads[p] is None:
                assert gp[p, k] == 0.0
                continue
            ref = float((grads[p].double() * tans[p][k].double()).sum())
            mag = float((grads[p].double().abs() * tans[p][k].double().abs()).sum())
            assert abs(gp[p, k] - ref) <= 1e-5 * max(mag, 1e-30), (p, k, gp[p, k], ref)
    s.close()


def test_autograd_function_backward_uses_the_adjoint():
    from paper_2606_07759_b300.synim import SynIM, IMFunction
    wl = W.scao_small()
    s = SynIM(wl.dms, wl.wfss)
    params = torch.tensor([wl.misregs[0].as_tuple()], dtype=torch.float64, requires_grad=True)
    (im,) = IMFunction.apply(params, s)
    wgt = torch.linspace(-1, 1, im.numel(), device="cuda").reshape(im.shape)
    loss = (im * wgt).sum()
    loss.backward()
    # the same derivative from the FP64 oracle: sum(wgt * dIM/dp_k)
    T = oracle.pair_tangent(wl, 0, 0, misreg=wl.misregs[0].as_tuple())
    w_np = wgt.cpu().numpy().astype(np.float64)
    ref = np.array([(w_np * T[k]).sum() for k in range(4)])
    mag = np.array([(np.abs(w_np) * np.abs(T[k])).sum() for k in range(4)])
    np.testing.assert_array_less(np.abs(params.grad.numpy()[0] - ref), 1e-4 * mag)
    s.close()


def test_autograd_gradient_follows_the_parameter_device():
    from paper_2606_07759_b300.synim import SynIM, IMFunction
    wl = W.scao_small()
    s = SynIM(wl.dms, wl.wfss)
    params = torch.tensor([wl.misregs[0].as_tuple()], dtype=torch.float32, device="cuda", requires_grad=True)
    (im,) = IMFunction.apply(params, s)
    im.sum().backward()
    assert params.grad.device == params.device and params.grad.dtype == params.dtype
    assert torch.isfinite(params.grad).all()
    s.close()

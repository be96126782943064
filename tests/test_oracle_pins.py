"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check is a closed form
worked out from the geometry (Sec. 2.1), an invariance of the method
(rotation, magnification, linearity), the exact telescoping identity of the
summed central differences (Sec. 2.2), the continuous-gradient limit of the
G-tilt at low spatial frequency (Sec. 2.2), hand-worked edge-repair cases
(Sec. 2.3, tests/golden/edge_repair_cases.json) or a finite-difference
definition of a derivative.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def geom(N, dd, M, D, h=0.0, H=0.0, th=(0.0, 0.0), wrot=0.0, wmag=(1.0, 1.0), wshift=(0.0, 0.0)):
    return [N, dd, h, M, D, H, th[0], th[1], wrot, wmag[0], wmag[1], wshift[0], wshift[1]]


def rot(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[c, -s], [s, c]])


# ---------------------------------------------------------------------------
# Composite affine (Sec. 2.1)
# ---------------------------------------------------------------------------
def test_composite_identity():
    A, b = oracle.composite(geom(64, 0.1, 64, 6.4), (0, 0, 0, 1))
    np.testing.assert_allclose(A, [1, 0, 0, 1], atol=1e-15)
    np.testing.assert_allclose(b, [0, 0], atol=1e-12)


def test_composite_closed_forms():
    N, dd, M, D = 100, 0.05, 64, 4.0
    dw, cM, cN = D / M, (M - 1) / 2, (N - 1) / 2

    def apply(A, b, j, i):
        return A[0] * j + A[1] * i + b[0], A[2] * j + A[3] * i + b[1]

    # footprint shift h * theta for a natural guide star: the pupil centre
    # lands h * theta / dd pixels off the DM centre.
    A, b = oracle.composite(geom(N, dd, M, D, h=5000.0, th=(1e-4, -2e-4)), (0, 0, 0, 1))
    x, y = apply(A, b, cM, cM)
    assert x == pytest.approx(cN + 5000 * 1e-4 / dd, abs=1e-9)
    assert y == pytest.approx(cN - 5000 * 2e-4 / dd, abs=1e-9)
    # LGS cone: a DM at h seen from a source at H shrinks the beam by 1 - h/H.
    A, b = oracle.composite(geom(N, dd, M, D, h=10e3, H=90e3), (0, 0, 0, 1))
    x, y = apply(A, b, M - 1, cM)
    assert x == pytest.approx(cN + (8.0 / 9.0) * cM * dw / dd, abs=1e-9)
    assert y == pytest.approx(cN, abs=1e-9)
    # positive DM shift moves the DM pattern +x/+y on the sensor, so a fixed
    # sensor pixel samples the DM shift pixels earlier.
    A0, b0 = oracle.composite(geom(N, dd, M, D), (0, 0, 0, 1))
    A, b = oracle.composite(geom(N, dd, M, D), (1.5, -0.25, 0, 1))
    np.testing.assert_allclose(A, A0, atol=1e-15)
    np.testing.assert_allclose(b - b0, [-1.5, 0.25], atol=1e-12)
    # DM rotation by +90 degrees (counter-clockwise in (x, y)): a sensor pixel
    # sees the DM point rotated by -90 degrees: A = (dw/dd) R(-90).
    A, b = oracle.composite(geom(N, dd, M, D), (0, 0, 90.0, 1))
    np.testing.assert_allclose(A, np.array([[0, 1], [-1, 0]]).ravel() * dw / dd, atol=1e-14)
    np.testing.assert_allclose(apply(A, b, cM, cM), (cN, cN), atol=1e-12)
    # DM magnification m > 1 makes the DM look larger: A = dw / (dd m) I.
    A, b = oracle.composite(geom(N, dd, M, D), (0, 0, 0, 1.25))
    np.testing.assert_allclose(A, [dw / (dd * 1.25), 0, 0, dw / (dd * 1.25)], atol=1e-15)
    np.testing.assert_allclose(apply(A, b, cM, cM), (cN, cN), atol=1e-12)
    # sensor rotation and anamorphic magnification: A = (dw/dd) R(tw) diag(mx, my)
    A, b = oracle.composite(geom(N, dd, M, D, wrot=30.0, wmag=(1.1, 0.9)), (0, 0, 0, 1))
    np.testing.assert_allclose(A.reshape(2, 2), (dw / dd) * rot(math.radians(30)) @ np.diag([1.1, 0.9]),
                               atol=1e-14)
    # sensor shift in metres moves the sampled DM point by s / dd (times the cone factor)
    A, b = oracle.composite(geom(N, dd, M, D, h=10e3, H=90e3, wshift=(0.2, -0.1)), (0, 0, 0, 1))
    A1, b1 = oracle.composite(geom(N, dd, M, D, h=10e3, H=90e3), (0, 0, 0, 1))
    np.testing.assert_allclose(b - b1, np.array([0.2, -0.1]) * (8.0 / 9.0) / dd, atol=1e-12)


def test_composite_jacobian_matches_central_differences():
    g = geom(480, 39 / 480, 544, 39.0, h=4000.0, H=90e3, th=(3e-5, -2e-5), wrot=2.0, wmag=(1.01, 0.99),
             wshift=(0.05, -0.03))
    p = np.array([0.7, -0.4, 0.8, 1.007])
    dA, db = oracle.composite_jac(g, p)
    steps = [1e-5, 1e-5, 1e-5, 1e-7]
    for k in range(4):
        e = np.zeros(4)
        e[k] = steps[k]
        Ap, bp = oracle.composite(g, p + e)
        Am, bm = oracle.composite(g, p - e)
        np.testing.assert_allclose(dA[k], (Ap - Am) / (2 * steps[k]), rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(db[k], (bp - bm) / (2 * steps[k]), rtol=1e-6, atol=1e-7)


# ---------------------------------------------------------------------------
# Valid subapertures
# ---------------------------------------------------------------------------
def test_valid_subaps_half_lit_rule():
    rng = np.random.default_rng(0)
    M, n = 48, 6
    k = M // n
    P = (rng.random((M, M)) < 0.55).astype(np.uint8)
    ros, lit, nv = oracle.valid_subaps(P, n)
    blocks = P.reshape(n, k, n, k).sum(axis=(1, 3))
    np.testing.assert_array_equal(lit, blocks)
    valid = 2 * blocks >= k * k
    assert nv == valid.sum()
    np.testing.assert_array_equal(ros >= 0, valid)
    np.testing.assert_array_equal(ros[valid], np.arange(nv))  # row-major ranks
    forced = np.zeros((n, n), np.uint8)
    forced[1, 2] = forced[4, 4] = 1
    ros2, _, nv2 = oracle.valid_subaps(P, n, forced)
    assert nv2 == 2 and ros2[1, 2] == 0 and ros2[4, 4] == 1


# ---------------------------------------------------------------------------
# Closed forms of the full forward (Sec. 2.1 + 2.2)
# ---------------------------------------------------------------------------
def _interior_pupil(M, n, margin=1):
    k = M // n
    P = np.zeros((M, M), np.uint8)
    P[margin * k:(n - margin) * k, margin * k:(n - margin) * k] = 1
    return P


@pytest.mark.parametrize("case", [
    dict(p=(0.0, 0.0, 0.0, 1.0)),
    dict(p=(0.4, -0.3, 7.0, 1.03)),
    dict(p=(-1.2, 0.9, -20.0, 0.97), wrot=15.0, wmag=(1.05, 0.95)),
    dict(p=(0.2, 0.1, 3.0, 1.01), h=8000.0, H=90e3, th=(2e-5, -1e-5), wshift=(0.03, 0.02)),
])
def test_tilt_gives_constant_closed_form_slopes(case):
    N, dd, M, n, D = 140, 0.05, 64, 8, 3.2
    g = geom(N, dd, M, D, h=case.get("h", 0.0), H=case.get("H", 0.0), th=case.get("th", (0, 0)),
             wrot=case.get("wrot", 0.0), wmag=case.get("wmag", (1, 1)), wshift=case.get("wshift", (0, 0)))
    p = case["p"]
    cN = (N - 1) / 2
    al, be = 0.25, -0.75  # dyadic: the FP32 cube holds the plane exactly
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    tilt = (al * (xx - cN) + be * (yy - cN)).astype(np.float32)[None]
    A, b = oracle.composite(g, p)
    P = _interior_pupil(M, n)
    out = oracle.im(tilt, None, M, n, P, None, A, b, D / M)[0]
    nv = out.size // 2
    # d(x, y)/d(u, v) = c / (dd m) R(-td) R(tw) diag(mw); slopes = its transpose times (al, be)
    cone = 1.0 - g[2] / g[5] if g[5] > 0 else 1.0
    J = cone / (dd * p[3]) * rot(-math.radians(p[2])) @ rot(math.radians(g[8])) @ np.diag([g[9], g[10]])
    sx, sy = J.T @ np.array([al, be])
    np.testing.assert_allclose(out[:nv], sx, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(out[nv:], sy, rtol=1e-10, atol=1e-12)


def test_magnification_scales_tilt_slopes():
    N, dd, M, n, D = 140, 0.05, 64, 8, 3.2
    cN = (N - 1) / 2
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    tilt = (0.5 * (xx - cN) + 0.25 * (yy - cN)).astype(np.float32)[None]
    P = _interior_pupil(M, n)
    g = geom(N, dd, M, D)
    A1, b1 = oracle.composite(g, (0, 0, 0, 1.0))
    A2, b2 = oracle.composite(g, (0, 0, 0, 1.02))
    s1 = oracle.im(tilt, None, M, n, P, None, A1, b1, D / M)[0]
    s2 = oracle.im(tilt, None, M, n, P, None, A2, b2, D / M)[0]
    np.testing.assert_allclose(s2, s1 / 1.02, rtol=1e-11)


@pytest.mark.parametrize("axis", ["x", "y"])
def test_quadratic_gives_linear_slopes(axis):
    # pure shift, dw = dd: the bilinear error of a parabola is a constant and
    # the central difference of a parabola is exact, so the slope of each
    # subaperture is 2 dd (pixel centroid - shift - centre) exactly.
    N = M = 64
    n, dd = 8, 0.1
    k = M // n
    sx, sy = 0.37, -0.21
    c = (N - 1) / 2
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    q = ((xx - c) * dd) ** 2 if axis == "x" else ((yy - c) * dd) ** 2
    A, b = oracle.composite(geom(N, dd, M, M * dd), (sx, sy, 0, 1))
    P = _interior_pupil(M, n)
    ros, lit, nv = oracle.valid_subaps(P, n)
    out = oracle.im(q.astype(np.float32)[None], None, M, n, P, None, A, b, dd)[0]
    for si in range(n):
        for sj in range(n):
            r = ros[si, sj]
            if r < 0:
                continue
            cj, ci = sj * k + (k - 1) / 2, si * k + (k - 1) / 2
            if axis == "x":
                exp_x, exp_y = 2 * dd * (cj - sx - c), 0.0
            else:
                exp_x, exp_y = 0.0, 2 * dd * (ci - sy - c)
            # FP32 storage of the parabola limits the match to ~1e-6 of its scale
            assert out[r] == pytest.approx(exp_x, abs=2e-5)
            assert out[nv + r] == pytest.approx(exp_y, abs=2e-5)


# ---------------------------------------------------------------------------
# Invariances
# ---------------------------------------------------------------------------
def _smooth_cube(rng, N, n_act, sigma):
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    cube = np.empty((n_act, N, N), np.float32)
    for a in range(n_act):
        x0, y0 = rng.uniform(0.3 * N, 0.7 * N, 2)
        cube[a] = np.exp(-((xx - x0) ** 2 + (yy - y0) ** 2) / (2 * sigma ** 2))
    return cube


def _disc(n, r_out, r_in=0.0):
    c = (n - 1) / 2
    yy, xx = np.mgrid[0:n, 0:n]
    r = np.hypot(xx - c, yy - c)
    return ((r <= r_out) & (r >= r_in)).astype(np.uint8)


def test_dm_rotation_by_90_degrees_equals_rotated_influence_functions():
    rng = np.random.default_rng(1)
    N, dd, M, n, D = 56, 0.1, 48, 6, 4.32
    cube = _smooth_cube(rng, N, 3, 3.0)
    mask = _disc(N, 0.45 * N, 0.1 * N)
    cube *= mask
    # IF rotated so that IF'(x', y') = IF(y', -x') about the grid centre
    rot_cube = np.ascontiguousarray(np.transpose(cube, (0, 2, 1))[:, :, ::-1])
    P = _disc(M, M / 2, 0.1 * M)
    g = geom(N, dd, M, D)
    A90, b90 = oracle.composite(g, (0, 0, 90.0, 1))
    A0, b0 = oracle.composite(g, (0, 0, 0.0, 1))
    im90 = oracle.im(cube, mask, M, n, P, None, A90, b90, D / M)
    im0 = oracle.im(rot_cube, mask, M, n, P, None, A0, b0, D / M)
    assert np.abs(im90).max() > 1e-3
    np.testing.assert_allclose(im90, im0, atol=1e-12 * np.abs(im0).max())


def test_sensor_rotation_by_90_degrees_permutes_and_rotates_slopes():
    rng = np.random.default_rng(2)
    N, dd, M, n, D = 60, 0.1, 48, 6, 4.8
    k = M // n
    cube = _smooth_cube(rng, N, 3, 3.5)
    mask = _disc(N, 0.48 * N, 0.1 * N)
    cube *= mask
    P = _disc(M, M / 2, 0.2 * M / 2)
    ros, _, nv = oracle.valid_subaps(P, n)
    g0 = geom(N, dd, M, D)
    g90 = geom(N, dd, M, D, wrot=90.0)
    p = (0.3, -0.2, 4.0, 1.01)
    im0 = oracle.im(cube, mask, M, n, P, None, *oracle.composite(g0, p), D / M)
    im90 = oracle.im(cube, mask, M, n, P, None, *oracle.composite(g90, p), D / M)
    assert np.abs(im0).max() > 1e-3
    tol = 1e-12 * np.abs(im0).max()
    for si in range(n):
        for sj in range(n):
            r = ros[si, sj]
            if r < 0:
                continue
            r0 = ros[sj, n - 1 - si]
            assert r0 >= 0
            np.testing.assert_allclose(im90[:, r], im0[:, nv + r0], atol=tol)
            np.testing.assert_allclose(im90[:, nv + r], -im0[:, r0], atol=tol)
    del k


def test_linearity_in_the_influence_function():
    rng = np.random.default_rng(3)
    w = __import__("paper_2606_07759_b300.workloads", fromlist=["scao_small"]).scao_small()
    dm, wfs = w.dms[0], w.wfss[0]
    a, bb = 17, 42
    combo = (0.5 * dm.ifs[a].astype(np.float64) - 2.0 * dm.ifs[bb].astype(np.float64)).astype(np.float32)
    cube = np.stack([dm.ifs[a], dm.ifs[bb], combo])
    A, b = oracle.composite(oracle.pair_geom(dm, wfs), w.pair(0, 0).as_tuple())
    out = oracle.im(cube, dm.mask, wfs.grid_m, wfs.n_sub, wfs.pupil_mask, None, A, b,
                    wfs.pupil_diam_m / wfs.grid_m)
    np.testing.assert_allclose(out[2], 0.5 * out[0] - 2.0 * out[1], atol=1e-6 * np.abs(out).max())
    del rng


# ---------------------------------------------------------------------------
# Derivative engine (Sec. 2.2)
# ---------------------------------------------------------------------------
def test_telescoping_identity_of_summed_central_differences():
    # For a fully lit subaperture the sum of central differences telescopes:
    # sum_j (phi[j+1] - phi[j-1]) = phi[j1+1] + phi[j1] - phi[j0] - phi[j0-1].
    from paper_2606_07759_b300 import workloads as W
    w = W.scao_small()
    dm, wfs = w.dms[0], w.wfss[0]
    M, n = wfs.grid_m, wfs.n_sub
    k, dw = M // n, wfs.pupil_diam_m / M
    A, b = oracle.composite(oracle.pair_geom(dm, wfs), w.pair(0, 0).as_tuple())
    ros, lit, nv = oracle.valid_subaps(wfs.pupil_mask, n)
    cols = [5, 33, 61]
    out = oracle.im(dm.ifs, dm.mask, M, n, wfs.pupil_mask, None, A, b, dw, cols=cols)
    checked = 0
    for c, a in enumerate(cols):
        phi, _ = oracle.phase(dm.ifs[a], dm.mask, M, A, b)
        pad = np.zeros((M + 2, M + 2))
        pad[1:-1, 1:-1] = phi
        for si in range(n):
            for sj in range(n):
                if ros[si, sj] < 0 or lit[si, sj] != k * k:
                    continue
                i0, j0 = si * k + 1, sj * k + 1  # padded indices
                rows = slice(i0, i0 + k)
                cols_ = slice(j0, j0 + k)
                tx = (pad[rows, j0 + k] + pad[rows, j0 + k - 1] - pad[rows, j0] - pad[rows, j0 - 1]).sum()
                ty = (pad[i0 + k, cols_] + pad[i0 + k - 1, cols_] - pad[i0, cols_] - pad[i0 - 1, cols_]).sum()
                r = ros[si, sj]
                scale = 1.0 / (2 * dw * k * k)
                assert out[c, r] == pytest.approx(tx * scale, rel=1e-11, abs=1e-13)
                assert out[c, nv + r] == pytest.approx(ty * scale, rel=1e-11, abs=1e-13)
                checked += 1
    assert checked > 100


def test_low_frequency_slopes_match_continuous_gradient():
    # A wide Gaussian: the subaperture mean of the aligned central differences
    # converges to the mean continuous gradient over the subaperture square,
    # i.e. the boundary integral of phi over the subaperture edges (Sec. 2.2).
    N, dd, M, n, D = 96, 0.05, 48, 6, 3.6   # dw = 0.075, A = 1.5 I
    k, dw = M // n, D / M
    s = 4 * k * dw                          # Gaussian width: four subapertures
    sx_px, sy_px = 0.3, -0.45
    x0, y0 = 0.3, -0.2                      # centre in DM metres
    cN = (N - 1) / 2
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    X, Y = (xx - cN) * dd, (yy - cN) * dd
    f = np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / (2 * s * s))
    A, b = oracle.composite(geom(N, dd, M, D), (sx_px, sy_px, 0, 1))
    P = np.ones((M, M), np.uint8)
    ros, lit, nv = oracle.valid_subaps(P, n)
    out = oracle.im(f.astype(np.float32)[None], None, M, n, P, None, A, b, dw)[0]
    # sensor metres (u, v) see DM metres (u - sx dd, v - sy dd)
    gl, gw = np.polynomial.legendre.leggauss(24)

    def phi(u, v):
        return np.exp(-((u - sx_px * dd - x0) ** 2 + (v - sy_px * dd - y0) ** 2) / (2 * s * s))

    peak = np.abs(out).max()
    for si in range(1, n - 1):
        for sj in range(1, n - 1):
            u0, u1 = (sj * k - 0.5 - (M - 1) / 2) * dw, ((sj + 1) * k - 0.5 - (M - 1) / 2) * dw
            v0, v1 = (si * k - 0.5 - (M - 1) / 2) * dw, ((si + 1) * k - 0.5 - (M - 1) / 2) * dw
            vq = 0.5 * (v1 - v0) * gl + 0.5 * (v1 + v0)
            uq = 0.5 * (u1 - u0) * gl + 0.5 * (u1 + u0)
            area = (u1 - u0) * (v1 - v0)
            ex = 0.5 * (v1 - v0) * np.sum(gw * (phi(u1, vq) - phi(u0, vq))) / area
            ey = 0.5 * (u1 - u0) * np.sum(gw * (phi(uq, v1) - phi(uq, v0))) / area
            r = ros[si, sj]
            assert abs(out[r] - ex) < 2e-3 * peak
            assert abs(out[nv + r] - ey) < 2e-3 * peak


# ---------------------------------------------------------------------------
# Edge repair (Sec. 2.3): hand-worked cases
# ---------------------------------------------------------------------------
def _golden_cases():
    with open(os.path.join(GOLDEN, "edge_repair_cases.json")) as fh:
        return json.load(fh)["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"][:1])
def test_edge_repair_hand_worked_cases(case):
    n = case["n"]
    mask = np.zeros((n, n), np.uint8)
    if case.get("core_rect"):
        r0, r1, c0, c1 = case["core_rect"]
        mask[r0:r1 + 1, c0:c1 + 1] = 1
    for i, j in case.get("core_pixels", []):
        mask[i, j] = 1
    for i, j in case["core_minus"]:
        mask[i, j] = 0
    ii, jj = np.mgrid[0:n, 0:n].astype(np.float64)
    field = case["cj"] * jj + case["ci"] * ii + case["cii"] * ii * ii
    phi, cls = oracle.phase(field.astype(np.float32), mask, n, [1, 0, 0, 1], [0, 0])
    np.testing.assert_array_equal(cls == 1, mask == 1)
    for i, j, v, why in case["expected"]:
        assert phi[i, j] == pytest.approx(v, abs=1e-12), why


def test_edge_repair_reproduces_a_plane_on_thick_cores():
    # 2 P1 - P2 is exact for a plane wherever two core pixels line up.
    n = 32
    mask = _disc(n, 12.0)
    ii, jj = np.mgrid[0:n, 0:n].astype(np.float64)
    plane = 0.25 * jj - 0.5 * ii + 3.0
    phi, cls = oracle.phase(plane.astype(np.float32), mask, n, [1, 0, 0, 1], [0, 0])
    ring = cls == 2
    assert ring.sum() > 20
    np.testing.assert_allclose(phi[ring], plane[ring], atol=1e-12)
    assert np.all(phi[cls == 0] == 0)


# ---------------------------------------------------------------------------
# Tangents: central finite differences of the forward
# ---------------------------------------------------------------------------
def _kink_free_rows(w, d, wfs_i, p, steps, k):
    """Rows of the IM whose finite-difference stencil (p +- h) crosses no
    bilinear cell line and no change of the core set for parameter k."""
    dm, wfs = w.dms[d], w.wfss[wfs_i]
    M, n = wfs.grid_m, wfs.n_sub
    kk = M // n
    g = oracle.pair_geom(dm, wfs)
    e = np.zeros(4)
    e[k] = steps[k]
    ii, jj = np.mgrid[0:M, 0:M].astype(np.float64)
    bad = np.zeros((M, M), bool)
    cells = []
    cores = []
    for q in (np.asarray(p) - e, np.asarray(p) + e):
        A, b = oracle.composite(g, q)
        x = A[0] * jj + A[1] * ii + b[0]
        y = A[2] * jj + A[3] * ii + b[1]
        cells.append((np.floor(x), np.floor(y)))
        cores.append(oracle.core(dm.mask, dm.grid_n, M, A, b)[0])
    bad |= (cells[0][0] != cells[1][0]) | (cells[0][1] != cells[1][1]) | (cores[0] != cores[1])
    # a pixel reaches the slopes of subapertures up to 3 pixels away (ring 2 + derivative 1)
    from scipy.ndimage import binary_dilation
    bad = binary_dilation(bad, iterations=3)
    ros, _, nv = oracle.valid_subaps(wfs.pupil_mask, n)
    badsub = bad.reshape(n, kk, n, kk).any(axis=(1, 3))
    good = np.zeros(2 * nv, bool)
    for si in range(n):
        for sj in range(n):
            r = ros[si, sj]
            if r >= 0 and not badsub[si, sj]:
                good[r] = good[nv + r] = True
    return good


def test_tangents_match_central_finite_differences():
    from paper_2606_07759_b300 import workloads as W
    w = W.scao_small()
    p = np.array(w.pair(0, 0).as_tuple())
    steps = [1e-3, 1e-3, 1e-3, 1e-5]
    cols = [3, 20, 40, 71]
    T = oracle.pair_tangent(w, 0, 0, cols=cols, misreg=tuple(p))
    for k in range(4):
        e = np.zeros(4)
        e[k] = steps[k]
        fp = oracle.pair_im(w, 0, 0, cols=cols, misreg=tuple(p + e))
        fm = oracle.pair_im(w, 0, 0, cols=cols, misreg=tuple(p - e))
        fd = (fp - fm) / (2 * steps[k])
        good = _kink_free_rows(w, 0, 0, p, steps, k)
        assert good.mean() > 0.5
        scale = np.abs(T[k]).max()
        err = np.abs(T[k][:, good] - fd[:, good]).max()
        assert err <= 1e-4 * scale, (k, err, scale)

"""Seeded synthetic inputs with the shapes of the paper's workloads.

This module is shared by the CUDA path's tests/benchmark and by the CPU
oracle's tests.  It holds none of the method's arithmetic: no composite
affine, no resampling, no edge repair, no slopes and no subaperture
validity rule.  It only lays out actuator lattices, samples Gaussian
influence functions, draws binary masks and returns the raw geometric
parameters (pupil size, pixel pitches, altitudes, guide-star directions,
misregistrations) from which each side builds its own transforms.

Workload shapes follow the paper's systems: an ELT-like 39 m pupil sampled
at 480 px, a 68x68 Shack-Hartmann LGS sensor, DMs conjugated at 0, 4 and
12.7 km seen by LGS at 90 km and by NGS far off axis (Sec. 3, Sec. 4.2).
The paper's MORFEO/M4 data are not public, so these seeded Gaussian cubes
stand in for them.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

ARCSEC = math.pi / (180.0 * 3600.0)

# Gaussian influence function with coupling c at one actuator pitch p:
# exp(-p^2 / (2 sigma^2)) = c  ->  sigma = p / sqrt(-2 ln c).
def coupling_sigma(pitch_px: float, coupling: float = 0.15) -> float:
    return pitch_px / math.sqrt(-2.0 * math.log(coupling))


def disc_mask(n: int, outer_radius_px: float, inner_radius_px: float = 0.0) -> np.ndarray:
    """Binary annulus on an n x n grid of pixel centres (centre at (n-1)/2).

    A pixel is set when its centre's radius r satisfies inner <= r <= outer.
    """
    c = (n - 1) / 2.0
    y, x = np.mgrid[0:n, 0:n]
    r = np.hypot(x - c, y - c)
    return ((r <= outer_radius_px) & (r >= inner_radius_px)).astype(np.uint8)


@dataclasses.dataclass
class DM:
    """One deformable mirror (or virtual layer): cube [n_act][N][N] FP32."""
    ifs: np.ndarray            # float32 [n_act, N, N], row = y, column = x
    mask: Optional[np.ndarray]  # uint8 [N, N] or None (all ones)
    pixel_pitch_m: float
    altitude_m: float
    act_xy_px: np.ndarray      # float64 [n_act, 2] actuator centres (x, y) in DM pixels
    pitch_px: float
    support_eps: float = 1e-9

    @property
    def n_act(self) -> int:
        return int(self.ifs.shape[0])

    @property
    def grid_n(self) -> int:
        return int(self.ifs.shape[1])


@dataclasses.dataclass
class WFS:
    """One Shack-Hartmann sensor on an M x M grid (M = k * n_sub)."""
    n_sub: int
    grid_m: int
    pupil_diam_m: float
    src_height_m: float        # 0 = natural guide star at infinity
    field_rad: tuple           # guide-star direction (x, y) in radians
    pupil_mask: np.ndarray     # uint8 [M, M]
    rot_deg: float = 0.0
    mag: tuple = (1.0, 1.0)
    shift_m: tuple = (0.0, 0.0)
    obstruction: float = 0.0
    slope_scale: float = 1.0
    subap_valid: Optional[np.ndarray] = None  # uint8 [n_sub, n_sub] or None (>= 50 % rule)


@dataclasses.dataclass
class Misreg:
    """DM misregistration relative to the WFS: shift in DM pixels, rotation in degrees."""
    shift_x_px: float = 0.0
    shift_y_px: float = 0.0
    rot_deg: float = 0.0
    mag: float = 1.0

    def as_tuple(self):
        return (self.shift_x_px, self.shift_y_px, self.rot_deg, self.mag)


@dataclasses.dataclass
class Workload:
    name: str
    dms: List[DM]
    wfss: List[WFS]
    misregs: List[Misreg]      # [n_dm * n_wfs], pair index = dm * n_wfs + wfs

    def pair(self, d: int, w: int) -> Misreg:
        return self.misregs[d * len(self.wfss) + w]


def actuator_lattice(n_side: int, span_m: float, grid_n: int, pixel_pitch_m: float):
    """Square lattice of n_side x n_side actuators spanning span_m, in DM pixels.

    Returns (xy_px [n_side^2, 2], radius_m [n_side^2], pitch_m).
    """
    pitch_m = span_m / (n_side - 1)
    idx = np.arange(n_side) - (n_side - 1) / 2.0
    gx, gy = np.meshgrid(idx * pitch_m, idx * pitch_m)
    xm, ym = gx.ravel(), gy.ravel()
    c = (grid_n - 1) / 2.0
    xy_px = np.stack([xm / pixel_pitch_m + c, ym / pixel_pitch_m + c], axis=1)
    return xy_px, np.hypot(xm, ym), pitch_m


def gaussian_cube(xy_px: np.ndarray, sigma_px: float, grid_n: int,
                  mask: Optional[np.ndarray]) -> np.ndarray:
    """Separable Gaussian influence functions, multiplied by the DM mask, FP32."""
    n_act = xy_px.shape[0]
    cube = np.empty((n_act, grid_n, grid_n), dtype=np.float32)
    ax = np.arange(grid_n, dtype=np.float64)
    inv = 1.0 / (2.0 * sigma_px * sigma_px)
    m = None if mask is None else mask.astype(np.float32)
    for a in range(n_act):
        gx = np.exp(-(ax - xy_px[a, 0]) ** 2 * inv).astype(np.float32)
        gy = np.exp(-(ax - xy_px[a, 1]) ** 2 * inv).astype(np.float32)
        plane = np.outer(gy, gx)
        if m is not None:
            plane *= m
        cube[a] = plane
    return cube


def _uniform_misreg(rng: np.random.Generator, shift_px: float, rot_deg: float,
                    mag_rel: float) -> Misreg:
    return Misreg(float(rng.uniform(-shift_px, shift_px)), float(rng.uniform(-shift_px, shift_px)),
                  float(rng.uniform(-rot_deg, rot_deg)), float(1.0 + rng.uniform(-mag_rel, mag_rel)))


def scao_small(seed: int = 1) -> Workload:
    """11x11 DM on an 80x80 grid, 10x10 SH (k = 8), obstruction 0.2."""
    D, N, n_side, obs = 8.0, 80, 11, 0.2
    dd = D / N
    mask = disc_mask(N, N / 2.0, obs * N / 2.0)
    xy, r, pitch_m = actuator_lattice(n_side, D, N, dd)
    R = D / 2.0
    keep = (r <= R + 1e-9) & (r >= obs * R - 1e-9)
    xy = xy[keep]
    pitch_px = pitch_m / dd
    cube = gaussian_cube(xy, coupling_sigma(pitch_px), N, mask)
    n_sub, M = 10, 80
    wfs = WFS(n_sub, M, D, 0.0, (0.0, 0.0), disc_mask(M, M / 2.0, obs * M / 2.0), obstruction=obs)
    dm = DM(cube, mask, dd, 0.0, xy, pitch_px)
    return Workload("scao_small", [dm], [wfs], [Misreg(0.3, -0.2, 0.5, 1.01)])


def _elt_ground_dm(D: float, N: int, n_side: int, obs: float) -> DM:
    dd = D / N
    mask = disc_mask(N, N / 2.0, obs * N / 2.0)
    xy, r, pitch_m = actuator_lattice(n_side, D, N, dd)
    keep = r <= D / 2.0 + pitch_m + 1e-9
    xy = xy[keep]
    pitch_px = pitch_m / dd
    return DM(gaussian_cube(xy, coupling_sigma(pitch_px), N, mask), mask, dd, 0.0, xy, pitch_px)


def elt_single(seed: int = 2, n_side: int = 81, grid_n: int = 480, n_sub: int = 68) -> Workload:
    """ELT-scale single WFS: 81x81 DM on 480x480 (obstruction 0.28), 68x68 SH, M = 544.

    Smaller n_side / grid_n / n_sub give the same geometry at parity-test sizes.
    """
    D, obs = 39.0, 0.28
    dm = _elt_ground_dm(D, grid_n, n_side, obs)
    k = -(-grid_n // n_sub)  # ceil
    M = k * n_sub
    wfs = WFS(n_sub, M, D, 0.0, (0.0, 0.0), disc_mask(M, M / 2.0, obs * M / 2.0), obstruction=obs)
    rng = np.random.default_rng(seed)
    return Workload("elt_single", [dm], [wfs], [_uniform_misreg(rng, 1.0, 1.0, 0.01)])


def dense(wl: Workload) -> Workload:
    """The same workload with support_eps = 0: every influence function is
    resampled over its whole plane (the dense-cube accounting)."""
    dms = [dataclasses.replace(dm, support_eps=0.0) for dm in wl.dms]
    return Workload(wl.name + "_dense", dms, wl.wfss, wl.misregs)


def cosine_modes(N: int, dd: float, D: float, mask: np.ndarray, n_modes: int) -> np.ndarray:
    """The first n_modes 2-D cosines cos(pi n (x / D + 1/2)) cos(pi m (y / D + 1/2))
    over the mask (pixel centres, x along columns), piston excluded, ordered by
    n + m then n: float32 [n_modes, N, N]."""
    c = (np.arange(N) + 0.5) * dd - D / 2.0
    orders = sorted(((n, m) for n in range(2 * int(np.sqrt(n_modes)) + 4)
                     for m in range(2 * int(np.sqrt(n_modes)) + 4) if n + m > 0), key=lambda t: (t[0] + t[1], t[0]))
    orders = orders[:n_modes]
    cube = np.empty((n_modes, N, N), np.float32)
    mf = mask.astype(np.float32)
    for q, (n, m) in enumerate(orders):
        cx = np.cos(np.pi * n * (c / D + 0.5)).astype(np.float32)
        cy = np.cos(np.pi * m * (c / D + 0.5)).astype(np.float32)
        np.multiply(np.outer(cy, cx), mf, out=cube[q])
    return cube


def modal_elt(n_modes: int = 4519, seed: int = 8, grid_n: int = 480, n_sub: int = 68) -> Workload:
    """A modal cube at ELT scale standing in for a mirror-mode set with global
    support: n_modes 2-D cosine modes over the 480x480 pupil (obstruction
    0.28), one 68x68 Shack-Hartmann (k = 8, M = 544), support_eps = 0."""
    D, obs = 39.0, 0.28
    N = grid_n
    dd = D / N
    mask = disc_mask(N, N / 2.0, obs * N / 2.0)
    cube = cosine_modes(N, dd, D, mask, n_modes)
    k = -(-N // n_sub)
    M = k * n_sub
    wfs = WFS(n_sub, M, D, 0.0, (0.0, 0.0), disc_mask(M, M / 2.0, obs * M / 2.0), obstruction=obs)
    xy = np.tile([N / 2.0, N / 2.0], (n_modes, 1))
    dm = DM(cube, mask, dd, 0.0, xy, float(N), support_eps=0.0)
    rng = np.random.default_rng(seed)
    return Workload("modal_elt", [dm], [wfs], [_uniform_misreg(rng, 1.0, 1.0, 0.01)])


def modal_scao(n_max: int = 8, seed: int = 7) -> Workload:
    """A modal cube on the SCAO small geometry: the 2-D cosine modes
    cos(pi n (x / D + 1/2)) cos(pi m (y / D + 1/2)) over the DM mask, 0 <= n, m
    <= n_max without piston, global support (support_eps = 0)."""
    D, N, obs = 8.0, 80, 0.2
    dd = D / N
    mask = disc_mask(N, N / 2.0, obs * N / 2.0)
    c = (np.arange(N) + 0.5) * dd - D / 2.0          # pixel centres in metres
    X, Y = np.meshgrid(c, c)
    modes, xy = [], []
    for n in range(n_max + 1):
        for m in range(n_max + 1):
            if n == 0 and m == 0:
                continue
            modes.append((np.cos(np.pi * n * (X / D + 0.5)) * np.cos(np.pi * m * (Y / D + 0.5)) * mask)
                         .astype(np.float32))
            xy.append((N / 2.0, N / 2.0))
    cube = np.stack(modes)
    n_sub, M = 10, 80
    wfs = WFS(n_sub, M, D, 0.0, (0.0, 0.0), disc_mask(M, M / 2.0, obs * M / 2.0), obstruction=obs)
    dm = DM(cube, mask, dd, 0.0, np.array(xy), float(N), support_eps=0.0)
    rng = np.random.default_rng(seed)
    return Workload("modal_scao", [dm], [wfs], [_uniform_misreg(rng, 1.0, 1.0, 0.01)])


def mcao_batched(seed: int = 3, scale: float = 1.0) -> Workload:
    """3 DMs (0, 4, 12.7 km) x (6 LGS 68x68 at 7.5" + 3 NGS 2x2 at 55"), 39 m pupil.

    ``scale`` < 1 shrinks every grid, lattice and subaperture count for
    parity tests while keeping the altitude / cone / field geometry.
    """
    D, obs, H_lgs = 39.0, 0.28, 90e3
    N0 = max(16, int(round(480 * scale)))
    dd = D / N0
    lgs_field, ngs_field = 7.5 * ARCSEC, 55.0 * ARCSEC
    dms = []
    specs = [(0.0, 81), (4000.0, 49), (12700.0, 41)]
    for h, n_side in specs:
        n_side = max(5, int(round((n_side - 1) * scale)) + 1)
        if h == 0.0:
            dms.append(_elt_ground_dm(D, N0, n_side, obs))
            continue
        d_meta = D + 2.0 * h * ngs_field
        N = int(math.ceil(d_meta / dd))
        N += N % 2
        mask = disc_mask(N, d_meta / (2.0 * dd))
        xy, r, pitch_m = actuator_lattice(n_side, d_meta, N, dd)
        keep = r <= d_meta / 2.0 + pitch_m + 1e-9
        xy = xy[keep]
        pitch_px = pitch_m / dd
        dms.append(DM(gaussian_cube(xy, coupling_sigma(pitch_px), N, mask), mask, dd, h, xy, pitch_px))
    wfss = []
    n_lgs = max(2, int(round(68 * scale)))
    k_lgs = -(-N0 // n_lgs)
    M_lgs = k_lgs * n_lgs
    for az in range(0, 360, 60):
        a = math.radians(az)
        wfss.append(WFS(n_lgs, M_lgs, D, H_lgs, (lgs_field * math.cos(a), lgs_field * math.sin(a)),
                        disc_mask(M_lgs, M_lgs / 2.0, obs * M_lgs / 2.0), obstruction=obs))
    k_ngs = N0 // 2
    M_ngs = 2 * k_ngs
    for az in (30, 150, 270):
        a = math.radians(az)
        wfss.append(WFS(2, M_ngs, D, 0.0, (ngs_field * math.cos(a), ngs_field * math.sin(a)),
                        disc_mask(M_ngs, M_ngs / 2.0, obs * M_ngs / 2.0), obstruction=obs))
    rng = np.random.default_rng(seed)
    mis = [_uniform_misreg(rng, 1.0, 1.0, 0.01) for _ in range(len(dms) * len(wfss))]
    return Workload("mcao_batched", dms, wfss, mis)


def gaussian_cube_device(xy_px: np.ndarray, sigma_px: float, grid_n: int, mask: Optional[np.ndarray], device):
    """gaussian_cube computed on a torch device (the same separable formula:
    FP64 exponentials, FP32 outer product times the mask), for cubes too large
    for host memory."""
    import torch
    ax = torch.arange(grid_n, dtype=torch.float64, device=device)
    xy = torch.as_tensor(xy_px, dtype=torch.float64, device=device)
    inv = 1.0 / (2.0 * sigma_px * sigma_px)
    gx = torch.exp(-(ax[None, :] - xy[:, 0:1]) ** 2 * inv).float()
    gy = torch.exp(-(ax[None, :] - xy[:, 1:2]) ** 2 * inv).float()
    cube = torch.empty((xy.shape[0], grid_n, grid_n), dtype=torch.float32, device=device)
    m = None if mask is None else torch.as_tensor(mask, dtype=torch.float32, device=device)
    for a0 in range(0, xy.shape[0], 256):
        a1 = min(xy.shape[0], a0 + 256)
        blk = gy[a0:a1, :, None] * gx[a0:a1, None, :]
        cube[a0:a1] = blk * m if m is not None else blk
    return cube


def mcao_dictionary(seed: int = 9, scale: float = 1.0, device=None) -> Workload:
    """An LGS tomographic dictionary in the shape of the paper's MCAO run: 12
    components (the 3 DMs of mcao_batched at 0, 4 and 12.7 km, plus 9 virtual
    layers at 0.2-22 km on meta-pupils D + 2 h 80", i.e. 480-690 px grids, 70x70
    actuator lattices) seen by the 6 LGS 68x68 sensors (7.5", 90 km): 72 IMs,
    about 44,600 modes.  With ``device`` the cubes are generated there as torch
    tensors (about 57 GB at full scale); otherwise as numpy arrays."""
    D, obs, H_lgs = 39.0, 0.28, 90e3
    N0 = max(16, int(round(480 * scale)))
    dd = D / N0
    lgs_field, meta_field = 7.5 * ARCSEC, 80.0 * ARCSEC
    make = (lambda xy, sig, N, m: gaussian_cube_device(xy, sig, N, m, device)) if device is not None else gaussian_cube
    dms = []
    specs = [(0.0, 81), (4000.0, 49), (12700.0, 41)] + \
            [(h, 70) for h in (200.0, 1000.0, 2000.0, 4500.0, 7000.0, 10000.0, 14000.0, 18000.0, 22000.0)]
    for q, (h, n_side) in enumerate(specs):
        n_side = max(5, int(round((n_side - 1) * scale)) + 1)
        if q == 0:
            mask = disc_mask(N0, N0 / 2.0, obs * N0 / 2.0)
            xy, r, pitch_m = actuator_lattice(n_side, D, N0, dd)
            xy = xy[r <= D / 2.0 + pitch_m + 1e-9]
            pitch_px = pitch_m / dd
            dms.append(DM(make(xy, coupling_sigma(pitch_px), N0, mask), mask, dd, 0.0, xy, pitch_px))
            continue
        d_meta = D + 2.0 * h * (55.0 * ARCSEC if q < 3 else meta_field)
        N = int(math.ceil(d_meta / dd))
        N += N % 2
        mask = disc_mask(N, d_meta / (2.0 * dd))
        xy, r, pitch_m = actuator_lattice(n_side, d_meta, N, dd)
        xy = xy[r <= d_meta / 2.0 + pitch_m + 1e-9]
        pitch_px = pitch_m / dd
        dms.append(DM(make(xy, coupling_sigma(pitch_px), N, mask), mask, dd, h, xy, pitch_px))
    wfss = []
    n_lgs = max(2, int(round(68 * scale)))
    k_lgs = -(-N0 // n_lgs)
    M_lgs = k_lgs * n_lgs
    for az in range(0, 360, 60):
        a = math.radians(az)
        wfss.append(WFS(n_lgs, M_lgs, D, H_lgs, (lgs_field * math.cos(a), lgs_field * math.sin(a)),
                        disc_mask(M_lgs, M_lgs / 2.0, obs * M_lgs / 2.0), obstruction=obs))
    rng = np.random.default_rng(seed)
    mis = [_uniform_misreg(rng, 1.0, 1.0, 0.01) for _ in range(len(dms) * len(wfss))]
    return Workload("mcao_dictionary", dms, wfss, mis)


def probe_modes(dm: DM, D_m: float, n_modes: int = 16) -> np.ndarray:
    """Low-order 2-D cosine probe commands sampled at the actuator positions.

    c[m, a] = cos(pi n (x_a/D + 1/2)) cos(pi l (y_a/D + 1/2)), (n, l) in
    {0..4}^2 without (0, 0), ordered by n + l then n; the first n_modes.
    Returns the command matrix [n_modes, n_act] (float64).
    """
    pairs = [(n, l) for n in range(5) for l in range(5) if (n, l) != (0, 0)]
    pairs.sort(key=lambda t: (t[0] + t[1], t[0]))
    pairs = pairs[:n_modes]
    c = (dm.grid_n - 1) / 2.0
    x = (dm.act_xy_px[:, 0] - c) * dm.pixel_pitch_m
    y = (dm.act_xy_px[:, 1] - c) * dm.pixel_pitch_m
    cmd = np.empty((len(pairs), dm.n_act))
    for m, (n, l) in enumerate(pairs):
        cmd[m] = np.cos(math.pi * n * (x / D_m + 0.5)) * np.cos(math.pi * l * (y / D_m + 0.5))
    return cmd


def learned(seed: int = 5):
    """40x40 SH (k = 8, M = 320, no obstruction), 41x41 DM (p = 8 px), 16 probes.

    The DM grid is N = 352 px (the 320 px pupil plus two pitches on each side)
    with no DM mask, so that a sensor misregistered by up to one subaperture
    and 2 % still sees only the DM's active area: a mask edge inside the
    pupil would make the probe responses jump with the misregistration
    (pixels entering and leaving the edge-repair ring) and no local fit
    could follow them.
    """
    D, M, n_side = 8.0, 320, 41
    dd = D / M
    N = M + 32
    xy, r, pitch_m = actuator_lattice(n_side, D, N, dd)
    keep = r <= D / 2.0 + pitch_m + 1e-9
    xy = xy[keep]
    pitch_px = pitch_m / dd
    dm = DM(gaussian_cube(xy, coupling_sigma(pitch_px), N, None), None, dd, 0.0, xy, pitch_px)
    wfs = WFS(40, M, D, 0.0, (0.0, 0.0), disc_mask(M, M / 2.0), obstruction=0.0)
    cmd = probe_modes(dm, D, 16)
    return Workload("learned", [dm], [wfs], [Misreg()]), cmd


def random_misregs(rng: np.random.Generator, n: int, shift_px: float, rot_deg: float,
                   mag_rel: float) -> np.ndarray:
    """[n, 4] float64 (shift_x_px, shift_y_px, rot_deg, mag) drawn uniformly."""
    out = np.empty((n, 4))
    out[:, 0] = rng.uniform(-shift_px, shift_px, n)
    out[:, 1] = rng.uniform(-shift_px, shift_px, n)
    out[:, 2] = rng.uniform(-rot_deg, rot_deg, n)
    out[:, 3] = 1.0 + rng.uniform(-mag_rel, mag_rel, n)
    return out

// synim_geom.h -- the composite affine transform of one (DM, sensor) pair
// and its derivative with respect to the misregistration, shared by host code
// (per-pair parameters) and device code (per-sample probe transforms).
#pragma once

#include <cmath>

#include "synim.h"

#if defined(__CUDACC__)
#define SYNIM_HD __host__ __device__ __forceinline__
#else
#define SYNIM_HD inline
#endif

namespace synim {

// Host-side geometry of one DM and one sensor.
struct DmHost {
    int n_act = 0, N = 0, W = 0, Wp = 0;
    double dd = 0, h = 0;
};

struct WfsHost {
    int n_sub = 0, M = 0, k = 0, nv = 0, CH = 1;
    double D = 0, H = 0, th[2] = {0, 0}, rot = 0, mag[2] = {1, 1}, shift[2] = {0, 0}, scale = 1;
};

constexpr double kPi = 3.14159265358979323846;

// Composite affine (Sec. 2.1): DM pixel (x, y) = A (j, i) + b for sensor
// pixel (i, j).  Sensor frame: pixel -> metres about the grid centre, sensor
// rotation and anamorphic magnification, sensor shift; projection to the DM
// plane (cone factor 1 - h/H, footprint shift h theta); DM frame: shift,
// rotation (counter-clockwise positive) and magnification of the DM
// relative to the sensor; metres -> DM pixels about the DM grid centre.
SYNIM_HD void composite(const DmHost &D, const WfsHost &W, const synim_misreg &m, double A[4], double b[2]) {
    const double cone = (W.H > 0.0 && isfinite(W.H)) ? 1.0 - D.h / W.H : 1.0;
    const double dw = W.D / W.M;
    const double s = cone * dw / (D.dd * m.mag);
    const double tw = W.rot * kPi / 180.0, td = m.rot_deg * kPi / 180.0;
    const double ct = cos(td), st = sin(td), cw = cos(tw), sw = sin(tw);
    // X = R(tw) diag(mw)
    const double X00 = cw * W.mag[0], X01 = -sw * W.mag[1], X10 = sw * W.mag[0], X11 = cw * W.mag[1];
    // R(-td) = [[ct, st], [-st, ct]]
    A[0] = s * (ct * X00 + st * X10);
    A[1] = s * (ct * X01 + st * X11);
    A[2] = s * (-st * X00 + ct * X10);
    A[3] = s * (-st * X01 + ct * X11);
    const double tx = cone * W.shift[0] + D.h * W.th[0] - m.shift_x_px * D.dd;
    const double ty = cone * W.shift[1] + D.h * W.th[1] - m.shift_y_px * D.dd;
    const double inv = 1.0 / (D.dd * m.mag);
    const double cN = (D.N - 1) * 0.5, cM = (W.M - 1) * 0.5;
    b[0] = cN + inv * (ct * tx + st * ty) - (A[0] + A[1]) * cM;
    b[1] = cN + inv * (-st * tx + ct * ty) - (A[2] + A[3]) * cM;
}

// d(A, b)/dp_k in closed form: the shifts translate by -R(-td) e / m; the
// rotation turns the map about the DM centre (dA = -J A, db = -J (b - cN),
// J = [[0, -1], [1, 0]], per radian); the magnification scales it about the
// DM centre (dA = -A / m, db = -(b - cN) / m).
SYNIM_HD void composite_jac(const DmHost &D, const synim_misreg &m, const double A[4], const double b[2],
                   double dA[16], double db[8]) {
    const double td = m.rot_deg * kPi / 180.0, ct = cos(td), st = sin(td);
    const double cN = (D.N - 1) * 0.5, rad = kPi / 180.0;
    for (int q = 0; q < 16; ++q) dA[q] = 0.0;
    db[0] = -ct / m.mag; db[1] = st / m.mag;
    db[2] = -st / m.mag; db[3] = -ct / m.mag;
    dA[8] = rad * A[2]; dA[9] = rad * A[3]; dA[10] = -rad * A[0]; dA[11] = -rad * A[1];
    db[4] = rad * (b[1] - cN); db[5] = -rad * (b[0] - cN);
    for (int q = 0; q < 4; ++q) dA[12 + q] = -A[q] / m.mag;
    db[6] = -(b[0] - cN) / m.mag; db[7] = -(b[1] - cN) / m.mag;
}

}  // namespace synim

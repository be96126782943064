"""Python front end of the CUDA library: device memory and streams from PyTorch,
every step of the IM computation in libsynim.so (include/synim.h).
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from . import abi


def _misreg_array(misregs) -> ctypes.Array:
    arr = (abi.synim_misreg * len(misregs))()
    for q, m in enumerate(misregs):
        t = m.as_tuple() if hasattr(m, "as_tuple") else tuple(m)
        arr[q] = abi.synim_misreg(*[float(v) for v in t])
    return arr


def _host_u8(a) -> Optional[np.ndarray]:
    if a is None:
        return None
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint8))


class SynIM:
    """Interaction matrices of n_dm DMs x n_wfs Shack-Hartmann sensors on one GPU.

    ``dms`` items need: ifs (numpy float32 [n_act, N, N] or a CUDA float32
    tensor), mask (uint8 [N, N] or None), pixel_pitch_m, altitude_m and
    optionally support_eps.  ``wfss`` items need: n_sub, grid_m,
    pupil_diam_m, src_height_m, field_rad, rot_deg, mag, shift_m,
    pupil_mask, subap_valid, obstruction, slope_scale.  ``slope_engine`` is
    "numerical" (central differences with edge repair) or "telescoping" (the
    edge-sum engine of Sec. 2.2; ``compute`` only).
    """

    def __init__(self, dms: Sequence, wfss: Sequence, threads_per_cta: int = 0, ctas_per_sm: int = 0,
                 use_graph: bool = True, profile: bool = False, device: Optional[torch.device] = None,
                 autotune: bool = False, device_mem_cap: int = 0, slope_engine: str = "numerical"):
        self._L = abi.load()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.n_dm, self.n_wfs = len(dms), len(wfss)
        keep = []
        dd = (abi.synim_dm_desc * self.n_dm)()
        for q, dm in enumerate(dms):
            ifs = dm.ifs
            if isinstance(ifs, torch.Tensor):
                if ifs.dtype != torch.float32 or not ifs.is_contiguous():
                    ifs = ifs.float().contiguous()
                on_dev = 1 if ifs.is_cuda else 0
                ptr = ifs.data_ptr()
                n_act, N = ifs.shape[0], ifs.shape[1]
            else:
                ifs = np.ascontiguousarray(ifs, dtype=np.float32)
                on_dev, ptr = 0, ifs.ctypes.data
                n_act, N = ifs.shape[0], ifs.shape[1]
            keep.append(ifs)
            mask = _host_u8(getattr(dm, "mask", None))
            keep.append(mask)
            dd[q] = abi.synim_dm_desc(n_act, N, float(dm.pixel_pitch_m), float(dm.altitude_m), ptr, on_dev,
                                      None if mask is None else mask.ctypes.data,
                                      float(getattr(dm, "support_eps", 1e-9)))
        ww = (abi.synim_wfs_desc * self.n_wfs)()
        for q, w in enumerate(wfss):
            pm = _host_u8(getattr(w, "pupil_mask", None))
            sv = _host_u8(getattr(w, "subap_valid", None))
            keep += [pm, sv]
            d = abi.synim_wfs_desc()
            d.n_sub, d.grid_m = int(w.n_sub), int(w.grid_m)
            d.pupil_diam_m, d.src_height_m = float(w.pupil_diam_m), float(w.src_height_m)
            d.field_rad[0], d.field_rad[1] = float(w.field_rad[0]), float(w.field_rad[1])
            d.rot_deg = float(getattr(w, "rot_deg", 0.0))
            mag = getattr(w, "mag", (1.0, 1.0))
            d.mag[0], d.mag[1] = float(mag[0]), float(mag[1])
            sh = getattr(w, "shift_m", (0.0, 0.0))
            d.shift_m[0], d.shift_m[1] = float(sh[0]), float(sh[1])
            d.pupil_mask = None if pm is None else pm.ctypes.data
            d.subap_valid = None if sv is None else sv.ctypes.data
            d.obstruction = float(getattr(w, "obstruction", 0.0))
            d.slope_scale = float(getattr(w, "slope_scale", 1.0))
            ww[q] = d
        engines = {"numerical": abi.ENGINE_NUMERICAL, "telescoping": abi.ENGINE_TELESCOPING}
        if slope_engine not in engines:
            raise ValueError(f"slope_engine must be one of {sorted(engines)}")
        opts = abi.synim_opts(int(threads_per_cta), int(ctas_per_sm), 1 if use_graph else 0, 1 if autotune else 0,
                              1 if profile else 0, int(device_mem_cap), engines[slope_engine])
        ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            abi.check(self._L.synim_im_create(dd, self.n_dm, ww, self.n_wfs, ctypes.byref(opts),
                                              ctypes.byref(ctx)))
        self._ctx = ctx
        self.shapes = {}
        for d in range(self.n_dm):
            for w in range(self.n_wfs):
                self.shapes[(d, w)] = self.query(d, w)

    # ------------------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            self._L.synim_im_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def query(self, d: int, w: int):
        """(n_rows, n_cols) of the IM of pair (d, w)."""
        r, c = ctypes.c_int64(), ctypes.c_int64()
        abi.check(self._L.synim_im_query(self._ctx, d, w, ctypes.byref(r), ctypes.byref(c)), self._ctx)
        return int(r.value), int(c.value)

    def dm_window(self, d: int) -> int:
        W = ctypes.c_int32()
        abi.check(self._L.synim_dm_window(self._ctx, d, ctypes.byref(W)), self._ctx)
        return int(W.value)

    def tuning(self, mode: int = 0):
        """(threads per CTA, lanes per segment, kernel ms) chosen by the autotuner, or None."""
        th, ln, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        st = self._L.synim_im_tuning(self._ctx, mode, ctypes.byref(th), ctypes.byref(ln), ctypes.byref(ms))
        return (int(th.value), int(ln.value), float(ms.value)) if st == 0 else None

    def kernel_ms(self):
        """(summed device ms, launches) of the IM kernel since the last call (profile=True)."""
        ms, n = ctypes.c_double(), ctypes.c_int32()
        abi.check(self._L.synim_im_kernel_ms(self._ctx, ctypes.byref(ms), ctypes.byref(n)), self._ctx)
        return float(ms.value), int(n.value)

    def pair_affine(self, d: int, w: int, misreg):
        A = (ctypes.c_double * 4)()
        b = (ctypes.c_double * 2)()
        m = _misreg_array([misreg])
        abi.check(self._L.synim_pair_affine(self._ctx, d, w, m, A, b), self._ctx)
        return np.array(A[:]), np.array(b[:])

    def alloc_outputs(self):
        """One FP32 tensor [n_act, 2 nv] per pair (row a = IM column a)."""
        return [torch.empty((self.shapes[(d, w)][1], self.shapes[(d, w)][0]), dtype=torch.float32,
                            device=self.device)
                for d in range(self.n_dm) for w in range(self.n_wfs)]

    def _stream(self, stream):
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        return ctypes.c_void_p(s.cuda_stream)

    def compute(self, misregs, out=None, stream=None):
        """All IMs for the per-pair misregistrations (pair index = d * n_wfs + w)."""
        np_ = self.n_dm * self.n_wfs
        if len(misregs) != np_:
            raise ValueError(f"need {np_} misregistrations")
        out = self.alloc_outputs() if out is None else out
        ptrs = (ctypes.c_void_p * np_)(*[None if t is None else t.data_ptr() for t in out])
        abi.check(self._L.synim_im_compute(self._ctx, _misreg_array(misregs), ptrs, self._stream(stream)),
                  self._ctx)
        return out

    def check(self, stream=None):
        abi.check(self._L.synim_im_check(self._ctx, self._stream(stream)), self._ctx)

    def wait_selftest(self, limit_clocks: int = 1 << 20, stream=None) -> int:
        """Status of the bounded-wait self-test (SYNIM_ERR_TIMEOUT = 5 when the wait gave up)."""
        return int(self._L.synim_wait_selftest(self._ctx, int(limit_clocks), self._stream(stream)))

    def sensitivity(self, misregs, out=None, d_out=None, stream=None):
        """IMs and their tangents dIM/dp_k, p = (shift_x_px, shift_y_px, rot_deg, mag).

        Returns (ims, tangents) with tangents[p][k] shaped like ims[p].
        """
        np_ = self.n_dm * self.n_wfs
        out = self.alloc_outputs() if out is None else out
        if d_out is None:
            d_out = [[torch.empty_like(t) for _ in range(4)] for t in out]
        ptrs = (ctypes.c_void_p * np_)(*[None if t is None else t.data_ptr() for t in out])
        dptrs = (ctypes.c_void_p * (4 * np_))(*[None if t is None else t.data_ptr() for ts in d_out for t in ts])
        abi.check(self._L.synim_im_sensitivity(self._ctx, _misreg_array(misregs), ptrs, dptrs,
                                               self._stream(stream)), self._ctx)
        return out, d_out

    def vjp(self, misregs, grad_ims, stream=None):
        """grad_p[p, k] = sum(grad_ims[p] * dIM_p / dp_k) as a float64 numpy array [n_pairs, 4]."""
        np_ = self.n_dm * self.n_wfs
        keep = [None if g is None else g.contiguous().float() for g in grad_ims]
        gptrs = (ctypes.c_void_p * np_)(*[None if g is None else g.data_ptr() for g in keep])
        gp = (ctypes.c_double * (4 * np_))()
        abi.check(self._L.synim_im_vjp(self._ctx, _misreg_array(misregs), gptrs, gp, self._stream(stream)),
                  self._ctx)
        return np.array(gp[:]).reshape(np_, 4)

    # ---- tomographic projection (Sec. 2.5) ----
    def projection_rows(self, w: int, n_dir: int, bin: int) -> int:
        r = ctypes.c_int64()
        abi.check(self._L.synim_projection_rows(self._ctx, w, n_dir, bin, ctypes.byref(r)), self._ctx)
        return int(r.value)

    @staticmethod
    def _dirs(dirs):
        d = np.ascontiguousarray(np.asarray(dirs, np.float64).reshape(-1, 2))
        return d, d.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), d.shape[0]

    @staticmethod
    def _ints(v):
        a = np.ascontiguousarray(np.asarray(v, np.int32).ravel())
        return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), a.size

    def projection_matrix(self, w: int, dirs, bin: int, comps, stream=None):
        """P_X of components comps as a tensor [n_cols, rows] (row c = actuator c's column)."""
        d, dp, nd = self._dirs(dirs)
        c, cp, nc = self._ints(comps)
        rows = self.projection_rows(w, nd, bin)
        ncols = sum(self.shapes[(int(q), 0)][1] for q in c)
        out = torch.empty((ncols, rows), dtype=torch.float32, device=self.device)
        abi.check(self._L.synim_projection_matrix(self._ctx, w, nd, dp, bin, nc, cp, ctypes.c_void_p(out.data_ptr()),
                                                  self._stream(stream)), self._ctx)
        return out

    def projection_opt(self, w: int, dirs, bin: int, dms, layers, lam: float, stream=None):
        """P_opt = (P_DM^T P_DM + lam I)^-1 P_DM^T P_Layer as a tensor [n_dm_cols, n_layer_cols]."""
        d, dp, nd = self._dirs(dirs)
        a, ap, na = self._ints(dms)
        b, bp, nb = self._ints(layers)
        nd_cols = sum(self.shapes[(int(q), 0)][1] for q in a)
        nl_cols = sum(self.shapes[(int(q), 0)][1] for q in b)
        out = torch.empty((nl_cols, nd_cols), dtype=torch.float32, device=self.device)
        abi.check(self._L.synim_projection_opt(self._ctx, w, nd, dp, bin, na, ap, nb, bp, float(lam),
                                               ctypes.c_void_p(out.data_ptr()), self._stream(stream)), self._ctx)
        return out.t()

    # ---- probe responses (input of the misregistration estimators) ----
    def probe_attach(self, d: int, w: int, cmd):
        """Attach probe commands cmd [n_modes, n_act] (float64) to pair (d, w)."""
        c = np.ascontiguousarray(cmd, dtype=np.float64)
        abi.check(self._L.synim_probe_attach(self._ctx, d, w, c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             c.shape[0]), self._ctx)
        n_sub, C = ctypes.c_int32(), ctypes.c_int32()
        abi.check(self._L.synim_probe_query(self._ctx, ctypes.byref(n_sub), ctypes.byref(C), None), self._ctx)
        self.probe_shape = (int(n_sub.value), int(n_sub.value), int(C.value))
        valid = np.zeros((n_sub.value, n_sub.value), np.uint8)
        abi.check(self._L.synim_probe_query(self._ctx, None, None, valid.ctypes.data), self._ctx)
        self.probe_valid = valid.astype(bool)

    @staticmethod
    def _params(params, device):
        t = torch.as_tensor(params, dtype=torch.float64)
        return t.to(device).contiguous().reshape(-1, 4)

    def probe_response(self, params, tangents: bool = False, stream=None):
        """Clean slope maps [n, n_sub, n_sub, C] (and tangents [4, n, ...]) for params [n, 4]."""
        p = self._params(params, self.device)
        n = p.shape[0]
        maps = torch.empty((n, *self.probe_shape), dtype=torch.float32, device=self.device)
        dmaps = torch.empty((4, n, *self.probe_shape), dtype=torch.float32, device=self.device) if tangents else None
        abi.check(self._L.synim_probe_response(self._ctx, ctypes.c_void_p(p.data_ptr()), n,
                                               ctypes.c_void_p(maps.data_ptr()),
                                               None if dmaps is None else ctypes.c_void_p(dmaps.data_ptr()),
                                               self._stream(stream)), self._ctx)
        return (maps, dmaps) if tangents else maps

    def probe_generate(self, params, seed: int, sample0: int = 0, noise_rel: float = 0.01, out=None,
                       stream=None):
        """Noisy bfloat16 probe inputs [n, n_sub, n_sub, C] for params [n, 4]."""
        p = self._params(params, self.device)
        n = p.shape[0]
        if out is None:
            out = torch.empty((n, *self.probe_shape), dtype=torch.bfloat16, device=self.device)
        abi.check(self._L.synim_probe_generate(self._ctx, ctypes.c_void_p(p.data_ptr()), n, seed, sample0,
                                               float(noise_rel), ctypes.c_void_p(out.data_ptr()),
                                               self._stream(stream)), self._ctx)
        return out

    # ---- misregistration estimators ----
    METHODS = {"gn": 0, "cnn": 1, "cnn+gn": 2}

    def gn_config(self, max_iter: int = 30, tol: float = 1e-4, scale=None):
        sc = None if scale is None else (ctypes.c_double * 4)(*[float(v) for v in scale])
        abi.check(self._L.synim_gn_config(self._ctx, int(max_iter), float(tol), sc), self._ctx)

    def estimate(self, slopes, method: str = "gn", init=None, stream=None):
        """Estimate the probed pair's misregistration from slope maps [n, n_sub, n_sub, C].

        Returns (params [n, 4] float64, relative residual [n], iterations [n], converged [n]).
        """
        y = torch.as_tensor(slopes)
        if y.device != self.device or y.dtype != torch.float32 or not y.is_contiguous():
            y = y.to(self.device, torch.float32).contiguous()
        n = y.shape[0]
        # synim_misreg is four doubles: an [n, 4] float64 array is its array
        # (default start: the prior centre nudged off the exact grid alignment)
        p = np.empty((max(n, 1), 4), np.float64)
        p[:n] = (1e-3, 1e-3, 1e-3, 1.0 + 1e-5) if init is None else np.asarray(init, np.float64).reshape(n, 4)
        res = np.zeros(max(n, 1))
        it = np.zeros(max(n, 1), np.int32)
        cv = np.zeros(max(n, 1), np.int32)
        abi.check(self._L.synim_misreg_estimate(self._ctx, ctypes.c_void_p(y.data_ptr()), n, self.METHODS[method],
                                                p.ctypes.data_as(ctypes.POINTER(abi.synim_misreg)),
                                                res.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                self._stream(stream)), self._ctx)
        abi.check(self._L.synim_misreg_estimate_stats(self._ctx, it.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                      cv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), self._ctx)
        return p[:n], res[:n], it[:n], cv[:n].astype(bool)

    # ---- the learned estimator ----
    def cnn_n_params(self) -> int:
        return int(self._L.synim_cnn_n_params(self.probe_shape[0], self.probe_shape[2]))

    def cnn_init(self, params, center, range_):
        """Create the network with initial parameters (float32 [n_params]) and the
        output normalisation (p - center) / range."""
        w = np.ascontiguousarray(params, np.float32)
        norm = np.ascontiguousarray(list(center) + list(range_), np.float64)
        abi.check(self._L.synim_cnn_init(self._ctx, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                         norm.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), self._ctx)

    def cnn_get(self):
        w = np.zeros(self.cnn_n_params(), np.float32)
        norm = np.zeros(8)
        abi.check(self._L.synim_cnn_get(self._ctx, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                        norm.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), self._ctx)
        return w, norm[:4], norm[4:]

    def cnn_save(self, path=None) -> bytes:
        """Checkpoint of the network and its Adam state (synim_cnn_save); written
        to path when given.  Returns the bytes."""
        n = ctypes.c_int64()
        abi.check(self._L.synim_cnn_save(self._ctx, None, 0, ctypes.byref(n)), self._ctx)
        buf = np.zeros(n.value, np.uint8)
        abi.check(self._L.synim_cnn_save(self._ctx, buf.ctypes.data_as(ctypes.c_void_p), n.value, ctypes.byref(n)),
                  self._ctx)
        data = buf.tobytes()
        if path is not None:
            with open(path, "wb") as f:
                f.write(data)
        return data

    def cnn_load(self, src):
        """Restore a checkpoint (bytes, or a path to a file written by cnn_save)."""
        if not isinstance(src, (bytes, bytearray)):
            with open(src, "rb") as f:
                src = f.read()
        buf = np.frombuffer(bytes(src), np.uint8)
        abi.check(self._L.synim_cnn_load(self._ctx, buf.ctypes.data_as(ctypes.c_void_p), buf.size), self._ctx)

    def cnn_forward(self, x, stream=None):
        """Normalised outputs [n, 4] for bfloat16 maps x [n, n_sub, n_sub, C]."""
        x = x.to(self.device, torch.bfloat16).contiguous()
        out = torch.empty((x.shape[0], 4), dtype=torch.float32, device=self.device)
        abi.check(self._L.synim_cnn_forward(self._ctx, ctypes.c_void_p(x.data_ptr()), x.shape[0],
                                            ctypes.c_void_p(out.data_ptr()), self._stream(stream)), self._ctx)
        return out

    def cnn_grad(self, x, target, stream=None):
        """(loss, gradient [n_params]) of one forward/backward pass without an update."""
        x = x.to(self.device, torch.bfloat16).contiguous()
        t = torch.as_tensor(target, dtype=torch.float32).to(self.device).contiguous()
        loss = ctypes.c_double()
        g = np.zeros(self.cnn_n_params(), np.float32)
        abi.check(self._L.synim_cnn_grad(self._ctx, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                         x.shape[0], ctypes.byref(loss),
                                         g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), self._stream(stream)),
                  self._ctx)
        return float(loss.value), g

    def cnn_train(self, params, epochs: int = 10, batch: int = 256, lr: float = 1e-3, lr_final: float = 0.0,
                  noise_rel: float = 0.01, seed: int = 0, sample0: int = 0, stream=None):
        """Train on samples with misregistrations params [n, 4]; returns the per-epoch loss."""
        p = self._params(params, self.device)
        o = abi.synim_train_opts(int(epochs), int(batch), float(lr), float(lr_final), 0.0, 0.0, 0.0,
                                 float(noise_rel), int(seed), int(sample0))
        loss = (ctypes.c_double * int(epochs))()
        abi.check(self._L.synim_cnn_train(self._ctx, ctypes.c_void_p(p.data_ptr()), p.shape[0], ctypes.byref(o),
                                          loss, self._stream(stream)), self._ctx)
        return np.array(loss[:])


def cnn_init_params(n_channels: int, seed: int = 0, input_scale: float = 1.0, side: int = 40) -> np.ndarray:
    """He-uniform initial parameters of the estimator network (seeded) for side x side
    maps, the first layer scaled by input_scale (1 / typical input magnitude), the
    dense layer Glorot-uniform; biases zero."""
    rng = np.random.default_rng(seed)
    out = []
    for cin, fan, sc in ((n_channels, 9 * n_channels, input_scale), (64, 576, 1.0), (64, 576, 1.0)):
        lim = np.sqrt(6.0 / fan) * sc
        out += [rng.uniform(-lim, lim, 64 * 9 * cin), np.zeros(64)]
    h3 = ((side - 1) // 2) // 2 + 1
    nf = h3 * h3 * 64
    lim = np.sqrt(6.0 / (nf + 4))
    out += [rng.uniform(-lim, lim, 4 * nf), np.zeros(4)]
    return np.concatenate(out).astype(np.float32)


class IMFunction(torch.autograd.Function):
    """IMs as a differentiable function of the misregistrations.

    forward(params [n_pairs, 4] tensor on any device, synim) -> tuple of IMs;
    backward uses the library's adjoint kernel (synim_im_vjp) and returns the
    parameter gradient on the device and with the dtype of ``params``.
    """

    @staticmethod
    def forward(ctx, params, synim):
        mis = params.detach().cpu().double().tolist()
        ctx.synim, ctx.mis, ctx.pdtype, ctx.pdevice = synim, mis, params.dtype, params.device
        return tuple(synim.compute(mis))

    @staticmethod
    def backward(ctx, *grads):
        gp = ctx.synim.vjp(ctx.mis, list(grads))
        return torch.from_numpy(gp).to(device=ctx.pdevice, dtype=ctx.pdtype), None

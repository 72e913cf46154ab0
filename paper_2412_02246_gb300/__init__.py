"""GB300 (sm_103a) visibility-based binned angular bispectrum estimator (arXiv 2412.02246).

Thin ctypes binding over the C ABI declared in ``include/abs.h`` (libabs.so).
Every step of the estimator runs in the library's CUDA kernels; this module
only marshals arguments (torch device tensors -> pointers, the current CUDA
stream).  There is no CPU fallback: if libabs.so is missing or cannot load,
every call raises.

Names follow the C ABI: ``abs_grid``, ``abs_filter_fft``, ``abs_triple``,
``abs_normalise``, ``abs_estimate``, ``abs_estimate_many``,
``abs_estimate_batched``, ``abs_estimate_host``; around the path ``abs_rebin``
((l1, mu, t) cells and ensemble statistics), ``abs_bana_d`` (the discretely
sampled prediction), ``abs_simulate_vis`` (the visibility simulator),
``autotune`` / ``tuned_shape`` (launch-shape autotuner) and ``profile`` /
``profile_read`` (stage tracing); plus the host helpers ``abs_ring_q``,
``abs_fft_size``, ``abs_triplets``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libabs.so")

ABS_OK, ABS_ERR_INVALID_ARG, ABS_ERR_CUDA, ABS_ERR_OOM, ABS_ERR_TIMEOUT, ABS_ERR_UNSUPPORTED, \
    ABS_ERR_DEVICE = range(7)
ABS_KERNEL_NGP, ABS_KERNEL_GAUSS = 0, 1
ABS_FP32, ABS_SPLIT_BF16 = 0, 1
ABS_W_MEAN_UNITMASK, ABS_W_PAPER_LITERAL, ABS_W_NOISE = 0, 1, 2
ABS_BEAM_NONE, ABS_BEAM_MWA_TILE, ABS_BEAM_GAUSS = 0, 1, 2
_STATUS = {0: "ABS_OK", 1: "ABS_ERR_INVALID_ARG", 2: "ABS_ERR_CUDA", 3: "ABS_ERR_OOM",
           4: "ABS_ERR_TIMEOUT", 5: "ABS_ERR_UNSUPPORTED", 6: "ABS_ERR_DEVICE"}


class AbsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class abs_stage_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("ms", ctypes.c_double), ("launches", ctypes.c_int64)]


class abs_config(ctypes.Structure):
    _fields_ = [("n_grid", ctypes.c_int32), ("du", ctypes.c_double), ("kernel", ctypes.c_int32),
                ("sigma_cells", ctypes.c_double), ("radius_cells", ctypes.c_int32),
                ("n_bins", ctypes.c_int32), ("ell_edges", ctypes.POINTER(ctypes.c_double)),
                ("n_fft", ctypes.c_int32), ("precision", ctypes.c_int32), ("norm_A", ctypes.c_double),
                ("weight_mode", ctypes.c_int32)]


class abs_config3d(ctypes.Structure):
    _fields_ = [("base", abs_config), ("n_chan", ctypes.c_int32), ("n_dbins", ctypes.c_int32),
                ("delay_edges", ctypes.POINTER(ctypes.c_int32)), ("n_z", ctypes.c_int32)]


class abs_item(ctypes.Structure):
    _fields_ = [("cfg", ctypes.POINTER(abs_config)), ("n_vis", ctypes.c_int64), ("d_uv", ctypes.c_void_p),
                ("d_vis", ctypes.c_void_p), ("n_trip", ctypes.c_int32), ("d_ijk", ctypes.c_void_p),
                ("d_B", ctypes.c_void_p), ("d_count", ctypes.c_void_p), ("d_ellbar", ctypes.c_void_p)]


_lib = None


def load(path: str | None = None):
    """Load libabs.so (built by ``paper_2412_02246_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libabs.so not built ({p}); run paper_2412_02246_gb300.build.build()")
    lib = ctypes.CDLL(p)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    C = ctypes.POINTER(abs_config)
    sig = {
        "abs_create": ([ctypes.POINTER(P), i32, P], ctypes.c_int),
        "abs_destroy": ([P], ctypes.c_int),
        "abs_last_error": ([P], ctypes.c_char_p),
        "abs_sync": ([P], ctypes.c_int),
        "abs_ring_q": ([C, P], ctypes.c_int),
        "abs_fft_size": ([C, P], ctypes.c_int),
        "abs_triplets": ([C, i32, P, P], ctypes.c_int),
        "abs_grid": ([P, C, i64, P, P, P, P, P], ctypes.c_int),
        "abs_filter_fft": ([P, C, P, P, P, P], ctypes.c_int),
        "abs_triple": ([P, C, P, P, i32, P, P, P], ctypes.c_int),
        "abs_normalise": ([P, C, i32, P, P, P, P, P], ctypes.c_int),
        "abs_estimate": ([P, C, i64, P, P, i32, P, P, P, P], ctypes.c_int),
        "abs_estimate_many": ([P, C, i64, P, i32, P, i32, P, P, P, P], ctypes.c_int),
        "abs_estimate_host": ([P, C, i64, P, i32, P, i32, P, P, P, P], ctypes.c_int),
        "abs_estimate_batched": ([P, i32, P], ctypes.c_int),
        "abs_estimate_batched_host": ([P, i32, P], ctypes.c_int),
        "abs_triple_sums_static": ([C, P, i32, P, P, P], ctypes.c_int),
        "abs_profile": ([P, i32], ctypes.c_int),
        "abs_profile_read": ([P, i32, P, P], ctypes.c_int),
        "abs_autotune": ([P, i32], ctypes.c_int),
        "abs_probe_timeout": ([P, i32], ctypes.c_int),
        "abs_inject_alloc_failures": ([P, i32], ctypes.c_int),
        "abs_rebin": ([P, P, i32, i32, P, P, P, P, i32, i32, P, P, P], ctypes.c_int),
        "abs_bana_d": ([P, P, P, P, i32, P, P, ctypes.c_double, P], ctypes.c_int),
        "abs_simulate_vis": ([P, i32, ctypes.c_double, P, i32, ctypes.c_double, i64, P, P], ctypes.c_int),
        "abs_tuned_shape": ([P, P, P, P, P], ctypes.c_int),
        "abs_triplets_3d": ([P, i32, P, P], ctypes.c_int),
        "abs_estimate_3d": ([P, P, i64, P, P, i32, P, P, P, P], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


# ------------------------------------------------------------------ config


@dataclass
class Config:
    n_grid: int
    du: float
    ell_edges: np.ndarray
    kernel: int = ABS_KERNEL_GAUSS
    sigma_cells: float = 1.0
    radius_cells: int = 3
    n_fft: int = 0
    precision: int = ABS_FP32
    norm_A: float = 1.0
    weight_mode: int = ABS_W_MEAN_UNITMASK

    def __post_init__(self):
        self.ell_edges = np.ascontiguousarray(self.ell_edges, np.float64)
        self._c = abs_config(int(self.n_grid), float(self.du), int(self.kernel), float(self.sigma_cells),
                             int(self.radius_cells), len(self.ell_edges) - 1,
                             self.ell_edges.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             int(self.n_fft), int(self.precision), float(self.norm_A),
                             int(self.weight_mode))

    @property
    def n_bins(self) -> int:
        return len(self.ell_edges) - 1

    @property
    def N(self) -> int:
        """The sky-grid side the library uses for this configuration (abs_fft_size)."""
        if not hasattr(self, "_N"):
            self._N = abs_fft_size(self)
        return self._N

    def ref(self):
        return ctypes.byref(self._c)

    @classmethod
    def from_workload(cls, wl, **kw):
        prec = ABS_SPLIT_BF16 if getattr(wl, "precision", "fp32") == "split_bf16" else ABS_FP32
        args = dict(n_grid=wl.n_grid, du=wl.du, ell_edges=wl.ell_edges,
                    kernel=ABS_KERNEL_NGP if wl.kernel == "ngp" else ABS_KERNEL_GAUSS,
                    sigma_cells=wl.sigma_cells, radius_cells=wl.radius_cells, precision=prec)
        args.update(kw)
        return cls(**args)


@dataclass
class Config3D:
    """abs_config3d: the per-channel configuration, the channel count, the delay-bin edges in
    |t| and the line-of-sight grid N_z (0: 3 t_max + 1)."""
    base: Config
    n_chan: int
    delay_edges: np.ndarray
    n_z: int = 0

    def __post_init__(self):
        self.delay_edges = np.ascontiguousarray(self.delay_edges, np.int32)
        self._c = abs_config3d(self.base._c, int(self.n_chan), len(self.delay_edges) - 1,
                               self.delay_edges.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(self.n_z))

    @property
    def n_dbins(self) -> int:
        return len(self.delay_edges) - 1

    @property
    def n_bins(self) -> int:
        return self.base.n_bins

    def ref(self):
        # the base's edges pointer is re-read, so a Config3D stays valid while its base lives
        self._c.base = self.base._c
        return ctypes.byref(self._c)

    @classmethod
    def from_cube(cls, ci, **kw):
        """From synth.CubeInputs (its workload's grid and rings, its channels and delay bins)."""
        return cls(Config.from_workload(ci.wl, **kw), int(ci.uv.shape[0]), ci.tau)


def _check(st: int, ctx=None, what: str = ""):
    if st != ABS_OK:
        msg = load().abs_last_error(ctx).decode() if ctx else ""
        raise AbsError(st, f"{what}: {msg}")


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


_DT = {"f32": "float32", "f64": "float64", "i32": "int32", "i64": "int64", "u8": "uint8"}


def _dev(t, dt: str, numel: int, name: str, device: int | None = None, optional: bool = False):
    """Pointer of a device-buffer argument, after checking what the C ABI cannot:
    a contiguous CUDA tensor of the documented element type, on the expected
    device, holding at least `numel` elements.  A wrong buffer would otherwise
    be read or written out of bounds by the kernels.  Raises ValueError."""
    import torch
    if t is None:
        if optional:
            return None
        raise ValueError(f"{name}: a CUDA tensor is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name}: expected a CUDA tensor, got {type(t).__name__}"
                         + ("" if not isinstance(t, torch.Tensor) else f" on {t.device}"))
    if t.dtype != getattr(torch, _DT[dt]):
        raise ValueError(f"{name}: dtype {t.dtype}, expected torch.{_DT[dt]}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: tensor must be contiguous")
    want = torch.cuda.current_device() if device is None else device
    if t.device.index != want:
        raise ValueError(f"{name}: on cuda:{t.device.index}, expected cuda:{want}")
    if t.numel() < numel:
        raise ValueError(f"{name}: {t.numel()} elements, at least {numel} required")
    return ctypes.c_void_p(t.data_ptr())


def _host(a, dt: str, numel: int, name: str, optional: bool = False):
    """Address (int) of a host-buffer argument: a C-contiguous numpy array or CPU torch tensor of
    the documented element type with at least `numel` elements.  Raises ValueError."""
    if a is None:
        if optional:
            return None
        raise ValueError(f"{name}: a host array is required")
    if hasattr(a, "data_ptr"):
        if a.is_cuda:
            raise ValueError(f"{name}: expected host memory, got a CUDA tensor")
        if str(a.dtype) != "torch." + _DT[dt] or not a.is_contiguous() or a.numel() < numel:
            raise ValueError(f"{name}: need a contiguous {_DT[dt]} tensor of >= {numel} elements")
        return a.data_ptr()
    a = np.asarray(a)
    if a.dtype != np.dtype(_DT[dt]) or not a.flags["C_CONTIGUOUS"] or a.size < numel:
        raise ValueError(f"{name}: need a C-contiguous {_DT[dt]} array of >= {numel} elements")
    return a.ctypes.data


def _ijk_rows(ijk, name="ijk", device=None):
    """(pointer, rows) of a triplet list: int32 [n][3] on the device."""
    if ijk.dim() != 2 or ijk.shape[1] != 3:
        raise ValueError(f"{name}: shape {tuple(ijk.shape)}, expected (n, 3)")
    return _dev(ijk, "i32", ijk.numel(), name, device), int(ijk.shape[0])


# ------------------------------------------------------------------ host helpers


def abs_ring_q(cfg: Config) -> np.ndarray:
    q = np.zeros(cfg.n_bins + 1, np.int64)
    _check(load().abs_ring_q(cfg.ref(), q.ctypes.data_as(ctypes.c_void_p)), what="abs_ring_q")
    return q


def abs_fft_size(cfg: Config) -> int:
    n = ctypes.c_int32(0)
    _check(load().abs_fft_size(cfg.ref(), ctypes.byref(n)), what="abs_fft_size")
    return n.value


def abs_triplets(cfg: Config) -> np.ndarray:
    n = ctypes.c_int32(0)
    _check(load().abs_triplets(cfg.ref(), 0, ctypes.byref(n), None), what="abs_triplets")
    out = np.zeros((max(n.value, 1), 3), np.int32)
    _check(load().abs_triplets(cfg.ref(), n.value, ctypes.byref(n), out.ctypes.data_as(ctypes.c_void_p)),
           what="abs_triplets")
    return out[:n.value]


def abs_triplets_3d(cfg: Config3D) -> np.ndarray:
    n = ctypes.c_int32(0)
    _check(load().abs_triplets_3d(cfg.ref(), 0, ctypes.byref(n), None), what="abs_triplets_3d")
    out = np.zeros((max(n.value, 1), 3), np.int32)
    _check(load().abs_triplets_3d(cfg.ref(), n.value, ctypes.byref(n), out.ctypes.data_as(ctypes.c_void_p)),
           what="abs_triplets_3d")
    return out[:n.value]


# ------------------------------------------------------------------ context


class Context:
    """An abs_ctx on one device, bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = ctypes.c_void_p()
        _check(load().abs_create(ctypes.byref(h), int(device), ctypes.c_void_p(stream.cuda_stream)),
               what="abs_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().abs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self):
        _check(load().abs_sync(self.h), self.h, "abs_sync")

    def profile(self, on: bool = True):
        """Turn the per-kernel CUDA-event profiler on (clearing totals) or off."""
        _check(load().abs_profile(self.h, 1 if on else 0), self.h, "abs_profile")

    def abs_rebin(self, cfg: "Config", B, counts, ellbar, ijk=None, n_mu: int = 5, n_t: int = 5,
                  mean=None, sigma=None, weight=None):
        """(l1, mu, t) cells of B ([R][n_trip] or [n_trip] CUDA FP64): count-weighted means per
        realisation, then their ensemble mean and spread; outputs [n_bins][n_mu][n_t] FP64."""
        n_real = B.shape[0] if B.dim() == 2 else 1
        n_trip = int(B.shape[-1])
        d, nc = self.device, cfg.n_bins * int(n_mu) * int(n_t)
        pijk = None
        if ijk is not None:
            pijk, rows = _ijk_rows(ijk, device=d)
            if rows < n_trip:
                raise ValueError(f"ijk: {rows} triplets, B has {n_trip}")
        _check(load().abs_rebin(self.h, cfg.ref(), int(n_real), n_trip, _dev(B, "f64", n_real * n_trip, "B", d),
                                _dev(counts, "i64", n_trip, "counts", d),
                                _dev(ellbar, "f64", cfg.n_bins, "ellbar", d), pijk, int(n_mu), int(n_t),
                                _dev(mean, "f64", nc, "mean", d, optional=True),
                                _dev(sigma, "f64", nc, "sigma", d, optional=True),
                                _dev(weight, "f64", nc, "weight", d, optional=True)), self.h, "abs_rebin")

    def abs_bana_d(self, cfg: "Config", C, mask, counts, out, ijk=None, f_over_sigma: float = 0.3):
        """[B_Ana]_d per triplet (CUDA FP64 out) from C(l_g) per uv cell (CUDA FP64 [n][n]),
        the filled mask (CUDA uint8 [n][n]) and the triangle counts of that mask."""
        d, c, nt = self.device, cfg.n_grid * cfg.n_grid, int(out.shape[0])
        pijk = None
        if ijk is not None:
            pijk, rows = _ijk_rows(ijk, device=d)
            if rows < nt:
                raise ValueError(f"ijk: {rows} triplets, out has {nt}")
        _check(load().abs_bana_d(self.h, cfg.ref(), _dev(C, "f64", c, "C", d), _dev(mask, "u8", c, "mask", d), nt,
                                 pijk, _dev(counts, "i64", nt, "counts", d), float(f_over_sigma),
                                 _dev(out, "f64", nt, "out", d)), self.h, "abs_bana_d")

    def abs_simulate_vis(self, sky, dtheta: float, uv, vis, beam: int = 0, beam_param: float = 0.0):
        """Eq. vis by direct DFT of the beam-weighted map (CUDA FP32 [m][m]) at the baselines uv
        (CUDA FP32 [n][2]) into vis (CUDA FP32 [n][2]); beam ABS_BEAM_NONE / MWA_TILE / GAUSS."""
        m, nv, d = int(sky.shape[0]), int(uv.shape[0]), self.device
        _check(load().abs_simulate_vis(self.h, m, float(dtheta), _dev(sky, "f32", m * m, "sky", d), int(beam),
                                       float(beam_param), nv, _dev(uv, "f32", 2 * nv, "uv", d),
                                       _dev(vis, "f32", 2 * nv, "vis", d)),
               self.h, "abs_simulate_vis")

    def probe_timeout(self, max_polls: int = 1000):
        """Queue a bounded device-side wait that runs out (see include/abs.h); the next sync raises
        ABS_ERR_TIMEOUT."""
        _check(load().abs_probe_timeout(self.h, int(max_polls)), self.h, "abs_probe_timeout")

    def inject_alloc_failures(self, count: int):
        """Make the next `count` workspace allocations fail (host-side failure injection)."""
        _check(load().abs_inject_alloc_failures(self.h, int(count)), self.h, "abs_inject_alloc_failures")

    def autotune(self, on: bool = True):
        """Turn the split-BF16 launch-shape autotuner on (default) or off (cost model)."""
        _check(load().abs_autotune(self.h, 1 if on else 0), self.h, "abs_autotune")

    def tuned_shape(self, cfg: "Config") -> dict:
        """The split-BF16 launch shape chosen for cfg: accumulator columns of a work item
        (0: none chosen yet), work items per SM, and whether the autotuner timed it."""
        sc, wv, me = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(load().abs_tuned_shape(self.h, cfg.ref(), ctypes.byref(sc), ctypes.byref(wv), ctypes.byref(me)),
               self.h, "abs_tuned_shape")
        return {"set_cols": sc.value, "waves": wv.value, "measured": bool(me.value)}

    def profile_read(self) -> dict:
        """{stage: (total ms, launches)} accumulated since profile(True); waits for the stream."""
        n = ctypes.c_int32(0)
        _check(load().abs_profile_read(self.h, 0, ctypes.byref(n), None), self.h, "abs_profile_read")
        arr = (abs_stage_time * max(n.value, 1))()
        _check(load().abs_profile_read(self.h, n.value, ctypes.byref(n), arr), self.h, "abs_profile_read")
        return {arr[i].name.decode(): (arr[i].ms, arr[i].launches) for i in range(n.value)}

    # ------------- stages (torch CUDA tensors in, torch CUDA tensors out)
    def abs_grid(self, cfg: Config, uv, vis, grid, wsum, mask):
        nv, c = int(uv.shape[0]), cfg.n_grid * cfg.n_grid
        d = self.device
        _check(load().abs_grid(self.h, cfg.ref(), nv, _dev(uv, "f32", 2 * nv, "uv", d),
                               _dev(vis, "f32", 2 * nv, "vis", d), _dev(grid, "f32", 2 * c, "grid", d),
                               _dev(wsum, "f32", c, "wsum", d), _dev(mask, "u8", c, "mask", d)),
               self.h, "abs_grid")

    def abs_filter_fft(self, cfg: Config, grid, wsum, mask, fields):
        c, d = cfg.n_grid * cfg.n_grid, self.device
        _check(load().abs_filter_fft(self.h, cfg.ref(), _dev(grid, "f32", 2 * c, "grid", d),
                                     _dev(wsum, "f32", c, "wsum", d), _dev(mask, "u8", c, "mask", d),
                                     _dev(fields, "f32", cfg.n_bins * cfg.N * cfg.N, "fields", d)),
               self.h, "abs_filter_fft")

    def abs_triple(self, cfg: Config, fields, mask, ijk, sums=None, counts=None):
        d = self.device
        pijk, nt = _ijk_rows(ijk, device=d)
        _check(load().abs_triple(self.h, cfg.ref(), _dev(fields, "f32", cfg.n_bins * cfg.N * cfg.N, "fields", d,
                                                                 optional=sums is None),
                                 _dev(mask, "u8", cfg.n_grid * cfg.n_grid, "mask", d, optional=counts is None),
                                 nt, pijk, _dev(sums, "f64", nt, "sums", d, optional=True),
                                 _dev(counts, "i64", nt, "counts", d, optional=True)), self.h, "abs_triple")

    def abs_normalise(self, cfg: Config, sums, counts, B, mask=None, ellbar=None):
        nt, d = int(sums.shape[0]), self.device
        _check(load().abs_normalise(self.h, cfg.ref(), nt, _dev(sums, "f64", nt, "sums", d),
                                    _dev(counts, "i64", nt, "counts", d), _dev(B, "f64", nt, "B", d),
                                    _dev(mask, "u8", cfg.n_grid * cfg.n_grid, "mask", d, optional=True),
                                    _dev(ellbar, "f64", cfg.n_bins, "ellbar", d, optional=True)),
               self.h, "abs_normalise")

    def _est_ptrs(self, cfg, uv, vis, n_real, n_trip, ijk, B, counts, ellbar):
        nv, d, nt = int(uv.shape[0]), self.device, int(n_trip)
        if ijk is not None:
            pijk, rows = _ijk_rows(ijk, device=d)
            if rows < nt:
                raise ValueError(f"ijk: {rows} triplets, n_trip = {nt}")
        else:
            pijk = None
        return (nv, _dev(uv, "f32", 2 * nv, "uv", d), _dev(vis, "f32", 2 * nv * n_real, "vis", d), pijk,
                _dev(B, "f64", nt * n_real, "B", d, optional=True),
                _dev(counts, "i64", nt, "counts", d, optional=True),
                _dev(ellbar, "f64", cfg.n_bins, "ellbar", d, optional=True))

    def abs_estimate(self, cfg: Config, uv, vis, n_trip, ijk=None, B=None, counts=None, ellbar=None):
        nv, puv, pvis, pijk, pB, pT, pE = self._est_ptrs(cfg, uv, vis, 1, n_trip, ijk, B, counts, ellbar)
        _check(load().abs_estimate(self.h, cfg.ref(), nv, puv, pvis, int(n_trip), pijk, pB, pT, pE),
               self.h, "abs_estimate")

    def abs_estimate_3d(self, cfg: Config3D, uv, vis, n_trip, uvw=None, B=None, counts=None, ellbar=None):
        """Multi-frequency estimate: uv, vis [n_chan][n_vis][2] float32 on the device."""
        d, nt, nc = self.device, int(n_trip), int(cfg.n_chan)
        if uv.dim() != 3 or uv.shape[0] != nc or uv.shape[2] != 2:
            raise ValueError(f"uv: shape {tuple(uv.shape)}, expected ({nc}, n_vis, 2)")
        nv = int(uv.shape[1])
        if uvw is not None:
            puvw, rows = _ijk_rows(uvw, "uvw", device=d)
            if rows < nt:
                raise ValueError(f"uvw: {rows} triplets, n_trip = {nt}")
        else:
            puvw = None
        _check(load().abs_estimate_3d(self.h, cfg.ref(), nv, _dev(uv, "f32", 2 * nv * nc, "uv", d),
                                      _dev(vis, "f32", 2 * nv * nc, "vis", d), nt, puvw,
                                      _dev(B, "f64", nt, "B", d, optional=True),
                                      _dev(counts, "i64", nt, "counts", d, optional=True),
                                      _dev(ellbar, "f64", cfg.n_bins, "ellbar", d, optional=True)),
               self.h, "abs_estimate_3d")

    def abs_estimate_many(self, cfg: Config, uv, vis, n_trip, ijk=None, B=None, counts=None, ellbar=None):
        n_real = int(vis.shape[0])
        nv, puv, pvis, pijk, pB, pT, pE = self._est_ptrs(cfg, uv, vis, n_real, n_trip, ijk, B, counts, ellbar)
        _check(load().abs_estimate_many(self.h, cfg.ref(), nv, puv, n_real, pvis, int(n_trip), pijk, pB, pT, pE),
               self.h, "abs_estimate_many")

    def abs_estimate_batched(self, items):
        """items: sequence of (cfg, uv, vis, n_trip, ijk, B, counts, ellbar), torch CUDA tensors or None,
        one independent estimate each (configurations may differ)."""
        arr = (abs_item * max(len(items), 1))()
        for a, (cfg, uv, vis, n_trip, ijk, B, counts, ellbar) in zip(arr, items):
            nv, puv, pvis, pijk, pB, pT, pE = self._est_ptrs(cfg, uv, vis, 1, n_trip, ijk, B, counts, ellbar)
            a.cfg = ctypes.pointer(cfg._c)
            a.n_vis = nv
            a.d_uv, a.d_vis = puv.value, pvis.value
            a.n_trip = int(n_trip)
            a.d_ijk, a.d_B, a.d_count, a.d_ellbar = [None if p is None else p.value for p in (pijk, pB, pT, pE)]
        _check(load().abs_estimate_batched(self.h, len(items), ctypes.cast(arr, ctypes.c_void_p)), self.h,
               "abs_estimate_batched")

    def abs_estimate_batched_host(self, items):
        """items: sequence of (cfg, uv, vis, n_trip, ijk, B, counts, ellbar) with uv / vis host inputs
        and B / counts / ellbar host outputs (numpy arrays or CPU torch tensors, pinned ones let the
        copies run inside the batch's graph; float32 [n_vis, 2], float64 [n_trip], int64 [n_trip],
        float64 [n_bins]) and ijk None or a device triplet list; blocks until the outputs are written."""
        arr = (abs_item * max(len(items), 1))()
        keep = []
        for a, (cfg, uv, vis, n_trip, ijk, B, counts, ellbar) in zip(arr, items):
            nv, nt = int(uv.shape[0]), int(n_trip)
            ptrs = []
            for name, t, dt, n in (("uv", uv, "f32", 2 * nv), ("vis", vis, "f32", 2 * nv), ("B", B, "f64", nt),
                                   ("counts", counts, "i64", nt), ("ellbar", ellbar, "f64", cfg.n_bins)):
                ptrs.append(_host(t, dt, n, name, optional=name not in ("uv", "vis")))
                keep.append(t)
            a.cfg = ctypes.pointer(cfg._c)
            a.n_vis = nv
            a.d_uv, a.d_vis = ptrs[0], ptrs[1]
            a.n_trip = nt
            a.d_ijk = None if ijk is None else _ijk_rows(ijk, device=self.device)[0].value
            a.d_B, a.d_count, a.d_ellbar = ptrs[2], ptrs[3], ptrs[4]
        _check(load().abs_estimate_batched_host(self.h, len(items), ctypes.cast(arr, ctypes.c_void_p)), self.h,
               "abs_estimate_batched_host")

    def abs_estimate_host(self, cfg: Config, uv: np.ndarray, vis: np.ndarray, n_trip: int, ijk=None,
                          B=None, counts=None, ellbar=None):
        """Host arrays in and out (numpy or pinned torch CPU tensors); blocks until done."""
        def hp(a):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):
                return ctypes.c_void_p(a.data_ptr())
            return a.ctypes.data_as(ctypes.c_void_p)
        n_real = vis.shape[0] if vis.ndim == 3 else 1
        _check(load().abs_estimate_host(self.h, cfg.ref(), uv.shape[0], hp(uv), n_real, hp(vis), int(n_trip),
                                        hp(ijk), hp(B), hp(counts), hp(ellbar)), self.h, "abs_estimate_host")


def abs_triple_sums_static(cfg: Config, fields, ijk, sums, stream=None):
    """FP32 triple sums without a context or any device allocation (see include/abs.h).

    fields, ijk, sums: torch CUDA tensors on the current device; the work is
    enqueued on `stream` (default: torch's current stream).  Calls share one
    fixed scratch array inside the library, so calls that overlap on the GPU
    must be serialised by the caller."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    pijk, nt = _ijk_rows(ijk)
    st = load().abs_triple_sums_static(cfg.ref(), _dev(fields, "f32", cfg.n_bins * cfg.N * cfg.N, "fields"), nt,
                                       pijk, _dev(sums, "f64", nt, "sums"), ctypes.c_void_p(stream.cuda_stream))
    _check(st, None, "abs_triple_sums_static")


def estimate(cfg: Config, uv, vis, ctx: Context | None = None):
    """Convenience: one realisation V -> (B, counts, ellbar) as torch CUDA tensors."""
    import torch
    ctx = ctx or Context(uv.device.index or 0)
    ijk = abs_triplets(cfg)
    nt = len(ijk)
    dev = uv.device
    B = torch.empty(nt, dtype=torch.float64, device=dev)
    T = torch.empty(nt, dtype=torch.int64, device=dev)
    E = torch.empty(cfg.n_bins, dtype=torch.float64, device=dev)
    ctx.abs_estimate(cfg, uv, vis, nt, None, B, T, E)
    return B, T, E, ijk

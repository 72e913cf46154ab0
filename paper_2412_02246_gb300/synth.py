"""Seeded synthetic inputs for the visibility-based binned angular bispectrum.

This module only *makes inputs*: baselines U, visibilities V and the l-bin
edges of each workload.  It contains none of the estimator's arithmetic
(gridding, ring filtering, transforms, triple sums, counts, normalisation),
so both the CUDA path and the FP64 oracle can take their inputs from here
without sharing any of the method.

Recipe (stands in for the MWA 154.25 MHz drift-scan data of Sec. 3, which is
not available):

* sky: a Gaussian random field g on an M x M periodic flat-sky grid with
  angular power C_l proportional to l^-alpha (alpha = 2.5), scaled to unit
  ensemble variance, then the local quadratic transform of Eq. (mb1),
  delta = g + f (g^2 - 1);
* visibilities: the map's Fourier modes with the sign of Eq. (vis)
  (exp(+i 2 pi U.theta)), on a uv lattice of spacing du (so that the map
  spans 1/du radians), read at each baseline by bilinear interpolation
  between the four surrounding lattice modes, plus complex Gaussian noise of
  rms `noise_frac` x rms|V|;
* baselines: either uniform in area inside an annulus, or an interferometer
  of n_ant antennas (n_ant (n_ant-1)/2 baselines) whose areal density falls
  as |U|^-1.5 between u_min and u_max, each baseline tracked over n_time
  samples of a rotation of `track_deg` degrees in the uv plane (a flat
  stand-in for Earth-rotation synthesis).

* multi-channel workload: 32 channels evenly over 139-169 MHz share one
  sky (the quadratic diffuse field plus 2,000 point sources on map pixels
  with dN/dS ~ S^-1.6 over S in [1, 1000]) and one baseline set drawn at
  154.25 MHz, scaled by nu / 154.25 MHz per channel; noise per channel.

All randomness is drawn from numpy's PCG64 seeded per workload and
realisation.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 24120224600


def seed_for(cfg_id: int, realisation: int = 0) -> int:
    return SEED_BASE + 1000 * cfg_id + realisation


@dataclass
class Workload:
    """Shape of one estimate: uv grid, gridding kernel, l bins, baselines."""

    name: str
    n_grid: int              # uv grid side (cells)
    du: float                # grid spacing Delta U_g (wavelengths)
    ell_edges: np.ndarray    # n_bins + 1 ascending bin edges in l = 2 pi |U|
    kernel: str = "gauss"    # "gauss" or "ngp"
    sigma_cells: float = 1.0
    radius_cells: int = 3
    map_side: int = 64       # sky map side M (pixels); map modes spaced by du
    f_ng: float = 0.3
    alpha: float = 2.5
    noise_frac: float = 0.05
    # baselines
    layout: str = "annulus"  # "annulus" or "array"
    n_vis: int = 5000
    u_min: float = 4.0
    u_max: float = 60.0
    n_ant: int = 128
    n_time: int = 120
    track_deg: float = 7.5
    precision: str = "fp32"
    extra: dict = field(default_factory=dict)

    @property
    def n_bins(self) -> int:
        return len(self.ell_edges) - 1


def _lin_edges(lo, hi, n):
    return np.linspace(lo, hi, n + 1)


def _log_edges(lo, hi, n):
    return np.geomspace(lo, hi, n + 1)


def workload(cfg_id: int) -> Workload:
    """The workload shapes: tiny (0), MWA-shaped (1), precision (2), multi-channel (4).

    The uneven batch items (3) come from `batch_item`; the channels of the
    multi-channel workload from `channel_inputs`.
    """
    if cfg_id == 0:
        return Workload("tiny-64sq-5k-8lin", 64, 2.0, _lin_edges(25.0, 375.0, 8),
                        map_side=64, layout="annulus", n_vis=5000, u_min=4.0, u_max=60.0)
    if cfg_id == 1:
        return Workload("mwa-512sq-975k-20log", 512, 2.3, _log_edges(46.0, 1320.0, 20),
                        map_side=512, layout="array", n_ant=128, n_time=120,
                        u_min=7.0, u_max=220.0)
    if cfg_id == 2:
        return Workload("precision-2048sq-4M-64log", 2048, 1.15, _log_edges(46.0, 1320.0, 64),
                        map_side=2048, layout="array", n_ant=128, n_time=0, n_vis=4_000_000,
                        u_min=7.0, u_max=220.0, precision="split_bf16")
    if cfg_id == 4:
        return Workload("channels-4096sq-10M-128log", 4096, 0.6, _log_edges(46.0, 1320.0, 128),
                        map_side=4096, layout="array", n_ant=128, n_time=0, n_vis=10_000_000,
                        u_min=7.0, u_max=220.0, precision="split_bf16",
                        extra={"n_chan": 32, "nu_lo_mhz": 139.0, "nu_hi_mhz": 169.0,
                               "nu_ref_mhz": 154.25, "n_src": 2000, "src_slope": 1.6,
                               "s_min": 1.0, "s_max": 1000.0})
    raise ValueError(f"unknown workload id {cfg_id}")


def batch_item(rng: np.random.Generator, idx: int) -> Workload:
    """One item of the uneven batch: grid in {256,512,1024}^2, 1e5-1e6 vis, 16-48 log bins.

    The uv extent is held fixed (du = 2.3 * 512 / n) so that l spans 46-1320
    for every grid size.
    """
    n = int(rng.choice([256, 512, 1024]))
    nv = int(rng.integers(100_000, 1_000_001))
    nb = int(rng.integers(16, 49))
    du = 2.3 * 512.0 / n
    return Workload(f"batch-{idx}-{n}sq-{nv}-{nb}log", n, du, _log_edges(46.0, 1320.0, nb),
                    map_side=n, layout="array", n_ant=128, n_time=0, n_vis=nv,
                    u_min=7.0, u_max=220.0, precision="split_bf16")


# ----------------------------------------------------------------------------- sky


def gaussian_field(m: int, rng: np.random.Generator, alpha: float = 2.5) -> np.ndarray:
    """Real Gaussian field on an m x m periodic grid, P(k) ~ |k|^-alpha, unit ensemble variance."""
    k = np.fft.fftfreq(m) * m
    kk = np.sqrt(k[None, :] ** 2 + k[:, None] ** 2)
    p = np.zeros_like(kk)
    nz = kk > 0
    p[nz] = kk[nz] ** (-alpha)
    p *= (m * m) / p.sum()          # (1/m^2) sum_k P(k) = 1  ->  <g^2> = 1
    white = rng.standard_normal((m, m))
    g = np.fft.ifft2(np.fft.fft2(white) * np.sqrt(p)).real
    return g


def power_spectrum_model(m: int, alpha: float = 2.5) -> np.ndarray:
    """The P(k) used by `gaussian_field` (same normalisation), for the closed-form tests."""
    k = np.fft.fftfreq(m) * m
    kk = np.sqrt(k[None, :] ** 2 + k[:, None] ** 2)
    p = np.zeros_like(kk)
    nz = kk > 0
    p[nz] = kk[nz] ** (-alpha)
    p *= (m * m) / p.sum()
    return p


def quadratic_sky(g: np.ndarray, f_ng: float) -> np.ndarray:
    """Eq. (mb1) with sigma_T = 1: delta = g + f (g^2 - 1)."""
    return g + f_ng * (g * g - 1.0)


def sky_modes(delta: np.ndarray) -> np.ndarray:
    """Fourier modes of the map with the exp(+i 2 pi U.theta) sign of Eq. (vis), FFT order."""
    m = delta.shape[0]
    return np.fft.ifft2(delta) * (m * m)


# ----------------------------------------------------------------------- baselines


def annulus_baselines(rng: np.random.Generator, n_vis: int, u_min: float, u_max: float) -> np.ndarray:
    r = np.sqrt(rng.uniform(u_min ** 2, u_max ** 2, n_vis))
    phi = rng.uniform(0.0, 2.0 * np.pi, n_vis)
    return np.stack([r * np.cos(phi), r * np.sin(phi)], axis=1)


def array_baselines(rng: np.random.Generator, n_base: int, n_time: int, u_min: float,
                    u_max: float, track_deg: float) -> np.ndarray:
    """Areal density ~ |U|^-1.5 on [u_min, u_max]: p(|U|) ~ |U|^-0.5, uniform angle.

    With n_time > 0 every baseline is repeated n_time times, rotated by
    track_deg * t / n_time (baseline-major order, as an interferometer writes
    its data); with n_time == 0 the n_base points are independent.
    """
    s = rng.uniform(0.0, 1.0, n_base)
    a, b = np.sqrt(u_min), np.sqrt(u_max)
    r = (a + s * (b - a)) ** 2
    phi = rng.uniform(0.0, 2.0 * np.pi, n_base)
    if n_time <= 0:
        return np.stack([r * np.cos(phi), r * np.sin(phi)], axis=1)
    rot = np.deg2rad(track_deg) * np.arange(n_time) / n_time
    ang = phi[:, None] + rot[None, :]
    return np.stack([(r[:, None] * np.cos(ang)).ravel(), (r[:, None] * np.sin(ang)).ravel()], axis=1)


def bilinear(modes: np.ndarray, uv_modes: np.ndarray) -> np.ndarray:
    """Bilinear read of a periodic complex mode lattice at fractional (u, v) mode coordinates."""
    m = modes.shape[0]
    x, y = uv_modes[:, 0], uv_modes[:, 1]
    x0, y0 = np.floor(x), np.floor(y)
    tx, ty = x - x0, y - y0
    ix0, iy0 = x0.astype(np.int64) % m, y0.astype(np.int64) % m
    ix1, iy1 = (ix0 + 1) % m, (iy0 + 1) % m
    return ((1 - tx) * (1 - ty) * modes[iy0, ix0] + tx * (1 - ty) * modes[iy0, ix1]
            + (1 - tx) * ty * modes[iy1, ix0] + tx * ty * modes[iy1, ix1])


@dataclass
class Inputs:
    uv: np.ndarray        # [n_vis, 2] float32, wavelengths
    vis: np.ndarray       # [n_vis] complex64
    ell_edges: np.ndarray
    wl: Workload


def make_baselines(wl: Workload, rng: np.random.Generator) -> np.ndarray:
    if wl.layout == "annulus":
        uv = annulus_baselines(rng, wl.n_vis, wl.u_min, wl.u_max)
    elif wl.n_time > 0:
        uv = array_baselines(rng, wl.n_ant * (wl.n_ant - 1) // 2, wl.n_time, wl.u_min,
                             wl.u_max, wl.track_deg)
    else:
        uv = array_baselines(rng, wl.n_vis, 0, wl.u_min, wl.u_max, wl.track_deg)
    return uv.astype(np.float32)


def make_visibilities(wl: Workload, uv: np.ndarray, rng: np.random.Generator,
                      f_ng: float | None = None) -> np.ndarray:
    f = wl.f_ng if f_ng is None else f_ng
    g = gaussian_field(wl.map_side, rng, wl.alpha)
    modes = sky_modes(quadratic_sky(g, f))
    v = bilinear(modes, uv.astype(np.float64) / np.float64(wl.du))
    if wl.noise_frac > 0:
        rms = np.sqrt(np.mean(np.abs(v) ** 2))
        s = wl.noise_frac * rms / np.sqrt(2.0)
        v = v + s * (rng.standard_normal(v.shape) + 1j * rng.standard_normal(v.shape))
    return v.astype(np.complex64)


def make_inputs(cfg_id: int, realisation: int = 0, wl: Workload | None = None,
                n_vis: int | None = None) -> Inputs:
    """Seeded (U, V) for one realisation of a workload.

    Baselines depend only on the workload seed (every realisation observes
    with the same array, as in the paper's 500-realisation ensemble); the
    sky and noise change with `realisation`.
    """
    wl = workload(cfg_id) if wl is None else wl
    if n_vis is not None:
        wl = Workload(**{**wl.__dict__, "n_vis": n_vis, "layout": "annulus"
                         if wl.layout == "annulus" else "array", "n_time": 0})
    rb = np.random.Generator(np.random.PCG64(seed_for(cfg_id, 0)))
    uv = make_baselines(wl, rb)
    rs = np.random.Generator(np.random.PCG64(seed_for(cfg_id, 1 + realisation)))
    vis = make_visibilities(wl, uv, rs)
    return Inputs(uv=uv, vis=vis, ell_edges=np.asarray(wl.ell_edges, np.float64), wl=wl)


# ------------------------------------------------------------------ channels


def channel_freqs_mhz(wl: Workload) -> np.ndarray:
    """Channel centre frequencies, evenly spaced over [nu_lo, nu_hi] (end points included)."""
    e = wl.extra
    return np.linspace(e["nu_lo_mhz"], e["nu_hi_mhz"], e["n_chan"])


def point_sources(m: int, rng: np.random.Generator, n_src: int, slope: float, s_min: float,
                  s_max: float) -> np.ndarray:
    """n_src sources on uniformly drawn pixels of an m x m map, fluxes drawn from
    dN/dS ~ S^-slope on [s_min, s_max] by inverting the cumulative count."""
    a = 1.0 - slope
    u = rng.uniform(0.0, 1.0, n_src)
    flux = (s_min ** a + u * (s_max ** a - s_min ** a)) ** (1.0 / a)
    img = np.zeros((m, m))
    np.add.at(img, (rng.integers(0, m, n_src), rng.integers(0, m, n_src)), flux)
    return img


_channel_sky: dict = {}


def channel_sky_modes(wl: Workload, realisation: int = 0) -> np.ndarray:
    """Fourier modes of the multi-channel sky: the quadratic diffuse field of the
    other workloads plus point sources (one flat-spectrum sky for every channel).
    The last one made is kept, since every channel reads it."""
    key = (wl.name, realisation)
    if key not in _channel_sky:
        _channel_sky.clear()
        e = wl.extra
        rng = np.random.Generator(np.random.PCG64(seed_for(4, 1 + realisation)))
        delta = quadratic_sky(gaussian_field(wl.map_side, rng, wl.alpha), wl.f_ng)
        delta += point_sources(wl.map_side, rng, e["n_src"], e["src_slope"], e["s_min"], e["s_max"])
        _channel_sky[key] = sky_modes(delta)
    return _channel_sky[key]


def channel_inputs(channel: int, realisation: int = 0, wl: Workload | None = None) -> Inputs:
    """Seeded (U, V) of one channel of the multi-channel workload.

    One set of baselines is drawn at the reference frequency and scaled by
    nu / nu_ref in every channel (a baseline's length in wavelengths grows
    with frequency); the sky is shared, the noise is drawn per channel.
    """
    wl = workload(4) if wl is None else wl
    nu = channel_freqs_mhz(wl)[channel]
    rb = np.random.Generator(np.random.PCG64(seed_for(4, 0)))
    uv = make_baselines(wl, rb).astype(np.float64) * (nu / wl.extra["nu_ref_mhz"])
    uv = uv.astype(np.float32)
    v = bilinear(channel_sky_modes(wl, realisation), uv.astype(np.float64) / np.float64(wl.du))
    rn = np.random.Generator(np.random.PCG64(seed_for(4, 500 + channel + 100 * realisation)))
    rms = np.sqrt(np.mean(np.abs(v) ** 2))
    s = wl.noise_frac * rms / np.sqrt(2.0)
    v = v + s * (rn.standard_normal(v.shape) + 1j * rn.standard_normal(v.shape))
    return Inputs(uv=uv, vis=v.astype(np.complex64), ell_edges=np.asarray(wl.ell_edges, np.float64), wl=wl)


def vis_as_float2(vis: np.ndarray) -> np.ndarray:
    """complex64 [n] -> float32 [n, 2] (re, im) view used by both implementations."""
    return np.ascontiguousarray(vis.astype(np.complex64)).view(np.float32).reshape(-1, 2)


# ------------------------------------------------------------------ multi-frequency cube


@dataclass
class CubeInputs:
    uv: np.ndarray        # [n_chan, n_vis, 2] float32, wavelengths at each channel's frequency
    vis: np.ndarray       # [n_chan, n_vis] complex64
    freqs_mhz: np.ndarray
    tau: np.ndarray       # delay-bin edges in |t| (int32, ascending)
    wl: Workload


def cube_workload(cfg_id: int) -> Workload:
    """Multi-frequency cubes for the 3-D form: tiny (5) and MWA-shaped (6).

    tiny: the tiny workload's grid and rings over 8 channels (150-157 MHz),
    delay bins {0}, {1}, {2, 3}.  MWA-shaped: the MWA-shaped workload's grid,
    array and rings over 32 channels evenly on 139-169 MHz, delay bins {0},
    [1, 4), [4, 8), [8, 16).  Baselines are drawn at 154.25 MHz and scaled by
    nu / 154.25 MHz in every channel.
    """
    if cfg_id == 5:
        return Workload("cube-tiny-64sq-8ch-5k-8lin", 64, 2.0, _lin_edges(25.0, 375.0, 8), map_side=64,
                        layout="annulus", n_vis=5000, u_min=4.0, u_max=60.0,
                        extra={"n_chan": 8, "nu_lo_mhz": 150.0, "nu_hi_mhz": 157.0, "nu_ref_mhz": 154.25,
                               "tau": [0, 1, 2, 4]})
    if cfg_id == 6:
        return Workload("cube-mwa-512sq-32ch-975k-20log", 512, 2.3, _log_edges(46.0, 1320.0, 20),
                        map_side=512, layout="array", n_ant=128, n_time=120, u_min=7.0, u_max=220.0,
                        extra={"n_chan": 32, "nu_lo_mhz": 139.0, "nu_hi_mhz": 169.0, "nu_ref_mhz": 154.25,
                               "tau": [0, 1, 4, 8, 16]})
    raise ValueError(f"unknown cube workload id {cfg_id}")


def cube_power_model(m: int, n_chan: int, alpha: float = 2.5) -> np.ndarray:
    """P(k) ~ |k|^-alpha on an m x m x n_chan grid (k in grid-index units on all three axes, FFT
    order, P(0) = 0), scaled so that (1 / size) sum_k P(k) = 1: the spectrum of `gaussian_cube`."""
    kx = np.fft.fftfreq(m) * m
    kz = np.fft.fftfreq(n_chan) * n_chan
    kk = np.sqrt(kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kz[None, None, :] ** 2)
    p = np.zeros_like(kk)
    nz = kk > 0
    p[nz] = kk[nz] ** (-alpha)
    return p * (p.size / p.sum())


def gaussian_cube(m: int, n_chan: int, rng: np.random.Generator, alpha: float = 2.5) -> np.ndarray:
    """Real Gaussian field on an m x m x n_chan periodic grid (axis 2 along frequency) with the
    spectrum of `cube_power_model`, unit ensemble variance."""
    p = cube_power_model(m, n_chan, alpha)
    white = rng.standard_normal((m, m, n_chan))
    return np.fft.ifftn(np.fft.fftn(white) * np.sqrt(p)).real


def cube_inputs(cfg_id: int, realisation: int = 0, wl: Workload | None = None) -> CubeInputs:
    """Seeded (U, V) of every channel of a multi-frequency cube.

    sky: the quadratic transform of Eq. (mb1) (f = 0.3) of a 3-D Gaussian field,
    one map per channel; visibilities: each channel's map modes read at that
    channel's baselines (one set drawn at the reference frequency, scaled by
    nu / nu_ref), plus 5 % complex Gaussian noise drawn per channel.
    """
    wl = cube_workload(cfg_id) if wl is None else wl
    e = wl.extra
    freqs = np.linspace(e["nu_lo_mhz"], e["nu_hi_mhz"], e["n_chan"])
    rb = np.random.Generator(np.random.PCG64(seed_for(cfg_id, 0)))
    uv0 = make_baselines(wl, rb).astype(np.float64)
    rs = np.random.Generator(np.random.PCG64(seed_for(cfg_id, 1 + realisation)))
    cube = quadratic_sky(gaussian_cube(wl.map_side, e["n_chan"], rs, wl.alpha), wl.f_ng)
    uvs, viss = [], []
    for c, nu in enumerate(freqs):
        uv = (uv0 * (nu / e["nu_ref_mhz"])).astype(np.float32)
        v = bilinear(sky_modes(np.ascontiguousarray(cube[:, :, c])), uv.astype(np.float64) / np.float64(wl.du))
        rms = np.sqrt(np.mean(np.abs(v) ** 2))
        s = wl.noise_frac * rms / np.sqrt(2.0)
        v = v + s * (rs.standard_normal(v.shape) + 1j * rs.standard_normal(v.shape))
        uvs.append(uv)
        viss.append(v.astype(np.complex64))
    return CubeInputs(uv=np.stack(uvs), vis=np.stack(viss), freqs_mhz=freqs,
                      tau=np.asarray(e["tau"], np.int32), wl=wl)

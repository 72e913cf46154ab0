"""The multi-channel workload's generator (no GPU): one baseline set scaled by
nu / nu_ref per channel, channel frequencies over 139-169 MHz, and point
sources drawn from dN/dS ~ S^-1.6 on [1, 1000]."""
import numpy as np

from paper_2412_02246_gb300 import synth


def test_channel_frequencies_and_baseline_scaling():
    wl = synth.workload(4)
    nu = synth.channel_freqs_mhz(wl)
    assert len(nu) == 32 and nu[0] == 139.0 and nu[-1] == 169.0
    small = synth.Workload(**{**wl.__dict__, "n_vis": 20000, "map_side": 64, "n_grid": 64})
    a = synth.channel_inputs(0, wl=small)
    b = synth.channel_inputs(31, wl=small)
    assert a.uv.shape == (20000, 2) and a.vis.dtype == np.complex64
    ratio = b.uv.astype(np.float64) / a.uv.astype(np.float64)
    assert np.allclose(ratio, 169.0 / 139.0, rtol=1e-6)
    r = np.hypot(*(a.uv.astype(np.float64) * (154.25 / 139.0)).T)
    assert r.min() >= 7.0 - 1e-3 and r.max() <= 220.0 + 1e-3
    assert not np.allclose(a.vis, b.vis)


def test_point_source_fluxes_follow_the_power_law():
    rng = np.random.default_rng(9)
    img = synth.point_sources(512, rng, 2000, 1.6, 1.0, 1000.0)
    s = img[img > 0]
    assert s.min() >= 1.0 and len(s) >= 1980        # a few sources may share a pixel
    # N(>S) ~ S^-0.6: the fraction above 10 is (10^-0.6 - 1000^-0.6) / (1 - 1000^-0.6)
    rng = np.random.default_rng(10)
    a = 1.0 - 1.6
    u = rng.uniform(0.0, 1.0, 20000)
    flux = (1.0 + u * (1000.0 ** a - 1.0)) ** (1.0 / a)
    want = (10 ** a - 1000 ** a) / (1 - 1000 ** a)
    assert abs((flux > 10).mean() - want) < 0.01
    img2 = synth.point_sources(4096, np.random.default_rng(10), 20000, 1.6, 1.0, 1000.0)
    assert abs((img2[img2 > 0] > 10).mean() - want) < 0.02

"""The C ABI library loads, exports every declared symbol, and its host-only
helpers (ring thresholds, sky-grid size, closing triplets, argument checks)
agree with the oracle.  No GPU needed: these entry points do no device work."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2412_02246_gb300 as absmod
from paper_2412_02246_gb300 import build as absbuild
from paper_2412_02246_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    absbuild.build()
    return absmod.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "abs.h")).read()
    return sorted(set(re.findall(r"^(?:abs_status|const char \*)\s*(abs_\w+)\s*\(", src, re.M)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


@pytest.mark.parametrize("cfg_id", [0, 1, 2])
def test_ring_q_fft_size_triplets_match_oracle(lib, cfg_id):
    wl = synth.workload(cfg_id)
    cfg = absmod.Config.from_workload(wl)
    q = absmod.abs_ring_q(cfg)
    assert np.array_equal(q, oracle.ring_q(wl.ell_edges, wl.du))
    assert absmod.abs_fft_size(cfg) == oracle.min_fft_size(q, wl.n_grid)
    assert np.array_equal(absmod.abs_triplets(cfg), oracle.triplets(q))


def test_known_sizes(lib):
    # N = smallest 2^a 3^b 5^c >= 3R + 1 for the three workload shapes
    sizes = [absmod.abs_fft_size(absmod.Config.from_workload(synth.workload(c))) for c in (0, 1, 2)]
    assert sizes == [90, 288, 576]
    assert len(absmod.abs_triplets(absmod.Config.from_workload(synth.workload(1)))) == 689


def test_random_edges_match_oracle(lib):
    rng = np.random.default_rng(5)
    for _ in range(30):
        n = int(rng.choice([16, 32, 64, 128]))
        du = float(rng.uniform(0.5, 3.0))
        nb = int(rng.integers(1, 12))
        edges = np.sort(rng.uniform(5.0, 2 * np.pi * du * n / 2, nb + 1))
        if np.any(np.diff(edges) <= 0):
            continue
        cfg = absmod.Config(n_grid=n, du=du, ell_edges=edges)
        q = absmod.abs_ring_q(cfg)
        assert np.array_equal(q, oracle.ring_q(edges, du))
        assert np.array_equal(absmod.abs_triplets(cfg), oracle.triplets(q))
        assert absmod.abs_fft_size(cfg) == oracle.min_fft_size(q, n)


@pytest.mark.parametrize("bad", [
    dict(n_grid=7), dict(n_grid=0), dict(n_grid=16386), dict(du=0.0), dict(du=-1.0),
    dict(du=float("nan")), dict(kernel=5), dict(sigma_cells=0.1), dict(sigma_cells=0.38), dict(radius_cells=4),
    dict(radius_cells=-1), dict(precision=3), dict(norm_A=0.0), dict(n_fft=7), dict(n_fft=80), dict(n_fft=91),
    dict(ell_edges=[10.0, 5.0]), dict(ell_edges=[0.0, 5.0]), dict(ell_edges=[5.0, float("inf")]),
    dict(weight_mode=3), dict(weight_mode=-1),
])
def test_invalid_configs_rejected(lib, bad):
    base = dict(n_grid=64, du=2.0, ell_edges=np.linspace(25, 375, 9))
    base.update(bad)
    cfg = absmod.Config(**base)
    with pytest.raises(absmod.AbsError) as ei:
        absmod.abs_ring_q(cfg) if "n_fft" not in bad else absmod.abs_fft_size(cfg)
    assert ei.value.status == absmod.ABS_ERR_INVALID_ARG


def test_fft_size_user_value(lib):
    cfg = absmod.Config(n_grid=64, du=2.0, ell_edges=np.linspace(25, 375, 9), n_fft=128)
    assert absmod.abs_fft_size(cfg) == 128
    cfg = absmod.Config(n_grid=64, du=2.0, ell_edges=np.linspace(25, 375, 9), n_fft=90)
    assert absmod.abs_fft_size(cfg) == 90


def test_product_path_has_no_cpu_fallback(monkeypatch, tmp_path):
    # with the library absent the binding raises instead of computing anything
    monkeypatch.setattr(absmod, "_lib", None)
    with pytest.raises(RuntimeError):
        absmod.load(str(tmp_path / "missing.so"))


def test_binding_rejects_wrong_buffers_before_the_call():
    """The binding checks device-buffer arguments (CUDA, dtype, contiguity, size)
    before any pointer crosses the ABI; CPU tensors and misshapen triplet lists
    are refused on the host."""
    import torch
    import paper_2412_02246_gb300 as m
    cfg = m.Config(n_grid=64, du=2.0, ell_edges=np.linspace(25.0, 375.0, 9))
    f = torch.zeros((8, cfg.N, cfg.N), dtype=torch.float32)
    with pytest.raises(ValueError, match="CUDA"):
        m.abs_triple_sums_static(cfg, f, torch.zeros((3, 3), dtype=torch.int32), torch.zeros(3, dtype=torch.float64),
                                 stream=type("S", (), {"cuda_stream": 0})())
    with pytest.raises(ValueError, match=r"\(n, 3\)"):
        m._ijk_rows(torch.zeros((3, 2), dtype=torch.int32))
    with pytest.raises(ValueError, match="required"):
        m._dev(None, "f32", 1, "x")
    assert m._dev(None, "f32", 1, "x", optional=True) is None


@pytest.mark.parametrize("cfg_id", [5, 6])
def test_cube_triplets_match_oracle(lib, cfg_id):
    wl = synth.cube_workload(cfg_id)
    cfg = absmod.Config3D(absmod.Config.from_workload(wl), wl.extra["n_chan"], wl.extra["tau"])
    q = oracle.ring_q(wl.ell_edges, wl.du)
    assert np.array_equal(absmod.abs_triplets_3d(cfg), oracle.triplets_3d(q, wl.extra["tau"]))


def test_cube_triplets_random_delay_bins_match_oracle(lib):
    rng = np.random.default_rng(11)
    wl = synth.workload(0)
    q = oracle.ring_q(wl.ell_edges, wl.du)
    for _ in range(6):
        n_chan = int(rng.integers(2, 40))
        t_top = int(rng.integers(1, (n_chan - 1) // 2 + 2))      # delay_edges[-1]: 2 (t_top - 1) < n_chan
        start = int(rng.integers(0, min(2, t_top)))              # 0, or 1 (drop t = 0) when t_top > 1
        inner = rng.integers(start + 1, t_top, int(rng.integers(0, 4))).tolist() if t_top > start + 1 else []
        tau = sorted(set([start, t_top] + inner))
        cfg = absmod.Config3D(absmod.Config.from_workload(wl), n_chan, tau)
        assert np.array_equal(absmod.abs_triplets_3d(cfg), oracle.triplets_3d(q, tau)), (n_chan, tau)


def test_cube_config_checks(lib):
    wl = synth.workload(0)
    base = absmod.Config.from_workload(wl)
    bad = [
        absmod.Config3D(base, 8, [0, 2, 1]),       # not ascending
        absmod.Config3D(base, 8, [0, 1, 5]),       # 2 t_max = 8 >= n_chan
        absmod.Config3D(base, 0, [0, 1]),          # no channels
        absmod.Config3D(base, 8, [-1, 1]),         # negative edge
        absmod.Config3D(base, 8, [0, 1, 4], n_z=9),   # n_z below 3 t_max + 1 = 10
        absmod.Config3D(absmod.Config.from_workload(wl, weight_mode=absmod.ABS_W_PAPER_LITERAL), 8, [0, 1]),
    ]
    for cfg in bad:
        with pytest.raises(absmod.AbsError):
            absmod.abs_triplets_3d(cfg)
    assert len(absmod.abs_triplets_3d(absmod.Config3D(base, 8, [0, 1, 4], n_z=10))) > 0


def test_binding_gives_every_declared_call_a_signature(lib):
    """Every call the header declares has explicit ctypes argument and result types in the binding
    (a call without them would be passed guessed C types)."""
    for n in declared_functions():
        f = getattr(lib, n)
        assert f.argtypes is not None, n
        assert f.restype is not None, n
    # and as many arguments as the declaration has parameters
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "abs.h")).read(), flags=re.S)
    decls = re.findall(r"^(?:abs_status|const char \*)\s*(abs_\w+)\s*\(([^;]*?)\)\s*;", src, re.M | re.S)
    assert len(decls) == len(declared_functions())
    for name, params in decls:
        params = params.strip()
        want = 0 if params in ("", "void") else len(params.split(","))
        assert len(getattr(lib, name).argtypes) == want, (name, want, len(getattr(lib, name).argtypes))

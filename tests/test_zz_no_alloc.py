"""The allocation-free triple-sum entry point (abs_triple_sums_static).

Callers that cannot allocate device memory where they need the sums (code
inside CUDA stream capture, frameworks whose own allocator must be the only
one to call cudaMalloc) use this variant: it keeps its scratch in one fixed
device array inside the library.  Here it must give the same sums as
abs_triple, through the C ABI, on two calls in a row (the array keeps the
previous call's contents, which must not leak into the next result).
"""
import numpy as np
import pytest

import paper_2412_02246_gb300 as absmod
from paper_2412_02246_gb300 import build as absbuild
from paper_2412_02246_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SUM_TOL = 1e-5   # the FP32 triple-sum tolerance of the parity tests


def _fields(ctx, cfg, inp):
    dev = torch.device("cuda:0")
    n = cfg.n_grid
    g = torch.empty((n, n, 2), dtype=torch.float32, device=dev)
    w = torch.empty((n, n), dtype=torch.float32, device=dev)
    m = torch.empty((n, n), dtype=torch.uint8, device=dev)
    uv = torch.from_numpy(inp.uv).to(dev)
    vis = torch.from_numpy(synth.vis_as_float2(inp.vis)).to(dev)
    ctx.abs_grid(cfg, uv, vis, g, w, m)
    N = absmod.abs_fft_size(cfg)
    f = torch.empty((cfg.n_bins, N, N), dtype=torch.float32, device=dev)
    ctx.abs_filter_fft(cfg, g, w, m, f)
    ctx.sync()
    return f, m


@pytest.mark.parametrize("cfg_id", [0, 1])
def test_static_triple_sums_match_abs_triple(cfg_id):
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    absbuild.build()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    ctx = absmod.Context(0)
    inp = synth.make_inputs(cfg_id)
    cfg = absmod.Config.from_workload(inp.wl, precision=absmod.ABS_FP32)
    fields, mask = _fields(ctx, cfg, inp)
    ijk = torch.from_numpy(absmod.abs_triplets(cfg)).to(dev)
    nt = ijk.shape[0]
    ref = torch.empty(nt, dtype=torch.float64, device=dev)
    ctx.abs_triple(cfg, fields, mask, ijk, ref, None)
    ctx.sync()
    ref = ref.cpu().numpy()
    scale = np.abs(ref).max()
    for call in range(2):
        out = torch.full((nt,), float("nan"), dtype=torch.float64, device=dev)
        absmod.abs_triple_sums_static(cfg, fields, ijk, out)
        torch.cuda.synchronize(dev)
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), f"call {call}: non-finite sums"
        assert np.allclose(got, ref, rtol=SUM_TOL, atol=SUM_TOL * 1e-3 * scale), f"call {call} differs"
    ctx.close()


def test_static_triple_sums_reject_oversize():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    absbuild.build()
    dev = torch.device("cuda:0")
    cfg = absmod.Config.from_workload(synth.workload(0))
    lib = absmod.load()
    import ctypes
    tiny = torch.zeros(4, dtype=torch.float64, device=dev)
    too_many = (8 << 20) // 8 + 1
    st = lib.abs_triple_sums_static(cfg.ref(), ctypes.c_void_p(tiny.data_ptr()), too_many,
                                    ctypes.c_void_p(tiny.data_ptr()), ctypes.c_void_p(tiny.data_ptr()), None)
    assert st == absmod.ABS_ERR_INVALID_ARG


def _all_triplets(nb):
    """Every i <= j <= k < nb in lexicographic order: a canonical list (closing or not)."""
    i, j, k = np.meshgrid(np.arange(nb), np.arange(nb), np.arange(nb), indexing="ij")
    sel = (i <= j) & (j <= k)
    return np.stack([i[sel], j[sel], k[sel]], axis=1).astype(np.int32)


def test_static_triple_sums_long_lists_and_capture():
    """Lists long enough that the fixed array holds only one or two pixel
    splits (160 rings, all 695,520 ordered triplets, and the first 500,000 of
    them), each against abs_triple on the same random fields; then a shorter
    list right after a longer one (stale partials must not leak in); then the
    call captured into a CUDA graph after a warm-up call, and the graph
    replayed on new field values."""
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    absbuild.build()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    ctx = absmod.Context(0)
    nb = 160
    cfg = absmod.Config(n_grid=64, du=2.0, ell_edges=np.linspace(25.0, 375.0, nb + 1), precision=absmod.ABS_FP32)
    N = cfg.N
    g = torch.Generator(device=dev).manual_seed(7)
    fields = torch.randn((nb, N, N), generator=g, device=dev, dtype=torch.float32)
    full = torch.from_numpy(_all_triplets(nb)).to(dev)
    cap = (8 << 20) // 8
    assert cap // full.shape[0] == 1 and cap // 500_000 == 2

    def ref_sums(ijk):
        out = torch.empty(ijk.shape[0], dtype=torch.float64, device=dev)
        ctx.abs_triple(cfg, fields, None, ijk, out, None)
        ctx.sync()
        return out.cpu().numpy()

    def static_sums(ijk):
        out = torch.full((ijk.shape[0],), float("nan"), dtype=torch.float64, device=dev)
        absmod.abs_triple_sums_static(cfg, fields, ijk, out)
        torch.cuda.synchronize(dev)
        return out.cpu().numpy()

    def close(got, ref, what):
        scale = np.abs(ref).max()
        assert np.all(np.isfinite(got)), what
        assert np.allclose(got, ref, rtol=SUM_TOL, atol=SUM_TOL * 1e-3 * scale), what

    for ijk in (full, full[:500_000].contiguous(), full[:9_000].contiguous()):
        close(static_sums(ijk), ref_sums(ijk), f"{ijk.shape[0]} triplets")

    # capture: one eager call first (it looks the array up), then the same call in a graph
    short = full[:20_000].contiguous()
    out = torch.full((short.shape[0],), float("nan"), dtype=torch.float64, device=dev)
    absmod.abs_triple_sums_static(cfg, fields, short, out)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(dev)
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            absmod.abs_triple_sums_static(cfg, fields, short, out)
    fields.copy_(torch.randn((nb, N, N), generator=g, device=dev, dtype=torch.float32))
    out.fill_(float("nan"))
    graph.replay()
    torch.cuda.synchronize(dev)
    close(out.cpu().numpy(), ref_sums(short), "captured call")
    ctx.close()

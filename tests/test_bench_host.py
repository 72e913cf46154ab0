"""Host-side helpers of bench.py that its roofline figures rest on (no GPU).

* ring_rmax: the largest |g_x| of a ring cell, which sizes the transforms'
  intermediate; it must give the library's own sky-grid side (N is the
  smallest 2^a 3^b 5^c >= 3 R + 1).
* ring_census / count_route_visits: the pair visits of the exact-count
  kernel's route, against a direct count on a small hand-made mask.
"""
import numpy as np
import pytest

import bench
import oracle
import paper_2412_02246_gb300 as absmod
from paper_2412_02246_gb300 import synth


def _smooth(v):
    for p in (2, 3, 5):
        while v % p == 0:
            v //= p
    return v == 1


@pytest.mark.parametrize("cfg_id", [0, 1, 2, 4])
def test_ring_rmax_gives_the_library_fft_size(cfg_id):
    wl = synth.workload(cfg_id)
    cfg = absmod.Config.from_workload(wl)
    q = absmod.abs_ring_q(cfg)
    R = max(bench.ring_rmax(q, wl.n_grid // 2 - 1))
    N = absmod.abs_fft_size(cfg)
    want = max(3 * R + 1, 8)
    while not _smooth(want):
        want += 1
    assert N == want


def test_route_visits_match_a_direct_count():
    """Direct route: sum over a <= b of floor(F_a / 2) F_b pairs; holes route:
    floor(H_a / 2) A_b + 2 floor(F_a / 2) H_b; the kernel takes the smaller."""
    n = 24
    edges = 2 * np.pi * np.array([1.5, 3.0, 5.0, 7.5])
    q = oracle.ring_q(edges, 1.0)
    rng = np.random.default_rng(3)
    for fill in (1.0, 0.9, 0.3):
        mask = (rng.random((n, n)) < fill).astype(np.uint8)
        A, F = bench.ring_census(mask, q, n)
        k = np.where(np.arange(n) > n // 2, np.arange(n) - n, np.arange(n))
        r2 = k[None, :] ** 2 + k[:, None] ** 2
        on = (np.abs(k) <= n // 2 - 1)
        for b in range(len(q) - 1):
            sel = (r2 >= q[b]) & (r2 < q[b + 1]) & on[None, :] & on[:, None]
            assert A[b] == sel.sum() and F[b] == (sel & (mask > 0)).sum()
        H = A - F
        direct = sum((F[a] // 2) * F[b] for a in range(len(A)) for b in range(a, len(A)))
        holes = sum((H[a] // 2) * A[b] + 2 * (F[a] // 2) * H[b] for a in range(len(A)) for b in range(a, len(A)))
        assert bench.count_route_visits(A, F) == (holes if holes < direct else direct)
        if fill == 1.0:
            assert bench.count_route_visits(A, F) == 0

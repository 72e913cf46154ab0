"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own code path: worked cases
written out by hand, closed forms, pure-Python enumeration on tiny grids, the
FFT identity through numpy's transform, and symmetries.  Each is chosen so
that a plausible mistake (a dropped term, a wrong sign or index, a
transposed operand) fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2412_02246_gb300 import synth


# ----------------------------------------------------------------- helpers


def full_mask(n):
    f = np.ones((n, n), np.uint8)
    f[n // 2, :] = 0          # the row/column at index n/2 is off the grid (|g| <= n/2-1)
    f[:, n // 2] = 0
    return f


def coords(n):
    k = np.arange(n)
    k = np.where(k > n // 2, k - n, k)
    gy, gx = np.meshgrid(k, k, indexing="ij")
    return gx, gy


def random_hermitian_grid(n, rng):
    """X with X(-g) = conj X(g) on the grid (|g| <= n/2-1), built by explicit mirroring."""
    gx, gy = coords(n)
    X = np.zeros((n, n), np.complex128)
    half = n // 2 - 1
    for y in range(-half, half + 1):
        for x in range(-half, half + 1):
            if (y, x) < (0, 0) or (y == 0 and x < 0):
                continue
            v = complex(rng.standard_normal(), rng.standard_normal())
            if x == 0 and y == 0:
                v = complex(v.real, 0.0)
            X[y % n, x % n] = v
            X[(-y) % n, (-x) % n] = np.conj(v)
    return X


# ----------------------------------------------------------------- cell index


def test_cell_rule_worked_cases():
    # nearest grid point, ties rounded up (floor(x + 1/2)), Eq. vg
    assert oracle.cell(0.0, 1.0) == 0
    assert oracle.cell(0.5, 1.0) == 1
    assert oracle.cell(-0.5, 1.0) == 0
    assert oracle.cell(1.49, 1.0) == 1
    assert oracle.cell(-1.5, 1.0) == -1
    assert oracle.cell(-1.51, 1.0) == -2
    assert oracle.cell(7.0, 2.0) == 4          # 3.5 -> 4
    assert oracle.cell(-7.0, 2.0) == -3        # -3.5 -> -3
    assert oracle.cell(219.9, 2.3) == 96


def test_cell_rule_is_binary32():
    # 0.3/0.2: in binary32 the quotient rounds to exactly 1.5 and goes up to 2;
    # in binary64 it is 1.4999999999999998 and would go to 1.  Masks (and hence
    # counts) depend on taking the binary32 reading on both sides.
    u, du = np.float32(0.3), np.float32(0.2)
    assert np.float32(u / du) == np.float32(1.5)
    assert float(u) / float(du) != 1.5
    assert oracle.cell(0.3, 0.2) == 2


# ----------------------------------------------------------------- rings, triplets


def test_ring_thresholds_against_membership_definition():
    # a_m holds the cells with l_m <= 2 pi |g| dU < l_{m+1}: Q_m is the smallest
    # integer |g|^2 in ring m.  Checked by scanning the integers directly.
    rng = np.random.default_rng(1)
    for _ in range(20):
        du = float(np.float32(rng.uniform(0.5, 3.0)))
        edges = np.sort(rng.uniform(10.0, 900.0, 6))
        q = oracle.ring_q(edges, du)
        for m, e in enumerate(edges):
            r2 = 0
            while 2.0 * math.pi * du * math.sqrt(r2) < e:
                r2 += 1
            # r2 is the first integer with l(r2) >= e (up to the last ulp of sqrt)
            assert abs(q[m] - r2) <= 1
            if q[m] != r2:        # only possible at an exact tie in floating point
                assert abs(2.0 * math.pi * du * math.sqrt(q[m]) - e) < 1e-9 * e


def test_ring_thresholds_known_values():
    # l = 2 pi dU r with r = 2.5 -> r^2 = 6.25 -> first integer 7; r = 4.1 -> 16.81 -> 17
    q = oracle.ring_q([2 * math.pi * 2.5, 2 * math.pi * 4.1], 1.0)
    assert list(q) == [7, 17]
    q = oracle.ring_q([2 * math.pi * 2.0 * 2.5], 2.0)
    assert list(q) == [7]


def test_paper_ring_set_has_2024_combinations():
    # Sec. 3: 22 rings in grid units ([1,5], nine in 5-50, five in 50-100, five
    # in 100-200, two in 200-250), "every possible combination of three rings".
    r = [1.0, 5.0] + list(np.linspace(5, 50, 10)[1:]) + list(np.linspace(50, 100, 6)[1:]) \
        + list(np.linspace(100, 200, 6)[1:]) + list(np.linspace(200, 250, 3)[1:])
    assert len(r) == 23
    edges = 2 * np.pi * np.asarray(r)       # dU_g = 1
    q = oracle.ring_q(edges, 1.0)
    nb = len(q) - 1
    assert nb == 22
    assert len(list(itertools.combinations_with_replacement(range(nb), 3))) == 2024
    t = oracle.triplets(q)
    assert 0 < len(t) < 2024


def test_triplets_are_a_superset_of_closing_rings():
    # Every (i<=j<=k) that holds at least one closed triangle on a full grid
    # must be listed; the list must be ordered i<=j<=k lexicographically.
    n = 40
    edges = np.array([6.0, 20.0, 37.0, 55.0, 80.0, 110.0])
    du = 1.0
    q = oracle.ring_q(edges, du)
    t = oracle.triplets(q)
    assert np.all(t[:, 0] <= t[:, 1]) and np.all(t[:, 1] <= t[:, 2])
    assert [tuple(x) for x in t] == sorted(tuple(x) for x in t)
    allc = np.array(list(itertools.combinations_with_replacement(range(len(q) - 1), 3)), np.int32)
    X = np.ones((n, n), np.complex128)
    _, _, T = oracle.triple_bruteforce(X, full_mask(n), q, allc)
    listed = {tuple(x) for x in t}
    for (i, j, k), cnt in zip(allc, T):
        if cnt > 0:
            assert (i, j, k) in listed
    # and the test is tight enough to drop most non-closing combinations
    assert len(t) < len(allc)


# ----------------------------------------------------------------- gridding


def test_grid_single_visibility_on_grid_point():
    # Gaussian kernel sigma = 1 cell, r = 3: weights exp(-|d|^2/2) at c + d,
    # mirrored with V* at -(c + d).  du = 1 so U_i is exactly the grid point.
    n = 64
    v = 0.75 - 0.5j
    gr = oracle.grid(n, 1.0, np.array([[10.0, 5.0]], np.float32), np.array([v], np.complex64))
    for dy in range(-3, 4):
        for dx in range(-3, 4):
            w = math.exp(-(dx * dx + dy * dy) / 2.0)
            gx, gy = 10 + dx, 5 + dy
            assert gr.wsum[gy % n, gx % n] == pytest.approx(w, rel=1e-15)
            assert gr.grid[gy % n, gx % n] == pytest.approx(w * v, rel=1e-15)
            assert gr.grid[(-gy) % n, (-gx) % n] == pytest.approx(w * np.conj(v), rel=1e-15)
            assert gr.ncontrib[gy % n, gx % n] == 1
    s1 = sum(math.exp(-k * k / 2.0) for k in range(-3, 4))
    assert gr.wsum.sum() == pytest.approx(2 * s1 * s1, rel=1e-14)
    assert gr.ncontrib.sum() == 2 * 49


def test_grid_single_visibility_off_grid():
    # U = (c + f) dU with f = (0.25, -0.375): w = exp(-((dx - fx)^2 + (dy - fy)^2)/2)
    n, du = 64, 2.0
    fx, fy = 0.25, -0.375
    u = np.array([[(7 + fx) * du, (-9 + fy) * du]], np.float32)
    gr = oracle.grid(n, du, u, np.array([1.0 + 0j], np.complex64))
    for dy in range(-3, 4):
        for dx in range(-3, 4):
            w = math.exp(-((dx - fx) ** 2 + (dy - fy) ** 2) / 2.0)
            assert gr.wsum[(-9 + dy) % n, (7 + dx) % n] == pytest.approx(w, rel=1e-14)


def test_grid_sigma_and_radius():
    n = 32
    gr = oracle.grid(n, 1.0, np.array([[3.0, 4.0]], np.float32), np.array([1.0], np.complex64),
                     sigma_cells=2.0, radius_cells=1)
    assert gr.ncontrib.sum() == 2 * 9
    assert gr.wsum[5 % n, 4 % n] == pytest.approx(math.exp(-2.0 / 8.0), rel=1e-15)


def test_grid_ngp_sums_and_mirror():
    # NGP: every visibility lands on its nearest cell with w = 1
    n, du = 32, 1.0
    uv = np.array([[2.2, 3.1], [1.8, 2.6], [-4.0, 0.4]], np.float32)
    vis = np.array([1 + 2j, 3 - 1j, 0.5 + 0.5j], np.complex64)
    gr = oracle.grid(n, du, uv, vis, kernel="ngp")
    assert gr.grid[3, 2] == pytest.approx(complex(vis[0]) + complex(vis[1]))
    assert gr.grid[(-3) % n, (-2) % n] == pytest.approx(np.conj(complex(vis[0]) + complex(vis[1])))
    assert gr.ncontrib[3, 2] == 2 and gr.ncontrib[0, (-4) % n] == 1 and gr.ncontrib[0, 4] == 1
    assert gr.ncontrib.sum() == 6


def test_grid_edge_cells_dropped():
    # cells with |g_x| or |g_y| > n/2 - 1 are not on the grid
    n = 16
    gr = oracle.grid(n, 1.0, np.array([[7.0, 0.0]], np.float32), np.array([1.0], np.complex64))
    # footprint x in 4..10, only 4..7 kept: 4 columns x 7 rows, twice (mirror)
    assert gr.ncontrib.sum() == 2 * 4 * 7
    assert gr.ncontrib[:, n // 2].sum() == 0 and gr.ncontrib[n // 2, :].sum() == 0


def test_grid_is_hermitian():
    inp = synth.make_inputs(0)
    gr = oracle.grid(64, inp.wl.du, inp.uv, inp.vis)
    flip = lambda a: np.roll(a[::-1, ::-1], 1, axis=(0, 1))   # a(-g)
    assert np.allclose(gr.grid, np.conj(flip(gr.grid)), rtol=0, atol=1e-12 * np.abs(gr.grid).max())
    assert np.array_equal(gr.ncontrib, flip(gr.ncontrib))
    X, f = oracle.mean_grid(gr)
    assert np.array_equal(f, (gr.ncontrib > 0).astype(np.uint8))
    sel = f > 0
    assert np.allclose(X[sel] * gr.wsum[sel], gr.grid[sel], rtol=1e-14, atol=0)


# ----------------------------------------------------------------- triple sums


def python_enumeration(X, filled, q):
    """All ordered triples (g1,g2,g3) of filled ring cells with g1+g2+g3 = 0: O(C^3)."""
    n = X.shape[0]
    half = n // 2 - 1
    cells = []
    for gy in range(-half, half + 1):
        for gx in range(-half, half + 1):
            if not filled[gy % n, gx % n]:
                continue
            r2 = gx * gx + gy * gy
            m = [b for b in range(len(q) - 1) if q[b] <= r2 < q[b + 1]]
            if m:
                cells.append((gx, gy, m[0], X[gy % n, gx % n]))
    S, T = {}, {}
    for a in cells:
        for b in cells:
            for c in cells:
                if a[0] + b[0] + c[0] == 0 and a[1] + b[1] + c[1] == 0:
                    key = (a[2], b[2], c[2])
                    S[key] = S.get(key, 0) + a[3] * b[3] * c[3]
                    T[key] = T.get(key, 0) + 1
    return S, T


def test_bruteforce_matches_python_enumeration_tiny():
    rng = np.random.default_rng(7)
    n = 14
    X = random_hermitian_grid(n, rng)
    filled = full_mask(n)
    gx, gy = coords(n)
    drop = rng.random((n, n)) < 0.2
    filled[drop] = 0
    filled[(-gy[drop]) % n, (-gx[drop]) % n] = 0      # holes come in +-g pairs
    edges = 2 * np.pi * np.array([1.2, 2.6, 4.0, 5.7])
    q = oracle.ring_q(edges, 1.0)
    allc = np.array(list(itertools.product(range(3), repeat=3)), np.int32)
    S, _, T = oracle.triple_bruteforce(X, filled, q, allc)
    Sp, Tp = python_enumeration(X, filled, q)
    for t, (i, j, k) in enumerate(allc):
        assert T[t] == Tp.get((i, j, k), 0)
        assert S[t] == pytest.approx(Sp.get((i, j, k), 0), rel=1e-12, abs=1e-12)
    assert T.sum() > 0
    # triple_one agrees with the all-pairs route
    for t in (0, 5, 13, 26):
        s1, _, t1 = oracle.triple_one(X, filled, q, *allc[t])
        assert t1 == T[t] and s1 == pytest.approx(S[t], rel=1e-12, abs=1e-12)


def test_literal_weights_reduce_to_counts_and_scale():
    """Eq. iFT_I as printed: with NGP and every filled cell holding one visibility
    (N_g = 1), W = 1 and S_W is the integer count T, so the literal B equals the
    unit-mask B; doubling every visibility's weight (each position entered twice)
    halves W, so S_W = T / 8 and the literal B is 8 times the unit-mask B (X, the
    weighted mean, does not change)."""
    rng = np.random.default_rng(3)
    n, du = 32, 1.0
    cells = set()
    uv = []
    while len(uv) < 60:   # distinct cells, none the mirror of another
        c = tuple(int(x) for x in rng.integers(-12, 13, 2))
        if c == (0, 0) or c in cells or (-c[0], -c[1]) in cells:
            continue
        cells.add(c)
        uv.append(c)
    uv = np.array(uv, np.float32) + rng.uniform(-0.3, 0.3, (60, 2)).astype(np.float32)
    vis = (rng.standard_normal(60) + 1j * rng.standard_normal(60)).astype(np.complex64)
    edges = 2 * np.pi * np.array([2.0, 5.0, 8.0, 11.0, 14.0])
    e0 = oracle.estimate(n, du, edges, uv, vis, kernel="ngp")
    e1 = oracle.estimate(n, du, edges, uv, vis, kernel="ngp", weight_mode="literal")
    gr = oracle.grid(n, du, uv, vis, kernel="ngp")
    X, f = oracle.mean_grid(gr)
    W = oracle.literal_weights(gr, f)
    assert np.all(W[f > 0] == 1.0) and np.all(W[f == 0] == 0.0)
    ok = e0.T > 0
    assert ok.sum() > 5
    assert np.allclose(e1.B[ok], e0.B[ok], rtol=1e-12) and np.all(np.isnan(e1.B[~ok]))
    uv2, vis2 = np.concatenate([uv, uv]), np.concatenate([vis, vis])
    e2 = oracle.estimate(n, du, edges, uv2, vis2, kernel="ngp", weight_mode="literal")
    assert np.allclose(e2.B[ok], 8 * e0.B[ok], rtol=1e-12)


def test_literal_sums_match_python_enumeration_tiny():
    """S_W by brute force equals the pure-Python enumeration of W1 W2 W3 over
    closed triangles on a tiny grid with uneven weights."""
    rng = np.random.default_rng(11)
    n = 14
    filled = full_mask(n)
    gx, gy = coords(n)
    drop = rng.random((n, n)) < 0.2
    filled[drop] = 0
    filled[(-gy[drop]) % n, (-gx[drop]) % n] = 0
    w = rng.uniform(0.5, 3.0, (n, n))
    w = 0.5 * (w + w[(-gy) % n, (-gx) % n])            # N_g = N_-g, as the mirror makes it
    W = np.where(filled > 0, 1.0 / w, 0.0)
    edges = 2 * np.pi * np.array([1.2, 2.6, 4.0, 5.7])
    q = oracle.ring_q(edges, 1.0)
    allc = np.array(list(itertools.product(range(3), repeat=3)), np.int32)
    SW, _, T = oracle.triple_bruteforce(W.astype(np.complex128), filled, q, allc)
    Sp, Tp = python_enumeration(W.astype(np.complex128), filled, q)
    for t, (i, j, k) in enumerate(allc):
        assert SW[t] == pytest.approx(Sp.get((i, j, k), 0), rel=1e-12, abs=1e-12)
        assert abs(SW[t].imag) == 0.0


def test_fft_identity_and_aliasing():
    # Sec. 2: sum_theta D_i D_j D_k (Eq. iFT) equals N^2 times the sum over closed
    # grid triangles when the sky grid is large enough (N >= 3R+1) to exclude
    # wrapped triangles; smaller N aliases.
    inp = synth.make_inputs(0)
    wl = inp.wl
    est = oracle.estimate(wl.n_grid, wl.du, wl.ell_edges, inp.uv, inp.vis)
    N = oracle.min_fft_size(est.q)
    assert N == 90
    S_fft, T_fft, T_raw = oracle.fft_form(est.X, est.filled, est.q, est.ijk, N)
    assert np.max(np.abs(S_fft - est.S.real) / np.maximum(est.absum, 1e-300)) < 1e-12
    assert np.array_equal(T_fft, est.T)
    assert np.max(np.abs(T_raw - est.T)) < 1e-6
    S_al, T_al, _ = oracle.fft_form(est.X, est.filled, est.q, est.ijk, 64)
    assert np.sum(T_al != est.T) > 0


def test_fft_form_all_matches_bruteforce():
    # The matrix-product route of fft_form_all is the same Eq. estimator_t sums:
    # against the brute-force closed-triangle sums of the tiny workload at the
    # smallest admissible N and at a larger one (results independent of N once
    # N >= 3R+1), sums to rounding of sum |X1 X2 X3|, counts exact; and entry
    # for entry against the per-triplet fft_form.  Triplets are taken in a
    # shuffled subset too, so that the (j, i, k) bookkeeping cannot hide behind
    # the canonical order (the matrix shapes change, so the sums agree to
    # rounding, the counts exactly).
    inp = synth.make_inputs(0)
    wl = inp.wl
    est = oracle.estimate(wl.n_grid, wl.du, wl.ell_edges, inp.uv, inp.vis)
    for N in (90, 128):
        S, T, T_raw, D, I = oracle.fft_form_all(est.X, est.filled, est.q, est.ijk, N)
        assert np.max(np.abs(S - est.S.real) / np.maximum(est.absum, 1e-300)) < 1e-12
        assert np.array_equal(T, est.T)
        assert np.max(np.abs(T_raw - est.T)) < 1e-6
    S1, T1, _ = oracle.fft_form(est.X, est.filled, est.q, est.ijk, 90)
    S, T, _, D, I = oracle.fft_form_all(est.X, est.filled, est.q, est.ijk, 90)
    assert np.allclose(S, S1, rtol=1e-12, atol=1e-12 * np.abs(S1).max()) and np.array_equal(T, T1)
    perm = np.random.default_rng(3).permutation(len(est.ijk))[:40]
    Sp, Tp, _, _, _ = oracle.fft_form_all(None, None, None, est.ijk[perm], 90, fields=(D, I))
    assert np.allclose(Sp, S[perm], rtol=1e-12, atol=1e-12 * np.abs(S).max()) and np.array_equal(Tp, T[perm])


def test_constant_visibilities_give_s_cubed():
    # V = s (real) everywhere -> every filled X_g = s (the gridded mean of a constant,
    # mirror included) -> B = s^3 on every triplet with T > 0, whatever the gridding
    # kernel (a point source at the phase centre).
    inp = synth.make_inputs(0)
    wl = inp.wl
    vis = np.full(len(inp.uv), 0.7, np.complex64)
    s = float(np.float32(0.7))
    for kernel in ("gauss", "ngp"):
        est = oracle.estimate(wl.n_grid, wl.du, wl.ell_edges, inp.uv, vis, kernel=kernel)
        ok = est.T > 0
        assert ok.sum() > 50
        assert np.allclose(est.B[ok], s ** 3, rtol=1e-12)
        assert np.all(np.isnan(est.B[~ok]))


def test_point_source_phase_closure():
    # X_g = s exp(-2 pi i g.p0 / M): the phases cancel on every closed triangle
    # (g1+g2+g3 = 0), so S = s^3 T exactly; a wrong closure sign would not cancel.
    n = 48
    gx, gy = coords(n)
    p0 = (5.0, -3.0)
    s = 1.3
    X = s * np.exp(-2j * np.pi * (gx * p0[0] + gy * p0[1]) / 37.0)
    q = oracle.ring_q(2 * np.pi * np.array([2.0, 6.0, 10.0, 15.0, 21.0]), 1.0)
    ijk = oracle.triplets(q)
    S, _, T = oracle.triple_bruteforce(X, full_mask(n), q, ijk)
    assert np.all(T > 0)
    assert np.allclose(S, s ** 3 * T, rtol=1e-11)
    B = oracle.normalise(S, T)
    assert np.allclose(B, s ** 3, rtol=1e-11)


def test_ring_constant_fields_give_products():
    n = 40
    gx, gy = coords(n)
    edges = 2 * np.pi * np.array([2.0, 5.0, 8.0, 12.0, 17.0])
    q = oracle.ring_q(edges, 1.0)
    r2 = gx.astype(np.int64) ** 2 + gy.astype(np.int64) ** 2
    xm = np.array([1.5, -0.5, 2.0, 0.25])
    X = np.zeros((n, n), np.complex128)
    for m in range(4):
        X[(r2 >= q[m]) & (r2 < q[m + 1])] = xm[m]
    ijk = oracle.triplets(q)
    S, _, T = oracle.triple_bruteforce(X, full_mask(n), q, ijk)
    B = oracle.normalise(S, T, norm_A=2.0)
    for t, (i, j, k) in enumerate(ijk):
        if T[t] > 0:
            assert B[t] == pytest.approx(xm[i] * xm[j] * xm[k] / 2.0, rel=1e-13)
        else:
            assert np.isnan(B[t])


def test_rotation_and_reflection_invariance():
    rng = np.random.default_rng(3)
    n = 32
    X = random_hermitian_grid(n, rng)
    q = oracle.ring_q(2 * np.pi * np.array([2.0, 4.5, 7.0, 10.0, 14.0]), 1.0)
    ijk = oracle.triplets(q)
    f = full_mask(n)
    S0, _, T0 = oracle.triple_bruteforce(X, f, q, ijk)
    gx, gy = coords(n)
    rot = X[(gx % n), (-gy) % n]           # X'(gx, gy) = X(-gy, gx): 90 degree rotation
    ref = X[(-gy) % n, gx % n]             # X'(gx, gy) = X(gx, -gy): reflection
    for Y in (rot, ref):
        S1, _, T1 = oracle.triple_bruteforce(Y, f, q, ijk)
        assert np.array_equal(T1, T0)
        assert np.allclose(S1, S0, rtol=1e-11, atol=1e-11 * np.abs(S0).max())


def test_counts_permutation_symmetric_and_real_sums():
    inp = synth.make_inputs(0)
    wl = inp.wl
    est = oracle.estimate(wl.n_grid, wl.du, wl.ell_edges, inp.uv, inp.vis)
    perms = []
    for (i, j, k) in est.ijk[:30]:
        perms += [(i, j, k), (k, j, i), (j, k, i), (i, k, j)]
    perms = np.array(perms, np.int32)
    S, A, T = oracle.triple_bruteforce(est.X, est.filled, est.q, perms)
    T4, S4 = T.reshape(-1, 4), S.reshape(-1, 4)
    assert np.all(T4 == T4[:, :1])
    assert np.allclose(S4, S4[:, :1], rtol=1e-11, atol=1e-12 * np.abs(S4).max())
    # Hermitian grid -> imaginary parts cancel to rounding
    assert np.max(np.abs(est.S.imag) / np.maximum(est.absum, 1e-300)) < 1e-13
    # sum over k of T_ijk is bounded by |a_i||a_j| (each pair closes at most once)
    assert np.all(T >= 0)


def test_ellbar_hand_mask():
    n = 32
    f = np.zeros((n, n), np.uint8)
    for (x, y) in [(3, 4), (-3, -4), (5, 0), (-5, 0), (1, 1), (-1, -1)]:
        f[y % n, x % n] = 1
    du = 2.0
    q = oracle.ring_q(2 * np.pi * du * np.array([1.0, 3.0, 6.0]), du)
    e = oracle.ellbar(f, q, du)
    assert e[0] == pytest.approx(2 * np.pi * du * math.sqrt(2.0), rel=1e-15)
    assert e[1] == pytest.approx(2 * np.pi * du * 5.0, rel=1e-15)


def test_normalise_nan_on_empty():
    B = oracle.normalise(np.array([6.0 + 0j, 1.0, 0.0]), np.array([3, 0, 2]), norm_A=2.0)
    assert B[0] == 1.0 and np.isnan(B[1]) and B[2] == 0.0


# ----------------------------------------------------------------- statistics


def _grid_direct_B(delta_modes, q, ijk):
    """Estimator on X_g = map modes directly (no gridding), full mask."""
    n = delta_modes.shape[0]
    S, _, T = oracle.triple_bruteforce(delta_modes, full_mask(n), q, ijk)
    return oracle.normalise(S, T), T


def _closed_form_expectation(P, q, ijk, f, M):
    """Discrete Eq. bsana: E[X1 X2 X3] = 2 f M^2 (P1P2 + P2P3 + P3P1) per closed
    triangle (Wick's theorem on the quadratic field, App. B, with sums for
    integrals), averaged over the closed triangles of each ring triplet."""
    n = P.shape[0]
    half = n // 2 - 1
    gx, gy = coords(n)
    r2 = gx.astype(np.int64) ** 2 + gy.astype(np.int64) ** 2
    inside = (np.abs(gx) <= half) & (np.abs(gy) <= half)
    binmap = np.full((n, n), -1)
    for m in range(len(q) - 1):
        binmap[inside & (r2 >= q[m]) & (r2 < q[m + 1])] = m
    cy, cx = np.nonzero(binmap >= 0)
    g = np.stack([gx[cy, cx], gy[cy, cx]], 1)
    bm = binmap[cy, cx]
    Pc = P[cy, cx]
    nb = len(q) - 1
    acc = np.zeros((nb, nb, nb))
    cnt = np.zeros((nb, nb, nb))
    for a in range(len(g)):
        h = -(g[a] + g)
        ok = (np.abs(h[:, 0]) <= half) & (np.abs(h[:, 1]) <= half)
        hk = np.full(len(g), -1)
        hk[ok] = binmap[h[ok, 1] % n, h[ok, 0] % n]
        sel = hk >= 0
        P3 = P[h[sel, 1] % n, h[sel, 0] % n]
        val = Pc[a] * Pc[sel] + Pc[sel] * P3 + P3 * Pc[a]
        np.add.at(acc, (bm[a], bm[sel], hk[sel]), val)
        np.add.at(cnt, (bm[a], bm[sel], hk[sel]), 1)
    out = np.array([acc[i, j, k] / cnt[i, j, k] if cnt[i, j, k] else np.nan for i, j, k in ijk])
    return 2.0 * f * M * M * out


@pytest.mark.slow
def test_gaussian_sky_has_zero_mean_and_quadratic_sky_matches_closed_form():
    M = 32
    q = oracle.ring_q(2 * np.pi * np.array([2.0, 4.0, 6.5, 9.0, 13.0]), 1.0)
    ijk = oracle.triplets(q)
    P = synth.power_spectrum_model(M)
    R = 300
    rng = np.random.default_rng(2024)
    res = {}
    for f in (0.0, 0.05):
        Bs = []
        for _ in range(R):
            g = synth.gaussian_field(M, rng)
            modes = synth.sky_modes(synth.quadratic_sky(g, f))
            B, T = _grid_direct_B(modes, q, ijk)
            Bs.append(B)
        Bs = np.array(Bs)
        res[f] = (Bs.mean(0), Bs.std(0, ddof=1) / np.sqrt(R))
    mean0, se0 = res[0.0]
    z0 = mean0 / se0
    assert np.all(np.abs(z0) < 5.0)
    expect = _closed_form_expectation(P, q, ijk, 0.05, M)
    mean1, se1 = res[0.05]
    z1 = (mean1 - expect) / se1
    assert np.all(np.abs(z1) < 5.0)
    # the pin has teeth: the signal is detected, and a halved or doubled
    # prediction (a dropped Wick pairing, a wrong factor 2) is rejected
    assert np.max(np.abs(mean1 / se1)) > 10.0
    assert np.max(np.abs((mean1 - 0.5 * expect) / se1)) > 5.0
    assert np.max(np.abs((mean1 - 2.0 * expect) / se1)) > 5.0


# ----------------------------------------------------------------- paper constants


def test_paper_constants():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")
    vals = {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            vals[k.strip()] = float(v)
    c = oracle.beam_constants(vals["theta_F_deg"])
    # Sec. 3 prints dU_g ~ 1 and a decorrelation factor of 0.89
    assert round(c["du_g"], 0) == vals["du_g_approx"]
    assert round(c["decorrelation"], 2) == vals["decorrelation"]
    assert c["A"] == pytest.approx(np.pi * (0.6 * np.deg2rad(vals["theta_F_deg"])) ** 2 / 3)


# ----------------------------------------------------------------- results layer: (l1, mu, t) rebinning


def test_shape_params_match_vector_triangles():
    """mu and t against triangles built as 2-D vectors l1 + l2 + l3 = 0: mu is
    -l1.l2 / (|l1||l2|) taken from the vectors' dot product, t = |l2| / |l1|;
    equilateral (0.5, 1), folded (1, 0.5) and a 3-4-5 triangle (0.8, 0.8)."""
    rng = np.random.default_rng(3)
    cases = []
    for _ in range(20):
        a = rng.uniform(0.2, 3.0, 2)
        b = rng.uniform(0.2, 3.0, 2)
        v = [a, b, -(a + b)]
        lens = np.array([np.hypot(*x) for x in v])
        o = np.argsort(-lens)                       # l1 >= l2 >= l3
        l1v, l2v = v[o[0]], v[o[1]]
        mu_ref = -np.dot(l1v, l2v) / (lens[o[0]] * lens[o[1]])
        cases.append((lens[o[2]], lens[o[1]], lens[o[0]], mu_ref, lens[o[1]] / lens[o[0]]))
    cases += [(1.0, 1.0, 1.0, 0.5, 1.0), (1.0, 1.0, 2.0, 1.0, 0.5), (3.0, 4.0, 5.0, 0.8, 0.8)]
    ell = np.array([x for c in cases for x in c[:3]])
    ijk = np.arange(len(ell)).reshape(-1, 3)
    l1, mu, t = oracle.shape_params(ell, ijk)
    for q, c in enumerate(cases):
        assert l1[q] == c[2]
        assert abs(mu[q] - c[3]) < 1e-12 and abs(t[q] - c[4]) < 1e-12


def test_shape_cell_edges_and_clamping():
    ijk = np.array([[0, 0, 2]] * 7)
    # bins of width 0.1 from 0.5; values away from the edges except the exact ones 0.5 and 1
    mu = np.array([0.5, 0.5999999, 0.625, 0.95, 1.0, 0.49, 1.02])
    t = np.array([1.0, 0.5, 0.55, 0.75, 0.9999, 0.3, np.nan])
    c = oracle.shape_cell(ijk, mu, t, 5, 5)
    want = [(0, 4), (0, 0), (1, 0), (4, 2), (4, 4), (0, 0), (4, 0)]
    assert [tuple(divmod(int(x) - 2 * 25, 5)) for x in c] == want


def _rebin_case(seed=4, nb=6, R=3):
    rng = np.random.default_rng(seed)
    ell = np.sort(rng.uniform(50.0, 400.0, nb))
    ijk = np.array([(i, j, k) for i in range(nb) for j in range(i, nb) for k in range(j, nb)
                    if ell[k] < ell[i] + ell[j]])
    T = rng.integers(0, 50, len(ijk))
    T[::5] = 0
    B = rng.normal(size=(R, len(ijk)))
    B[:, T == 0] = np.nan
    return ell, ijk, T, B, nb


def test_rebin_constant_and_weights():
    ell, ijk, T, B, nb = _rebin_case()
    mean, sig, w = oracle.rebin(np.full_like(B, 2.5), T, ell, ijk, nb)
    live = w > 0
    assert np.allclose(mean[live], 2.5, rtol=0, atol=1e-14) and np.all(sig[live] < 1e-7)
    assert np.all(np.isnan(mean[~live])) and w.sum() == T.sum()


def test_rebin_is_linear_and_symmetric_ensembles_spread():
    ell, ijk, T, B, nb = _rebin_case(R=1)
    m1, _, w = oracle.rebin(B, T, ell, ijk, nb)
    m2, _, _ = oracle.rebin(3.0 * B - 1.0, T, ell, ijk, nb)
    live = w > 0
    assert np.allclose(m2[live], 3.0 * m1[live] - 1.0, rtol=1e-12, atol=1e-12)
    # two realisations +B and -B: mean 0, spread |count-weighted mean of B|
    mean, sig, _ = oracle.rebin(np.vstack([B, -B]), T, ell, ijk, nb)
    assert np.allclose(mean[live], 0.0, atol=1e-14)
    assert np.allclose(sig[live], np.abs(m1[live]), rtol=1e-9, atol=1e-14)


# ----------------------------------------------------------------- discretely sampled prediction [B_Ana]_d


def _bana_case(seed=12, n=14):
    rng = np.random.default_rng(seed)
    filled = full_mask(n)
    gx, gy = coords(n)
    drop = rng.random((n, n)) < 0.2
    filled[drop] = 0
    filled[(-gy[drop]) % n, (-gx[drop]) % n] = 0
    ell = 2 * np.pi * np.hypot(gx, gy)
    with np.errstate(divide="ignore"):
        C = np.where(ell > 0, ell ** -2.5, 0.0) * 1e4
    edges = 2 * np.pi * np.array([1.2, 2.6, 4.0, 5.7])
    return C, filled, oracle.ring_q(edges, 1.0)


def test_bana_d_matches_python_enumeration_tiny():
    """Sum of C1 C2 + C2 C3 + C3 C1 over every ordered closed triangle of filled
    ring cells, enumerated in pure Python, on a tiny grid with holes; all 27
    ring orders (the sum is symmetric in them, so the permuted triplets agree)."""
    C, filled, q = _bana_case()
    n = C.shape[0]
    half = n // 2 - 1
    cells = []
    for gy in range(-half, half + 1):
        for gx in range(-half, half + 1):
            r2 = gx * gx + gy * gy
            m = [b for b in range(len(q) - 1) if q[b] <= r2 < q[b + 1]]
            if filled[gy % n, gx % n] and m:
                cells.append((gx, gy, m[0], C[gy % n, gx % n]))
    S, T = {}, {}
    for a in cells:
        for b in cells:
            for c in cells:
                if a[0] + b[0] + c[0] == 0 and a[1] + b[1] + c[1] == 0:
                    key = (a[2], b[2], c[2])
                    S[key] = S.get(key, 0.0) + a[3] * b[3] + b[3] * c[3] + c[3] * a[3]
                    T[key] = T.get(key, 0) + 1
    allc = np.array(list(itertools.product(range(3), repeat=3)), np.int32)
    out, Tb = oracle.bana_d(C, filled, q, allc, 0.05)
    for t, (i, j, k) in enumerate(allc):
        assert Tb[t] == T.get((i, j, k), 0)
        if Tb[t]:
            assert out[t] == pytest.approx(2 * 0.05 * S[(i, j, k)] / T[(i, j, k)], rel=1e-12)
            assert out[t] == pytest.approx(out[list(map(tuple, allc)).index((k, i, j))], rel=1e-12)
        else:
            assert np.isnan(out[t])


def test_bana_d_constant_spectrum():
    """C = c on every cell: each triangle contributes 3 c^2, so [B_Ana]_d = 6 (f/sigma) c^2
    (the equilateral form of Eq. bsana) on every triplet with triangles."""
    _, filled, q = _bana_case()
    C = np.full(filled.shape, 0.7)
    ijk = oracle.triplets(q)
    out, T = oracle.bana_d(C, filled, q, ijk, 0.2)
    assert np.all(T[T > 0] > 0) and (T > 0).sum() >= 3
    assert np.allclose(out[T > 0], 6 * 0.2 * 0.49, rtol=1e-14)


# ----------------------------------------------------------------- visibility simulator (Eqs. vis, beam)


def test_simulator_single_pixel_closed_forms():
    """One bright pixel: at the phase centre V(U) = dtheta^2 A(0) T for every U; at
    theta_0 V(U) = dtheta^2 A(theta_0) T exp(+i 2 pi U.theta_0) (the sign of Eq. vis)."""
    m, dth = 32, 0.01
    rng = np.random.default_rng(2)
    uv = rng.uniform(-60, 60, (50, 2))
    sky = np.zeros((m, m))
    sky[m // 2, m // 2] = 3.0
    V = oracle.simulate_vis(sky, dth, uv, "gauss", 0.2)
    assert np.allclose(V, 3.0 * dth ** 2, rtol=1e-13, atol=0)
    sky[:] = 0
    a0, b0 = m // 2 + 5, m // 2 - 3
    sky[b0, a0] = 2.0
    th0 = np.array([5 * dth, -3 * dth])
    A0 = np.sinc(1.7 * th0[0]) ** 2 * np.sinc(1.7 * th0[1]) ** 2
    V = oracle.simulate_vis(sky, dth, uv, "mwa", 1.7)
    want = 2.0 * dth ** 2 * A0 * np.exp(2j * np.pi * (uv @ th0))
    assert np.allclose(V, want, rtol=1e-12, atol=1e-18)


def test_simulator_real_sky_is_hermitian():
    rng = np.random.default_rng(8)
    sky = rng.normal(size=(24, 24))
    uv = rng.uniform(-40, 40, (30, 2))
    V = oracle.simulate_vis(sky, 0.02, uv, "mwa", 2.0)
    Vm = oracle.simulate_vis(sky, 0.02, -uv, "mwa", 2.0)
    assert np.allclose(Vm, np.conj(V), rtol=1e-12, atol=1e-15)


def test_mwa_tile_beam_fwhm_is_the_printed_one():
    """Eq. beam for a d = 4 m tile at 154.25 MHz has the FWHM quoted beside it (24.68 deg)."""
    lam = 299792458.0 / 154.25e6
    d_over_lam = 4.0 / lam
    m, dth = 1501, np.deg2rad(0.02)                  # a 30 deg wide grid
    A = oracle.sky_weights(np.ones((m, m)), dth, "mwa", d_over_lam)[m // 2] / dth ** 2
    th = (np.arange(m) - m // 2) * dth
    i = np.nonzero(A >= 0.5)[0].max()                # last sample above half power, then interpolate
    x_half = th[i] + (A[i] - 0.5) / (A[i] - A[i + 1]) * (th[i + 1] - th[i])
    assert abs(np.rad2deg(2 * x_half) - 24.68) < 0.05


def _py_grid(n, du, uv, vis, sigma, r):
    """Eq. vg written out in Python: every visibility at its nearest grid point's
    (2r+1)^2 footprint and, conjugated, at the mirror; per cell the weighted sum V_g,
    the weight sum, the squared-weight sum and the count N_g of entries."""
    half = n // 2 - 1
    V = np.zeros((n, n), np.complex128)
    ws = np.zeros((n, n))
    w2 = np.zeros((n, n))
    N = np.zeros((n, n), np.int64)
    for (u, v), z in zip(uv.astype(np.float64), vis.astype(np.complex128)):
        cx, cy = int(np.floor(u / du + 0.5)), int(np.floor(v / du + 0.5))
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                gx, gy = cx + dx, cy + dy
                if abs(gx) > half or abs(gy) > half:
                    continue
                w = np.exp(-((gx * du - u) ** 2 + (gy * du - v) ** 2) / (2 * sigma ** 2 * du ** 2))
                for sx, sy, val in ((gx, gy, z), (-gx, -gy, np.conj(z))):
                    V[sy % n, sx % n] += w * val
                    ws[sy % n, sx % n] += w
                    w2[sy % n, sx % n] += w * w
                    N[sy % n, sx % n] += 1
    return V, ws, w2, N


@pytest.mark.parametrize("mode", ["literal", "noise"])
def test_weighted_estimators_match_python_definition_gaussian(mode):
    """The weighted estimators against Eqs. vg, iFT, iFT_I and estimator_t written out
    in Python on a tiny Gaussian-gridded case where cells collect several visibilities,
    so the count N_g, the weight sum and (sum w)^2 / sum w^2 all differ.  literal: D from
    V_g / N_g, I from 1 / N_g (Sec. 2's W_g = N_g^-1).  noise: D from the weighted mean
    times N_eff = (sum w)^2 / sum w^2, I from N_eff."""
    rng = np.random.default_rng(21)
    n, du, sigma, r = 16, 1.0, 1.0, 1
    base = rng.integers(-5, 6, (36, 2)).astype(np.float64)
    uv = (base + rng.uniform(-0.4, 0.4, base.shape)).astype(np.float32)
    vis = (rng.standard_normal(36) + 1j * rng.standard_normal(36)).astype(np.complex64)
    edges = 2 * np.pi * np.array([1.5, 3.0, 4.5, 6.0])
    est = oracle.estimate(n, du, edges, uv, vis, kernel="gauss", sigma_cells=sigma, radius_cells=r,
                          weight_mode=mode)
    V, ws, w2, N = _py_grid(n, du, uv, vis, sigma, r)
    filled = (N > 0).astype(np.uint8)
    assert np.any((N > 1) & (np.abs(ws - N) > 0.1))           # count and weight sum differ
    if mode == "literal":
        Y = np.where(N > 0, V / np.maximum(N, 1), 0)
        W = np.where(N > 0, 1.0 / np.maximum(N, 1), 0.0)
    else:
        neff = np.where(N > 0, ws ** 2 / np.where(w2 > 0, w2, 1.0), 0.0)
        Y = np.where(N > 0, V / np.where(ws > 0, ws, 1.0), 0) * neff
        W = neff
    q = oracle.ring_q(edges, du)
    Sp, _ = python_enumeration(Y, filled, q)
    Wp, _ = python_enumeration(W.astype(np.complex128), filled, q)
    checked = 0
    for t, (i, j, k) in enumerate(est.ijk):
        sw = Wp.get((i, j, k), 0)
        if sw == 0:
            assert np.isnan(est.B[t])
            continue
        assert est.B[t] == pytest.approx(Sp[(i, j, k)].real / sw.real, rel=1e-10, abs=1e-12)
        checked += 1
    assert checked >= 5


def test_noise_weights_reduce_to_natural_weighting_ngp():
    """With nearest-grid-point gridding every weight is 1, so N_eff = N_g and the
    noise-weighted D fields carry the plain sums V_g (natural weighting): the noise
    B equals sum V1 V2 V3 / sum N1 N2 N3 over the closed triangles, computed here from
    the oracle's own grid sums by the brute-force triple sum."""
    rng = np.random.default_rng(5)
    n, du = 24, 1.0
    base = rng.integers(-8, 9, (80, 2)).astype(np.float64)
    uv = (base + rng.uniform(-0.3, 0.3, base.shape)).astype(np.float32)
    vis = (rng.standard_normal(80) + 1j * rng.standard_normal(80)).astype(np.complex64)
    edges = 2 * np.pi * np.array([2.0, 4.5, 7.0, 9.5])
    est = oracle.estimate(n, du, edges, uv, vis, kernel="ngp", weight_mode="noise")
    gr = oracle.grid(n, du, uv, vis, kernel="ngp")
    f = (gr.ncontrib > 0).astype(np.uint8)
    assert np.array_equal(gr.wsum, gr.ncontrib.astype(np.float64))
    assert np.array_equal(gr.wsum2, gr.ncontrib.astype(np.float64))
    assert gr.ncontrib.max() > 1
    S, _, _ = oracle.triple_bruteforce(gr.grid, f, est.q, est.ijk)
    SN, _, _ = oracle.triple_bruteforce(gr.ncontrib.astype(np.complex128), f, est.q, est.ijk)
    ok = SN.real > 0
    assert ok.sum() >= 5
    assert np.allclose(est.B[ok], S.real[ok] / SN.real[ok], rtol=1e-12)


@pytest.mark.slow
def test_pure_noise_visibilities_give_zero_mean_B():
    """Uncorrelated visibility noise adds no bias (Sec. 2, the end of the estimator's description): with
    complex Gaussian noise alone at the tiny workload's baselines, gridded with the Gaussian kernel and the
    Hermitian mirror, every term of E[X1 X2 X3] is a third moment of zero-mean Gaussians, so the mean of B
    over realisations is 0 within its standard error on every triplet.  Teeth: a constant visibility
    s = 0.15 under the same noise is detected (its B is s^3)."""
    inp = synth.make_inputs(0)
    wl = inp.wl
    rng = np.random.default_rng(2026)
    R = 150
    res = {}
    for s in (0.0, 0.15):
        Bs = []
        for _ in range(R):
            n = rng.standard_normal(len(inp.uv)) + 1j * rng.standard_normal(len(inp.uv))
            est = oracle.estimate(wl.n_grid, wl.du, wl.ell_edges, inp.uv, (s + n).astype(np.complex64))
            Bs.append(est.B)
        Bs = np.array(Bs)
        res[s] = (np.nanmean(Bs, 0), np.nanstd(Bs, 0, ddof=1) / np.sqrt(R))
    m0, se0 = res[0.0]
    ok = np.isfinite(m0)
    assert ok.sum() >= 50
    assert np.all(np.abs(m0[ok] / se0[ok]) < 5.0)
    m1, se1 = res[0.15]
    assert np.max(np.abs(m1[ok] / se1[ok])) > 10.0

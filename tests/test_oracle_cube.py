"""Pins of the oracle's multi-frequency (3-D) form.

The 3-D form (a reading of the generalisation named as future work in Sec. 1
and Sec. 5) grids every channel on one uv grid, transforms the cells filled in
every channel along frequency into delay modes t, bins the voxels (g, t) by
ring and by |t|, and sums Xt Xt Xt over the voxel triangles that close in g and
in t.  These tests pin the oracle's brute force, its delay counts, its
canonical triplet list and its FFT form against what the definitions fix:
reduction to the (separately pinned) 2-D form, factorisation of a separable
cube through numpy's FFT along frequency, invariance under shifts and reversal
of the channel order, real sums, closed-form delay counts, and agreement of the
two routes.
"""
import numpy as np
import pytest

import oracle
from paper_2412_02246_gb300 import synth


def _tiny(n_rings: int | None = None):
    ci = synth.cube_inputs(5)
    wl = ci.wl
    X, F = oracle.cube_means(wl.n_grid, wl.du, ci.uv, ci.vis)
    edges = wl.ell_edges if n_rings is None else wl.ell_edges[: n_rings + 1]
    q = oracle.ring_q(edges, wl.du)
    return ci, X, F, q


def _B(S, T):
    return oracle.normalise(S, T)


def test_one_channel_is_the_2d_form():
    ci, X, F, q = _tiny()
    Xt, common = oracle.delay_modes(X[:1], F[:1], 0)
    assert np.array_equal(common, F[0])
    assert np.array_equal(Xt[0], X[0])
    ijk = oracle.triplets(q)
    tau = [0, 1]
    uvw = oracle.triplets_3d(q, tau)
    assert np.array_equal(uvw, ijk)   # one delay bin: bin u is ring u
    S3, A3, T3 = oracle.triple3d_bruteforce(Xt, common, q, tau, uvw)
    S2, A2, T2 = oracle.triple_bruteforce(X[0], F[0], q, ijk)
    assert np.array_equal(T3, T2)
    assert np.max(np.abs(S3 - S2) / np.maximum(A2, 1e-300)) < 1e-13


def test_separable_cube_factorises():
    """X_c(g) = x(g) f(c): the delay modes are x(g) F(t) with F numpy's FFT of f, so
    S_uvw = S2(rings) x sum over closed (t1, t2, t3) in the delay bins of F1 F2 F3."""
    ci, X, F, q = _tiny(n_rings=5)
    n_chan = X.shape[0]
    rng = np.random.default_rng(7)
    f = rng.standard_normal(n_chan)
    x = X[0]
    Xs = x[None] * f[:, None, None]
    Fs = np.repeat(F[:1], n_chan, axis=0)
    tau = [int(v) for v in ci.tau]
    t_max = tau[-1] - 1
    Xt, common = oracle.delay_modes(Xs, Fs, t_max)
    uvw = oracle.triplets_3d(q, tau)
    S3, A3, T3 = oracle.triple3d_bruteforce(Xt, common, q, tau, uvw)
    Ff = np.fft.fft(f)
    na = len(tau) - 1
    S1 = np.zeros((na, na, na), np.complex128)
    T1 = np.zeros((na, na, na), np.int64)
    for t1 in range(-t_max, t_max + 1):
        for t2 in range(-t_max, t_max + 1):
            t3 = -(t1 + t2)
            if abs(t3) > t_max:
                continue
            b = [oracle.delay_bin(t, tau) for t in (t1, t2, t3)]
            if min(b) < 0:
                continue
            S1[b[0], b[1], b[2]] += Ff[t1 % n_chan] * Ff[t2 % n_chan] * Ff[t3 % n_chan]
            T1[b[0], b[1], b[2]] += 1
    rings = np.sort(uvw // na, axis=1)
    S2, A2, T2 = oracle.triple_bruteforce(x, F[0], q, rings)
    d = uvw % na
    want_S = S2 * S1[d[:, 0], d[:, 1], d[:, 2]]
    want_T = T2 * T1[d[:, 0], d[:, 1], d[:, 2]]
    assert np.array_equal(T3, want_T)
    scale = np.maximum(A3, 1e-300)
    assert np.max(np.abs(S3 - want_S) / scale) < 1e-12
    # teeth: dropping the closure in t (every delay triple of the bins) gives other sums
    S1o = np.zeros((na, na, na), np.complex128)
    for t1 in range(-t_max, t_max + 1):
        for t2 in range(-t_max, t_max + 1):
            for t3 in range(-t_max, t_max + 1):
                b = [oracle.delay_bin(t, tau) for t in (t1, t2, t3)]
                if min(b) >= 0:
                    S1o[b[0], b[1], b[2]] += Ff[t1 % n_chan] * Ff[t2 % n_chan] * Ff[t3 % n_chan]
    wrong = S2 * S1o[d[:, 0], d[:, 1], d[:, 2]]
    assert np.max(np.abs(S3 - wrong) / scale) > 1e-3


def test_channel_shift_and_reversal_leave_B_unchanged():
    """A cyclic shift of the channels multiplies Xt(g, t) by exp(2 pi i s t / n_chan) and a
    reversal maps t to -t with a phase; both phases cancel on t1 + t2 + t3 = 0."""
    ci, X, F, q = _tiny(n_rings=5)
    tau = [int(v) for v in ci.tau]
    t_max = tau[-1] - 1
    uvw = oracle.triplets_3d(q, tau)

    def est(Xc, Fc):
        Xt, common = oracle.delay_modes(Xc, Fc, t_max)
        S, A, T = oracle.triple3d_bruteforce(Xt, common, q, tau, uvw)
        return _B(S, T), T, A

    B0, T0, A0 = est(X, F)
    ok = np.isfinite(B0) & (np.abs(B0) >= 1e-3 * np.nanmax(np.abs(B0)))
    for Xc, Fc in ((np.roll(X, 3, axis=0), np.roll(F, 3, axis=0)), (X[::-1].copy(), F[::-1].copy())):
        B1, T1, _ = est(Xc, Fc)
        assert np.array_equal(T0, T1)
        assert np.max(np.abs(B1[ok] - B0[ok]) / np.abs(B0[ok])) < 1e-9
    # teeth: swapping two channels is not a symmetry
    Xs = X.copy()
    Xs[[0, 2]] = Xs[[2, 0]]
    B2, _, _ = est(Xs, F)
    assert np.max(np.abs(B2[ok] - B0[ok]) / np.abs(B0[ok])) > 1e-3


def test_cube_sums_are_real():
    ci, X, F, q = _tiny()
    tau = [int(v) for v in ci.tau]
    Xt, common = oracle.delay_modes(X, F, tau[-1] - 1)
    uvw = oracle.triplets_3d(q, tau)
    S, A, T = oracle.triple3d_bruteforce(Xt, common, q, tau, uvw)
    assert (T > 0).all()
    assert np.max(np.abs(S.imag) / A) < 1e-12


@pytest.mark.parametrize("t_max", [0, 1, 2, 5, 15])
def test_delay_counts_closed_forms(t_max):
    # one bin holding every |t| <= t_max: pairs (t1, t2) with |t1 + t2| <= t_max
    T = oracle.delay_counts([0, t_max + 1], t_max)
    assert T.shape == (1, 1, 1)
    assert T[0, 0, 0] == (2 * t_max + 1) ** 2 - t_max * (t_max + 1)
    if t_max >= 1:
        T2 = oracle.delay_counts([0, 1, t_max + 1], t_max)
        assert T2[0, 0, 0] == 1                 # (0, 0, 0)
        assert T2[0, 1, 1] == 2 * t_max         # (0, t, -t)
        assert T2[0, 0, 1] == 0                 # 0 + 0 + t = 0 has no t != 0
        assert T2.sum() == T[0, 0, 0]


def test_triplets_3d_cover_every_closing_triplet_and_counts_factorise():
    """On a fully filled grid: every bin triplet with a closed voxel triangle is listed,
    and the factorised counts (2-D count x delay count) equal the brute-force counts."""
    ci, X, F, q = _tiny(n_rings=4)
    n = X.shape[1]
    tau = [0, 1, 2, 4]
    t_max = 3
    full = np.ones((n, n), np.uint8)
    Xt = np.ones((2 * t_max + 1, n, n), np.complex128)
    na, nb = len(tau) - 1, len(q) - 1
    nb3 = na * nb
    allt = np.array([(u, v, w) for u in range(nb3) for v in range(u, nb3) for w in range(v, nb3)], np.int32)
    _, _, T = oracle.triple3d_bruteforce(Xt, full, q, tau, allt)
    listed = {tuple(r) for r in oracle.triplets_3d(q, tau).tolist()}
    closing = {tuple(r) for r, t in zip(allt.tolist(), T) if t > 0}
    assert closing <= listed
    assert len(closing) > 10
    uvw = np.array(sorted(listed), np.int32)
    _, _, Tb = oracle.triple3d_bruteforce(Xt, full, q, tau, uvw)
    assert np.array_equal(oracle.counts_3d(full, q, tau, uvw), Tb)


def test_fft_form_3d_matches_bruteforce_and_aliases_when_delays_wrap():
    ci, X, F, q = _tiny(n_rings=5)
    tau = [int(v) for v in ci.tau]
    t_max = tau[-1] - 1
    Xt, common = oracle.delay_modes(X, F, t_max)
    uvw = oracle.triplets_3d(q, tau)
    S, A, _ = oracle.triple3d_bruteforce(Xt, common, q, tau, uvw)
    N = oracle.min_fft_size(q, X.shape[1])
    Sf, D = oracle.fft_form_3d(Xt, common, q, tau, uvw, N, 3 * t_max + 1)
    assert np.max(np.abs(Sf - S.real) / A) < 1e-12
    _, im = oracle.cube_fields(Xt, common, q, tau, N, 3 * t_max + 1)
    assert im < 1e-9 * np.abs(D).max()
    # at N_z = 2 t_max + 1 delay triples with t1 + t2 + t3 = +-N_z, such as (3, 3, 1), wrap
    # onto listed bin triplets
    Sa, _ = oracle.fft_form_3d(Xt, common, q, tau, uvw, N, 2 * t_max + 1)
    assert np.max(np.abs(Sa - S.real) / A) > 1e-6


def _cube_closed_form(P, q, tau, uvw, f, V):
    """First order in f of the quadratic cube's bispectrum (Wick's theorem as in App. B, with sums for
    integrals, in three dimensions): E[Xt1 Xt2 Xt3] = 2 f V (P1 P2 + P2 P3 + P3 P1) per voxel triangle
    closed in g and t, with <|Xt(g, t)|^2> = V P(g, t), averaged over the closed triangles of each bin
    triplet."""
    M, _, n_chan = P.shape
    half = M // 2 - 1
    t_max = tau[-1] - 1
    na = len(tau) - 1
    vox = []
    for gy in range(-half, half + 1):
        for gx in range(-half, half + 1):
            r2 = gx * gx + gy * gy
            if r2 < q[0] or r2 >= q[-1]:
                continue
            m = int(np.searchsorted(q, r2, side="right") - 1)
            for t in range(-t_max, t_max + 1):
                a = oracle.delay_bin(t, tau)
                if a >= 0:
                    vox.append((gx, gy, t, m * na + a))
    vox = np.array(vox)
    key = {(int(v[0]), int(v[1]), int(v[2])): int(v[3]) for v in vox}
    Pv = np.array([P[v[1] % M, v[0] % M, v[2] % n_chan] for v in vox])
    nb3 = (len(q) - 1) * na
    acc = np.zeros((nb3, nb3, nb3))
    cnt = np.zeros((nb3, nb3, nb3))
    for a in range(len(vox)):
        third = -(vox[a, :3] + vox[:, :3])
        u3 = np.array([key.get((int(x), int(y), int(z)), -1) for x, y, z in third])
        sel = u3 >= 0
        P3 = np.array([P[y % M, x % M, z % n_chan] for x, y, z in third[sel]])
        val = Pv[a] * Pv[sel] + Pv[sel] * P3 + P3 * Pv[a]
        np.add.at(acc, (vox[a, 3], vox[sel, 3], u3[sel]), val)
        np.add.at(cnt, (vox[a, 3], vox[sel, 3], u3[sel]), 1)
    out = np.array([acc[u, v, w] / cnt[u, v, w] if cnt[u, v, w] else np.nan for u, v, w in uvw])
    return 2.0 * f * V * out


@pytest.mark.slow
def test_gaussian_cube_has_zero_mean_and_quadratic_cube_matches_closed_form():
    """Grid-direct cubes (each channel's map modes taken as its gridded data, every cell filled): a
    Gaussian cube gives B = 0 within sampling error, and the quadratic cube g + f (g^2 - 1) at f = 0.05
    gives the three-dimensional analogue of the discrete Eq. bsana."""
    M, n_chan = 16, 8
    q = oracle.ring_q(2 * np.pi * np.array([1.5, 3.0, 4.5, 6.5]), 1.0)
    tau = [0, 1, 2, 4]
    uvw = oracle.triplets_3d(q, tau)
    P = synth.cube_power_model(M, n_chan)
    filled = np.ones((n_chan, M, M), np.uint8)
    filled[:, M // 2, :] = 0   # the row and column at index M/2 are off the grid
    filled[:, :, M // 2] = 0
    R = 1200
    rng = np.random.default_rng(2025)
    res = {}
    for f in (0.0, 0.05):
        Bs = []
        for _ in range(R):
            cube = synth.quadratic_sky(synth.gaussian_cube(M, n_chan, rng), f)
            X = np.stack([synth.sky_modes(np.ascontiguousarray(cube[:, :, c])) for c in range(n_chan)])
            Xt, common = oracle.delay_modes(X, filled, tau[-1] - 1)
            S, _, T = oracle.triple3d_bruteforce(Xt, common, q, tau, uvw)
            Bs.append(oracle.normalise(S, T))
        Bs = np.array(Bs)
        res[f] = (Bs.mean(0), Bs.std(0, ddof=1) / np.sqrt(R))
    mean0, se0 = res[0.0]
    assert np.all(np.abs(mean0 / se0) < 5.0)
    expect = _cube_closed_form(P, q, tau, uvw, 0.05, M * M * n_chan)
    mean1, se1 = res[0.05]
    assert np.all(np.abs((mean1 - expect) / se1) < 5.0)
    # teeth: the signal is detected, and a halved or doubled prediction is rejected
    assert np.max(np.abs(mean1 / se1)) > 10.0
    assert np.max(np.abs((mean1 - 0.5 * expect) / se1)) > 5.0
    assert np.max(np.abs((mean1 - 2.0 * expect) / se1)) > 5.0

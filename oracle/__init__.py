"""FP64 oracle for the visibility-based binned angular bispectrum (Sec. 2).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users.  The product path never
imports this package, and this package never imports the product.

The heavy loops (gridding, brute-force triple sums) are plain C in
``abs_oracle.c``; this module loads it with ctypes and adds the numpy glue.
``fft_form`` is a second, independent route to the same sums through numpy's
FFT (the identity the fast estimator of Sec. 2 relies on); the tests check
the two against each other and against closed forms.

Parity status per function (what pins it, see ``tests/test_oracle_*.py``):

* cell / ring thresholds / triplets: explicit worked cases, integer brute force
* grid: single-visibility closed forms, Hermitian mirror, NGP exact sums
* fft_form / fft_form_all: against brute force on tiny grids (sums to rounding,
  counts exact), at two admissible sky-grid sizes, aliasing below 3R+1
* triple_bruteforce / triple_one: pure-Python enumeration on tiny grids,
  FFT identity, constant-sky B = s^3, point-source phase closure,
  ring-constant product, rotation/reflection invariance, permutation
  symmetry of counts, Gaussian-sky zero mean, quadratic-sky closed form
  (discrete Eq. bsana), zero mean under pure gridded visibility noise
* ellbar: direct closed form on a hand-built mask
* normalise: closed forms above
* bana_d (discretely sampled prediction): constant C, a pure-Python
  enumeration on a tiny grid, symmetry in the three rings
* sky_weights / simulate_vis (visibility simulator): single-pixel closed
  forms, Hermitian symmetry of a real sky, the MWA tile beam's printed FWHM
* shape_params / rebin (results layer): hand-worked triangle shapes
  (equilateral, squeezed, folded), the bin edges, count-weighted means of a
  constant and of a linear B, and the ensemble mean / spread of +-B
* cube_means / delay_modes / triple3d_bruteforce (multi-frequency form):
  one channel reduces to the 2-D brute force; a separable cube x(g) f(c)
  factorises into the 2-D sums times the delay sums of numpy's FFT of f;
  cyclic shifts and reversal of the channel order leave B unchanged;
  Im S vanishes; a Gaussian cube gives B = 0 and the quadratic cube the
  three-dimensional analogue of the discrete Eq. bsana (teeth at 1/2x, 2x)
* delay_counts / triplets_3d: closed form of the one-bin delay count,
  against the brute-force 3-D counts on a fully filled tiny grid
* fft_form_3d: against the 3-D brute force (sums to rounding), aliasing
  below N_z = 3 t_max + 1
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "abs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle in place (gcc, FP contraction off, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    i32, i64, f32, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
    lib.orc_cell.argtypes = [f32, f32]
    lib.orc_cell.restype = i32
    lib.orc_ring_q.argtypes = [i32, P, f32, P]
    lib.orc_ring_q.restype = None
    lib.orc_triplets.argtypes = [i32, P, i32, P]
    lib.orc_triplets.restype = i32
    lib.orc_grid.argtypes = [i32, f32, i32, f64, i32, i64, P, P, P, P, P, P]
    lib.orc_grid.restype = ctypes.c_int
    lib.orc_mean_grid.argtypes = [i32, P, P, P, P, P]
    lib.orc_mean_grid.restype = None
    lib.orc_triple_bruteforce.argtypes = [i32, P, P, i32, P, i32, P, P, P, P]
    lib.orc_triple_bruteforce.restype = ctypes.c_int
    lib.orc_bana_bruteforce.argtypes = [i32, P, P, i32, P, i32, P, P, P]
    lib.orc_bana_bruteforce.restype = ctypes.c_int
    lib.orc_triple_one.argtypes = [i32, P, P, i32, P, i32, i32, i32, P, P, P]
    lib.orc_triple_one.restype = ctypes.c_int
    lib.orc_ellbar.argtypes = [i32, f32, P, i32, P, P]
    lib.orc_ellbar.restype = None
    lib.orc_normalise.argtypes = [i32, P, P, f64, P]
    lib.orc_normalise.restype = None
    lib.orc_delay_modes.argtypes = [i32, i32, P, P, i32, P, P]
    lib.orc_delay_modes.restype = ctypes.c_int
    lib.orc_triple3d_bruteforce.argtypes = [i32, i32, P, P, i32, P, i32, P, i32, P, P, P, P]
    lib.orc_triple3d_bruteforce.restype = ctypes.c_int
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------ small pieces


def cell(u: float, du: float) -> int:
    """Nearest grid index of one coordinate, binary32 rule floor(fl(fl(u/dU)+0.5))."""
    return int(_load().orc_cell(float(np.float32(u)), float(np.float32(du))))


def ring_q(ell_edges, du: float) -> np.ndarray:
    e = np.ascontiguousarray(ell_edges, np.float64)
    q = np.zeros(len(e), np.int64)
    _load().orc_ring_q(len(e) - 1, _p(e), float(np.float32(du)), _p(q))
    return q


def triplets(q: np.ndarray) -> np.ndarray:
    q = np.ascontiguousarray(q, np.int64)
    nb = len(q) - 1
    n = _load().orc_triplets(nb, _p(q), 0, None)
    out = np.zeros((max(n, 1), 3), np.int32)
    _load().orc_triplets(nb, _p(q), n, _p(out))
    return out[:n]


# ------------------------------------------------------------------ gridding


@dataclass
class Grid:
    grid: np.ndarray      # complex128 [n, n] (FFT order), Eq. vg sums incl. mirror
    wsum: np.ndarray      # float64 [n, n]: sum of the weights
    ncontrib: np.ndarray  # int64 [n, n]: N_g, the visibilities entered at the cell (Eq. vg)
    wsum2: np.ndarray = None   # float64 [n, n]: sum of the squared weights

    @property
    def n(self):
        return self.grid.shape[0]


def grid(n: int, du: float, uv: np.ndarray, vis: np.ndarray, kernel: str = "gauss",
         sigma_cells: float = 1.0, radius_cells: int = 3) -> Grid:
    uv = np.ascontiguousarray(uv, np.float32)
    v2 = np.ascontiguousarray(np.asarray(vis, np.complex64)).view(np.float32)
    g = np.zeros((n, n, 2), np.float64)
    w = np.zeros((n, n), np.float64)
    w2 = np.zeros((n, n), np.float64)
    c = np.zeros((n, n), np.int64)
    rc = _load().orc_grid(n, float(np.float32(du)), 0 if kernel == "ngp" else 1, float(sigma_cells),
                          int(radius_cells), len(uv), _p(uv), _p(v2), _p(g), _p(w), _p(w2), _p(c))
    if rc != 0:
        raise ValueError(f"orc_grid rejected its arguments (code {rc})")
    return Grid(g[..., 0] + 1j * g[..., 1], w, c, w2)


def mean_grid(gr: Grid):
    """X_g = V_g / sum w on filled cells (complex128 [n,n]) and the filled mask (uint8)."""
    n = gr.n
    g2 = np.ascontiguousarray(np.stack([gr.grid.real, gr.grid.imag], -1))
    X = np.zeros((n, n, 2), np.float64)
    f = np.zeros((n, n), np.uint8)
    _load().orc_mean_grid(n, _p(g2), _p(np.ascontiguousarray(gr.wsum)),
                          _p(np.ascontiguousarray(gr.ncontrib)), _p(X), _p(f))
    return X[..., 0] + 1j * X[..., 1], f


# ------------------------------------------------------------------ triple sums


def _x2(X):
    return np.ascontiguousarray(np.stack([np.real(X), np.imag(X)], -1).astype(np.float64))


def triple_bruteforce(X: np.ndarray, filled: np.ndarray, q: np.ndarray, ijk: np.ndarray):
    """(S complex128 [t], |.|-sum float64 [t], T int64 [t]) over all closed grid triangles."""
    n = X.shape[0]
    ijk = np.ascontiguousarray(ijk, np.int32).reshape(-1, 3)
    nt = len(ijk)
    S = np.zeros((max(nt, 1), 2))
    A = np.zeros(max(nt, 1))
    T = np.zeros(max(nt, 1), np.int64)
    rc = _load().orc_triple_bruteforce(n, _p(_x2(X)), _p(np.ascontiguousarray(filled, np.uint8)),
                                       len(q) - 1, _p(np.ascontiguousarray(q, np.int64)), nt,
                                       _p(ijk), _p(S), _p(A), _p(T))
    if rc != 0:
        raise MemoryError("orc_triple_bruteforce: allocation failed")
    return (S[:nt, 0] + 1j * S[:nt, 1]), A[:nt], T[:nt]


def triple_one(X, filled, q, i, j, k):
    n = X.shape[0]
    S = np.zeros(2)
    A = np.zeros(1)
    T = np.zeros(1, np.int64)
    _load().orc_triple_one(n, _p(_x2(X)), _p(np.ascontiguousarray(filled, np.uint8)), len(q) - 1,
                           _p(np.ascontiguousarray(q, np.int64)), int(i), int(j), int(k),
                           _p(S), _p(A), _p(T))
    return complex(S[0], S[1]), float(A[0]), int(T[0])


def ellbar(filled: np.ndarray, q: np.ndarray, du: float) -> np.ndarray:
    n = filled.shape[0]
    out = np.zeros(len(q) - 1)
    _load().orc_ellbar(n, float(np.float32(du)), _p(np.ascontiguousarray(filled, np.uint8)),
                       len(q) - 1, _p(np.ascontiguousarray(q, np.int64)), _p(out))
    return out


def normalise(S: np.ndarray, T: np.ndarray, norm_A: float = 1.0) -> np.ndarray:
    S = np.asarray(S)
    nt = len(S)
    s2 = np.ascontiguousarray(np.stack([S.real, S.imag], -1).reshape(-1, 2), np.float64)
    B = np.zeros(max(nt, 1))
    _load().orc_normalise(nt, _p(s2), _p(np.ascontiguousarray(T, np.int64)), float(norm_A), _p(B))
    return B[:nt]


# ------------------------------------------------------------------ FFT form


def _fft2(Z):
    """Unnormalised forward 2-D DFT (numpy's convention), on every host core when scipy is there."""
    try:
        import scipy.fft
        return scipy.fft.fft2(Z, workers=os.cpu_count() or 1)
    except ImportError:
        return np.fft.fft2(Z)


def ring_fields(X: np.ndarray, filled: np.ndarray, q: np.ndarray, N: int, unit: bool = False):
    """Real fields D_m(p) = sum_{g in a_m} X_g exp(-2 pi i g.p / N) (Eq. iFT) on an N x N
    sky grid, via numpy's FFT; with unit=True the unit-mask fields (X = 1 on filled
    ring cells).  Returns float64 [n_bins, N, N] (imaginary parts dropped) and the
    largest |imaginary part| seen."""
    n = filled.shape[0]
    half = n // 2 - 1
    gy, gx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    gy = np.where(gy > n // 2, gy - n, gy)
    gx = np.where(gx > n // 2, gx - n, gx)
    r2 = gx.astype(np.int64) ** 2 + gy.astype(np.int64) ** 2
    inside = (np.abs(gx) <= half) & (np.abs(gy) <= half) & (filled > 0) & (r2 >= q[0]) & (r2 < q[-1])
    # the filled cells of every ring, ring by ring (ring m: Q_m <= |g|^2 < Q_{m+1})
    cells = np.nonzero(inside.ravel())[0]
    ring = np.searchsorted(np.asarray(q), r2.ravel()[cells], side="right") - 1
    order = np.argsort(ring, kind="stable")
    cells, ring = cells[order], ring[order]
    nb = len(q) - 1
    start = np.searchsorted(ring, np.arange(nb + 1))
    D = np.zeros((nb, N, N))
    im = 0.0
    for m in range(nb):
        c = cells[start[m]:start[m + 1]]
        Z = np.zeros((N, N), np.complex128)
        vals = np.ones(len(c)) if unit else X.ravel()[c]
        np.add.at(Z, (gy.ravel()[c] % N, gx.ravel()[c] % N), vals)
        F = _fft2(Z)
        im = max(im, float(np.abs(F.imag).max()) if F.size else 0.0)
        D[m] = F.real
    return D, im


def fft_form(X, filled, q, ijk, N: int):
    """S_ijk = N^-2 sum_p D_i D_j D_k and T_ijk = N^-2 sum_p I_i I_j I_k (rounded), Eq. estimator_t."""
    D, _ = ring_fields(X, filled, q, N)
    I, _ = ring_fields(X, filled, q, N, unit=True)
    S = np.array([np.sum(D[i] * D[j] * D[k]) for i, j, k in ijk]) / (N * N)
    T = np.array([np.sum(I[i] * I[j] * I[k]) for i, j, k in ijk]) / (N * N)
    return S, np.rint(T).astype(np.int64), T


def fft_form_all(X, filled, q, ijk, N: int, fields=None, block: int = 65536):
    """fft_form for a whole triplet list at large sizes (Eq. estimator_t).

    The same sums, S_ijk = N^-2 sum_p D_i D_j D_k and T_ijk = N^-2 sum_p I_i I_j I_k,
    with the sum over pixels taken by matrix products: for every middle ring j, the
    fields D_i(p) of the rings i that pair with j, one row per i, times the products
    (D_j D_k)(p) of its rings k, one column per k; entry (i, k) is the sum for (i, j, k).
    The pixels are taken `block` at a time (the products for every block added up),
    which only bounds the memory.  fields: optional (D, I) from ring_fields, to reuse.
    Returns (S, T rounded, T before rounding, D, I)."""
    ijk = np.asarray(ijk, np.int64).reshape(-1, 3)
    if fields is None:
        D, _ = ring_fields(X, filled, q, N)
        I, _ = ring_fields(X, filled, q, N, unit=True)
    else:
        D, I = fields
    nb = D.shape[0]
    Df, If = D.reshape(nb, -1), I.reshape(nb, -1)
    P = Df.shape[1]
    js = np.unique(ijk[:, 1])
    span = {}
    for j in js:
        sel = np.nonzero(ijk[:, 1] == j)[0]
        span[j] = (sel, int(ijk[sel, 0].min()), int(ijk[sel, 0].max()) + 1, int(ijk[sel, 2].min()),
                   int(ijk[sel, 2].max()) + 1)
    MS = {j: np.zeros((span[j][2] - span[j][1], span[j][4] - span[j][3])) for j in js}
    MT = {j: np.zeros_like(MS[j]) for j in js}
    for p0 in range(0, P, block):
        Db, Ib = Df[:, p0:p0 + block], If[:, p0:p0 + block]
        for j in js:
            _, i0, i1, k0, k1 = span[j]
            MS[j] += Db[i0:i1] @ (Db[k0:k1] * Db[j]).T
            MT[j] += Ib[i0:i1] @ (Ib[k0:k1] * Ib[j]).T
    S = np.zeros(len(ijk))
    T = np.zeros(len(ijk))
    for j in js:
        sel, i0, _, k0, _ = span[j]
        S[sel] = MS[j][ijk[sel, 0] - i0, ijk[sel, 2] - k0]
        T[sel] = MT[j][ijk[sel, 0] - i0, ijk[sel, 2] - k0]
    S /= N * N
    T /= N * N
    return S, np.rint(T).astype(np.int64), T, D, I


def min_fft_size(q: np.ndarray, n: int | None = None) -> int:
    """Smallest 2^a 3^b 5^c >= max(3 R + 1, 8), R the largest |g_x| of any ring cell
    on an n x n grid (|g_x|, |g_y| <= n/2 - 1), found by scanning the cells."""
    half = (n // 2 - 1) if n else int(np.sqrt(float(q[-1]))) + 1
    k = np.arange(-half, half + 1)
    gx, gy = np.meshgrid(k, k)
    r2 = gx.astype(np.int64) ** 2 + gy.astype(np.int64) ** 2
    inring = (r2 >= q[0]) & (r2 < q[-1])
    R = int(np.abs(gx[inring]).max()) if inring.any() else 0
    N = max(3 * R + 1, 8)
    while True:
        m = N
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        if m == 1:
            return N
        N += 1


# ------------------------------------------------------------------ whole estimate


@dataclass
class Estimate:
    B: np.ndarray         # float64 [t]
    S: np.ndarray         # complex128 [t]
    absum: np.ndarray     # float64 [t]
    T: np.ndarray         # int64 [t]
    ellbar: np.ndarray    # float64 [n_bins]
    ijk: np.ndarray       # int32 [t, 3]
    q: np.ndarray         # int64 [n_bins + 1]
    X: np.ndarray         # complex128 [n, n]
    filled: np.ndarray    # uint8 [n, n]
    grid: Grid


def literal_weights(gr: Grid, filled: np.ndarray) -> np.ndarray:
    """W_g = 1 / N_g on filled cells, 0 elsewhere, with N_g the number of visibilities
    entered at the cell (Eq. vg; Sec. 2 takes W_g = N_g^-1 on filled cells): the weights
    of the literal D and I fields (Eqs. iFT, iFT_I)."""
    W = np.zeros(gr.wsum.shape)
    W[filled > 0] = 1.0 / gr.ncontrib[filled > 0]
    return W


def noise_weights(gr: Grid, filled: np.ndarray) -> np.ndarray:
    """N_eff,g = (sum w)^2 / sum w^2 on filled cells, 0 elsewhere: the inverse noise
    variance of the weighted mean X_g = V_g / sum w when every visibility carries
    the same uncorrelated noise (Sec. 2), in units of one visibility's inverse
    variance.  The noise-optimised form weights X_g by it in the D fields and uses
    it as the I-field weight."""
    W = np.zeros(gr.wsum.shape)
    m = filled > 0
    W[m] = gr.wsum[m] ** 2 / gr.wsum2[m]
    return W


def normalise_literal(S: np.ndarray, SW: np.ndarray, norm_A: float = 1.0) -> np.ndarray:
    """B = Re S / (A S_W), NaN where S_W = 0 (Eq. estimator_t with the I fields of Eq. iFT_I)."""
    S, SW = np.asarray(S), np.asarray(SW, np.float64)
    B = np.full(len(S), np.nan)
    ok = SW != 0
    B[ok] = np.real(S[ok]) / (norm_A * SW[ok])
    return B


def estimate(n, du, ell_edges, uv, vis, kernel="gauss", sigma_cells=1.0, radius_cells=3,
             norm_A=1.0, ijk=None, weight_mode="unitmask") -> Estimate:
    """V -> B for one realisation: Eq. vg, ring membership, closed-triangle sums, Eq. estimator_t.

    weight_mode "unitmask": D fields of the weighted mean X_g, denominator A T with T
    the count of closed triangles (unit-mask I fields).  "literal": Eqs. iFT and
    iFT_I as printed with W_g = 1 / N_g, N_g the visibilities entered at the cell:
    D fields of W_g V_g, denominator A S_W with S_W the sum of W1 W2 W3 over the closed
    triangles.  "noise": D fields of N_eff X_g, denominator A S_W with W = N_eff
    (noise_weights).  S is always the numerator sum of the D-field values."""
    q = ring_q(ell_edges, du)
    if ijk is None:
        ijk = triplets(q)
    gr = grid(n, du, uv, vis, kernel, sigma_cells, radius_cells)
    X, f = mean_grid(gr)
    if weight_mode == "unitmask":
        S, A, T = triple_bruteforce(X, f, q, ijk)
        B = normalise(S, T, norm_A)
    elif weight_mode in ("literal", "noise"):
        W = literal_weights(gr, f) if weight_mode == "literal" else noise_weights(gr, f)
        Y = gr.grid * W if weight_mode == "literal" else X * W
        S, A, T = triple_bruteforce(Y, f, q, ijk)
        SW, _, _ = triple_bruteforce(W, f, q, ijk)
        B = normalise_literal(S, SW.real, norm_A)
    else:
        raise ValueError(f"unknown weight_mode {weight_mode!r}")
    return Estimate(B, S, A, T, ellbar(f, q, du), np.asarray(ijk, np.int32), q, X, f, gr)


# ------------------------------------------------------------------ paper constants


def beam_constants(theta_f_deg: float = 24.68):
    """theta_0 = 0.6 theta_F (Eq. A_G), dU_g = sqrt(ln 2)/(pi theta_0) and the
    decorrelation exp(-pi^2 theta_0^2 dU^2/3) at dU^2 = dU_g^2/2 (Sec. 3), and the
    normalisation A = pi theta_0^2 / 3 of Eq. estimator_t."""
    th0 = 0.6 * np.deg2rad(theta_f_deg)
    dug = np.sqrt(np.log(2.0)) / (np.pi * th0)
    decor = np.exp(-np.pi ** 2 * th0 ** 2 * (dug ** 2 / 2.0) / 3.0)
    A = np.pi * th0 ** 2 / 3.0
    return {"theta0": th0, "du_g": dug, "decorrelation": decor, "A": A}


# ------------------------------------------------------------------ results layer


def shape_params(ellbar: np.ndarray, ijk: np.ndarray):
    """The triangle shape of every ring triplet in the (l1, mu, t) form of Sec. 1.

    The paper orders l1 >= l2 >= l3, which for a canonical triplet (i <= j <= k,
    rings ascending in l) is (k, j, i); each side is its ring's mean l.  With
    l1 + l2 + l3 = 0 as vectors, mu = -l1.l2 / (l1 l2) = (l1^2 + l2^2 - l3^2) /
    (2 l1 l2) and t = l2 / l1, both evaluated left to right in FP64 without
    fused operations (the kernel takes the same decisions from the same values).
    """
    ijk = np.asarray(ijk).reshape(-1, 3)
    l3, l2, l1 = (np.asarray(ellbar, np.float64)[ijk[:, c]] for c in range(3))
    with np.errstate(invalid="ignore", divide="ignore"):
        mu = ((l1 * l1 + l2 * l2) - l3 * l3) / ((2.0 * l1) * l2)
        t = l2 / l1
    return l1, mu, t


def shape_cell(ijk: np.ndarray, mu: np.ndarray, t: np.ndarray, n_mu: int, n_t: int):
    """Cell (ring of l1, mu bin, t bin) of every triplet: n_mu x n_t equal bins over
    [0.5, 1] (the range of closed triangles with l1 >= l2 >= l3, Sec. 4); ring means
    can put a shape just outside it, which is clamped into the edge bins."""
    ijk = np.asarray(ijk).reshape(-1, 3)
    def b(x, n):
        v = np.floor((x - 0.5) * (2.0 * n))
        v = np.where(np.isfinite(v), v, 0)
        return np.clip(v, 0, n - 1).astype(np.int64)
    return (ijk[:, 2] * n_mu + b(mu, n_mu)) * n_t + b(t, n_t)


def rebin(B: np.ndarray, T: np.ndarray, ellbar: np.ndarray, ijk: np.ndarray, n_bins: int,
          n_mu: int = 5, n_t: int = 5):
    """Count-weighted (l1, mu, t) averages of B and their ensemble statistics (Sec. 4).

    Per realisation r, cell c: B_r(c) = sum T B_r / sum T over the cell's triplets
    with T > 0 and finite B (the triangle count is the weight, Sec. 4); then over
    the R realisations the mean and the spread sigma^2 = <B_r(c)^2> - <B_r(c)>^2.
    Returns (mean, sigma, weight = sum T) as [n_bins][n_mu][n_t]; cells without
    triangles are NaN (weight 0).
    """
    B = np.atleast_2d(np.asarray(B, np.float64))
    T = np.asarray(T, np.int64)
    _, mu, t = shape_params(ellbar, ijk)
    cell = shape_cell(ijk, mu, t, n_mu, n_t)
    nc = n_bins * n_mu * n_t
    den = np.zeros(nc)
    num = np.zeros((B.shape[0], nc))
    for r in range(B.shape[0]):
        for q in range(len(T)):
            if T[q] > 0 and np.isfinite(B[r, q]):
                num[r, cell[q]] += float(T[q]) * B[r, q]
                if r == 0:
                    den[cell[q]] += float(T[q])
    with np.errstate(invalid="ignore", divide="ignore"):
        v = num / den
        mean = v.mean(axis=0)
        var = (v * v).mean(axis=0) - mean * mean
    sigma = np.sqrt(np.maximum(var, 0.0))
    sigma[den == 0] = np.nan
    shape = (n_bins, n_mu, n_t)
    return mean.reshape(shape), sigma.reshape(shape), den.reshape(shape)


def bana_d(C: np.ndarray, filled: np.ndarray, q: np.ndarray, ijk: np.ndarray, f_over_sigma: float):
    """[B_Ana]_d of Sec. 4 (Fig. 2): Eq. bsana's 2 (f_NG / sigma_T) (C1 C2 + C2 C3 + C3 C1)
    averaged over the closed triangles of filled cells in each ring triplet, with C the
    angular power spectrum at each cell's l (real [n][n], FFT order).  NaN where T = 0.
    Returns (bana_d, T)."""
    n = filled.shape[0]
    ijk = np.ascontiguousarray(np.asarray(ijk, np.int32).reshape(-1, 3))
    nt = len(ijk)
    S = np.zeros(max(nt, 1))
    T = np.zeros(max(nt, 1), np.int64)
    rc = _load().orc_bana_bruteforce(n, _p(np.ascontiguousarray(C, np.float64)),
                                     _p(np.ascontiguousarray(filled, np.uint8)), len(q) - 1,
                                     _p(np.ascontiguousarray(q, np.int64)), nt, _p(ijk), _p(S), _p(T))
    if rc != 0:
        raise MemoryError("oracle bana_d")
    S, T = S[:nt], T[:nt]
    with np.errstate(invalid="ignore", divide="ignore"):
        out = np.where(T > 0, 2.0 * f_over_sigma * S / T, np.nan)
    return out, T


# ------------------------------------------------------------------ visibility simulator


def sky_weights(sky: np.ndarray, dtheta: float, beam: str = "none", beam_param: float = 0.0) -> np.ndarray:
    """dtheta^2 A(theta) T(theta) on an m x m flat-sky grid (Sec. 3): pixel (row b, column a)
    at theta = ((a - m/2) dtheta, (b - m/2) dtheta).  beam "mwa": Eq. beam, sinc^2(pi (d/lambda)
    theta_x) sinc^2(pi (d/lambda) theta_y) with beam_param = d / lambda; "gauss": Eq. A_G,
    exp(-theta^2 / theta_0^2) with beam_param = theta_0 (radians); "none": A = 1."""
    m = sky.shape[0]
    th = (np.arange(m) - m // 2) * float(dtheta)
    tx, ty = th[None, :], th[:, None]
    if beam == "mwa":
        A = np.sinc(beam_param * tx) ** 2 * np.sinc(beam_param * ty) ** 2   # np.sinc(x) = sin(pi x)/(pi x)
    elif beam == "gauss":
        A = np.exp(-(tx * tx + ty * ty) / (beam_param * beam_param))
    else:
        A = np.ones((m, m))
    return float(dtheta) ** 2 * A * np.asarray(sky, np.float64)


def simulate_vis(sky: np.ndarray, dtheta: float, uv: np.ndarray, beam: str = "none",
                 beam_param: float = 0.0) -> np.ndarray:
    """Eq. vis with Q = 1 (map units): V(U) = sum over pixels of dtheta^2 A T exp(+i 2 pi U.theta),
    the direct DFT of Sec. 3, in FP64.  Returns complex128 [n_vis]."""
    W = sky_weights(sky, dtheta, beam, beam_param)
    m = W.shape[0]
    th = (np.arange(m) - m // 2) * float(dtheta)
    uv = np.asarray(uv, np.float64)
    out = np.zeros(len(uv), np.complex128)
    for s0 in range(0, len(uv), 256):
        u = uv[s0:s0 + 256, 0][:, None, None]
        v = uv[s0:s0 + 256, 1][:, None, None]
        ph = np.exp(2j * np.pi * (u * th[None, None, :] + v * th[None, :, None]))
        out[s0:s0 + 256] = (ph * W[None]).sum(axis=(1, 2))
    return out



# ------------------------------------------------------------------ multi-frequency (3-D) form
#
# A reading of the generalisation that Sec. 1 and Sec. 5 name as future work:
# the channels are gridded one by one on the same uv grid, the cells filled in
# every channel are transformed along frequency (delay modes t), and the voxels
# (g, t) are binned by ring and by |t|; a bin triplet sums over the voxel
# triangles that close in both g and t.  See abs_oracle.c for the definitions.


def cube_means(n: int, du: float, uvs, viss, kernel: str = "gauss", sigma_cells: float = 1.0,
               radius_cells: int = 3, threads: int | None = None):
    """Per-channel gridding (Eq. vg) and means: X complex128 [n_chan, n, n], filled uint8.
    The channels are independent; they are gridded on host threads (the C loops run
    outside the interpreter lock)."""
    from concurrent.futures import ThreadPoolExecutor

    def one(c):
        return mean_grid(grid(n, du, uvs[c], viss[c], kernel, sigma_cells, radius_cells))

    with ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 1) as ex:
        out = list(ex.map(one, range(len(uvs))))
    return np.stack([o[0] for o in out]), np.stack([o[1] for o in out])


def delay_modes(X: np.ndarray, filled: np.ndarray, t_max: int):
    """Delay modes Xt[t + t_max] = sum_c X_c exp(-2 pi i c t / n_chan) on the cells filled in
    every channel (0 elsewhere), |t| <= t_max, and that common mask."""
    n_chan, n = X.shape[0], X.shape[1]
    Xt = np.zeros((2 * t_max + 1, n, n, 2))
    common = np.zeros((n, n), np.uint8)
    rc = _load().orc_delay_modes(n, n_chan, _p(_x2(X)), _p(np.ascontiguousarray(filled, np.uint8)),
                                 int(t_max), _p(Xt), _p(common))
    if rc != 0:
        raise ValueError("delay_modes needs 0 <= 2 t_max < n_chan")
    return Xt[..., 0] + 1j * Xt[..., 1], common


def delay_bin(t: int, tau) -> int:
    """Delay bin a of a delay index t: tau_a <= |t| < tau_{a+1}, or -1."""
    for a in range(len(tau) - 1):
        if tau[a] <= abs(t) < tau[a + 1]:
            return a
    return -1


def delay_counts(tau, t_max: int) -> np.ndarray:
    """T1[a][b][c] = number of ordered (t1, t2, t3), |t| <= t_max, t1 + t2 + t3 = 0, with
    t1, t2, t3 in the delay bins a, b, c (pure-Python enumeration)."""
    na = len(tau) - 1
    T1 = np.zeros((na, na, na), np.int64)
    for t1 in range(-t_max, t_max + 1):
        for t2 in range(-t_max, t_max + 1):
            t3 = -(t1 + t2)
            if abs(t3) > t_max:
                continue
            a, b, c = delay_bin(t1, tau), delay_bin(t2, tau), delay_bin(t3, tau)
            if min(a, b, c) >= 0:
                T1[a, b, c] += 1
    return T1


def triplets_3d(q: np.ndarray, tau) -> np.ndarray:
    """Canonical bin triplets u <= v <= w (u = m n_dbins + a) of the 3-D form: the rings
    (sorted) close a triangle in the 2-D test of `triplets`, and the delay bins close one
    (their delay count is > 0)."""
    na = len(tau) - 1
    T1 = delay_counts(tau, int(tau[-1]) - 1)
    ring_ok = {tuple(r) for r in np.asarray(triplets(q)).reshape(-1, 3).tolist()}
    nb3 = (len(q) - 1) * na
    out = []
    for u in range(nb3):
        for v in range(u, nb3):
            for w in range(v, nb3):
                if tuple(sorted((u // na, v // na, w // na))) in ring_ok and T1[u % na, v % na, w % na] > 0:
                    out.append((u, v, w))
    return np.asarray(out, np.int32).reshape(-1, 3)


def triple3d_bruteforce(Xt: np.ndarray, common: np.ndarray, q: np.ndarray, tau, uvw: np.ndarray):
    """(S complex128 [t], |.|-sum float64 [t], T int64 [t]) over all closed voxel triangles."""
    t_max = (Xt.shape[0] - 1) // 2
    n = Xt.shape[1]
    uvw = np.ascontiguousarray(uvw, np.int32).reshape(-1, 3)
    nt = len(uvw)
    S = np.zeros((max(nt, 1), 2))
    A = np.zeros(max(nt, 1))
    T = np.zeros(max(nt, 1), np.int64)
    tau = np.ascontiguousarray(tau, np.int32)
    xt2 = np.ascontiguousarray(np.stack([Xt.real, Xt.imag], -1))
    rc = _load().orc_triple3d_bruteforce(n, int(t_max), _p(xt2), _p(np.ascontiguousarray(common, np.uint8)),
                                         len(q) - 1, _p(np.ascontiguousarray(q, np.int64)), len(tau) - 1,
                                         _p(tau), nt, _p(uvw), _p(S), _p(A), _p(T))
    if rc != 0:
        raise MemoryError("orc_triple3d_bruteforce: allocation failed")
    return (S[:nt, 0] + 1j * S[:nt, 1]), A[:nt], T[:nt]


def counts_3d(common: np.ndarray, q: np.ndarray, tau, uvw: np.ndarray) -> np.ndarray:
    """T_uvw = T2(rings of u, v, w) x T1(delay bins of u, v, w): the voxel triangles close
    in g and in t independently and the common mask does not depend on t, so the 3-D count
    is the 2-D count of `triple_bruteforce` on the common mask times `delay_counts`."""
    na = len(tau) - 1
    uvw = np.asarray(uvw, np.int64).reshape(-1, 3)
    rings = np.sort(uvw // na, axis=1)
    uniq, inv = np.unique(rings, axis=0, return_inverse=True)
    n = common.shape[0]
    _, _, T2 = triple_bruteforce(np.ones((n, n), np.complex128), common, q, uniq.astype(np.int32))
    T1 = delay_counts(tau, int(tau[-1]) - 1)
    d = uvw % na
    return T2[inv.ravel()] * T1[d[:, 0], d[:, 1], d[:, 2]]


def _fftn(Z):
    try:
        import scipy.fft
        return scipy.fft.fftn(Z, workers=os.cpu_count() or 1)
    except ImportError:
        return np.fft.fftn(Z)


def cube_fields(Xt: np.ndarray, common: np.ndarray, q: np.ndarray, tau, N: int, Nz: int):
    """Real 3-D fields D_u(z, p) = sum over the voxels (g, t) of bin u of
    Xt(g, t) exp(-2 pi i (t z / N_z + g.p / N)) by numpy's FFT, float64 [n_bins n_dbins,
    N_z, N, N] (imaginary parts dropped), and the largest |imaginary part| seen."""
    t_max = (Xt.shape[0] - 1) // 2
    n = common.shape[0]
    half = n // 2 - 1
    gy, gx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    gy = np.where(gy > n // 2, gy - n, gy)
    gx = np.where(gx > n // 2, gx - n, gx)
    r2 = gx.astype(np.int64) ** 2 + gy.astype(np.int64) ** 2
    na = len(tau) - 1
    nb = len(q) - 1
    D = np.zeros((nb * na, Nz, N, N))
    im = 0.0
    for m in range(nb):
        cells = np.nonzero(((np.abs(gx) <= half) & (np.abs(gy) <= half) & (common > 0)
                            & (r2 >= q[m]) & (r2 < q[m + 1])).ravel())[0]
        for a in range(na):
            Z = np.zeros((Nz, N, N), np.complex128)
            for t in range(-t_max, t_max + 1):
                if delay_bin(t, tau) != a:
                    continue
                Z[t % Nz, gy.ravel()[cells] % N, gx.ravel()[cells] % N] += Xt[t + t_max].ravel()[cells]
            F = _fftn(Z)
            im = max(im, float(np.abs(F.imag).max()))
            D[m * na + a] = F.real
    return D, im


def fft_form_3d(Xt, common, q, tau, uvw, N: int, Nz: int, fields=None, block: int = 65536):
    """S_uvw = (N^2 N_z)^-1 sum over voxels of D_u D_v D_w (the FFT route of Sec. 2 in three
    dimensions), the sum over voxels by matrix products as in `fft_form_all` (per middle
    bin v, rows u, columns w; voxels `block` at a time).  Returns (S, D)."""
    uvw = np.asarray(uvw, np.int64).reshape(-1, 3)
    D = cube_fields(Xt, common, q, tau, N, Nz)[0] if fields is None else fields
    nb3 = D.shape[0]
    Df = D.reshape(nb3, -1)
    P = Df.shape[1]
    vs = np.unique(uvw[:, 1])
    span = {}
    for v in vs:
        sel = np.nonzero(uvw[:, 1] == v)[0]
        span[v] = (sel, int(uvw[sel, 0].min()), int(uvw[sel, 0].max()) + 1, int(uvw[sel, 2].min()),
                   int(uvw[sel, 2].max()) + 1)
    MS = {v: np.zeros((span[v][2] - span[v][1], span[v][4] - span[v][3])) for v in vs}
    for p0 in range(0, P, block):
        Db = Df[:, p0:p0 + block]
        for v in vs:
            _, u0, u1, w0, w1 = span[v]
            MS[v] += Db[u0:u1] @ (Db[w0:w1] * Db[v]).T
    S = np.zeros(len(uvw))
    for v in vs:
        sel, u0, _, w0, _ = span[v]
        S[sel] = MS[v][uvw[sel, 0] - u0, uvw[sel, 2] - w0]
    return S / (float(N) * N * Nz), D

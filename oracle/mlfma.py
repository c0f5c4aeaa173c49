"""Plain CPU MLFMA in FP64 (numpy): the oracle for every stage of the GPU path.

TEST INFRASTRUCTURE (CPU oracle).  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import it; the product path never does.

What it computes, stage by stage, in the paper's order (Sec. 2, five stages;
Sec. 3.2.1-3.2.5): C2M, M2M (interpolate -> shift -> aggregate, Sec. 3.2.2),
M2L (Alg. 2: for each observer, sum the translated far-field sources,
Sec. 3.2.3), L2L (shift -> anterpolate -> add, Sec. 3.2.4), L2O (Sec. 3.2.5),
plus the near-field direct sums at the leaves (Sec. 2).  The paper omits the
mathematics (Sec. 2 defers it to its references), so the formulas below are the
standard diagonal plane-wave form derived from the Gegenbauer addition theorem
(expanding e^{ik|X+d|}/|X+d| over spherical Bessel and Hankel functions) and the
Funk-Hecke identity (replacing each j_n(k|d|) P_n by a quadrature of plane waves
over the unit sphere):

  e^{ik|X+d|}/|X+d| ~= (ik/4pi) sum_p w_p e^{ik khat_p.d} T_X(khat_p),
  T_X(khat) = sum_{n=0}^{L} i^n (2n+1) h_n(k|X|) P_n(khat.Xhat)

  C2M  F_b(p)  = sum_{j in b} q_j e^{-ik khat_p.(r_j - c_b)}
  M2M  F_P(p') = sum_c e^{-ik khat_p'.(c_c - c_P)} [I_{c->P} F_c](p')
  M2L  G_t(p)  = sum_{s in V(t)} T_{c_t - c_s}(p) F_s(p)
  L2L  G_c    += W_c^{-1} I^T W_P [e^{+ik khat.(c_c - c_P)} G_P]
  L2O  phi_i  += (ik/4pi) sum_p w_p e^{ik khat_p.(r_i - c_b)} G_b(p)

Readings where the paper is silent: kernel e^{+ikR}/R without 1/(4 pi), self term and
coincident points excluded; sampling grid = (L+1) Gauss-Legendre nodes in
cos(theta) (ascending) x nph uniform phi nodes (nph = smallest even 7-smooth number
>= 2L+2), sample p = i nph + j, weights w_p = w_i^GL 2pi/nph; global interpolation by spherical-harmonic
projection per Fourier mode (the 'global interpolation' the paper insists on,
Sec. 2 Related Work); truncation L = ceil(kD + 1.8 d0^(2/3) (kD)^(1/3)) with
D = sqrt(3) * edge, d0 = digits + DIGIT_MARGIN (excess-bandwidth rule, not
printed in the paper); M2L starts at the highest level with a non-empty V list.
Optional sampled translation operators (Sec. 3.2.3, "Translation Operators"): T tabulated in
the angle psi between khat and X and interpolated by P-point Lagrange weights
(sampled_translation_operator), at the levels with boxes of a wavelength or more.
"""
from __future__ import annotations

import math

import numpy as np

from . import special
from . import tree as tr

# d0 = digits + DIGIT_MARGIN in the truncation rule.  Calibrated once on the
# 4,096-point sphere (radius 2, 3 digits) so that the relative L2 error against the
# FP64 direct sum stays below 10^-digits, then frozen.
DIGIT_MARGIN = 1


def truncation_L(edge: float, k: float, digits: int, margin: int = DIGIT_MARGIN) -> int:
    kD = k * math.sqrt(3.0) * edge
    d0 = float(digits + margin)
    return int(math.ceil(kD + 1.8 * d0 ** (2.0 / 3.0) * kD ** (1.0 / 3.0)))


def smooth_even(m: int) -> int:
    """Smallest even number >= m whose prime factors are all in {2, 3, 5, 7}."""
    while True:
        t = m
        for r in (2, 3, 5, 7):
            while t % r == 0:
                t //= r
        if t == 1 and m % 2 == 0:
            return m
        m += 1


class Grid:
    """theta-phi sampling grid of one level.

    (L+1) Gauss-Legendre nodes in cos(theta) and nph uniform phi nodes, with nph the
    smallest even 7-smooth number >= 2L+2 (>= 2L+2 keeps the phi quadrature exact
    for the degree-2L products it integrates; the smooth size lets the GPU path use
    mixed-radix FFTs in phi).
    """

    def __init__(self, L: int):
        self.L = L
        self.nth = L + 1
        self.nph = smooth_even(2 * L + 2)
        self.K = self.nth * self.nph
        self.x, self.wgl = special.gauss_legendre(self.nth)
        self.phi = 2.0 * math.pi * np.arange(self.nph) / self.nph
        st = np.sqrt(1.0 - self.x * self.x)
        dirs = np.empty((self.nth, self.nph, 3))
        dirs[:, :, 0] = st[:, None] * np.cos(self.phi)[None, :]
        dirs[:, :, 1] = st[:, None] * np.sin(self.phi)[None, :]
        dirs[:, :, 2] = self.x[:, None]
        self.dirs = dirs.reshape(self.K, 3)
        self.w = np.repeat(self.wgl, self.nph) * (2.0 * math.pi / self.nph)


def translation_operator(grid: Grid, k: float, X: np.ndarray) -> np.ndarray:
    """T_X(khat_p) = sum_{n<=L} i^n (2n+1) h_n(k|X|) P_n(khat_p . Xhat), p over the grid."""
    X = np.asarray(X, dtype=np.float64)
    r = float(np.linalg.norm(X))
    L = grid.L
    h = special.spherical_hn_all(L, k * r)
    n = np.arange(L + 1)
    coef = (1j ** n) * (2 * n + 1) * h
    P = special.legendre_all(L, grid.dirs @ (X / r))        # [L+1, K]
    return coef @ P


# Sampled translation operators (Sec. 3.2.3, "Translation Operators": where the operators do
# not fit in memory they are sampled and interpolated).  T_X(khat) depends on khat only through
# the angle psi between khat and Xhat: T = sum_n i^n (2n+1) h_n(k|X|) P_n(cos psi).  Each
# P_n(cos psi) is a cosine polynomial of degree n, so T is an even, 2 pi-periodic trigonometric
# polynomial of degree L in psi.  Reading (the paper defers the technique to its reference):
# tabulate T at the equispaced angles psi_i = i pi / S, S = s L (s: oversampling over the
# Nyquist spacing pi / L), for i = -P .. S + P, and evaluate it at each sample's psi with the
# P-point Lagrange interpolant whose nodes straddle psi (P even, psi in the middle interval).
# The padded entries are T at cos(psi_i): by evenness and periodicity they are the reflections
# across psi = 0 and psi = pi.  Only levels whose boxes are at least one wavelength wide
# (k edge >= 2 pi) are sampled: their tables are the large ones, while at sub-wavelength boxes
# |T| grows far above the signatures it produces (low-frequency growth of h_n), which would
# magnify the interpolation error; those levels keep their exact operators.
SAMPLED_ORDER = 10


def level_is_sampled(k: float, edge: float, s: int) -> bool:
    """Sampled operators apply at levels with k edge >= 2 pi (relative slack 1e-9)."""
    return s > 0 and k * edge >= 2.0 * math.pi * (1.0 - 1e-9)


def lagrange_weights(t, P: int) -> np.ndarray:
    """l_j(t) = prod_{m != j} (t - m) / (j - m), j = 0..P-1: the P-point Lagrange basis on the
    nodes 0..P-1 evaluated at t (any shape); returns [P, *shape(t)]."""
    t = np.asarray(t, dtype=np.float64)
    w = np.ones((P,) + t.shape)
    for j in range(P):
        for m in range(P):
            if m != j:
                w[j] *= (t - m) / (j - m)
    return w


def operator_samples(L: int, k: float, r: float, s: int, P: int = SAMPLED_ORDER) -> np.ndarray:
    """T at psi_i = i pi / (s L), i = -P .. s L + P, for |X| = r: [s L + 2 P + 1] complex."""
    S = s * L
    h = special.spherical_hn_all(L, k * r)
    n = np.arange(L + 1)
    coef = (1j ** n) * (2 * n + 1) * h
    psi = np.arange(-P, S + P + 1) * (math.pi / S)
    return coef @ special.legendre_all(L, np.cos(psi))


def sampled_translation_operator(grid: Grid, k: float, X: np.ndarray, s: int, P: int = SAMPLED_ORDER) -> np.ndarray:
    """T_X(khat_p) interpolated from operator_samples at psi_p = angle(khat_p, Xhat)."""
    X = np.asarray(X, dtype=np.float64)
    r = float(np.linalg.norm(X))
    tab = operator_samples(grid.L, k, r, s, P)
    xh = X / r
    psi = np.arctan2(np.linalg.norm(np.cross(grid.dirs, xh), axis=1), grid.dirs @ xh)
    return interpolate_samples(tab, psi, s * grid.L, P)


def interpolate_samples(tab: np.ndarray, psi: np.ndarray, S: int, P: int = SAMPLED_ORDER) -> np.ndarray:
    """sum_j l_j(t) tab[psi_{i0 + j}]: nodes i0 .. i0 + P - 1, i0 = floor(psi / h) - P/2 + 1,
    t = psi / h - i0 (the middle interval), h = pi / S; tab[i + P] holds the value at psi_i."""
    u = np.asarray(psi, dtype=np.float64) / (math.pi / S)
    i0 = np.floor(u).astype(np.int64) - (P // 2 - 1)         # first node: psi_{i0}
    w = lagrange_weights(u - i0, P)
    out = np.zeros(u.shape, dtype=np.result_type(tab.dtype, np.float64))
    for j in range(P):
        out += w[j] * tab[i0 + j + P]
    return out


def theta_maps(gc: Grid, gp: Grid):
    """A_m[i', i] = sum_{n=|m|}^{L_c} Pbar_n^m(x'_i') Pbar_n^m(x_i) w_i, m = 0..L_c."""
    out = []
    for m in range(gc.L + 1):
        pc = special.assoc_legendre_normalized(gc.L, m, gc.x)   # [nn, nth_c]
        pp = special.assoc_legendre_normalized(gc.L, m, gp.x)   # [nn, nth_p]
        out.append(pp.T @ (pc * gc.wgl[None, :]))
    return out


def interpolate(Fc: np.ndarray, gc: Grid, gp: Grid, A) -> np.ndarray:
    """Global interpolation of child-grid samples to the parent grid.

    Fc: [..., K_c].  Forward DFT in phi (modes |m| <= L_c, the Nyquist mode is
    dropped), per-mode Legendre projection/evaluation A_|m|, inverse DFT in phi.
    """
    lead = Fc.shape[:-1]
    F = Fc.reshape(lead + (gc.nth, gc.nph))
    m = np.arange(-gc.L, gc.L + 1)
    Efwd = np.exp(-1j * np.outer(gc.phi, m)) / gc.nph          # [nph_c, 2Lc+1]
    Xm = F @ Efwd                                               # [..., nth_c, 2Lc+1]
    Y = np.empty(lead + (gp.nth, m.shape[0]), dtype=np.complex128)
    for mi, mm in enumerate(m):
        Y[..., :, mi] = Xm[..., :, mi] @ A[abs(mm)].T
    Einv = np.exp(1j * np.outer(m, gp.phi))                     # [2Lc+1, nph_p]
    return (Y @ Einv).reshape(lead + (gp.K,))


def anterpolate(Gp: np.ndarray, gc: Grid, gp: Grid, A) -> np.ndarray:
    """W_c^{-1} I^T W_p applied to parent-grid samples (bilinear weighted transpose).

    Factored form: (1/nph_p) sum_j' g e^{+i m phi'_j'}, then B_m = (A_m^T scaled by
    w'_i' / w_i), then sum_m e^{-i m phi_j}.  tests/test_oracle_mlfma.py pins it to
    the literal W_c^{-1} I^T W_p built from ``interpolate``.
    """
    lead = Gp.shape[:-1]
    G = Gp.reshape(lead + (gp.nth, gp.nph))
    m = np.arange(-gc.L, gc.L + 1)
    E1 = np.exp(1j * np.outer(gp.phi, m)) / gp.nph               # [nph_p, 2Lc+1]
    Gh = G @ E1                                                  # [..., nth_p, 2Lc+1]
    H = np.empty(lead + (gc.nth, m.shape[0]), dtype=np.complex128)
    for mi, mm in enumerate(m):
        B = A[abs(mm)].T * gp.wgl[None, :] / gc.wgl[:, None]     # [nth_c, nth_p]
        H[..., :, mi] = Gh[..., :, mi] @ B.T
    E3 = np.exp(-1j * np.outer(m, gc.phi))                       # [2Lc+1, nph_c]
    return (H @ E3).reshape(lead + (gc.K,))


def direct_pairs(tr_pos, src_pos, q, k, same_index=None):
    """sum_j q_j e^{ikR}/R over a block of pairs; R = 0 (self / coincident) is skipped."""
    d = tr_pos[:, None, :] - src_pos[None, :, :]
    R = np.sqrt(np.sum(d * d, axis=-1))
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.where(R > 0.0, np.exp(1j * k * R) / np.where(R > 0.0, R, 1.0), 0.0)
    return g @ q


class OracleMLFMA:
    """Plain FP64 MLFMA with per-stage dumps.  Level-uniform or adaptive tree."""

    def __init__(self, points, k: float, digits: int, leaf_max: int = 0, leaf_edge: float | None = None,
                 max_depth: int = 12, margin: int = DIGIT_MARGIN, sampled_operators: int = 0):
        # sampled_operators = s > 0: M2L of the levels with k edge >= 2 pi uses
        # sampled_translation_operator with oversampling s
        self.sampled = int(sampled_operators)
        self.k = float(k)
        self.digits = int(digits)
        self.points = np.asarray(points, dtype=np.float64)
        self.leaf_edge = 0.25 * 2.0 * math.pi / self.k if leaf_edge is None else float(leaf_edge)
        self.tree = tr.build_tree(self.points, self.leaf_edge, leaf_max, max_depth)
        t = self.tree
        self.coll = {l: tr.colleagues(t, l) for l in range(1, t.nlev + 1)}
        self.V = tr.v_lists(t, self.coll)
        # highest level with a non-empty V list starts the far field (Sec. 3.2.3)
        self.top = None
        for l in range(2, t.nlev + 1):
            if self.V[l][1].shape[0] > 0:
                self.top = l
                break
        self.uniform = leaf_max == 0
        if self.uniform:
            self.U = tr.uniform_u_lists(t, self.coll)
        else:
            U, W, X = tr.near_lists_general(t, self.coll)
            self.Ud, self.Wd, self.Xd = U, W, X
            self.near = tr.near_source_ranges(t, U, W, X)
        self.L = {}
        self.grid = {}
        if self.top is not None:
            for l in range(self.top, t.nlev + 1):
                self.L[l] = truncation_L(t.levels[l].edge, self.k, self.digits, margin)
                self.grid[l] = Grid(self.L[l])
        self.A = {}
        if self.top is not None:
            for l in range(self.top, t.nlev):
                self.A[l] = theta_maps(self.grid[l + 1], self.grid[l])
        self._T = {}

    # ---- operators ---------------------------------------------------------
    def T(self, l: int, off):
        key = (l, tuple(int(v) for v in off))
        if key not in self._T:
            X = np.asarray(off, dtype=np.float64) * self.tree.levels[l].edge
            if level_is_sampled(self.k, self.tree.levels[l].edge, self.sampled):
                self._T[key] = sampled_translation_operator(self.grid[l], self.k, X, self.sampled)
            else:
                self._T[key] = translation_operator(self.grid[l], self.k, X)
        return self._T[key]

    def shift_m2m(self, l: int, dc: np.ndarray) -> np.ndarray:
        """e^{-ik khat_p'.(c_c - c_P)} on the parent grid of level l; dc [nb, 3]."""
        return np.exp(-1j * self.k * (dc @ self.grid[l].dirs.T))

    # ---- stages ------------------------------------------------------------
    def c2m(self, l: int, qs: np.ndarray) -> np.ndarray:
        """F_b(p) = sum_{j in b} q_j e^{-ik khat_p.(r_j - c_b)} for the leaves of level l."""
        t, g = self.tree, self.grid[l]
        lev = t.levels[l]
        F = np.zeros((lev.nbox, g.K), dtype=np.complex128)
        for b in np.nonzero(lev.leaf)[0]:
            b0, b1 = lev.begin[b], lev.end[b]
            rel = self.sorted_pts[b0:b1] - lev.center[b]
            F[b] = qs[b0:b1] @ np.exp(-1j * self.k * (rel @ g.dirs.T))
        return F

    def m2m(self, l: int, Fchild: np.ndarray, F: np.ndarray) -> None:
        """F_P for the non-leaf boxes of level l from their children at level l+1."""
        t = self.tree
        lev, ch = t.levels[l], t.levels[l + 1]
        Fi = interpolate(Fchild, self.grid[l + 1], self.grid[l], self.A[l])
        dc = ch.center - lev.center[ch.parent]
        Fi = Fi * self.shift_m2m(l, dc)
        for b in np.nonzero(~lev.leaf)[0]:
            F[b] = Fi[lev.child_begin[b]:lev.child_end[b]].sum(axis=0)

    def m2l(self, l: int, F: np.ndarray) -> np.ndarray:
        """G_t(p) = sum_{s in V(t)} T_{c_t - c_s}(p) F_s(p) (Alg. 2, one level)."""
        lev = self.tree.levels[l]
        offs, cols = self.V[l]
        G = np.zeros_like(F)
        for tb in range(lev.nbox):
            for s in cols[offs[tb]:offs[tb + 1]]:
                G[tb] += self.T(l, lev.ijk[tb] - lev.ijk[s]) * F[s]
        return G

    def l2l(self, l: int, Gpar: np.ndarray, G: np.ndarray) -> None:
        """G_c += anterpolate(e^{+ik khat.(c_c - c_P)} G_P) for the boxes of level l+1."""
        t = self.tree
        lev, ch = t.levels[l], t.levels[l + 1]
        dc = ch.center - lev.center[ch.parent]
        sh = np.conj(self.shift_m2m(l, dc)) * Gpar[ch.parent]
        G += anterpolate(sh, self.grid[l + 1], self.grid[l], self.A[l])

    def l2o(self, l: int, G: np.ndarray, phi: np.ndarray) -> None:
        """phi_i += (ik/4pi) sum_p w_p e^{ik khat_p.(r_i - c_b)} G_b(p), leaves of level l."""
        t, g = self.tree, self.grid[l]
        lev = t.levels[l]
        for b in np.nonzero(lev.leaf)[0]:
            b0, b1 = lev.begin[b], lev.end[b]
            rel = self.sorted_pts[b0:b1] - lev.center[b]
            E = np.exp(1j * self.k * (rel @ g.dirs.T))
            phi[b0:b1] += (1j * self.k / (4.0 * math.pi)) * (E @ (g.w * G[b]))

    def p2p(self, qs: np.ndarray) -> np.ndarray:
        """Near-field direct sums at the leaves (Sec. 2)."""
        t = self.tree
        phi = np.zeros(t.n, dtype=np.complex128)
        P = self.sorted_pts
        if self.uniform:
            lev = t.levels[t.nlev]
            offs, cols = self.U
            for b in range(lev.nbox):
                b0, b1 = lev.begin[b], lev.end[b]
                srcs = cols[offs[b]:offs[b + 1]]
                idx = np.concatenate([np.arange(lev.begin[s], lev.end[s]) for s in srcs])
                phi[b0:b1] = direct_pairs(P[b0:b1], P[idx], qs[idx], self.k)
        else:
            for (l, b), srcs in self.near.items():
                lev = t.levels[l]
                b0, b1 = lev.begin[b], lev.end[b]
                if not srcs:
                    continue
                idx = np.concatenate([np.arange(t.levels[ls].begin[s], t.levels[ls].end[s]) for ls, s in srcs])
                phi[b0:b1] = direct_pairs(P[b0:b1], P[idx], qs[idx], self.k)
        return phi

    @property
    def sorted_pts(self):
        if not hasattr(self, "_sp"):
            self._sp = self.points[self.tree.perm]
        return self._sp

    def apply(self, q: np.ndarray, dump: bool = False):
        """phi = A q in the caller's point order (q: [n] complex)."""
        t = self.tree
        qs = np.asarray(q, dtype=np.complex128)[t.perm]
        near = self.p2p(qs)
        far = np.zeros(t.n, dtype=np.complex128)
        F, G = {}, {}
        if self.top is not None:
            for l in range(t.nlev, self.top - 1, -1):
                F[l] = self.c2m(l, qs)
                if l < t.nlev:
                    self.m2m(l, F[l + 1], F[l])
            for l in range(self.top, t.nlev + 1):
                G[l] = self.m2l(l, F[l])
                if l > self.top:
                    self.l2l(l - 1, G[l - 1], G[l])
                self.l2o(l, G[l], far)
        phi_s = near + far
        phi = np.empty_like(phi_s)
        phi[t.perm] = phi_s
        if dump:
            return phi, dict(F=F, G=G, near=near, far=far)
        return phi

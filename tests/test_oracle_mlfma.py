"""Pins for the oracle MLFMA stages and the FP64 direct sum (CPU only).

Independent references: scipy's spherical Bessel/Hankel functions and
spherical harmonics, closed forms (single source, two points), the
Funk-Hecke identity, the Gegenbauer series, brute-force literal operators
(weighted transpose), central finite differences, and invariants
(reciprocity, linearity).
"""
import math

import numpy as np
import pytest
import scipy.special as sp

import synth
from oracle import direct, mlfma, special

K = 2.0 * math.pi


# --------------------------------------------------------------------------- direct sum
def test_direct_two_points_closed_form():
    pts = np.array([[0.0, 0.0, 0.0], [0.3, -0.4, 1.2]])
    q = np.array([1.0 + 2.0j, -0.5 + 0.25j])
    R = np.linalg.norm(pts[1] - pts[0])
    phi = direct.direct(pts, q, K)
    g = np.exp(1j * K * R) / R
    assert abs(phi[0] - q[1] * g) < 1e-15 * abs(g)
    assert abs(phi[1] - q[0] * g) < 1e-15 * abs(g)


def test_direct_skips_self_and_coincident():
    pts = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    q = np.array([1.0, 1.0, 1.0], dtype=complex)
    phi = direct.direct(pts, q, K)
    g = np.exp(1j * K) / 1.0
    assert np.allclose(phi, [g, g, 2 * g], rtol=1e-15, atol=0)


def test_direct_matches_brute_python_and_sample_targets():
    pts = synth.sphere(200, 1.0, seed=3)
    q = synth.complex_normal(4, 200)[0]
    ref = np.zeros(200, dtype=complex)
    for i in range(200):
        for j in range(200):
            if i != j:
                R = math.dist(pts[i], pts[j])
                ref[i] += q[j] * complex(math.cos(K * R), math.sin(K * R)) / R
    assert np.max(np.abs(direct.direct(pts, q, K) - ref)) < 1e-12 * np.max(np.abs(ref))
    tg = np.array([5, 17, 199])
    assert np.max(np.abs(direct.direct(pts, q, K, targets=tg) - ref[tg])) < 1e-12 * np.max(np.abs(ref))


def test_direct_gradient_finite_difference():
    pts = synth.sphere(60, 1.0, seed=8)
    q = synth.complex_normal(9, 60)[0]
    g = direct.direct_grad(pts, q, K)
    h = 1e-5
    for i in (0, 7, 33):
        for a in range(3):
            pp, pm = pts.copy(), pts.copy()
            pp[i, a] += h
            pm[i, a] -= h
            # only phi_i as a function of r_i (sources fixed)
            fp = direct.direct(np.vstack([pp[i:i + 1], np.delete(pts, i, 0)]),
                               np.concatenate([[0], np.delete(q, i)]), K, targets=[0])
            fm = direct.direct(np.vstack([pm[i:i + 1], np.delete(pts, i, 0)]),
                               np.concatenate([[0], np.delete(q, i)]), K, targets=[0])
            fd = (fp[0] - fm[0]) / (2 * h)
            assert abs(fd - g[i, a]) < 1e-6 * max(1.0, abs(g[i, a]))


# --------------------------------------------------------------------------- far-field math
@pytest.mark.parametrize("L", [10, 25])
def test_funk_hecke_quadrature(L):
    """sum_p w_p e^{ik khat_p.d} P_n(khat_p.Xhat) = 4 pi i^n j_n(k|d|) P_n(dhat.Xhat)."""
    g = mlfma.Grid(L)
    rng = np.random.default_rng(L)
    d = rng.normal(size=3)
    d *= (0.25 * L / K) / np.linalg.norm(d)           # k|d| well inside the band
    X = rng.normal(size=3)
    X /= np.linalg.norm(X)
    P = special.legendre_all(L, g.dirs @ X)
    e = np.exp(1j * K * (g.dirs @ d))
    lhs = (P * (g.w * e)[None, :]).sum(axis=1)
    n = np.arange(L + 1)
    rhs = 4 * np.pi * (1j ** n) * sp.spherical_jn(n, K * np.linalg.norm(d)) * \
        sp.eval_legendre(n, d @ X / np.linalg.norm(d))
    # exact while n + (band of the plane wave) <= 2L+1; small aliasing above
    assert np.max(np.abs(lhs - rhs)[: L // 2 + 1]) < 1e-12
    assert np.max(np.abs(lhs - rhs)) < 1e-7


def _plane_wave_pair(L, X, d):
    g = mlfma.Grid(L)
    T = mlfma.translation_operator(g, K, X)
    return (1j * K / (4 * np.pi)) * np.sum(g.w * np.exp(1j * K * (g.dirs @ d)) * T)


def _gegenbauer(L, X, d):
    """ik sum_{n<=L} (-1)^n (2n+1) j_n(kd) h_n(kX) P_n(dhat.Xhat) with scipy's functions."""
    n = np.arange(L + 1)
    x, r = np.linalg.norm(X), np.linalg.norm(d)
    h = sp.spherical_jn(n, K * x) + 1j * sp.spherical_yn(n, K * x)
    return 1j * K * np.sum((-1.0) ** n * (2 * n + 1) * sp.spherical_jn(n, K * r) * h *
                           sp.eval_legendre(n, (d @ X) / (r * x)))


@pytest.mark.parametrize("a,tol,nL", [(0.5, 1e-4, 2), (1.0, 1e-6, 3), (2.0, 1e-8, 3)])
def test_addition_theorem_vs_gegenbauer_and_exact(a, tol, nL):
    """Two-box factorisation = truncated Gegenbauer series; its error falls with L.

    Once the grid integrates the plane wave (L >= k|d| + 8), the quadrature adds
    little: at a = lambda/2 (k|X| = 2 pi) the growth of |T| with L (low-frequency
    breakdown) amplifies the aliasing of the top degrees, hence the looser bound.
    """
    X = np.array([2 * a, 0.0, 0.0])                   # nearest far-field offset
    d = np.array([-a, a, a]) * 0.999                  # |d| close to the box diagonal
    exact = np.exp(1j * K * np.linalg.norm(X + d)) / np.linalg.norm(X + d)
    errs = []
    kd = K * np.linalg.norm(d)
    for L in range(int(kd) + 8, int(kd) + 8 + 3 * nL, 3):
        g = mlfma.Grid(L)
        T = mlfma.translation_operator(g, K, X)
        pw = (1j * K / (4 * np.pi)) * np.sum(g.w * np.exp(1j * K * (g.dirs @ d)) * T)
        gg = _gegenbauer(L, X, d)
        assert abs(pw - gg) < tol * abs(exact) + 0.1 * abs(gg - exact)
        errs.append(abs(gg - exact) / abs(exact))
    if a >= 1.0:                                      # slow, oscillating tail at lambda/2
        assert errs[-1] < errs[0]


@pytest.mark.parametrize("digits,edge", [(3, 0.5), (3, 1.0), (3, 4.0), (6, 1.0), (6, 4.0)])
def test_truncation_rule_meets_digits_worst_case(digits, edge):
    """The excess-bandwidth L meets 10^-d for the nearest far offsets of a level.

    Separations |d| <= sqrt(3) a / 2 (the bulk of point pairs); the extreme
    corner pairs (|d| -> sqrt(3) a, |X| = 2a) converge slowly for any L and are
    left to the end-to-end comparisons with the direct sum.
    """
    L = mlfma.truncation_L(edge, K, digits)
    worst = 0.0
    for X in (np.array([2.0, 0, 0]), np.array([2.0, 2.0, 0]), np.array([2.0, 2.0, 2.0])):
        X = X * edge
        for s in ([-1, 1, 1], [-1, -1, -1], [-1, 0.3, -0.7]):
            d = np.array(s, dtype=float) * 0.5 * edge * 0.999
            ex = np.exp(1j * K * np.linalg.norm(X + d)) / np.linalg.norm(X + d)
            worst = max(worst, abs(_plane_wave_pair(L, X, d) - ex) / abs(ex))
    assert worst < 10.0 ** (-digits)


def _random_bandlimited(Lc, grid, rng):
    """sum_{n<=Lc,|m|<=n} a_nm Y_nm sampled on ``grid`` (scipy's spherical harmonics)."""
    th = np.arccos(grid.dirs[:, 2])
    ph = np.mod(np.arctan2(grid.dirs[:, 1], grid.dirs[:, 0]), 2 * np.pi)
    f = np.zeros(grid.K, dtype=complex)
    for n in range(Lc + 1):
        for m in range(-n, n + 1):
            a = rng.normal() + 1j * rng.normal()
            f += a * sp.sph_harm_y(n, m, th, ph)
    return f


@pytest.mark.parametrize("Lc,Lp", [(6, 11), (13, 20)])
def test_interpolation_exact_on_bandlimited(Lc, Lp):
    rng = np.random.default_rng(Lc)
    gc, gp = mlfma.Grid(Lc), mlfma.Grid(Lp)
    A = mlfma.theta_maps(gc, gp)
    st = rng.bit_generator.state
    fc = _random_bandlimited(Lc, gc, rng)
    rng.bit_generator.state = st
    fp = _random_bandlimited(Lc, gp, rng)
    assert np.max(np.abs(mlfma.interpolate(fc, gc, gp, A) - fp)) < 1e-11 * np.max(np.abs(fp))


@pytest.mark.parametrize("Lc,Lp", [(5, 9), (8, 13)])
def test_anterpolation_is_weighted_transpose(Lc, Lp):
    gc, gp = mlfma.Grid(Lc), mlfma.Grid(Lp)
    A = mlfma.theta_maps(gc, gp)
    I = mlfma.interpolate(np.eye(gc.K, dtype=complex), gc, gp, A).T      # [Kp, Kc]
    lit = np.diag(1.0 / gc.w) @ I.T @ np.diag(gp.w)
    rng = np.random.default_rng(1)
    g = rng.normal(size=gp.K) + 1j * rng.normal(size=gp.K)
    assert np.max(np.abs(mlfma.anterpolate(g, gc, gp, A) - lit @ g)) < 1e-11 * np.max(np.abs(lit @ g))


def test_m2m_equals_direct_aggregation_at_parent(sphere4k):
    """F_P from the children (interpolate, shift, sum) ~= C2M evaluated at the parent."""
    pts, q, prm = sphere4k
    o = mlfma.OracleMLFMA(pts, prm["k"], 4)
    t = o.tree
    qs = q[0][t.perm]
    l = t.nlev - 1
    F = o.c2m(t.nlev, qs)
    Fp = np.zeros((t.levels[l].nbox, o.grid[l].K), dtype=complex)
    o.m2m(l, F, Fp)
    lev = t.levels[l]
    g = o.grid[l]
    for b in range(0, lev.nbox, 37):
        rel = o.sorted_pts[lev.begin[b]:lev.end[b]] - lev.center[b]
        ref = qs[lev.begin[b]:lev.end[b]] @ np.exp(-1j * prm["k"] * (rel @ g.dirs.T))
        assert np.max(np.abs(Fp[b] - ref)) < 1e-4 * np.max(np.abs(ref))


def test_mlfma_single_source_closed_form(sphere4k):
    pts, _, prm = sphere4k
    q = np.zeros(pts.shape[0], dtype=complex)
    q[123] = 1.0
    phi = mlfma.OracleMLFMA(pts, prm["k"], 3).apply(q)
    R = np.linalg.norm(pts - pts[123], axis=1)
    ref = np.where(R > 0, np.exp(1j * prm["k"] * R) / np.where(R > 0, R, 1), 0)
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-3


@pytest.mark.parametrize("digits,leaf", [(3, 0.25), (6, 0.5)])
def test_mlfma_vs_direct(sphere4k, digits, leaf):
    pts, q, prm = sphere4k
    o = mlfma.OracleMLFMA(pts, prm["k"], digits, leaf_edge=leaf)
    phi = o.apply(q[0])
    ref = direct.direct(pts, q[0], prm["k"])
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 10.0 ** (-digits)


def test_mlfma_reciprocity_and_linearity(sphere4k):
    pts, q, prm = sphere4k
    o = mlfma.OracleMLFMA(pts, prm["k"], 3)
    p = synth.complex_normal(77, pts.shape[0])[0]
    Aq, Ap = o.apply(q[0]), o.apply(p)
    assert abs(p @ Aq - q[0] @ Ap) <= 1e-3 * np.linalg.norm(p) * np.linalg.norm(Aq)
    Apq = o.apply(2.0 * q[0] - 1j * p)
    assert np.max(np.abs(Apq - (2.0 * Aq - 1j * Ap))) < 1e-12 * np.max(np.abs(Apq))


def test_mlfma_adaptive_vs_direct():
    pts = np.concatenate([synth.sphere(1500, 1.5, seed=41),
                          synth.normal(42, 3 * 600).reshape(600, 3) * 0.05 + np.array([0.9, 0.0, 0.0])])
    q = synth.complex_normal(43, pts.shape[0])[0]
    o = mlfma.OracleMLFMA(pts, K, 3, leaf_max=16)
    assert len({l for (l, _) in o.Ud}) > 1
    phi = o.apply(q)
    ref = direct.direct(pts, q, K)
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-3


def test_sample_count_quadruples_per_level():
    """K_l grows about four times per level up the tree (Sec. 2, H-FMM bullet)."""
    Ks = [mlfma.Grid(mlfma.truncation_L(0.25 * 2 ** j, K, 3)).K for j in range(10)]
    ratios = [Ks[j + 1] / Ks[j] for j in range(len(Ks) - 1)]
    # the excess bandwidth O((kD)^(1/3)) makes the ratio approach 4 from below
    assert all(r > 1.5 for r in ratios) and ratios[-1] > ratios[0] and abs(ratios[-1] - 4.0) < 0.3


def test_smooth_even_matches_enumerated_products():
    """The phi-grid length rule: the smallest even 7-smooth number >= m, against the 7-smooth
    numbers enumerated as products 2^a 3^b 5^c 7^d (not by trial division)."""
    bound = 4096
    smooth = set()
    p2 = 1
    while p2 <= bound:
        p3 = p2
        while p3 <= bound:
            p5 = p3
            while p5 <= bound:
                p7 = p5
                while p7 <= bound:
                    smooth.add(p7)
                    p7 *= 7
                p5 *= 5
            p3 *= 3
        p2 *= 2
    even = sorted(v for v in smooth if v % 2 == 0)
    for m in range(1, 2000):
        want = next(v for v in even if v >= m)
        assert mlfma.smooth_even(m) == want, m


def test_direct_pairs_matches_the_c_direct_sum():
    """The oracle MLFMA's near-field block sum (numpy) against the C direct sum on the same set,
    with a coincident pair that both must skip."""
    pts = synth.sphere(300, 1.0, seed=31)
    pts[5] = pts[9]
    q = synth.complex_normal(32, 300)[0]
    ref = direct.direct(pts, q, K)
    got = mlfma.direct_pairs(pts, pts, q, K)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("L", [3, 8, 13, 20])
def test_grid_quadrature_exact_and_antipodally_symmetric(L):
    """The level grid integrates (a . khat)^n over the sphere exactly for n <= 2L + 1 (closed form
    4 pi / (n + 1) for even n, 0 for odd n; any unit a), and is antipodally symmetric: -khat of
    sample (i, j) is sample (L - i, j + nph / 2) with the same weight."""
    g = mlfma.Grid(L)
    assert np.allclose(np.linalg.norm(g.dirs, axis=1), 1.0, atol=1e-14)
    rng = np.random.default_rng(L)
    for _ in range(3):
        a = rng.standard_normal(3)
        a /= np.linalg.norm(a)
        t = g.dirs @ a
        for n in range(2 * L + 2):
            want = 4.0 * math.pi / (n + 1) if n % 2 == 0 else 0.0
            assert abs(np.sum(g.w * t ** n) - want) < 1e-12 * 4.0 * math.pi
    i = np.arange(g.nth)[:, None]
    j = np.arange(g.nph)[None, :]
    anti = ((L - i) * g.nph + (j + g.nph // 2) % g.nph).reshape(-1)
    assert np.allclose(g.dirs[anti], -g.dirs, atol=1e-14)
    assert np.allclose(g.w[anti], g.w, rtol=1e-14)


# --------------------------------------------------------------------------- sampled operators
@pytest.mark.parametrize("P", [4, 10])
def test_lagrange_weights_reproduce_polynomials(P):
    """The P-point interpolant is exact on polynomials of degree < P and is a delta at the nodes."""
    rng = np.random.default_rng(5)
    c = rng.standard_normal(P)                          # degree P - 1
    t = rng.uniform(P // 2 - 1, P // 2, 7)
    w = mlfma.lagrange_weights(t, P)
    vals = np.polyval(c, np.arange(P, dtype=float))
    assert np.allclose(vals @ w, np.polyval(c, t), rtol=1e-11, atol=1e-11 * np.max(np.abs(vals)))
    for j in range(P):
        assert np.array_equal(mlfma.lagrange_weights(float(j), P), np.eye(P)[j])


def test_interpolation_stencil_is_centred():
    """On u^P (u = psi / h) the P-point interpolant errs by exactly prod_j (t - j) (the P-th
    derivative over P! is 1), with t = u - i0 in the middle interval [P/2 - 1, P/2): this fixes
    where the stencil sits around each angle."""
    P, S = mlfma.SAMPLED_ORDER, 40
    i = np.arange(-P, S + P + 1, dtype=float)
    for u in (0.3, 5.5, 17.25, 39.9):
        c = math.floor(u) + 0.5                        # (u - c)^P: same P-th derivative, no cancellation
        got = mlfma.interpolate_samples((i - c) ** P, np.array([u * math.pi / S]), S, P)[0]
        t = u - math.floor(u) + (P // 2 - 1)
        omega = np.prod([t - j for j in range(P)])
        assert abs((u - c) ** P - got - omega) < 1e-9 * abs(omega), u


class _Dirs:
    """A sampling 'grid' of given directions (translation_operator reads L, K and dirs)."""

    def __init__(self, L, dirs):
        self.L, self.dirs, self.K = L, dirs, dirs.shape[0]


def _bound(s, P):
    """sqrt(2) (pi / s)^P max_{t in middle interval} prod_j |t - j| / P!: the Lagrange remainder
    with Bernstein's inequality |f^(P)| <= L^P |f| for a trigonometric polynomial of degree L
    (node spacing pi / (s L)), real and imaginary parts apart."""
    t = np.linspace(P // 2 - 1, P // 2, 2001)
    om_max = np.max(np.abs(np.prod([t - j for j in range(P)], axis=0)))
    return math.sqrt(2.0) * (math.pi / s) ** P * om_max / math.factorial(P)


@pytest.mark.parametrize("edge,digits", [(0.25, 3), (2.0, 3), (1.0, 6)])
def test_sampled_operator_within_interpolation_bound(edge, digits):
    """Sampled-and-interpolated operators against the exact (Gegenbauer-pinned) ones: within the
    Lagrange-Bernstein bound relative to max |T|, and converging at order P in the oversampling.
    The axis offsets put samples next to psi = 0 and psi = pi, where the stencil reads the
    reflected entries of the table."""
    L = mlfma.truncation_L(edge, K, digits)
    g = mlfma.Grid(L)
    P = mlfma.SAMPLED_ORDER
    errs = {}
    for s in (3, 4, 6):
        worst = 0.0
        for off in ((0, 0, 2), (0, 0, -3), (2, 1, 3), (3, 3, 3), (-2, 2, 1)):
            X = np.array(off, float) * edge
            T = mlfma.translation_operator(g, K, X)
            Ts = mlfma.sampled_translation_operator(g, K, X, s)
            tmax = np.max(np.abs(mlfma.operator_samples(L, K, np.linalg.norm(X), 16)))
            e = np.max(np.abs(Ts - T)) / tmax
            assert e <= _bound(s, P), (s, off, e)
            worst = max(worst, e)
        errs[s] = worst
    assert errs[3] / errs[6] > 2.0 ** (P - 3)


def test_sampled_operator_exact_at_table_angles():
    """Directions at the tabulated angles psi_i (both ends included) reproduce T exactly."""
    L, s, edge = 12, 4, 0.5
    S = s * L
    i = np.array([0, 1, 7, S // 2, S - 1, S])
    psi = i * math.pi / S
    X = np.array([0.0, 0.0, 2.0]) * edge                 # Xhat = z: psi is the polar angle
    d = np.stack([np.sin(psi), np.zeros_like(psi), np.cos(psi)], axis=1)
    g = _Dirs(L, d)
    Ts = mlfma.sampled_translation_operator(g, K, X, s)
    T = mlfma.translation_operator(g, K, X)
    assert np.max(np.abs(Ts - T)) < 1e-12 * np.max(np.abs(T))


def test_operator_samples_hold_the_reflections():
    """Padding entries: T(-psi) = T(psi) and T(pi + psi) = T(pi - psi)."""
    L, s, P = 9, 3, mlfma.SAMPLED_ORDER
    S = s * L
    tab = mlfma.operator_samples(L, K, 1.3, s)
    assert tab.shape == (S + 2 * P + 1,)
    for m in range(1, P + 1):
        assert abs(tab[P - m] - tab[P + m]) < 1e-12 * np.max(np.abs(tab))
        assert abs(tab[P + S + m] - tab[P + S - m]) < 1e-12 * np.max(np.abs(tab))


def test_sampled_levels_are_the_wavelength_sized_boxes():
    assert mlfma.level_is_sampled(K, 1.0, 6) and mlfma.level_is_sampled(K, 1.0 - 1e-12, 6)
    assert not mlfma.level_is_sampled(K, 0.5, 6) and not mlfma.level_is_sampled(K, 4.0, 0)


def test_mlfma_with_sampled_operators_vs_direct(sphere4k):
    """The far field with sampled operators (oversampling 6; on this sphere level 3, edge one
    wavelength, is sampled) meets 3 digits and stays within the operator interpolation error
    of the full-table MLFMA."""
    pts, q, prm = sphere4k
    o = mlfma.OracleMLFMA(pts, prm["k"], 3, sampled_operators=6)
    assert [l for l in o.L if mlfma.level_is_sampled(o.k, o.tree.levels[l].edge, 6)] == [3]
    phi_s = o.apply(q[0])
    phi = mlfma.OracleMLFMA(pts, prm["k"], 3).apply(q[0])
    ref = direct.direct(pts, q[0], prm["k"])
    assert np.linalg.norm(phi_s - ref) / np.linalg.norm(ref) < 1e-3
    assert 0 < np.linalg.norm(phi_s - phi) / np.linalg.norm(phi) < 1e-4


@pytest.mark.parametrize("Lc,Lp", [(10, 19), (11, 20), (33, 57)])
def test_theta_maps_are_centrosymmetric(Lc, Lp):
    """Gauss-Legendre nodes come in pairs (x, -x) with equal weights and Pbar_n^m(-x) =
    (-1)^(n+m) Pbar_n^m(x), so every per-mode map satisfies A[n'-1-i', n-1-i] = A[i', i]: the
    property that lets the GPU path apply each map as an even and an odd half of a quarter of
    its size (odd and even grid lengths both covered)."""
    gc, gp = mlfma.Grid(Lc), mlfma.Grid(Lp)
    assert np.allclose(gc.x, -gc.x[::-1], atol=1e-15) and np.allclose(gc.wgl, gc.wgl[::-1], rtol=1e-13)
    for m, A in enumerate(mlfma.theta_maps(gc, gp)):
        assert np.max(np.abs(A[::-1, ::-1] - A)) <= 1e-13 * np.max(np.abs(A)), m

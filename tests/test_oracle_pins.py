"""Pins for the CPU oracle, against things other than itself.

* closed forms: the unit square's self integral (textbook), and 4-D corner
  sums of antiderivatives F (parallel panels) and H (perpendicular panels)
  whose defining derivatives are checked symbolically and which are then
  evaluated at 40 digits with mpmath;
* a library routine: numpy's Gauss-Legendre rule for well separated pairs;
* invariants: reciprocity with roles swapped, translation, h^3 scaling.

The paper (Sec. 3.4) reduces every entry to corner sums of antiderivatives
(its Eqs. "int1", "int2" for coplanar parallel panels and "int4", "int5" for
perpendicular ones).  The closed forms here are complete versions of those
reductions, derived independently; the oracle itself uses neither.
"""
import math
import random

import numpy as np
import pytest

from oracle import oracle as O

mpmath = pytest.importorskip("mpmath")
mp = mpmath.mp


# ---------------------------------------------------------------- closed forms

def _xlog(coef, t, r2, rho):
    if coef == 0:
        return mp.mpf(0)
    if t >= 0:
        return coef * mp.log(t + rho)
    return coef * mp.log(r2 / (rho - t))


def F_par(u, v, w):
    """d^4 F / du^2 dv^2 = 1/sqrt(u^2+v^2+w^2)."""
    rho = mp.sqrt(u * u + v * v + w * w)
    r = (_xlog((v / 2) * (u * u - w * w), v, u * u + w * w, rho)
         + _xlog((u / 2) * (v * v - w * w), u, v * v + w * w, rho)
         - (u * u + v * v - 2 * w * w) * rho / 6)
    if u * v * w != 0:
        r -= u * v * w * mp.atan(u * v / (w * rho))
    return r


def H_orth(u, v, w):
    """d^4 H / du^2 dv dw = 1/sqrt(u^2+v^2+w^2)."""
    rho = mp.sqrt(u * u + v * v + w * w)
    r = (_xlog(u * v * w, u, v * v + w * w, rho)
         + _xlog((w / 6) * (3 * u * u - w * w), v, u * u + w * w, rho)
         + _xlog((v / 6) * (3 * u * u - v * v), w, u * u + v * v, rho)
         - v * w * rho / 3)
    if u * w != 0 and v != 0:
        r -= (u * w * w / 2) * mp.atan(u * v / (w * rho))
    if u * v != 0 and w != 0:
        r -= (u * v * v / 2) * mp.atan(u * w / (v * rho))
    if u != 0 and v * w != 0:
        r -= (u ** 3 / 6) * mp.atan(v * w / (u * rho))
    return r


def _inplane(k):
    return [a for a in range(3) if a != k]


def closed_form(ax_i, gi, ax_j, gj):
    """int_{I_i} int_{I_j} 1/|x-y| by corner sums, at mp precision."""
    gi = [mp.mpf(repr(float(x))) for x in gi]
    gj = [mp.mpf(repr(float(x))) for x in gj]
    if ax_i == ax_j:
        w = gi[0] - gj[0]
        s = mp.mpf(0)
        for a in range(2):
            for b in range(2):
                for c in range(2):
                    for d in range(2):
                        sg = (-1) ** (a + b + c + d)
                        s += sg * F_par(gi[1 + a] - gj[1 + b], gi[3 + c] - gj[3 + d], w)
        return s
    # perpendicular: shared axis s, I_i spans s and ax_j, I_j spans s and ax_i
    sh = 3 - ax_i - ax_j
    pi, pj = _inplane(ax_i), _inplane(ax_j)
    ext_i = {pi[0]: (gi[1], gi[2]), pi[1]: (gi[3], gi[4])}
    ext_j = {pj[0]: (gj[1], gj[2]), pj[1]: (gj[3], gj[4])}
    p = ext_i[sh]
    q = ext_i[ax_j]
    r = ext_j[sh]
    t = ext_j[ax_i]
    ci, cj = gi[0], gj[0]
    s = mp.mpf(0)
    for a in range(2):
        for b in range(2):
            for c in range(2):
                for d in range(2):
                    sg = (-1) ** (a + b + c + d)
                    s += sg * H_orth(p[a] - r[b], q[c] - cj, ci - t[d])
    return s


def test_antiderivatives_symbolic():
    sp = pytest.importorskip("sympy")
    u, v, w = sp.symbols("u v w", real=True)
    rho = sp.sqrt(u ** 2 + v ** 2 + w ** 2)
    F = ((v / 2) * (u ** 2 - w ** 2) * sp.log(v + rho) + (u / 2) * (v ** 2 - w ** 2) * sp.log(u + rho)
         - (u ** 2 + v ** 2 - 2 * w ** 2) * rho / 6 - u * v * w * sp.atan(u * v / (w * rho)))
    H = (u * v * w * sp.log(u + rho) + (w / 6) * (3 * u ** 2 - w ** 2) * sp.log(v + rho)
         + (v / 6) * (3 * u ** 2 - v ** 2) * sp.log(w + rho) - v * w * rho / 3
         - (u * w ** 2 / 2) * sp.atan(u * v / (w * rho)) - (u * v ** 2 / 2) * sp.atan(u * w / (v * rho))
         - (u ** 3 / 6) * sp.atan(v * w / (u * rho)))
    dF = sp.lambdify((u, v, w), sp.diff(F, u, 2, v, 2) - 1 / rho, "mpmath")
    dH = sp.lambdify((u, v, w), sp.diff(H, u, 2, v, 1, w, 1) - 1 / rho, "mpmath")
    rng = random.Random(5)
    with mp.workdps(40):
        for _ in range(8):
            pt = [mp.mpf(rng.uniform(-2, 2)) for _ in range(3)]
            assert abs(dF(*pt)) < mp.mpf(10) ** -30
            assert abs(dH(*pt)) < mp.mpf(10) ** -30
    # the mpmath evaluators used below are the same expressions
    with mp.workdps(30):
        pt = (mp.mpf("0.3"), mp.mpf("-1.1"), mp.mpf("0.7"))
        assert abs(F_par(*pt) - sp.N(F.subs(dict(zip((u, v, w), pt))), 30)) < 1e-25
        assert abs(H_orth(*pt) - sp.N(H.subs(dict(zip((u, v, w), pt))), 30)) < 1e-25


# ---------------------------------------------------------------- textbook values

def test_unit_square_self_textbook():
    # self energy of the uniformly charged unit square:
    # int int 1/|x-y| = 4 ln(1+sqrt 2) - (4/3)(sqrt 2 - 1)
    exact = 4 * math.log(1 + math.sqrt(2)) - (4.0 / 3.0) * (math.sqrt(2) - 1)
    v, nf = O.pair_integral(2, [0, 0, 1, 0, 1], 2, [0, 0, 1, 0, 1])
    assert nf == 0
    assert v == pytest.approx(exact, rel=1e-14)
    with mp.workdps(40):
        assert float(closed_form(2, [0, 0, 1, 0, 1], 2, [0, 0, 1, 0, 1])) == pytest.approx(exact, rel=1e-15)


NAMED = [
    ("1x2 rectangle self", (2, [0, 0, 1, 0, 2]), (2, [0, 0, 1, 0, 2])),
    ("unit squares stacked at distance 1", (2, [0, 0, 1, 0, 1]), (2, [1, 0, 1, 0, 1])),
    ("coplanar edge-adjacent unit squares", (2, [0, 0, 1, 0, 1]), (2, [0, 1, 2, 0, 1])),
    ("coplanar corner-adjacent unit squares", (2, [0, 0, 1, 0, 1]), (2, [0, 1, 2, 1, 2])),
    ("parallel unit squares at distance 10", (2, [0, 0, 1, 0, 1]), (2, [10, 0, 1, 0, 1])),
    ("L-shape sharing an edge", (2, [0, 0, 1, 0, 1]), (1, [0, 0, 1, 0, 1])),
    ("perpendicular, face y=-1 vs face z=0", (1, [-1, 0, 1, 0, 1]), (2, [0, 0, 1, 0, 1])),
]


@pytest.mark.parametrize("name,pi,pj", NAMED, ids=[n for n, _, _ in NAMED])
def test_named_configurations(name, pi, pj):
    with mp.workdps(40):
        ref = float(closed_form(pi[0], pi[1], pj[0], pj[1]))
    v, nf = O.pair_integral(pi[0], pi[1], pj[0], pj[1])
    assert nf == 0
    assert v == pytest.approx(ref, rel=2e-14)


# ---------------------------------------------------------------- random closed-form pins

def _rand_rect(rng, scale=1.0):
    a0 = rng.uniform(-1, 1) * scale
    b0 = rng.uniform(-1, 1) * scale
    return [a0, a0 + rng.uniform(0.1, 1.0) * scale, b0, b0 + rng.uniform(0.1, 1.0) * scale]


def _cases(seed, n):
    rng = random.Random(seed)
    out = []
    for t in range(n):
        kind = t % 6
        k = rng.randrange(3)
        if kind == 0:      # coplanar, random overlap/adjacency/separation
            gi = [0.25] + _rand_rect(rng)
            gj = [0.25] + _rand_rect(rng)
            if t % 12 == 0:   # exact edge adjacency
                gj[1], gj[2] = gi[2], gi[2] + 0.4
            out.append((k, gi, k, gj))
        elif kind == 1:    # parallel offset
            gi = [0.0] + _rand_rect(rng)
            gj = [rng.choice([0.05, 0.3, 1.0])] + _rand_rect(rng)
            out.append((k, gi, k, gj))
        elif kind == 2:    # self
            gi = [0.1] + _rand_rect(rng)
            out.append((k, gi, k, list(gi)))
        else:              # perpendicular, touching along an edge or separated
            kj = (k + rng.choice([1, 2])) % 3
            pi, pj = _inplane(k), _inplane(kj)
            gi = [0.0] + _rand_rect(rng)
            gj = [0.0] + _rand_rect(rng)
            # I_j's plane: at an edge of I_i (touching) or beyond it
            ext_i = {pi[0]: (gi[1], gi[2]), pi[1]: (gi[3], gi[4])}
            lo_i, hi_i = ext_i[kj]
            gj[0] = hi_i if kind == 3 else hi_i + rng.uniform(0.05, 0.5)
            # I_j spans along I_i's normal starting at I_i's plane (an L) or above it
            slot = 1 if pj[0] == k else 3
            base = 0.0 if kind in (3, 4) else rng.uniform(0.05, 0.5)
            gj[slot], gj[slot + 1] = base, base + rng.uniform(0.1, 1.0)
            out.append((k, gi, kj, gj))
    return out


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_oracle_matches_closed_forms(seed):
    with mp.workdps(40):
        for (ki, gi, kj, gj) in _cases(seed, 18):
            ref = float(closed_form(ki, gi, kj, gj))
            v, nf = O.pair_integral(ki, gi, kj, gj)
            assert nf == 0
            assert v == pytest.approx(ref, rel=2e-13), (ki, gi, kj, gj)


def test_closed_form_catches_plausible_mistakes():
    """The pin would fail if the oracle dropped a corner, flipped a sign or
    swapped the roles of the two panels' extents."""
    with mp.workdps(30):
        gi, gj = [0.0, 0, 1, 0, 0.5], [0.2, 0.3, 1.1, -0.2, 0.4]
        ref = float(closed_form(2, gi, 2, gj))
        v, _ = O.pair_integral(2, gi, 2, gj)
        assert v == pytest.approx(ref, rel=1e-13)
        swapped = [0.2, -0.2, 0.4, 0.3, 1.1]
        v2, _ = O.pair_integral(2, gi, 2, swapped)
        assert abs(v2 - ref) > 1e-3 * ref


# ---------------------------------------------------------------- library routine

def test_gauss_legendre_nodes_match_numpy():
    for n in (1, 2, 3, 5, 8, 12, 16, 24):
        x, w = O.gauss_legendre(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        assert np.allclose(x, xr, atol=2e-15, rtol=0)
        assert np.allclose(w, wr, atol=2e-15, rtol=0)


def _numpy_gl4(ki, gi, kj, gj, n=14):
    xr, wr = np.polynomial.legendre.leggauss(n)

    def pts(k, g):
        p, q = _inplane(k)
        a = 0.5 * (g[1] + g[2]) + 0.5 * (g[2] - g[1]) * xr
        b = 0.5 * (g[3] + g[4]) + 0.5 * (g[4] - g[3]) * xr
        P = np.zeros((n, n, 3))
        P[..., k] = g[0]
        P[..., p] = a[:, None]
        P[..., q] = b[None, :]
        W = np.outer(wr, wr) * 0.25 * (g[2] - g[1]) * (g[4] - g[3])
        return P.reshape(-1, 3), W.reshape(-1)

    X, WX = pts(ki, gi)
    Y, WY = pts(kj, gj)
    D = np.sqrt(((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1))
    return float(WX @ (1.0 / D) @ WY)


def test_far_pairs_match_numpy_gauss_legendre():
    rng = random.Random(11)
    for _ in range(20):
        ki, kj = rng.randrange(3), rng.randrange(3)
        gi = [0.0] + _rand_rect(rng, 0.2)
        gj = [rng.uniform(3, 6)] + _rand_rect(rng, 0.2)
        ref = _numpy_gl4(ki, gi, kj, gj)
        v, nf = O.pair_integral(ki, gi, kj, gj)
        assert nf == 0
        assert v == pytest.approx(ref, rel=1e-13)


# ---------------------------------------------------------------- invariants

def test_reciprocity_roles_swapped():
    for (ki, gi, kj, gj) in _cases(7, 24):
        a, _ = O.pair_integral(ki, gi, kj, gj, method=1)
        b, _ = O.pair_integral(kj, gj, ki, gi, method=1)
        assert a == pytest.approx(b, rel=2e-13)


def test_translation_and_scaling():
    rng = random.Random(3)
    for (ki, gi, kj, gj) in _cases(9, 12):
        base, _ = O.pair_integral(ki, gi, kj, gj)
        # translate along every axis by the same vector
        sh = [rng.uniform(-3, 3) for _ in range(3)]

        def move(k, g):
            p, q = _inplane(k)
            return [g[0] + sh[k], g[1] + sh[p], g[2] + sh[p], g[3] + sh[q], g[4] + sh[q]]

        t, _ = O.pair_integral(ki, move(ki, gi), kj, move(kj, gj))
        assert t == pytest.approx(base, rel=1e-12)
        s = 2.5
        sc, _ = O.pair_integral(ki, [x * s for x in gi], kj, [x * s for x in gj])
        assert sc == pytest.approx(base * s ** 3, rel=1e-12)


def test_far_field_asymptote():
    # two unit squares, parallel, centres R apart along the normal:
    # int int 1/r = 1/R * (1 - 1/(6 R^2) * (1/2+1/2)... ) -> R * value -> 1
    for R in (50.0, 200.0):
        v, _ = O.pair_integral(2, [0, 0, 1, 0, 1], 2, [R, 0, 1, 0, 1])
        # second moments of a unit square are 1/12 per axis, so the leading
        # correction is -(1/R^3) * (2 * 1/12 + 2 * 1/12) / 2 * ... ; compare to
        # the multipole series through 1/R^3
        approx = 1.0 / R - (1.0 / 6.0) / R ** 3
        assert v == pytest.approx(approx, rel=1e-6 / R)

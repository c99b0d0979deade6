"""Numerical soundness of the sparse elimination that the GPU Newton kernels
use for the alpha chain (host logic; restated here in numpy, independent of
the CUDA source).

The chain network's Newton matrix M = c I - dt_m dR/dw (section 2, Eq.
sdc:general: the implicit reaction update) is lower bidiagonal in the chain
species X_1..X_{ns-1}, bordered by the alpha (X_0) and energy rows and
columns.  Eliminating the chain columns first, with row exchanges only between
the row carried from the previous column and the next chain row, keeps the
band and costs O(n); the 2 x 2 border block is then solved with partial
pivoting.  These tests check, on systems built from the oracle's analytic
Jacobian, that the elimination's forward error stays within a small factor of
LAPACK's partially pivoted LU, and that it is exact on the structure it
assumes.
"""
import numpy as np
import pytest

import oracle as O
from paper_1910_12578_gb300 import workloads as W


def chain_elimination(M, g, zero=0.0):
    n = M.shape[0]
    nc = n - 2
    ci = [2 + k for k in range(nc)]
    bd = [M[ci[k], ci[k]] for k in range(nc)]
    bs = [zero] + [M[ci[k], ci[k - 1]] for k in range(1, nc)]
    uE = [M[ci[k], 0] for k in range(nc)]
    uA = [M[ci[k], 1] for k in range(nc)]
    vE = [M[0, ci[k]] for k in range(nc)]
    vA = [M[1, ci[k]] for k in range(nc)]
    dEE, dEA, dAE, dAA = M[0, 0], M[0, 1], M[1, 0], M[1, 1]
    gE, gA = g[0], g[1]
    gc = [g[ci[k]] for k in range(nc)]
    cur = [bd[0], uE[0], uA[0], gc[0]]
    wE, wA = vE[0], vA[0]
    rows = []
    for k in range(nc):
        if k + 1 < nc:
            nxt = [bs[k + 1], bd[k + 1], uE[k + 1], uA[k + 1], gc[k + 1]]
            sw = abs(nxt[0]) > abs(cur[0])
        else:
            sw = False
        if sw:
            p, e, qE, qA, qg = nxt
            l = cur[0] / p
            cur = [-l * e, cur[1] - l * qE, cur[2] - l * qA, cur[3] - l * qg]
        else:
            p, e, qE, qA, qg = cur[0], zero, cur[1], cur[2], cur[3]
            if k + 1 < nc:
                l = nxt[0] / p
                cur = [nxt[1], nxt[2] - l * qE, nxt[3] - l * qA, nxt[4] - l * qg]
        lE, lA = wE / p, wA / p
        dEE, dEA, gE = dEE - lE * qE, dEA - lE * qA, gE - lE * qg
        dAE, dAA, gA = dAE - lA * qE, dAA - lA * qA, gA - lA * qg
        if k + 1 < nc:
            wE, wA = vE[k + 1] - lE * e, vA[k + 1] - lA * e
        rows.append((p, e, qE, qA, qg))
    if abs(dAE) > abs(dEE):
        dEE, dEA, dAE, dAA, gE, gA = dAE, dAA, dEE, dEA, gA, gE
    l = dAE / dEE
    xA = (gA - l * gE) / (dAA - l * dEA)
    xE = (gE - dEA * xA) / dEE
    x = [zero] * n
    x[0], x[1] = xE, xA
    xn = zero
    for k in range(nc - 1, -1, -1):
        p, e, qE, qA, qg = rows[k]
        xn = (qg - e * xn - qE * xE - qA * xA) / p
        x[ci[k]] = xn
    return np.array(x, dtype=np.float64) if isinstance(zero, float) else x


def accurate_solve(M, g):
    """LAPACK solve plus two steps of refinement with an extended-precision residual."""
    x = np.linalg.solve(M, g)
    for _ in range(2):
        r = g.astype(np.longdouble) - M.astype(np.longdouble) @ x.astype(np.longdouble)
        x = x + np.linalg.solve(M, r.astype(np.float64))
    return x


@pytest.mark.parametrize("nspec", [5, 7, 13])
def test_chain_matrix_has_the_bordered_band_structure(nspec):
    net = W.alpha_chain(nspec, np.random.default_rng(nspec))
    P = W.Problem(dim=1, n=(4, 1, 1), dx=(0.25, 1, 1), gamma=5 / 3, net=net)
    o = O.Oracle(P)
    rng = np.random.default_rng(1)
    X = rng.dirichlet(np.ones(nspec))
    w = np.concatenate([[1.0 / (P.gamma - 1)], X])
    _, J = o.rates(1.0, np.zeros(1), w)
    for a in range(nspec - 1):
        for b in range(nspec - 1):
            if b not in (a, a - 1):
                assert J[2 + a, 2 + b] == 0.0


@pytest.mark.parametrize("nspec", [5, 7, 13])
def test_chain_elimination_matches_pivoted_lu(nspec):
    """Stressed systems: density 0.1-10, T 0.3-3, dt_m 1e-8-1e2, negative alpha
    and product abundances down to -0.011, pseudo-transient shifts c = 1 + 1/h."""
    net = W.alpha_chain(nspec, np.random.default_rng(nspec))
    P = W.Problem(dim=1, n=(4, 1, 1), dx=(0.25, 1, 1), gamma=5 / 3, net=net)
    o = O.Oracle(P)
    rng = np.random.default_rng(7)
    worst_ratio = 0.0
    for _ in range(600):
        rho = 10 ** rng.uniform(-1, 1)
        T = rng.uniform(0.3, 3.0)
        X = rng.dirichlet(np.ones(nspec) * rng.uniform(0.1, 2))
        if rng.random() < 0.4:
            X[0] = rng.uniform(-0.011, 0.0)
        if rng.random() < 0.2:
            X[rng.integers(1, nspec)] = rng.uniform(-0.011, 0.0)
        w = np.concatenate([[rho * T / (P.gamma - 1)], rho * X])
        _, J = o.rates(rho, np.zeros(1), w)
        dtm = 10 ** rng.uniform(-8, 2)
        c = 1.0 if rng.random() < 0.7 else 1.0 + 10 ** rng.uniform(-3, 12)
        M = c * np.eye(nspec + 1) - dtm * J
        if not np.all(np.isfinite(M)):
            continue
        g = rng.standard_normal(nspec + 1) * np.concatenate([[w[0]], [rho] * nspec])
        xr = accurate_solve(M, g)
        scale = np.abs(xr).max()
        e_lu = max(np.abs(np.linalg.solve(M, g) - xr).max() / scale, 1e-16)
        e_ch = np.abs(chain_elimination(M, g) - xr).max() / scale
        assert np.isfinite(e_ch)
        # within the forward-error bound of a backward-stable solve, n cond(M) eps
        assert e_ch <= (nspec + 1) * np.linalg.cond(M) * 2.2e-16, (e_ch, e_lu)
        worst_ratio = max(worst_ratio, e_ch / e_lu)
    # and within a modest factor of LU's own error on every system
    assert worst_ratio < 1e4, worst_ratio


# ---- the same elimination in float pairs (double-float arithmetic in FP32)
F32 = np.float32


def _exact_prod(a, b):
    """p + e = a b exactly for floats a, b (their product is exact in FP64)."""
    p64 = np.float64(a) * np.float64(b)
    p = F32(p64)
    return p, F32(p64 - np.float64(p))


def _fma32(x, y, z):
    """x y + z rounded once to float (FP64 holds x y exactly)."""
    return F32(np.float64(x) * np.float64(y) + np.float64(z))


def _fast_two_sum(a, b):
    s = F32(a + b)
    return s, F32(b - F32(s - a))


def _two_sum(a, b):
    s = F32(a + b)
    bb = F32(s - a)
    return s, F32(F32(a - F32(s - bb)) + F32(b - bb))


class Pair:
    """hi + lo in two floats: Knuth's TwoSum, Dekker's Fast2Sum and the exact
    product (restated from those published definitions, not from the CUDA
    source)."""

    def __init__(self, hi, lo=0.0):
        self.hi, self.lo = F32(hi), F32(lo)

    @classmethod
    def of(cls, x):
        h = F32(x)
        return cls(h, F32(np.float64(x) - np.float64(h)))

    def value(self):
        return np.float64(self.hi) + np.float64(self.lo)

    def __neg__(self):
        return Pair(-self.hi, -self.lo)

    def __add__(self, o):
        s, e = _two_sum(self.hi, o.hi)
        return Pair(*_fast_two_sum(s, F32(e + F32(self.lo + o.lo))))

    def __sub__(self, o):
        return self + (-o)

    def __mul__(self, o):
        p, e = _exact_prod(self.hi, o.hi)
        e = _fma32(self.hi, o.lo, e)
        e = _fma32(self.lo, o.hi, e)
        return Pair(*_fast_two_sum(p, e))

    def inv(self):
        y = F32(1.0 / np.float64(self.hi))
        r = _fma32(-self.hi, y, F32(1.0))
        r = _fma32(-self.lo, y, r)
        return Pair(*_fast_two_sum(y, F32(y * _fma32(r, r, r))))

    def __truediv__(self, o):
        return self * o.inv()

    def __abs__(self):
        return abs(self.hi)

    def __gt__(self, o):
        return self.hi > o.hi


def chain_elimination_pairs(M, g):
    """chain_elimination with every entry, multiplier and sum a float pair."""
    n = M.shape[0]
    Mp = [[Pair.of(M[i, j]) for j in range(n)] for i in range(n)]
    gp = [Pair.of(v) for v in g]
    x = chain_elimination(np.array(Mp, dtype=object), gp, zero=Pair(0.0))
    return np.array([v.value() for v in x])


@pytest.mark.parametrize("nspec", [5, 7, 13])
def test_float_pair_elimination_is_accurate_to_about_2_pow_minus_44(nspec):
    """The float-pair Jacobian mode forms Newton's step by this elimination in
    double-float arithmetic on the FP32 pipe.  On the stressed systems of
    test_chain_elimination_matches_pivoted_lu (condition numbers up to 1e12)
    its forward error stays within n cond(M) 2^-44; typically it is a few tens
    of times the FP64 elimination's (2^-48 against 2^-53) and a million times
    below the FP32 elimination's, so for Newton's convergence test the step is
    as good as an FP64 one."""
    net = W.alpha_chain(nspec, np.random.default_rng(nspec))
    P = W.Problem(dim=1, n=(4, 1, 1), dx=(0.25, 1, 1), gamma=5 / 3, net=net)
    o = O.Oracle(P)
    rng = np.random.default_rng(11)
    e_pair, e_64, e_32 = [], [], []
    for _ in range(120):
        rho = 10 ** rng.uniform(-1, 1)
        T = rng.uniform(0.3, 3.0)
        X = rng.dirichlet(np.ones(nspec) * rng.uniform(0.1, 2))
        if rng.random() < 0.4:
            X[0] = rng.uniform(-0.011, 0.0)
        w = np.concatenate([[rho * T / (P.gamma - 1)], rho * X])
        _, J = o.rates(rho, np.zeros(1), w)
        dtm = 10 ** rng.uniform(-8, 2)
        c = 1.0 if rng.random() < 0.7 else 1.0 + 10 ** rng.uniform(-3, 6)
        M = c * np.eye(nspec + 1) - dtm * J
        if not np.all(np.isfinite(M)) or np.abs(M).max() > 1e30:
            continue
        g = rng.standard_normal(nspec + 1) * np.concatenate([[w[0]], [rho] * nspec])
        xr = accurate_solve(M, g)
        scale = np.abs(xr).max()
        ep = np.abs(chain_elimination_pairs(M, g) - xr).max() / scale
        assert ep <= (nspec + 1) * np.linalg.cond(M) * 2.0 ** -44, ep
        with np.errstate(all="ignore"):
            e32 = np.abs(chain_elimination(M.astype(F32), g.astype(F32)) - xr).max() / scale
        e_pair.append(ep)
        e_64.append(max(np.abs(chain_elimination(M, g) - xr).max() / scale, 2.0 ** -53))
        if np.isfinite(e32):
            e_32.append(e32)
    e_pair, e_64 = np.array(e_pair), np.array(e_64)
    assert np.median(e_pair / e_64) <= 64
    assert np.median(e_pair) <= 1e-6 * np.median(e_32)

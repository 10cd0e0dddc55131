"""Pins of the oracle's lattice tables and equilibria (Appendix B; Eqs. feq-3,
feq-4, macro).  Nothing here re-types the oracle's formulas: the tables are
checked against the Gauss-Hermite isotropy conditions and the paper's printed
weights, the equilibria against the moments of the Maxwellian they expand."""
import math
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def gauss_moment(n, mean=0.0, var=1.0):
    """E[X^n] for X ~ N(mean, var), by the binomial sum over central moments."""
    tot = 0.0
    for k in range(0, n + 1, 2):
        dfact = 1.0
        for j in range(k - 1, 0, -2):
            dfact *= j
        tot += math.comb(n, k) * mean ** (n - k) * var ** (k / 2) * dfact
    return tot


def class_of(c):
    a, b = sorted((abs(int(c[0])), abs(int(c[1]))), reverse=True)
    return (a, b)


@pytest.mark.parametrize("lat,q,M,degree", [("D2Q9", 9, 1, 5), ("D2Q37", 37, 3, 9),
                                            ("D2Q17", 17, 3, 7)])
def test_quadrature_isotropy(lat, q, M, degree):
    """sum_i w_i xi_x^a xi_y^b equals the standard-normal moments E[Z^a] E[Z^b]
    for every a + b <= degree (a Gauss-Hermite rule of that degree)."""
    L = oracle.lattice_info(lat)
    assert L["q"] == q and L["M"] == M
    assert np.abs(L["c"]).max() == M
    assert len({tuple(c) for c in L["c"]}) == q
    xi = L["c"] / math.sqrt(L["cs2"])
    worst = 0.0
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            got = np.sum(L["w"] * xi[:, 0] ** a * xi[:, 1] ** b)
            want = gauss_moment(a) * gauss_moment(b)
            worst = max(worst, abs(got - want) / max(1.0, abs(want)))
    assert worst < 2e-14, worst
    # one order beyond the rule must fail (the rule is not of higher degree)
    a = degree + 1 if (degree + 1) % 2 == 0 else degree + 2
    got = np.sum(L["w"] * xi[:, 0] ** a)
    assert abs(got - gauss_moment(a)) > 1e-3


def test_d2q37_weights_match_printed_table():
    """Appendix B, Tab. d2q37 prints the weights truncated to 14 decimals."""
    L = oracle.lattice_info("D2Q37")
    rows = np.loadtxt(os.path.join(GOLD, "d2q37_weights_printed.txt"))
    printed = {(int(r[0]), int(r[1])): r[2] for r in rows}
    counts = {}
    for c, w in zip(L["c"], L["w"]):
        k = class_of(c)
        assert abs(w - printed[k]) < 1e-14
        counts[k] = counts.get(k, 0) + 1
    assert counts == {(0, 0): 1, (1, 0): 4, (1, 1): 4, (2, 0): 4, (2, 1): 8,
                      (2, 2): 4, (3, 0): 4, (3, 1): 8}
    # The printed c_s formula of Tab. d2q37 evaluates to 0.8665..., which fails
    # the fourth-moment condition with the printed weights; the oracle's c_s
    # (0.835436...) satisfies it (checked above).
    printed_cs = math.sqrt(49 - (119 + (469 + 252 * math.sqrt(30)) ** (2 / 3))
                           / (469 + 252 * math.sqrt(30)) ** (1 / 3)) / 6
    xi = L["c"][:, 0] / printed_cs
    assert abs(np.sum(L["w"] * xi ** 4) - 3.0) > 0.1


def test_d2q17_weights_match_printed_table():
    """Appendix B, Tab. d2q17 prints the weights as closed forms.  Its printed
    c_s^2 = 5 (25 + sqrt 193) / 72 fails the second-moment condition with
    those weights; its reciprocal, which the oracle uses, satisfies it."""
    L = oracle.lattice_info("D2Q17")
    rows = np.loadtxt(os.path.join(GOLD, "d2q17_weights_printed.txt"))
    r = math.sqrt(193.0)
    printed = {(int(x[0]), int(x[1])): (x[2] + x[3] * r) / x[4] for x in rows}
    counts = {}
    for c, w in zip(L["c"], L["w"]):
        k = class_of(c)
        assert abs(w - printed[k]) < 1e-16
        counts[k] = counts.get(k, 0) + 1
    assert counts == {(0, 0): 1, (1, 0): 4, (1, 1): 4, (2, 2): 4, (3, 0): 4}
    printed_cs2 = 5.0 * (25.0 + r) / 72.0
    assert abs(np.sum(L["w"] * L["c"][:, 0] ** 2) - printed_cs2) > 1.0
    assert abs(L["cs2"] * printed_cs2 - 1.0) < 1e-15


def test_d2q9_weights_match_printed_table():
    L = oracle.lattice_info("D2Q9")
    rows = np.loadtxt(os.path.join(GOLD, "d2q9_weights_printed.txt"))
    printed = {(int(r[0]), int(r[1])): r[2] / r[3] for r in rows}
    for c, w in zip(L["c"], L["w"]):
        assert abs(w - printed[class_of(c)]) < 1e-16
    assert abs(L["cs2"] - 1.0 / 3.0) < 1e-16


def random_states(rng, n, thermal):
    out = []
    for _ in range(n):
        drho = rng.uniform(-0.2, 0.2)
        ux, uy = rng.uniform(-0.15, 0.15, 2)
        dT = rng.uniform(-0.1, 0.1) if thermal else 0.0
        out.append(np.array([drho, ux, uy, dT]))
    return out


@pytest.mark.parametrize("lat,order", [("D2Q9", 2), ("D2Q37", 4), ("D2Q17", 3)])
def test_equilibrium_reproduces_maxwellian_moments(lat, order):
    """Eq. feq-4 (D2Q37) / Eq. feq-3 (D2Q17) / the second-order isothermal
    expansion (D2Q9) must carry every velocity moment of the Maxwellian
    through its expansion order:
    sum f^eq xi_x^a xi_y^b = rho E[X^a] E[Y^b], X ~ N(u~_x, theta)."""
    L = oracle.lattice_info(lat)
    thermal = lat != "D2Q9"
    xi = L["c"] / math.sqrt(L["cs2"])
    rng = np.random.default_rng(1)
    rho0 = 1.0
    for U in random_states(rng, 20, thermal):
        f = oracle.feq(lat, rho0, U) + L["w"] * rho0
        rho = rho0 + U[0]
        th = 1.0 + U[3]
        ut = U[1:3] / math.sqrt(L["cs2"])
        for a in range(order + 1):
            for b in range(order + 1 - a):
                got = np.sum(f * xi[:, 0] ** a * xi[:, 1] ** b)
                want = rho * gauss_moment(a, ut[0], th) * gauss_moment(b, ut[1], th)
                assert abs(got - want) < 1e-13 * max(1.0, abs(want)), (a, b, got, want)


def test_fourth_order_misprint_breaks_mass():
    """The coefficient printed in Eq. feq-4 for the (u.c)^2 (T-1) term,
    (c^2 - 4), does not conserve mass; the oracle's reading (xi^2 - 6) does.
    The difference between the two readings is 6 (T-1)(u.c)^2 * 2/24 w rho;
    its zeroth moment must be non-zero, so the printed form is excluded."""
    L = oracle.lattice_info("D2Q37")
    xi = L["c"] / math.sqrt(L["cs2"])
    U = np.array([0.1, 0.13 * math.sqrt(L["cs2"]), -0.07 * math.sqrt(L["cs2"]), 0.05])
    g = oracle.feq("D2Q37", 1.0, U)
    assert abs(np.sum(g) - U[0]) < 1e-15
    xu = xi @ (U[1:3] / math.sqrt(L["cs2"]))
    delta = L["w"] * (1.0 + U[0]) * (6.0 * U[3] * xu ** 2 * 2.0) / 24.0
    assert abs(np.sum(delta)) > 1e-4


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q37", "D2Q17"])
def test_moments_invert_equilibrium(lat):
    """U(f^eq(U)) = U (Eq. macro applied to Eqs. feq-3/4)."""
    rng = np.random.default_rng(2)
    for U in random_states(rng, 30, lat != "D2Q9"):
        got = oracle.moments(lat, 1.0, oracle.feq(lat, 1.0, U))
        assert np.allclose(got, U, rtol=0, atol=2e-15), (got, U)


@pytest.mark.parametrize("lat", ["D2Q37", "D2Q17"])
def test_equilibrium_heat_flux_vanishes(lat):
    """The central third moment of f^eq is zero on D2Q37 and D2Q17 (the
    oracle computes the heat flux of Eq. heatflux from f - f^eq on that
    basis)."""
    L = oracle.lattice_info(lat)
    rng = np.random.default_rng(3)
    for U in random_states(rng, 10, True):
        f = oracle.feq(lat, 1.0, U) + L["w"]
        e = L["c"] - U[1:3]
        q = 0.5 * np.sum(f[:, None] * (e ** 2).sum(1)[:, None] * e, axis=0)
        assert np.abs(q).max() < 1e-14

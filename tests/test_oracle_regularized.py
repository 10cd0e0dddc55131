"""Pins of the regularised non-equilibrium Dirichlet condition (the Hermite
projection of f^neq(x_f), a scheme the paper names for future work).  The
checks are properties of an orthogonal projection, computed here from the
lattice tables, not from the oracle's formula."""
import math

import numpy as np
import pytest

import oracle
import lbm_workloads as W


def hermite_moments(L, g, order):
    """a2 = sum H2 g (xx, xy, yy) and a3 = sum H3 g (xxx, xxy, xyy, yyy)."""
    c = L["c"].astype(float)
    cs2 = L["cs2"]
    cx, cy = c[:, 0], c[:, 1]
    H = [cx * cx - cs2, cx * cy, cy * cy - cs2]
    if order >= 3:
        H += [cx ** 3 - 3 * cs2 * cx, cx * cx * cy - cs2 * cy, cx * cy * cy - cs2 * cx,
              cy ** 3 - 3 * cs2 * cy]
    return np.array([np.sum(h * g) for h in H])


def random_neq(L, rng, thermal):
    """A random vector with no mass, momentum (and, thermal, energy)."""
    q = L["q"]
    c = L["c"].astype(float)
    g = rng.normal(size=q) * L["w"]
    cons = [np.ones(q), c[:, 0], c[:, 1]] + ([(c ** 2).sum(1)] if thermal else [])
    A = np.array(cons)
    # remove the conserved components in the w-weighted sense
    Wm = np.diag(L["w"])
    coef = np.linalg.solve(A @ Wm @ A.T, A @ g)
    return g - Wm @ A.T @ coef


ORDERS = {"D2Q9": 2, "D2Q17": 3, "D2Q37": 3}


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q17", "D2Q37"])
def test_projection_keeps_hermite_moments_and_conserved_zero(lat):
    L = oracle.lattice_info(lat)
    rng = np.random.default_rng(5)
    order = ORDERS[lat]
    c = L["c"].astype(float)
    for _ in range(10):
        g = random_neq(L, rng, lat != "D2Q9")
        r = oracle.regularize(lat, g)
        scale = np.abs(g).max()
        assert np.allclose(hermite_moments(L, r, order), hermite_moments(L, g, order), atol=1e-14 * scale)
        assert abs(r.sum()) < 1e-15 * scale * L["q"]
        assert np.abs(c.T @ r).max() < 1e-14 * scale * L["q"]


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q17", "D2Q37"])
def test_projection_is_idempotent_and_keeps_hermite_polynomials(lat):
    L = oracle.lattice_info(lat)
    rng = np.random.default_rng(6)
    g = random_neq(L, rng, lat != "D2Q9")
    r = oracle.regularize(lat, g)
    assert np.allclose(oracle.regularize(lat, r), r, rtol=0, atol=1e-15 * np.abs(r).max())
    # a pure second-order Hermite polynomial w_i H2_i : A is returned unchanged
    c = L["c"].astype(float)
    cs2 = L["cs2"]
    A = np.array([[0.3, -0.2], [-0.2, 0.7]])
    H2A = A[0, 0] * (c[:, 0] ** 2 - cs2) + 2 * A[0, 1] * c[:, 0] * c[:, 1] + A[1, 1] * (c[:, 1] ** 2 - cs2)
    p = L["w"] * H2A
    assert np.allclose(oracle.regularize(lat, p), p, rtol=0, atol=1e-15)


def test_projection_drops_what_the_hermite_basis_does_not_carry():
    """On D2Q37 a generic non-equilibrium vector has higher-order content:
    the projection removes it, so the result differs from the input."""
    L = oracle.lattice_info("D2Q37")
    g = random_neq(L, np.random.default_rng(7), True)
    r = oracle.regularize("D2Q37", g)
    assert np.abs(r - g).max() > 0.1 * np.abs(g).max()


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q17", "D2Q37"])
def test_regularised_dirichlet_keeps_targets_and_uniform_states(lat):
    """The regularised write, like NEEP, adds no mass or momentum: boundary
    layers carry the target macros, and a uniform moving state stays."""
    n = 2 * W.M_OF[lat] + 8
    T = 1.01 if lat != "D2Q9" else 1.0
    P = W.CS2[lat] * 1.02 * T
    cfg = W.run(lat, n, n + 1, 0.7, sides=("cbc",) * 4, schemes=("cbc_relax",) * 4,
                dirichlet="reg", alpha_T=0.3, beta_P=0.4, p_inf=[P] * 4)
    s = oracle.Sim(cfg).init(*W.uniform(n, n + 1, 1.02, 0.03, -0.015, T))
    s.step(30)
    for got, want in zip(s.macros(), (1.02, 0.03, -0.015, T)):
        assert np.abs(got - want).max() < 5e-15

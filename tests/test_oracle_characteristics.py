"""Pins of the oracle's characteristic analysis (Sec. 3.1-3.2) and RK4 (Sec. 3.3).

The normal-flux matrix A is derived here from the Euler equations in
primitive variables (continuity, momentum with P = rho c_s^2 T, and energy
with c_v = 1), not copied from the oracle.  Left eigenvectors come from
numpy, so each check is independent of the oracle's S and S^-1."""
import math

import numpy as np
import pytest

import oracle
from lbm_workloads import CS2


def euler_A(lat, Ul, rho0=1.0):
    """d/dt U = -A dU/dn + ... for U = (rho, u_n, u_t, T) (thermal) or
    (rho, u_n, u_t) (isothermal), from
      rho_t + u rho_n + rho u_n,n = 0
      u_t + u u_n + (1/rho) P_n = 0,  P = c_s^2 rho T
      v_t + u v_n = 0
      rho c_v (T~_t + u T~_n) = -P u_n,n  with T~ = c_s^2 T, c_v = 1."""
    cs2 = CS2[lat]
    rho, un = rho0 + Ul[0], Ul[1]
    if lat != "D2Q9":
        T = 1.0 + Ul[3]
        return np.array([[un, rho, 0, 0],
                         [cs2 * T / rho, un, 0, cs2],
                         [0, 0, un, 0],
                         [0, T, 0, un]], dtype=float)
    return np.array([[un, rho, 0], [cs2 / rho, un, 0], [0, 0, un]], dtype=float)


def rand_local(rng, lat):
    return np.array([rng.uniform(-0.2, 0.2), rng.uniform(-0.3, 0.3),
                     rng.uniform(-0.3, 0.3), rng.uniform(-0.1, 0.1) if lat != "D2Q9" else 0.0])


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q37", "D2Q17"])
def test_S_diagonalises_A(lat):
    rng = np.random.default_rng(4)
    for _ in range(25):
        Ul = rand_local(rng, lat)
        S, Si, lam = oracle.char_matrices(lat, 1.0, Ul)
        A = euler_A(lat, Ul)
        n = A.shape[0]
        assert np.abs(S @ Si - np.eye(n)).max() < 1e-14
        assert np.abs(S @ A - np.diag(lam) @ S).max() < 1e-14
        assert np.allclose(np.sort(lam), np.sort(np.linalg.eigvals(A).real), atol=1e-14)


def test_sound_speed_is_sqrt_2_T():
    """Lambda_33/44 = u_n -+ sqrt(2 T~) (Sec. 3.1; gamma = c_p/c_v = 2)."""
    cs2 = CS2["D2Q37"]
    S, Si, lam = oracle.char_matrices("D2Q37", 1.0, [0.0, 0.0, 0.0, 0.0])
    assert abs(lam[3] - math.sqrt(2 * cs2)) < 1e-15 and abs(lam[2] + math.sqrt(2 * cs2)) < 1e-15


def left_eigs(A):
    w, V = np.linalg.eig(A.T)
    return w.real, V.real.T        # rows: left eigenvectors l_i, l_i A = w_i l_i


def cfg_for(lat, **kw):
    d = dict(lattice=lat, nx=16, ny=16, tau=0.8, rho0=1.0, alpha_T=0.0, beta_P=0.0, t_inf=0.0)
    d.update(kw)
    return d


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q37", "D2Q17"])
@pytest.mark.parametrize("scheme", ["lodi", "lodi_relax", "cbc", "cbc_relax"])
@pytest.mark.parametrize("alpha_V", [0.0, 0.6])
def test_char_rhs_projections(lat, scheme, alpha_V):
    """Eqs. PNR / LODI-Relax / CBC-PNR / CBC-Relax seen through independent
    left eigenvectors l_i of A:
      outgoing i:  l_i.k = -lambda_i l_i.dU_n + [CBC] l_i.(T + V)
      incoming i:  l_i.k = [LODI] 0, [CBC] 0,
                           [RELAX, alpha=1, T_inf=0] l_i.T  (+ beta dP term)
                           + [CBC-RELAX] alpha_V l_i.V: the viscous term
                           relaxed towards 0 at rate alpha_V in the incoming
                           amplitude (0: the paper's equation) leaves that
                           share of V in the incoming characteristic."""
    rng = np.random.default_rng(5)
    n = 3 if lat == "D2Q9" else 4
    alpha = 1.0 if scheme.endswith("relax") else 0.0
    cfg = cfg_for(lat, alpha_T=alpha, beta_P=0.0, alpha_V=alpha_V)
    cbc = scheme.startswith("cbc")
    for trial in range(30):
        Ul = rand_local(rng, lat)
        dUn = rng.normal(size=4) * 1e-3
        TT = rng.normal(size=4) * 1e-3
        VV = rng.normal(size=4) * 1e-3
        if n == 3:
            dUn[3] = TT[3] = VV[3] = 0.0
        mask = int(rng.integers(0, 1 << n))
        S, Si, lam = oracle.char_matrices(lat, 1.0, Ul)
        # the mask addresses the oracle's wave order; translate to eigenvalues
        incoming_vals = [lam[i] for i in range(n) if mask >> i & 1]
        outgoing_vals = [lam[i] for i in range(n) if not mask >> i & 1]
        # degenerate pair (u_n twice): only masks treating both alike are meaningful
        if lat != "D2Q9" and ((mask >> 0) & 1) != ((mask >> 1) & 1):
            continue
        k = oracle.char_rhs(cfg, Ul, dUn, TT, VV, mask, 0.0, scheme)[:n]
        A = euler_A(lat, Ul)
        w, Lv = left_eigs(A)
        for wi, li in zip(w, Lv):
            if any(abs(wi - v) < 1e-12 for v in incoming_vals):
                want = 0.0
                if alpha == 1.0:
                    want = li @ TT[:n]
                if scheme == "cbc_relax":
                    want += alpha_V * (li @ VV[:n])
            else:
                assert any(abs(wi - v) < 1e-12 for v in outgoing_vals)
                want = -wi * (li @ dUn[:n]) + ((li @ (TT[:n] + VV[:n])) if cbc else 0.0)
            assert abs(li @ k - want) < 1e-15 + 1e-12 * np.abs(li).max() * 1e-3, (trial, wi)


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q37", "D2Q17"])
def test_all_outgoing_is_normal_euler_flux(lat):
    """With no incoming wave, LODI gives dU/dt = -A dU/dn and CBC adds T + V."""
    rng = np.random.default_rng(6)
    n = 3 if lat == "D2Q9" else 4
    for _ in range(10):
        Ul = rand_local(rng, lat)
        dUn, TT, VV = (rng.normal(size=4) * 1e-3 for _ in range(3))
        if n == 3:
            dUn[3] = TT[3] = VV[3] = 0
        A = euler_A(lat, Ul)
        k = oracle.char_rhs(cfg_for(lat), Ul, dUn, TT, VV, 0, 0.0, "lodi")[:n]
        assert np.abs(k + A @ dUn[:n]).max() < 1e-16
        k = oracle.char_rhs(cfg_for(lat), Ul, dUn, TT, VV, 0, 0.0, "cbc")[:n]
        assert np.abs(k + A @ dUn[:n] - TT[:n] - VV[:n]).max() < 1e-16


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q37", "D2Q17"])
def test_pressure_relaxation_restores(lat):
    """beta (Z - Z_inf) on the incoming acoustic wave pulls P back to P_inf:
    with P > P_inf and nothing else, dP/dt < 0 (Eq. LODI-Relax)."""
    cs2 = CS2[lat]
    Ul = np.array([0.0, 0.05, 0.0, 0.0])
    S, Si, lam = oracle.char_matrices(lat, 1.0, Ul)
    mask = sum(1 << i for i in range(len(lam)) if lam[i] < 0)
    z = np.zeros(4)
    k = oracle.char_rhs(cfg_for(lat, beta_P=0.5), Ul, z, z, z, mask, 1e-3, "lodi_relax")
    rho, T = 1.0 + Ul[0], 1.0 + Ul[3]
    dP = cs2 * (k[0] * T + rho * k[3]) if lat == "D2Q37" else cs2 * k[0]
    assert dP < 0 and k[0] < 0


def test_rk4_is_classical_fourth_order():
    """One step on y' = lam y multiplies by 1 + z + z^2/2 + z^3/6 + z^4/24
    (z = lam h), and the global error at t = 1 falls as h^4."""
    for z in (-0.3, -1.0, 0.25):
        got = oracle.rk4_scalar(z, 1.0, 1.0, 1)
        assert abs(got - (1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24)) < 1e-15
    e1 = abs(oracle.rk4_scalar(-2.0, 1.0, 0.1, 10) - math.exp(-2.0))
    e2 = abs(oracle.rk4_scalar(-2.0, 1.0, 0.05, 20) - math.exp(-2.0))
    assert 14.0 < e1 / e2 < 18.0


def _corner_frame(cid):
    """Outward diagonal n of corner cid (0 SW, 1 SE, 2 NW, 3 NE) and t = n
    turned by +90 degrees."""
    sx = 1.0 if cid & 1 else -1.0
    sy = 1.0 if cid & 2 else -1.0
    n = np.array([sx, sy]) / math.sqrt(2.0)
    return n, np.array([-n[1], n[0]]), np.array([sx, sy])


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q37", "D2Q17"])
@pytest.mark.parametrize("cid", [0, 1, 2, 3])
def test_corner_lodi_along_the_diagonal(lat, cid):
    """Sec. 3.3 / Fig. Layer-Multispeed-BC: the corner node takes LODI
    (Eq. PNR) along the outward diagonal, with the normal derivative by the
    one-sided Eq. FD-dx-bw through the node and the two diagonal nodes inward
    (spacing sqrt(2)).  On a field linear in space (exact for that
    difference) the right-hand side must be dU/dt = -A_out dU/dn, A_out the
    outgoing part of the Euler flux matrix along n (numpy eigenvectors): a
    spacing of 1, a sign flip or the inward diagonal all fail."""
    rng = np.random.default_rng(40 + cid)
    cs2 = CS2[lat]
    n, t, s = _corner_frame(cid)
    cfg = cfg_for(lat)
    for _ in range(6):
        # lab state at the corner node and a small lab-frame gradient G (4 x 2)
        U = np.array([rng.uniform(-0.05, 0.05), rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2),
                      rng.uniform(-0.05, 0.05) if lat != "D2Q9" else 0.0])
        G = 1e-3 * rng.standard_normal((4, 2))
        if lat == "D2Q9":
            G[3] = 0.0
        U1, U2 = U - G @ s, U - 2.0 * G @ s
        k = oracle.corner_rhs(cfg, cid, U, U1, U2)
        # expected, from the local frame (rho, u_n, u_t, T)
        Ul = np.array([U[0], U[1:3] @ n, U[1:3] @ t, U[3]])
        dlab = G @ n                                   # d/dn of the lab components
        dUn = np.array([dlab[0], dlab[1:3] @ n, dlab[1:3] @ t, dlab[3]])
        A = euler_A(lat, Ul)
        m = A.shape[0]
        w, R = np.linalg.eig(A)
        w, R = w.real, R.real
        Lm = np.linalg.inv(R)
        Aout = R @ np.diag(np.where(w >= 0.0, w, 0.0)) @ Lm
        kl = np.zeros(4)
        kl[:m] = -Aout @ dUn[:m]
        want = np.array([kl[0], kl[1] * n[0] + kl[2] * t[0], kl[1] * n[1] + kl[2] * t[1], kl[3]])
        scale = np.abs(want).max()
        assert np.abs(k - want).max() <= 1e-12 * scale + 1e-18, (k, want)
        # the same corner with unit spacing would be sqrt(2) off
        assert np.abs(k * math.sqrt(2.0) - want).max() > 1e-3 * scale

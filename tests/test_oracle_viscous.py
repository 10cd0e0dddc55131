"""Pins of the mesoscopic viscous terms on the paper's own benchmark.

Sec. 3.3 ("Evaluation of viscous terms") evaluates the viscous vector from
the non-equilibrium moments of Eqs. LaplaceU / LaplaceT with one-sided
normal differences next to the boundary, and Sec. 4.2 ("Treatment of
viscous terms") reports that, on the thermal vortex carried out through a
CBC-RELAX outlet, this mesoscopic form is stable at every viscosity tried
and at least as accurate as the "-FD" form, which becomes unstable at
nu = 0.3.  The oracle starts the one-sided stencil M nodes below x_f, at
the first node none of whose populations was streamed from a boundary
layer; read literally at x_f, the moments there mix in the populations the
equilibrium Dirichlet condition wrote into the layers, and an odd-even mode
along the outlet grows from the corners until the run leaves finite values.
These tests hold the oracle to the paper's statements."""
import math

import numpy as np
import pytest

import lbm_workloads as W
import oracle

L = 150          # Sec. 4.2: 150 x 150, Ma = 0.1, alpha = Ma, beta = 0, T_inf = 0
MA = 0.1
LAT = "D2Q17"
EVERY = 50


def _tau(nu):
    return 0.5 + nu / W.CS2[LAT]


def _vortex_cfg(nu, viscous, meso_depth=-1, outlet="cbc_relax"):
    cfg = W.run(LAT, L, L, _tau(nu), sides=("cbc",) * 4, schemes=("lodi", outlet, "lodi", "lodi"),
                viscous=viscous, alpha_T=MA, beta_P=0.0, t_inf=0.0)
    cfg["meso_depth"] = meso_depth
    return cfg


def _fields():
    return W.thermal_vortex(L, L, LAT, Ma=MA)


def _run(cfg, steps, ref=None):
    """Step `steps` steps; return (max |rho - 1| over the last E-side
    columns per block of EVERY steps, e_Z (Eq. errors) per block against ref
    crops when given)."""
    s = oracle.Sim(cfg).init(*_fields())
    edge, errs = [], []
    for k in range(steps // EVERY):
        s.step(EVERY)
        rho, ux, uy, T = s.macros()
        edge.append(float(np.max(np.abs(rho[:, -6:] - 1.0))))
        if ref is not None:
            r = ref[k]
            errs.append([math.sqrt(float(np.sum(((z - rz) / rz) ** 2)))
                         for z, rz in ((rho, r[0]), (ux, r[1]), (T, r[3]))])
    return np.array(edge), np.array(errs)


@pytest.fixture(scope="module")
def reference_nu01():
    """Crops of a periodic run large enough that no periodic image re-enters
    the 150 x 150 window within 1000 steps (Sec. 4: fully periodic reference
    on an extended grid)."""
    steps = 1000
    c = math.sqrt(2.0 * W.CS2[LAT]) + MA * math.sqrt(W.CS2[LAT])
    n = L + int(c * steps) + 20
    o = (n - L) // 2
    cfg = W.run(LAT, n, n, _tau(0.1))
    s = oracle.Sim(cfg).init(*W.thermal_vortex(n, L, LAT, Ma=MA, offset=o))
    crops = []
    for _ in range(steps // EVERY):
        s.step(EVERY)
        m = s.macros()
        crops.append([a[o:o + L, o:o + L].copy() for a in m])
    return crops


def test_mesoscopic_cbc_relax_beats_fd_on_the_vortex(reference_nu01):
    """nu = 0.1, 1000 steps: the mesoscopic form stays finite and its mean
    e_rho, e_ux and e_T are below those of the -FD form (Sec. 4.2: the
    mesoscopic Laplacian follows the ground truth closely, -FD departs)."""
    edge_m, e_m = _run(_vortex_cfg(0.1, "meso"), 1000, reference_nu01)
    edge_f, e_f = _run(_vortex_cfg(0.1, "fd"), 1000, reference_nu01)
    assert np.all(np.isfinite(e_m)) and np.all(np.isfinite(e_f))
    assert edge_m.max() < 2e-3, edge_m.max()
    mean_m, mean_f = e_m.mean(axis=0), e_f.mean(axis=0)
    assert np.all(mean_m < mean_f), (mean_m, mean_f)
    # and both improve on plain LODI at the outlet (Fig. L2-Vortex)
    _, e_l = _run(_vortex_cfg(0.1, "meso", outlet="lodi"), 1000, reference_nu01)
    assert mean_m[0] < e_l.mean(axis=0)[0]


def test_literal_x_f_stencil_grows_on_the_vortex():
    """The same run with the stencil at x_f itself: an odd-even mode along
    the outlet grows (max |rho - 1| at the outlet passes 1e-2 within 1000
    steps, from 1e-3), while the stencil M nodes deeper stays below 2e-3."""
    s = oracle.Sim(_vortex_cfg(0.1, "meso", meso_depth=0)).init(*_fields())
    s.step(700)
    # the growing mode alternates in sign along the outlet, next to the
    # south-east corner where it starts
    d = s.macros()[0][4:16, L - 1] - 1.0
    flips = np.mean(np.sign(d[1:]) != np.sign(d[:-1]))
    assert flips > 0.8, (flips, d)
    s.step(300)
    edge_lit = np.max(np.abs(s.macros()[0][:, -6:] - 1.0))
    assert not (edge_lit < 1e-2), edge_lit
    edge_adj, _ = _run(_vortex_cfg(0.1, "meso"), 1000)
    assert edge_adj.max() < 2e-3, edge_adj


def test_fd_fails_at_nu_03_where_mesoscopic_holds():
    """Sec. 4.2: the -FD form becomes unstable at nu = 0.3; the mesoscopic
    form stays finite and bounded there."""
    edge_f, _ = _run(_vortex_cfg(0.3, "fd"), 300)
    assert not np.all(np.isfinite(edge_f)) or edge_f[-1] > 1.0, edge_f
    edge_m, _ = _run(_vortex_cfg(0.3, "meso"), 1000)
    assert np.all(np.isfinite(edge_m)) and edge_m.max() < 2e-3, edge_m


def test_viscous_heating_of_a_shear_wave():
    """The viscous-heating part of the fourth component of the viscous
    vector (Sec. 3.1: (nu / c_s^2) ((d_x u_x - d_y u_y)^2 + (d_y u_x +
    d_x u_y)^2), with the velocity derivatives by the stencil's differences)
    on a plane shear wave u_y = A sin(k x): averaged over a wavelength, where
    the heat-flux divergence of the other part of V_4 sums to zero,
    V_4 = (nu / c_s^2) (A k)^2 / 2; its cos(2 k x) component carries the same
    amplitude less what conduction has smoothed; both quadratic in A."""
    lat, n, tau = "D2Q37", 48, 0.8
    cs2 = W.CS2[lat]
    nu = (tau - 0.5) * cs2
    k = 2.0 * math.pi / n
    x = np.arange(n)

    def V4_modes(A):
        cfg = W.run(lat, n, n, tau)
        s = oracle.Sim(cfg).init(*W.shear_wave(n, n, A, k_axis="x"))
        s.step(10)
        amp = np.abs(s.macros()[2][5]).max()
        V4 = np.array([s.vis_meso_at(1, xx, 5)[3] for xx in x])
        return V4.mean(), 2.0 * np.mean(V4 * np.cos(2.0 * k * x)), amp

    mean, c2, amp = V4_modes(0.02)
    heat = nu / cs2 * (amp * k) ** 2 / 2.0
    assert abs(mean - heat) < 0.03 * heat, (mean, heat)
    assert 0.8 * heat < c2 < 1.0 * heat, (c2, heat)
    mean2, _, amp2 = V4_modes(0.04)
    assert abs(mean2 / mean - (amp2 / amp) ** 2) < 0.03 * (amp2 / amp) ** 2

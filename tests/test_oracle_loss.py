"""The pressure loss of the relaxation-parameter gradients and its FP64
finite-difference gradient, on the oracle: closed forms for the sum itself
(region, step count, reference), and second-order convergence of the
central differences."""
import numpy as np

import lbm_workloads as W
import oracle


def _pulse(lat="D2Q37", n=32, m=24, u=(0.04, 0.03)):
    """A pulse carried by a mean flow oblique to every side: |u_n| >= 0.03
    on the sides and corners keeps every wave on one side of the
    incoming/outgoing switch (at rest the switch makes the loss only
    piecewise smooth in the parameters: Sec. 3.2 classifies the waves by
    the sign of Lambda)."""
    cs2 = W.CS2[lat]
    cfg = W.run(lat, n, m, 0.8, sides=("cbc",) * 4, schemes=("cbc_relax",) * 4, viscous="off",
                alpha_T=0.5, beta_P=0.3, p_inf=[cs2 * 1.0002] * 4)
    f = list(W.gaussian_pulse(n, m, 1e-3, 1e-3 if lat != "D2Q9" else 0.0, 3.0, center=(15.3, 11.6)))
    f[1] = f[1] + u[0]
    f[2] = f[2] + u[1]
    return cfg, tuple(f)


def test_loss_of_a_state_at_rest_is_the_reference_offset():
    """Uniform state at rest with P_inf = c_s^2 rho0 stays uniform, so
    J = steps x (nodes off the layers) x c^2 for a constant reference c."""
    for lat in ("D2Q9", "D2Q37"):
        n, m, steps = 20, 16, 7
        cfg = W.run(lat, n, m, 0.7, sides=("cbc",) * 4, schemes=("cbc_relax",) * 4, viscous="off",
                    alpha_T=0.4, beta_P=0.2)
        f = W.uniform(n, m)
        M = W.M_OF[lat]
        assert oracle.pressure_loss(cfg, f, steps) == 0.0
        c = 3e-4
        ref = np.full((steps, m, n), c)
        J = oracle.pressure_loss(cfg, f, steps, ref)
        assert abs(J - steps * (n - 2 * M) * (m - 2 * M) * c * c) <= 1e-15 * J
    # a periodic axis keeps all its rows
    cfg = W.run("D2Q37", 20, 16, 0.7, sides=("cbc", "cbc", "periodic", "periodic"),
                schemes=("cbc_relax",) * 4, viscous="off")
    J = oracle.pressure_loss(cfg, W.uniform(20, 16), 3, np.full((3, 16, 20), c))
    assert abs(J - 3 * (20 - 6) * 16 * c * c) <= 1e-15 * J


def test_loss_against_its_own_run_is_zero():
    cfg, f = _pulse()
    info = oracle.lattice_info("D2Q37")
    s = oracle.Sim(cfg).init(*f)
    ref = []
    for _ in range(12):
        s.step(1)
        rho, ux, uy, T = s.macros()
        dr = rho - 1.0
        ref.append(info["cs2"] * (dr + (T - 1.0) + dr * (T - 1.0)))
    assert oracle.pressure_loss(cfg, f, 12, np.array(ref)) == 0.0
    assert oracle.pressure_loss(cfg, f, 12) > 0.0


def test_central_differences_converge_at_second_order():
    """Dividing h by 10 divides the change of the central differences by
    about 100: the loss is smooth in the three parameters here."""
    cfg, f = _pulse()
    steps = 60
    cs2 = W.CS2["D2Q37"]
    g = [oracle.pressure_loss_fd_gradient(cfg, f, steps, (h, h, h * cs2)) for h in (1e-3, 1e-4, 1e-5)]
    for k in range(3):
        a, b, c = g[0][k], g[1][k], g[2][k]
        assert c != 0.0
        assert abs(b - c) <= 1e-3 * abs(c), g
    # P_inf has the largest curvature: the ratio of successive changes is
    # the order of the scheme (2) over a factor 10 in h
    d1, d2 = abs(g[0][2] - g[1][2]), abs(g[1][2] - g[2][2])
    assert 30.0 < d1 / d2 < 300.0, (d1, d2)

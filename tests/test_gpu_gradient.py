"""Gradients of the pressure loss with respect to the relaxation parameters
(alpha_T, beta_P, P_inf, alpha_V, t_inf) by tangent-linear steps on the
GPU, against the FP64 oracle: its loss, and its central differences."""
import numpy as np
import pytest

import lbm_workloads as W
import oracle

pytestmark = pytest.mark.gpu


def lbm():
    import paper_2307_16766_gb300 as m
    return m


def _case(lat="D2Q37", n=32, m=24, u=(0.04, 0.03), sides=("cbc",) * 4):
    """A pulse carried by a mean flow oblique to every side, so that no wave
    changes between incoming and outgoing (the loss is smooth there)."""
    cs2 = W.CS2[lat]
    cfg = W.run(lat, n, m, 0.8, sides=sides, schemes=("cbc_relax",) * 4, viscous="off",
                alpha_T=0.5, beta_P=0.3, p_inf=[cs2 * 1.0002] * 4)
    f = list(W.gaussian_pulse(n, m, 1e-3, 1e-3 if lat != "D2Q9" else 0.0, 3.0,
                              center=(n / 2 - 0.7, m / 2 - 0.4)))
    f[1] = f[1] + u[0]
    f[2] = f[2] + u[1]
    return cfg, tuple(f)


def _loss_by_steps(cfg, f, steps):
    """The same loss from ordinary steps and the macros after each."""
    m = lbm()
    cs2, M = W.CS2[cfg["lattice"]], W.M_OF[cfg["lattice"]]
    sim = m.Simulation(cfg).init_fields(*f)
    J = 0.0
    for _ in range(steps):
        sim.step(1)
        rho, ux, uy, T = sim.macros()
        dr = rho - 1.0
        dP = cs2 * (dr + (T - 1.0) + dr * (T - 1.0)) if cfg["lattice"] != "D2Q9" else cs2 * dr
        ys = slice(0, cfg["ny"]) if cfg["sides"][2] == "periodic" else slice(M, cfg["ny"] - M)
        xs = slice(0, cfg["nx"]) if cfg["sides"][0] == "periodic" else slice(M, cfg["nx"] - M)
        J += float(np.sum(dP[ys, xs] ** 2))
    sim.close()
    return J


@pytest.mark.parametrize("storage,tol", [("f64", 1e-10), ("f32", 1e-4)])
@pytest.mark.parametrize("viscous", ["off", "fd", "meso"])
def test_tangent_steps_carry_the_ordinary_step(storage, tol, viscous):
    cfg, f = _case()
    c = dict(cfg, storage=storage, viscous=viscous, alpha_V=0.3)
    J, _ = lbm().pressure_loss_and_gradient(c, f, 60)
    Js = _loss_by_steps(c, f, 60)
    assert abs(J - Js) <= tol * Js, (J, Js)


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q17", "D2Q37"])
def test_gradient_matches_oracle_central_differences(lat):
    cfg, f = _case(lat)
    steps = 60
    cs2 = W.CS2[lat]
    J, dJ = lbm().pressure_loss_and_gradient(dict(cfg, storage="f64"), f, steps)
    Jo = oracle.pressure_loss(cfg, f, steps)
    assert abs(J - Jo) <= 1e-10 * Jo, (J, Jo)
    fd = oracle.pressure_loss_fd_gradient(cfg, f, steps, (1e-4, 1e-4, 1e-4 * cs2))
    for k in range(3):
        assert abs(dJ[k] - fd[k]) <= 1e-4 * abs(fd[k]), (k, dJ, fd)


def test_gradient_on_periodic_sides_with_a_reference_field():
    """Characteristic W/E sides, periodic S/N, a seeded reference pressure
    field per step: loss and gradient against the oracle's."""
    import torch
    cfg, f = _case("D2Q37", 40, 20, u=(0.05, 0.0), sides=("cbc", "cbc", "periodic", "periodic"))
    steps = 50
    rng = np.random.default_rng(3)
    ref = 1e-5 * rng.standard_normal((steps, 20, 40))
    J, dJ = lbm().pressure_loss_and_gradient(dict(cfg, storage="f64"), f, steps,
                                             torch.tensor(ref, device="cuda"))
    Jo = oracle.pressure_loss(cfg, f, steps, ref)
    assert abs(J - Jo) <= 1e-10 * Jo
    fd = oracle.pressure_loss_fd_gradient(cfg, f, steps, (1e-4, 1e-4, 1e-4 * W.CS2["D2Q37"]), ref)
    for k in range(3):
        assert abs(dJ[k] - fd[k]) <= 1e-4 * abs(fd[k]), (k, dJ, fd)


def test_fp32_gradient_against_fp64(capsys):
    cfg, f = _case()
    _, g64 = lbm().pressure_loss_and_gradient(dict(cfg, storage="f64"), f, 60)
    _, g32 = lbm().pressure_loss_and_gradient(dict(cfg, storage="f32"), f, 60)
    rel = [abs(a - b) / abs(b) for a, b in zip(g32, g64)]
    with capsys.disabled():
        print("\nFP32 storage gradient vs FP64, rel. errors (alpha_T, beta_P, P_inf):",
              ["%.1e" % r for r in rel])
    assert max(rel) < 1e-4


def test_gradient_matches_gpu_central_differences_and_a_random_direction():
    """Central differences of the loss from ordinary GPU steps (FP64
    storage, h = 1e-4) per parameter, and along one seeded random direction
    v of the parameters the directional difference equals dJ . v (the
    forward-mode counterpart of an adjoint's dot-product test)."""
    cfg, f = _case()
    c = dict(cfg, storage="f64")
    steps = 60
    cs2 = W.CS2["D2Q37"]
    J, dJ = lbm().pressure_loss_and_gradient(c, f, steps)

    def loss(d):
        q = dict(c, alpha_T=c["alpha_T"] + d[0], beta_P=c["beta_P"] + d[1],
                 p_inf=[p + d[2] for p in c["p_inf"]])
        return _loss_by_steps(q, f, steps)

    hs = (1e-4, 1e-4, 1e-4 * cs2)
    for k in range(3):
        e = [0.0, 0.0, 0.0]
        e[k] = hs[k]
        fd = (loss(e) - loss([-x for x in e])) / (2 * hs[k])
        assert abs(dJ[k] - fd) <= 1e-4 * abs(fd), (k, dJ[k], fd)
    v = np.random.default_rng(5).standard_normal(3) * np.array(hs)
    fd_v = (loss(v) - loss(-v)) / 2.0
    assert abs(float(np.dot(dJ, v)) - fd_v) <= 1e-4 * abs(fd_v), (np.dot(dJ, v), fd_v)


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q37"])
def test_gradient_in_alpha_V_and_t_inf_with_fd_viscous_terms(lat):
    """With the "-FD" viscous vector (frozen at t) in CBC-RELAX: dJ/d(alpha_T,
    alpha_V, t_inf) against the oracle's central differences."""
    cfg, f = _case(lat)
    cfg = dict(cfg, viscous="fd", alpha_V=0.4, t_inf=0.0)
    params = ("alpha_T", "alpha_V", "t_inf")
    steps = 60
    J, dJ = lbm().pressure_loss_gradient_in(dict(cfg, storage="f64"), f, steps, params)
    Jo = oracle.pressure_loss(cfg, f, steps)
    assert abs(J - Jo) <= 1e-10 * Jo, (J, Jo)
    fd = oracle.pressure_loss_fd_gradient(cfg, f, steps, (1e-4, 1e-4, 1e-7), params=params)
    for k in range(3):
        assert fd[k] != 0.0
        assert abs(dJ[k] - fd[k]) <= 1e-4 * abs(fd[k]), (k, dJ, fd)


@pytest.mark.parametrize("lat", ["D2Q17", "D2Q37"])
def test_gradient_with_mesoscopic_viscous_terms(lat):
    """With the mesoscopic viscous vector (Eqs. LaplaceU, LaplaceT; strips'
    non-equilibrium moments carried with their derivatives):
    dJ/d(alpha_T, beta_P, alpha_V) against the oracle's central
    differences."""
    cfg, f = _case(lat)
    cfg = dict(cfg, viscous="meso", alpha_V=0.4)
    params = ("alpha_T", "beta_P", "alpha_V")
    steps = 60
    J, dJ = lbm().pressure_loss_gradient_in(dict(cfg, storage="f64"), f, steps, params)
    Jo = oracle.pressure_loss(cfg, f, steps)
    assert abs(J - Jo) <= 1e-10 * Jo, (J, Jo)
    fd = oracle.pressure_loss_fd_gradient(cfg, f, steps, (1e-4, 1e-4, 1e-4), params=params)
    for k in range(3):
        assert fd[k] != 0.0
        assert abs(dJ[k] - fd[k]) <= 1e-4 * abs(fd[k]), (k, dJ, fd)


def test_gradient_directions_combine_linearly():
    """A direction that mixes parameters gives the same combination of the
    unit-direction derivatives (forward mode is linear in the seed, up to
    the FP32 rounding of the boundary state's derivative parts)."""
    cfg, f = _case()
    cfg = dict(cfg, viscous="fd", alpha_V=0.2, storage="f64")
    m = lbm()
    _, unit = m.pressure_loss_gradient_in(cfg, f, 40, m.THETA)
    rng = np.random.default_rng(8)
    dirs = rng.standard_normal((3, 5))
    _, mixed = m.pressure_loss_and_gradient(cfg, f, 40, directions=dirs.tolist())
    want = dirs @ np.array(unit)
    assert np.allclose(mixed, want, rtol=1e-5, atol=1e-6 * np.abs(want).max()), (mixed, want)


def test_autograd_function_returns_the_tangent_gradient():
    import torch
    m = lbm()
    cfg, f = _case()
    cs2 = W.CS2["D2Q37"]
    theta = torch.tensor([0.5, 0.3, cs2 * 1.0002], dtype=torch.float64, requires_grad=True)
    J = m.cbc_loss(theta, dict(cfg, storage="f64"), f, 40)
    J.backward()
    Jr, dJ = m.pressure_loss_and_gradient(dict(cfg, storage="f64"), f, 40)
    assert abs(J.item() - Jr) <= 1e-14 * Jr
    assert np.allclose(theta.grad.numpy(), dJ, rtol=1e-14, atol=0.0)
    # all five parameters (two runs of gradient steps)
    c5 = dict(cfg, storage="f64", viscous="fd", alpha_V=0.3)
    th5 = torch.tensor([0.5, 0.3, cs2 * 1.0002, 0.3, 0.0], dtype=torch.float64, requires_grad=True)
    J5 = m.cbc_loss(th5, c5, f, 30, params=m.THETA)
    J5.backward()
    _, g5 = m.pressure_loss_gradient_in(c5, f, 30, m.THETA)
    assert np.allclose(th5.grad.numpy(), g5, rtol=1e-14, atol=0.0)


def test_gradient_steps_are_checked_and_fence_ordinary_steps():
    m = lbm()
    cfg, f = _case()
    sim = m.Simulation(dict(cfg, storage="f64", dirichlet="neep")).init_fields(*f)
    with pytest.raises(m.LbmError, match="Dirichlet"):
        m.lbm_grad_begin(sim.handle)
    sim.close()
    sim = m.Simulation(dict(cfg, storage="f64")).init_fields(*f)
    with pytest.raises(m.LbmError, match="finite"):
        m.lbm_grad_begin_along(sim.handle, [[float("nan")] * 5] * 3)
    with pytest.raises(ValueError):
        m.lbm_grad_begin_along(sim.handle, [[1.0] * 4] * 3)
    sim.close()
    sim = m.Simulation(dict(cfg, storage="f16")).init_fields(*f)
    with pytest.raises(m.LbmError, match="storage"):
        m.lbm_grad_begin(sim.handle)
    sim.close()
    sim = m.Simulation(dict(cfg, storage="f64")).init_fields(*f)
    with pytest.raises(m.LbmError):
        m.lbm_grad_step(sim.handle, 1)          # before lbm_grad_begin
    m.lbm_grad_begin(sim.handle)
    m.lbm_grad_step(sim.handle, 3)
    m.lbm_grad_end(sim.handle)
    with pytest.raises(m.LbmError, match="lbm_init_fields"):
        sim.step(1)
    rho, _, _, _ = sim.macros()                  # the populations the gradient steps made
    assert np.all(np.isfinite(rho)) and sim.steps_done == 3
    sim.init_fields(*f)
    sim.step(1)
    sim.close()

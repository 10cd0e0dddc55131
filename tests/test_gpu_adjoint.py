"""Reverse-mode (adjoint) gradients of the pressure loss with respect to the
incoming-wave relaxation parameters (Eqs. LODI-Relax, CBC-Relax) and the
extension alpha_V, with segment checkpointing (lbm_adj_*).

Checked against two independent derivatives: the forward-mode
(tangent-linear) steps, whose directional derivative along v must equal
<grad J, v> from the reverse sweep (the dot-product identity of the whole
step map), and the FP64 oracle's central differences."""
import numpy as np
import pytest

import lbm_workloads as W
import oracle

pytestmark = pytest.mark.gpu

THETA = ("alpha_T", "beta_P", "p_inf", "alpha_V", "t_inf")


def lbm():
    import paper_2307_16766_gb300 as m
    return m


def _case(lat="D2Q37", n=32, m=24, u=(0.04, 0.03), sides=("cbc",) * 4, viscous="off", alpha_V=0.3,
          t_inf=0.0):
    """A pulse carried by a mean flow oblique to every side (no wave changes
    between incoming and outgoing, so J is smooth in the parameters)."""
    cs2 = W.CS2[lat]
    cfg = W.run(lat, n, m, 0.8, sides=sides, schemes=("cbc_relax",) * 4, viscous=viscous,
                alpha_T=0.5, beta_P=0.3, p_inf=[cs2 * 1.0002] * 4, alpha_V=alpha_V, t_inf=t_inf)
    f = list(W.gaussian_pulse(n, m, 1e-3, 1e-3 if lat != "D2Q9" else 0.0, 3.0,
                              center=(n / 2 - 0.7, m / 2 - 0.4)))
    f[1] = f[1] + u[0]
    f[2] = f[2] + u[1]
    return cfg, tuple(f)


def _tangent_all(cfg, f, steps, dP_ref=None):
    """dJ along the five unit directions by the tangent-linear steps."""
    J, g = lbm().pressure_loss_gradient_in(cfg, f, steps, THETA, dP_ref)
    return J, np.array(g)


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


@pytest.mark.parametrize("lat,viscous", [("D2Q37", "off"), ("D2Q37", "fd"), ("D2Q37", "meso"),
                                         ("D2Q17", "meso"), ("D2Q9", "fd")])
def test_adjoint_equals_tangent_linear(lat, viscous):
    """FP64 storage: the loss and all five derivatives from one reverse sweep
    equal the forward-mode ones (exact up to rounding; the tangent-linear
    steps keep the boundary state's derivatives in FP32, hence 1e-6)."""
    cfg, f = _case(lat, n=36 if viscous == "meso" else 32, m=26, viscous=viscous)
    cfg = dict(cfg, storage="f64")
    steps = 60
    Ja, ga = lbm().pressure_loss_gradient_adjoint(cfg, f, steps, checkpoint_every=25)
    Jt, gt = _tangent_all(cfg, f, steps)
    assert abs(Ja - Jt) <= 1e-10 * Jt, (Ja, Jt)
    scale = np.abs(gt).max()
    for k, name in enumerate(THETA):
        assert abs(ga[k] - gt[k]) <= 1e-6 * max(abs(gt[k]), 1e-6 * scale), (name, ga, gt)


def test_adjoint_dot_product_with_a_random_direction():
    """<grad J, v> from the reverse sweep equals the tangent-linear
    derivative along a seeded random direction v of the five parameters (the
    adjoint identity <J v, 1> = <v, J^T 1> for the whole run of steps),
    with the mesoscopic viscous vector and a reference field."""
    import torch
    cfg, f = _case("D2Q37", 36, 26, viscous="meso")
    cfg = dict(cfg, storage="f64")
    steps = 50
    rng = np.random.default_rng(17)
    ref = torch.tensor(2e-6 * rng.standard_normal((steps, 26, 36)), device="cuda")
    v = rng.standard_normal(5)
    v[2] *= W.CS2["D2Q37"]
    J, g = lbm().pressure_loss_gradient_adjoint(cfg, f, steps, ref, checkpoint_every=16)
    dirs = [list(v), [0.0] * 5, [0.0] * 5]
    Jt, dJt = lbm().pressure_loss_and_gradient(cfg, f, steps, ref, directions=dirs)
    lhs = float(np.dot(g, v))
    assert abs(J - Jt) <= 1e-10 * Jt
    # the tangent-linear steps hold the boundary state's derivatives in FP32
    assert abs(lhs - dJt[0]) <= 1e-6 * abs(dJt[0]), (lhs, dJt[0])


@pytest.mark.parametrize("K", [1, 7, 60])
def test_checkpoint_interval_does_not_change_the_gradient(K):
    """Segments of 1, 7 and 60 steps (the recompute restarts from each
    checkpoint): the same gradient as with segments of 20 steps."""
    cfg, f = _case("D2Q37", 36, 26, viscous="meso")
    cfg = dict(cfg, storage="f64")
    J0, g0 = lbm().pressure_loss_gradient_adjoint(cfg, f, 60, checkpoint_every=20)
    J1, g1 = lbm().pressure_loss_gradient_adjoint(cfg, f, 60, checkpoint_every=K)
    # sums of block partials by atomics: equal up to the order of the additions
    assert abs(J1 - J0) <= 1e-14 * J0
    assert np.all(_rel(g1, g0) <= 1e-11), (g0, g1)


def test_adjoint_matches_oracle_central_differences():
    """dJ/d(alpha_T, beta_P, P_inf, alpha_V, t_inf) with the mesoscopic
    viscous vector against the FP64 oracle's central differences (h = 1e-4
    in alpha_T, beta_P, alpha_V, 1e-4 c_s^2 in P_inf; t_inf, which moves the
    incoming amplitudes directly, takes h = 1e-5 c_s^2, where the difference
    quotient's third-order term is below 1e-6 of the derivative)."""
    cfg, f = _case("D2Q37", 36, 26, viscous="meso", alpha_V=0.3, t_inf=1e-5)
    steps = 60
    cs2 = W.CS2["D2Q37"]
    J, g = lbm().pressure_loss_gradient_adjoint(dict(cfg, storage="f64"), f, steps, checkpoint_every=30)
    Jo = oracle.pressure_loss(cfg, f, steps)
    assert abs(J - Jo) <= 1e-10 * Jo, (J, Jo)
    fd = oracle.pressure_loss_fd_gradient(cfg, f, steps, (1e-4, 1e-4, 1e-4 * cs2, 1e-4, 1e-5 * cs2),
                                          params=THETA)
    for k, name in enumerate(THETA):
        assert abs(g[k] - fd[k]) <= 1e-4 * abs(fd[k]), (name, g, fd)


def test_fp32_storage_gradient_close_to_fp64():
    """FP32 storage (adjoint populations and boundary arithmetic in FP32,
    parameter sums in FP64): within 1e-4 of the FP64 gradient."""
    cfg, f = _case("D2Q37", 36, 26, viscous="meso")
    _, g64 = lbm().pressure_loss_gradient_adjoint(dict(cfg, storage="f64"), f, 60, checkpoint_every=20)
    _, g32 = lbm().pressure_loss_gradient_adjoint(dict(cfg, storage="f32"), f, 60, checkpoint_every=20)
    scale = np.abs(g64).max()
    for k, name in enumerate(THETA):
        assert abs(g32[k] - g64[k]) <= 1e-4 * max(abs(g64[k]), 1e-3 * scale), (name, g32, g64)


def test_autograd_backward_is_the_reverse_sweep():
    import torch
    cfg, f = _case("D2Q37", 36, 26, viscous="meso")
    cfg = dict(cfg, storage="f64")
    theta = torch.tensor([0.5, 0.3, W.CS2["D2Q37"] * 1.0002, 0.3, 0.0], dtype=torch.float64,
                         requires_grad=True)
    J = lbm().cbc_loss_adjoint(theta, cfg, f, 40, checkpoint_every=15)
    J.backward()
    Jr, gr = lbm().pressure_loss_gradient_adjoint(cfg, f, 40, checkpoint_every=15)
    assert abs(float(J.detach()) - Jr) <= 1e-12 * Jr
    assert np.all(_rel(theta.grad.cpu().numpy(), gr) <= 1e-12)


def test_adjoint_leaves_the_state_after_the_forward_steps():
    cfg, f = _case("D2Q37", 32, 24, viscous="fd")
    cfg = dict(cfg, storage="f64")
    L = lbm()
    a = L.Simulation(cfg).init_fields(*f)
    L.lbm_adj_begin(a.handle, 9, 30)
    L.lbm_adj_forward(a.handle, 30)
    L.lbm_adj_backward(a.handle)
    L.lbm_adj_end(a.handle)
    a.step(5)
    b = L.Simulation(cfg).init_fields(*f)
    b.step(35)
    for x, y in zip(a.macros(), b.macros()):
        assert np.array_equal(x, y)
    a.close()
    b.close()


@pytest.mark.parametrize("change", [dict(dirichlet="neep"), dict(storage="f16"),
                                    dict(sides=("inflow", "cbc", "periodic", "periodic"))])
def test_adjoint_rejects_unsupported_configurations(change):
    cfg, f = _case("D2Q37", 32, 24)
    cfg = dict(cfg, storage="f64")
    cfg.update(change)
    sim = lbm().Simulation(cfg).init_fields(*f)
    with pytest.raises(lbm().LbmError) as e:
        lbm().lbm_adj_begin(sim.handle, 10, 20)
    assert e.value.code == -1
    sim.close()

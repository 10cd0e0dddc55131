"""The allocation-free boundary step (for callers that cannot allocate device
memory) gives the same boundary state as the solver's own boundary phase.

Collected last on purpose, so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

import lbm_workloads as W

pytestmark = pytest.mark.gpu

M = 3


def side_arrays(macros, nx):
    """East-side layers [ny][M][4] and bulk strips [3][ny][4] as deviations."""
    rho, ux, uy, T = macros
    dev = np.stack([rho - 1.0, ux, uy, T - 1.0], -1)
    layers = np.stack([dev[:, nx - 1 - M + j] for j in range(1, M + 1)], axis=1)
    strips = np.stack([dev[:, nx - 1 - M - d] for d in range(3)], axis=0)
    return np.ascontiguousarray(layers), np.ascontiguousarray(strips)


def test_noalloc_side_step_matches_solver_on_two_calls():
    import torch
    import paper_2307_16766_gb300 as lbm

    nx, ny = 96, 64
    cfg = W.run("D2Q37", nx, ny, 0.8, sides=("inflow", "cbc", "periodic", "periodic"),
                schemes=("cbc_relax",) * 4, alpha_T=0.3, beta_P=0.2, viscous="fd",
                storage="f64", inflow=(1.0, 0.05, 0.0, 1.0))
    fields = W.smooth_random(nx, ny, seed=21, amp=1e-3, u0=(0.05, 0.0))
    sim = lbm.Simulation(cfg).init_fields(*fields)
    params = lbm.params_from_run(cfg)
    stream = torch.cuda.current_stream()

    layers0, _ = side_arrays(sim.macros(), nx)
    ub = torch.tensor(layers0, device="cuda")
    for call in range(2):
        _, st = side_arrays(sim.macros(), nx)
        sim.step(1)
        ref_layers, st1 = side_arrays(sim.macros(), nx)
        st_d = torch.tensor(st, device="cuda")
        st1_d = torch.tensor(st1, device="cuda")
        lbm.lbm_cbc_side_step_noalloc(lbm.LBM_D2Q37, 1, ny, cfg["tau"], params, ub.data_ptr(),
                                      st_d.data_ptr(), st1_d.data_ptr(), 0, stream.cuda_stream)
        torch.cuda.synchronize()
        got = ub.cpu().numpy()
        # same bars as the FP64 parity tests: 1e-12 of the field scale
        for c, scale in ((0, 1.0), (3, 1.0)):
            assert np.abs(got[..., c] - ref_layers[..., c]).max() < 1e-12 * scale, (call, c)
        umax = np.abs(ref_layers[..., 1:3]).max()
        assert np.abs(got[..., 1:3] - ref_layers[..., 1:3]).max() < 1e-12 * umax, call
    sim.close()


def deep_strip(orc, macros, nx):
    """The nodes of the mesoscopic stencil of the east side, depths M, M+1,
    M+2 below x_f: [3][ny][9] = (sigma'_xx, sigma'_xy, sigma'_yy, q_x, q_y,
    rho - rho0, u_x, u_y, T - 1) of time t.  The moments come from the FP64
    oracle stepped beside the solver (its sigma' and q carry the
    (1 - 1/(2 tau)) factor the entry point expects)."""
    rho, ux, uy, T = macros
    dev = np.stack([rho - 1.0, ux, uy, T - 1.0], -1)
    ny = dev.shape[0]
    out = np.zeros((3, ny, 9))
    for k in range(3):
        x = nx - 1 - M - (M + k)
        for y in range(ny):
            out[k, y, :5] = orc.neq_moments(x, y)
        out[k, :, 5:] = dev[:, x]
    return out


def test_noalloc_side_step_mesoscopic_viscous_terms():
    """The same with the mesoscopic viscous vector (Eqs. LaplaceU,
    LaplaceT), whose stencil the caller supplies as the deep strip."""
    import torch
    import oracle
    import paper_2307_16766_gb300 as lbm

    nx, ny = 96, 64
    cfg = W.run("D2Q37", nx, ny, 0.8, sides=("inflow", "cbc", "periodic", "periodic"),
                schemes=("cbc_relax",) * 4, alpha_T=0.3, beta_P=0.2, alpha_V=0.25, viscous="meso",
                storage="f64", inflow=(1.0, 0.05, 0.0, 1.0))
    fields = W.smooth_random(nx, ny, seed=23, amp=1e-3, u0=(0.05, 0.0))
    sim = lbm.Simulation(cfg).init_fields(*fields)
    orc = oracle.Sim(cfg).init(*fields)
    # a few steps first, so that the non-equilibrium moments are not zero
    sim.step(5)
    orc.step(5)
    params = lbm.params_from_run(cfg)
    stream = torch.cuda.current_stream()
    layers0, _ = side_arrays(sim.macros(), nx)
    ub = torch.tensor(layers0, device="cuda")
    for call in range(2):
        mac = sim.macros()
        _, st = side_arrays(mac, nx)
        neq = deep_strip(orc, mac, nx)
        assert np.abs(neq[..., :5]).max() > 1e-9        # the viscous terms are in play
        sim.step(1)
        orc.step(1)
        ref_layers, st1 = side_arrays(sim.macros(), nx)
        st_d = torch.tensor(st, device="cuda")
        st1_d = torch.tensor(st1, device="cuda")
        neq_d = torch.tensor(neq, device="cuda")
        lbm.lbm_cbc_side_step_noalloc(lbm.LBM_D2Q37, 1, ny, cfg["tau"], params, ub.data_ptr(),
                                      st_d.data_ptr(), st1_d.data_ptr(), neq_d.data_ptr(),
                                      stream.cuda_stream)
        torch.cuda.synchronize()
        got = ub.cpu().numpy()
        for c in (0, 3):
            assert np.abs(got[..., c] - ref_layers[..., c]).max() < 1e-12, (call, c)
        umax = np.abs(ref_layers[..., 1:3]).max()
        assert np.abs(got[..., 1:3] - ref_layers[..., 1:3]).max() < 1e-12 * umax, call
    sim.close()


def test_noalloc_rejects_oversized_side():
    import paper_2307_16766_gb300 as lbm
    params = lbm.lbm_params_default()
    params.viscous = 2
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_cbc_side_step_noalloc(lbm.LBM_D2Q37, 1, 5000, 0.8, params, 1, 1, 1, 0, 0)
    assert e.value.code == -1

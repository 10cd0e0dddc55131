"""Pins of the oracle's bulk dynamics on periodic boxes (Sec. 2): conservation,
sound speed, shear and thermal diffusion, and the mesoscopic viscous terms of
Eqs. LaplaceU / LaplaceT, against closed forms of the Navier-Stokes-Fourier
equations (Eq. NSF) with nu = alpha = (tau - 1/2) c_s^2."""
import math

import numpy as np
import pytest

import oracle
import lbm_workloads as W
from lbm_workloads import CS2


def periodic(lat, nx, ny, tau):
    return W.run(lat, nx, ny, tau)


def totals(lat, rho, ux, uy, T):
    cs2 = CS2[lat]
    mass = rho.sum()
    px, py = (rho * ux).sum(), (rho * uy).sum()
    # (1/2) sum_i f_i |c_i|^2 = rho |u|^2 / 2 + rho c_s^2 T  (Eq. macro, d = 2)
    energy = (0.5 * rho * (ux ** 2 + uy ** 2) + rho * cs2 * T).sum()
    return mass, px, py, energy


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q37", "D2Q17"])
def test_periodic_conservation(lat):
    nx, ny = 40, 36
    cfg = periodic(lat, nx, ny, 0.7)
    f = W.smooth_random(nx, ny, seed=11, amp=2e-2, lattice=lat, u0=(0.03, -0.02))
    s = oracle.Sim(cfg).init(*f)
    t0 = totals(lat, *s.macros())
    s.step(1000)
    t1 = totals(lat, *s.macros())
    N = nx * ny
    assert abs(t1[0] - t0[0]) < 1e-12 * N
    assert abs(t1[1] - t0[1]) < 1e-13 * N and abs(t1[2] - t0[2]) < 1e-13 * N
    if lat != "D2Q9":
        assert abs(t1[3] - t0[3]) < 1e-12 * N


def right_centroid(v, x0):
    x = np.arange(v.size, dtype=float)
    m = (x > x0) & (v > 0)
    return (v[m] * x[m]).sum() / v[m].sum()


@pytest.mark.parametrize("lat,speed", [("D2Q9", math.sqrt(1 / 3)),
                                       ("D2Q37", math.sqrt(2 * CS2["D2Q37"])),
                                       ("D2Q17", math.sqrt(2 * CS2["D2Q17"]))])
def test_acoustic_pulse_speed(lat, speed):
    """An isentropic pulse splits into two waves travelling at
    sqrt(gamma T~) = sqrt(2) c_s (thermal, gamma = 2) or c_s (isothermal)."""
    nx, ny, w, a = 400, 2, 6.0, 1e-4
    x = np.arange(nx, dtype=float)
    x0 = nx / 2.0
    G = np.exp(-((x - x0) ** 2) / (2 * w * w))[None, :].repeat(ny, 0)
    rho = 1.0 + a * G
    T = 1.0 + a * G if lat != "D2Q9" else np.ones_like(G)    # T ~ rho^(gamma-1)
    s = oracle.Sim(periodic(lat, nx, ny, 0.55)).init(rho, 0 * G, 0 * G, T)
    n = 100
    s.step(n)
    r = s.macros()[0][0] - 1.0
    c = (right_centroid(r, x0) - x0) / n
    assert abs(c - speed) < 0.01 * speed, (c, speed)


def fourier_amp(v, axis_len, axis=1):
    x = np.arange(axis_len)
    k = 2 * math.pi / axis_len
    s = np.sin(k * x)
    prof = v.mean(axis=0) if axis == 1 else v.mean(axis=1)
    return 2.0 * (prof * s).sum() / axis_len


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q37", "D2Q17"])
def test_shear_wave_decay(lat):
    """u_y = A sin(kx) decays as exp(-nu k^2 t), nu = (tau - 1/2) c_s^2."""
    nx, ny, tau, A, n = 64, 2, 0.8, 1e-3, 400
    s = oracle.Sim(periodic(lat, nx, ny, tau)).init(*W.shear_wave(nx, ny, A))
    s.step(n)
    a = fourier_amp(s.macros()[2], nx)
    nu_meas = -math.log(a / A) / ((2 * math.pi / nx) ** 2 * n)
    nu = (tau - 0.5) * CS2[lat]
    assert abs(nu_meas - nu) < 0.01 * nu, (nu_meas, nu)


@pytest.mark.parametrize("lat", ["D2Q37", "D2Q17"])
def test_thermal_diffusion(lat):
    """At uniform pressure, T - 1 = A sin(kx) decays as exp(-alpha k^2 t) with
    the thermal diffusivity alpha = kappa / (rho c_p) = (tau - 1/2) c_s^2."""
    nx, ny, tau, A, n = 64, 2, 0.8, 1e-3, 300
    s = oracle.Sim(periodic(lat, nx, ny, tau)).init(*W.temperature_wave(nx, ny, A))
    s.step(n)
    a = fourier_amp(s.macros()[3] - 1.0, nx)
    al_meas = -math.log(a / A) / ((2 * math.pi / nx) ** 2 * n)
    al = (tau - 0.5) * CS2[lat]
    assert abs(al_meas - al) < 0.02 * al, (al_meas, al)


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q37", "D2Q17"])
def test_viscous_stress_sign_and_factor(lat):
    """sigma'_xy from Eq. LaplaceU equals mu du_y/dx = rho nu du_y/dx on a
    developed shear wave (fixes f^neq = f - f^eq and the 1 - 1/(2 tau) factor)."""
    nx, ny, tau, A = 64, 2, 0.8, 1e-3
    s = oracle.Sim(periodic(lat, nx, ny, tau)).init(*W.shear_wave(nx, ny, A))
    s.step(40)
    uy = s.macros()[2][0]
    k = 2 * math.pi / nx
    amp = fourier_amp(s.macros()[2], nx)
    nu = (tau - 0.5) * CS2[lat]
    x = np.arange(nx)
    for xx in (0, 5, 16, 40):
        want = 1.0 * nu * amp * k * math.cos(k * xx)
        got = s.neq_moments(xx, 0)[1]
        assert abs(got - want) < 0.02 * nu * amp * k, (xx, got, want)
    assert np.abs(uy).max() > 0.5 * A


def test_heat_flux_factor():
    """q from Eq. LaplaceT with the (1 - 1/(2 tau)) factor equals Fourier's law
    q = -kappa dT~/dx, kappa = rho c_p alpha, c_p = 2, T~ = c_s^2 T."""
    nx, ny, tau, A = 64, 2, 0.8, 1e-3
    cs2 = CS2["D2Q37"]
    s = oracle.Sim(periodic("D2Q37", nx, ny, tau)).init(*W.temperature_wave(nx, ny, A))
    s.step(40)
    amp = fourier_amp(s.macros()[3] - 1.0, nx)
    k = 2 * math.pi / nx
    kappa = 1.0 * 2.0 * (tau - 0.5) * cs2
    for xx in (0, 7, 16, 33):
        want = -kappa * cs2 * amp * k * math.cos(k * xx)
        got = s.neq_moments(xx, 0)[3]
        assert abs(got - want) < 0.03 * kappa * cs2 * amp * k, (xx, got, want)


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q37"])
@pytest.mark.parametrize("side", [0, 1, 2, 3])
def test_mesoscopic_viscous_vector(lat, side):
    """The viscous vector the boundary solver uses at x_f (Eqs. LaplaceU,
    LaplaceT with Eqs. FD-dx-bw / FD-dx-center) approximates
    V = (0, nu Lap u_n, nu Lap u_t, 2 nu Lap T) (Sec. 3.1) on plane waves,
    through both the normal (one-sided) and the tangential (central) paths."""
    n = 48
    tau = 0.8
    nu = (tau - 0.5) * CS2[lat]
    k = 2 * math.pi / n
    normal_is_x = side < 2
    sgn = -1.0 if side in (0, 2) else 1.0
    # wave varying along the normal carries the tangential velocity (u_t)
    along_n = W.shear_wave(n, n, 1e-3, k_axis="x" if normal_is_x else "y")
    # wave varying along the tangent carries the normal velocity (u_n)
    along_t = W.shear_wave(n, n, 1e-3, k_axis="y" if normal_is_x else "x")
    for fields, comp in ((along_n, 2), (along_t, 1)):
        s = oracle.Sim(periodic(lat, n, n, tau)).init(*fields)
        s.step(30)
        rho, ux, uy, T = s.macros()
        for pos in (3, 17, 30):
            x, y = (pos, 11) if normal_is_x else (11, pos)
            V = s.vis_meso_at(side, x, y)
            vel = ux if normal_is_x else uy   # normal-axis velocity component
            other = uy if normal_is_x else ux
            if comp == 1:
                u_n = sgn * vel[y, x]
                want = -nu * k * k * u_n
            else:
                u_t = other[y, x]
                want = -nu * k * k * u_t
            scale = nu * k * k * 1e-3
            assert abs(V[comp] - want) < 0.05 * scale, (comp, pos, V, want)
    if lat == "D2Q37":
        s = oracle.Sim(periodic(lat, n, n, tau)).init(*W.temperature_wave(n, n, 1e-3))
        s.step(30)
        T = s.macros()[3]
        for pos in (3, 17, 30):
            x, y = (pos, 11) if normal_is_x else (11, pos)
            V = s.vis_meso_at(side, x, y)
            want = -2.0 * nu * k * k * (T[y, x] - 1.0)
            assert abs(V[3] - want) < 0.05 * 2 * nu * k * k * 1e-3, (pos, V, want)

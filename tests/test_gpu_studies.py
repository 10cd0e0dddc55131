"""The paper's benchmark studies (Sec. 4) on the CUDA path, with the claims
the paper makes about them that this implementation reproduces (the ones it
does not reproduce are measured and reported, not asserted)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def S():
    from paper_2307_16766_gb300 import studies
    return studies


def _mean(e, lo=None, hi=None):
    t = e["t"]
    m = np.ones_like(t, dtype=bool)
    if lo is not None:
        m &= t >= lo
    if hi is not None:
        m &= t <= hi
    return {z: float(np.mean(e[z][m])) for z in ("rho", "ux", "T")}


def _show(capsys, title, table):
    with capsys.disabled():
        print("\n" + title)
        for k, v in table.items():
            print("   %-16s %s" % (k, {z: "%.2e" % x for z, x in v.items()} if isinstance(v, dict) else v))


def test_temperature_step_sec_4_1(capsys):
    """Any characteristic condition lowers e_Z by about two orders of
    magnitude on average against zero gradient; LODI and CBC, and the
    equilibrium and NEEP Dirichlet conditions, give similar errors."""
    st = S().TemperatureStep()
    m = {v: _mean(st.run(v)) for v in st.VARIANTS}
    _show(capsys, "Sec. 4.1 temperature step, mean e_Z over 1500 steps (D2Q17 200x20):", m)
    for v in ("lodi", "lodi_neep", "cbc", "cbc_neep"):
        for z in ("rho", "ux", "T"):
            assert m["zg"][z] / m[v][z] > 50.0, (v, z, m)
    for a, b in (("lodi", "lodi_neep"), ("cbc", "cbc_neep"), ("lodi", "cbc")):
        for z in ("rho", "ux", "T"):
            assert 0.5 < m[b][z] / m[a][z] < 2.0, (a, b, z, m)


@pytest.fixture(scope="module")
def vortex17():
    return S().ThermalVortex(lattice="D2Q17")


def test_thermal_vortex_sec_4_2(vortex17, capsys):
    """Zero gradient gives the largest errors; relaxing the transversal
    waves in the incoming amplitude (LODI-RELAX) lowers the errors of the
    LODI outlet severalfold between 400 and 1000 iterations (the paper:
    about tenfold).  CBC-RELAX with the -FD viscous vector is on a par with
    LODI-RELAX (the paper: similar error levels)."""
    vt = vortex17
    runs = {"zg": dict(zg=True), "lodi": dict(outlet="lodi"), "lodi_relax": dict(outlet="lodi_relax"),
            "cbc_relax_fd": dict(outlet="cbc_relax", viscous="fd"),
            "cbc_relax_meso": dict(outlet="cbc_relax", viscous="meso")}
    e = {k: vt.run(**kw) for k, kw in runs.items()}
    m = {k: _mean(v) for k, v in e.items()}
    w = {k: _mean(v, 400, 1000) for k, v in e.items()}
    _show(capsys, "Sec. 4.2 thermal vortex D2Q17 150x150, mean e_Z over 1200 steps:", m)
    _show(capsys, "   ... over steps 400-1000:", w)
    for k in ("lodi", "lodi_relax", "cbc_relax_fd", "cbc_relax_meso"):
        for z in ("rho", "T"):
            assert m["zg"][z] > m[k][z], (k, z, m)
    for z in ("rho", "ux", "T"):
        assert w["lodi"][z] / w["lodi_relax"][z] > 3.0, (z, w)
        assert 0.33 < w["cbc_relax_fd"][z] / w["lodi_relax"][z] < 3.0, (z, w)
        # the mesoscopic viscous vector (Eqs. LaplaceU, LaplaceT) stays
        # finite and is at least as accurate as -FD (Sec. 4.2)
        assert math.isfinite(m["cbc_relax_meso"][z]) and m["cbc_relax_meso"][z] < m["cbc_relax_fd"][z], (z, m)


def test_stencils_and_lodi_sec_4_2_table(vortex17, capsys):
    """Tab. CBCs-17-vs-37: the errors in rho and T are about the same for
    D2Q17 and D2Q37, and switching from zero gradient to LODI lowers them by
    roughly a factor of two on both."""
    v37 = S().ThermalVortex(lattice="D2Q37")
    tab = {}
    for lat, vt in (("D2Q17", vortex17), ("D2Q37", v37)):
        for k, kw in (("zg", dict(zg=True)), ("lodi", dict(outlet="lodi"))):
            tab[lat + " " + k] = _mean(vt.run(**kw))
    z17 = tab["D2Q17 zg"]
    _show(capsys, "Tab. CBCs-17-vs-37 (mean e_Z normalised to D2Q17 ZG):",
          {k: {z: v[z] / z17[z] for z in v} for k, v in tab.items()})
    for lat in ("D2Q17", "D2Q37"):
        for z in ("rho", "T"):
            assert tab[lat + " zg"][z] / tab[lat + " lodi"][z] > 1.5, (lat, z, tab)
    for k in ("zg", "lodi"):
        for z in ("rho", "T"):
            assert 0.5 < tab["D2Q37 " + k][z] / tab["D2Q17 " + k][z] < 2.0, (k, z, tab)


def test_fd_viscous_terms_unstable_at_high_viscosity_sec_4_2(vortex17, capsys):
    """The -FD viscous vector with CBC-RELAX runs at nu = 0.1 and 0.2 and
    becomes numerically unstable at nu = 0.3, as the paper reports; the
    mesoscopic vector stays finite at all three, with mean errors below the
    -FD form's."""
    res, meso = {}, {}
    for nu in (0.1, 0.2, 0.3):
        vt = vortex17 if nu == 0.1 else S().ThermalVortex(nu=nu, ref_side=vortex17.Lref)
        e = vt.run(outlet="cbc_relax", viscous="fd")
        res["nu=%.1f" % nu] = {z: float(e[z][-1]) for z in ("rho", "ux", "T")}
        meso["nu=%.1f" % nu] = _mean(vt.run(outlet="cbc_relax", viscous="meso"))
    _show(capsys, "Sec. 4.2 CBC-RELAX-FD, e_Z at the last step:", res)
    _show(capsys, "Sec. 4.2 CBC-RELAX (mesoscopic), mean e_Z over 1200 steps:", meso)
    for nu in ("nu=0.1", "nu=0.2"):
        assert all(math.isfinite(v) for v in res[nu].values()), res
        assert res[nu]["rho"] < 0.05, res
    assert not math.isfinite(res["nu=0.3"]["rho"]) or res["nu=0.3"]["rho"] > 10 * res["nu=0.1"]["rho"], res
    for nu in ("nu=0.1", "nu=0.2", "nu=0.3"):
        assert all(math.isfinite(v) and v < 0.1 for v in meso[nu].values()), meso


def test_angular_wave_reflection_sec_4_3(capsys):
    """Zero gradient reflects a few percent of a plane pulse; at small
    angles the characteristic conditions reflect several times less."""
    R = {"phi=%d" % p: S().angular_wave(p) for p in (0, 10, 20, 30, 40)}
    _show(capsys, "Sec. 4.3 angular wave, R_rho (D2Q17 200x700):", R)
    assert 0.01 < R["phi=0"]["zg"] < 0.08, R
    for p in ("phi=0", "phi=10"):
        for v in ("lodi", "cbc"):
            assert R[p][v] < R[p]["zg"] / 5.0, (p, v, R)


def test_corners_iso_thermal_vortex_sec_4_4(capsys):
    """Iso-thermal vortex with D2Q9 (-FD viscous vector), D2Q17 and D2Q37 at
    t* = floor(150 c_s^17 / c_s^q): pointwise errors near the outlet
    corners against those near the middle of the outlet (reported)."""
    cs17 = math.sqrt(S().CS2["D2Q17"])
    out = {}
    for lat in ("D2Q9", "D2Q17", "D2Q37"):
        ts = int(math.floor(150 * cs17 / math.sqrt(S().CS2[lat]))) // 10 * 10
        vt = S().ThermalVortex(lattice=lat, isothermal=True, steps=ts)
        er, eu = vt.pointwise(ts, outlet="cbc_relax", viscous="fd" if lat == "D2Q9" else "meso")
        L, c = vt.L, 12
        corner = max(er[:c, L - c:].max(), er[L - c:, L - c:].max())
        middle = er[L // 2 - 20:L // 2 + 20, L - c:].max()
        cu = max(eu[:c, L - c:].max(), eu[L - c:, L - c:].max())
        mu = eu[L // 2 - 20:L // 2 + 20, L - c:].max()
        out[lat] = {"t*": ts, "rho corner/middle": corner / middle, "ux corner/middle": cu / mu}
        assert np.isfinite(er).all() and np.isfinite(eu).all()
    with capsys.disabled():
        print("\nSec. 4.4 iso-thermal vortex, max pointwise error near the outlet corners / near its middle:")
        for k, v in out.items():
            print("   %s %s" % (k, {a: ("%.2f" % b if isinstance(b, float) else b) for a, b in v.items()}))

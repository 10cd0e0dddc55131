"""The C-ABI library builds, loads and exports what include/lbm_cbc.h declares;
the ctypes mirror matches the C struct layout; host-side validation rejects
invalid configurations.  No CUDA kernel is launched here."""
import ctypes as C
import os
import re
import subprocess

import pytest

import paper_2307_16766_gb300 as lbm
from paper_2307_16766_gb300 import build as gpu_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm_cbc.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    path = gpu_build.build()
    names = declared_functions()
    assert len(names) >= 15
    L = C.CDLL(path)
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (lbm_\w+)", out))
    assert set(names) <= exported, set(names) - exported


def test_params_struct_layout_matches_header(tmp_path):
    """Compile a probe against the header and compare sizeof / offsets with
    the ctypes mirror used by the binding."""
    fields = [f[0] for f in lbm.LbmCbcParams._fields_]
    probe = tmp_path / "probe.c"
    body = "\n".join('printf("%%s %%zu\\n", "%s", offsetof(lbm_cbc_params, %s));' % (f, f) for f in fields)
    probe.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbm_cbc.h"\nint main(void){\n'
                     'printf("sizeof %zu\\n", sizeof(lbm_cbc_params));\n' + body + "\nreturn 0;}\n")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(probe), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    assert int(got["sizeof"]) == C.sizeof(lbm.LbmCbcParams)
    for f in fields:
        assert int(got[f]) == getattr(lbm.LbmCbcParams, f).offset, f


def cfg_params(**kw):
    p = lbm.lbm_params_default()
    for k, v in kw.items():
        if k in ("side", "scheme", "p_inf", "inflow", "u_ref"):
            for i, x in enumerate(v):
                getattr(p, k)[i] = x
        else:
            setattr(p, k, v)
    return p


def test_defaults_and_workspace_size():
    p = lbm.lbm_params_default()
    assert list(p.side) == [0, 0, 0, 0] and p.storage == lbm.LBM_F32 and p.rho0 == 1.0
    n32 = lbm.lbm_workspace_bytes(lbm.LBM_D2Q37, 1024, 512, p)
    # two population buffers dominate: 2 * 37 * 512 * 1024 * 4 bytes
    assert 2 * 37 * 512 * 1024 * 4 <= n32 < 2 * 37 * 512 * 1024 * 4 * 1.5
    p.storage = lbm.LBM_F64
    assert lbm.lbm_workspace_bytes(lbm.LBM_D2Q37, 1024, 512, p) > 1.9 * n32 - 64 * 1024 * 1024


@pytest.mark.parametrize("lattice,nx,ny,kw,ok", [
    (lbm.LBM_D2Q37, 9, 9, dict(side=[1, 1, 1, 1], viscous=1), True),    # minimal 2M+3
    (lbm.LBM_D2Q37, 8, 9, dict(side=[1, 1, 1, 1], viscous=1), False),   # too small
    (lbm.LBM_D2Q37, 12, 12, dict(side=[1, 1, 1, 1]), True),        # mesoscopic stencil: 3M+3
    (lbm.LBM_D2Q37, 11, 12, dict(side=[1, 1, 1, 1]), False),
    (lbm.LBM_D2Q37, 12, 11, dict(side=[1, 1, 1, 1]), False),
    (lbm.LBM_D2Q37, 11, 16, dict(side=[1, 1, 0, 0]), False),       # ... across a CBC side
    (lbm.LBM_D2Q37, 11, 16, dict(side=[3, 3, 0, 0]), True),        # zero gradient: 2M+3
    (lbm.LBM_D2Q9, 5, 5, dict(side=[1, 1, 1, 1], viscous=2), True),
    (lbm.LBM_D2Q9, 6, 6, dict(side=[1, 1, 1, 1]), True),
    (lbm.LBM_D2Q9, 5, 6, dict(side=[1, 1, 1, 1]), False),
    (lbm.LBM_D2Q9, 4, 5, dict(side=[3, 3, 3, 3]), False),
    (lbm.LBM_D2Q37, 16, 3, dict(side=[1, 1, 0, 0]), True),         # periodic axis of length M
    (lbm.LBM_D2Q37, 16, 2, dict(side=[1, 1, 0, 0]), False),
    (lbm.LBM_D2Q37, 16, 16, dict(side=[1, 0, 0, 0]), False),       # unpaired periodic side
    (lbm.LBM_D2Q37, 16, 16, dict(side=[1, 3, 1, 1]), False),       # mixed corners
    (lbm.LBM_D2Q37, 16, 16, dict(side=[2, 1, 0, 0]), True),        # inflow | CBC
    (lbm.LBM_D2Q37, 16, 16, dict(side=[2, 3, 3, 3]), True),        # inflow + ZG corners
    (lbm.LBM_D2Q37, 16, 16, dict(storage=7), False),
    (lbm.LBM_D2Q37, 16, 16, dict(viscous=3), False),
    (lbm.LBM_D2Q37, 16, 16, dict(rho0=0.0), False),
    (lbm.LBM_D2Q17, 9, 9, dict(side=[1, 1, 1, 1], viscous=2), True),    # D2Q17: M = 3 as well
    (lbm.LBM_D2Q17, 9, 8, dict(side=[1, 1, 1, 1], viscous=2), False),
    (lbm.LBM_D2Q17, 12, 12, dict(side=[1, 1, 1, 1]), True),
    (lbm.LBM_D2Q37, 7616, 7616, dict(side=[1, 1, 1, 1]), True),    # 37 x 7616^2 < 2^31 values
    (lbm.LBM_D2Q37, 7680, 7616, dict(side=[1, 1, 1, 1]), False),   # 37 x 7616 x 7680 > 2^31
    (lbm.LBM_D2Q9, 15360, 15360, dict(), True),                    # 9 x 15360^2 < 2^31
    (lbm.LBM_D2Q9, 16384, 15360, dict(), False),
    (lbm.LBM_D2Q37, 16, 16, dict(alpha_V=float("nan")), False),    # relaxation parameters finite
    (lbm.LBM_D2Q37, 16, 16, dict(alpha_T=float("inf")), False),
    (lbm.LBM_D2Q37, 16, 16, dict(u_ref=[0.3, 0.2]), True),          # reference velocity below c_s
    (lbm.LBM_D2Q37, 16, 16, dict(u_ref=[0.8, 0.3]), False),         # |u_ref| >= c_s
    (lbm.LBM_D2Q37, 16, 16, dict(u_ref=[float("nan"), 0.0]), False),
    (lbm.LBM_D2Q9, 16, 16, dict(u_ref=[0.5, 0.3]), False),          # c_s^2 = 1/3 on D2Q9
    (lbm.LBM_D2Q37, 64, 64, dict(side=[1, 1, 1, 1], band_ctas=3), True),
    (lbm.LBM_D2Q37, 64, 64, dict(side=[1, 1, 1, 1], band_ctas=10 ** 6), True),
    (lbm.LBM_D2Q37, 16, 16, dict(band_ctas=-1), False),
    (3, 16, 16, dict(), False),                                    # unknown lattice
    (-1, 16, 16, dict(), False),
])
def test_configuration_validation(lattice, nx, ny, kw, ok):
    p = cfg_params(**kw)
    if ok:
        assert lbm.lbm_workspace_bytes(lattice, nx, ny, p) > 0
    else:
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_workspace_bytes(lattice, nx, ny, p)
        assert e.value.code == -1


def test_create_rejects_bad_tau_without_touching_the_device():
    p = cfg_params()
    for tau in (0.5, 0.2, float("nan")):
        with pytest.raises(lbm.LbmError):
            lbm.lbm_create(lbm.LBM_D2Q37, 16, 16, tau, p)

"""GB300 (sm_103a) thermal lattice Boltzmann solver with the layer-wise
characteristic boundary condition of Klass, Gabbana & Bartel (arXiv 2307.16766).

A thin ctypes binding of the C ABI declared in ``include/lbm_cbc.h``: the
functions below carry the C names and only marshal arguments; every step of
the method runs in the CUDA kernels of ``csrc/``.  PyTorch is used only to
provide device memory (the solver workspace) and the CUDA stream.

Quick use::

    import lbm_workloads as W, paper_2307_16766_gb300 as lbm
    cfg, fields = W.pulse_d2q37(256, alpha_T=0.5, steps=100)
    sim = lbm.Simulation(cfg)          # workspace from torch, torch's stream
    sim.init_fields(*fields)
    sim.step(100)
    rho, ux, uy, T = sim.macros()      # numpy [ny, nx] arrays
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

__all__ = [
    "LbmCbcParams", "LBM_D2Q9", "LBM_D2Q37", "LBM_D2Q17", "LBM_F64", "LBM_F32", "LBM_F16",
    "lbm_params_default", "lbm_workspace_bytes", "lbm_create", "lbm_create_in",
    "lbm_set_stream", "lbm_init_fields", "lbm_step", "lbm_step_phase", "lbm_set_kernel_events",
    "lbm_get_macros",
    "lbm_state_bytes", "lbm_get_state", "lbm_set_state", "lbm_steps_done",
    "lbm_last_error", "lbm_destroy", "lbm_cbc_side_step_noalloc", "Simulation",
    "params_from_run", "LbmError",
]

LBM_D2Q9, LBM_D2Q37, LBM_D2Q17 = 0, 1, 2
LBM_F64, LBM_F32, LBM_F16 = 0, 1, 2
LATTICES = {"D2Q9": LBM_D2Q9, "D2Q37": LBM_D2Q37, "D2Q17": LBM_D2Q17}
STORAGES = {"f64": LBM_F64, "f32": LBM_F32, "f16": LBM_F16}
SIDES = {"periodic": 0, "cbc": 1, "inflow": 2, "zg": 3}
SCHEMES = {"lodi": 0, "lodi_relax": 1, "cbc": 2, "cbc_relax": 3}
VISCOUS = {"meso": 0, "fd": 1, "off": 2}
DIRICHLET = {"eq": 0, "neep": 1, "reg": 2}
ERRORS = {-1: "LBM_ERR_ARG", -2: "LBM_ERR_ALLOC", -3: "LBM_ERR_CUDA",
          -4: "LBM_ERR_NUMERICAL", -5: "LBM_ERR_STATE", -6: "LBM_ERR_TIMEOUT"}


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "error"), code, msg))
        self.code = code


class LbmCbcParams(C.Structure):
    """Mirror of ``lbm_cbc_params``."""
    _fields_ = [
        ("side", C.c_int * 4), ("scheme", C.c_int * 4), ("viscous", C.c_int),
        ("dirichlet", C.c_int), ("alpha_T", C.c_double), ("beta_P", C.c_double),
        ("t_inf", C.c_double), ("p_inf", C.c_double * 4), ("inflow", C.c_double * 4),
        ("storage", C.c_int), ("rho0", C.c_double), ("alpha_V", C.c_double),
        ("u_ref", C.c_double * 2), ("band_ctas", C.c_int),
    ]


_lib = None


def lib():
    """Load the CUDA library, building it in-tree if needed.  There is no
    fallback: without the library nothing in this package runs."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            path = _build.build()
        L = C.CDLL(path)
        vp, dp, sz = C.c_void_p, C.POINTER(C.c_double), C.c_size_t
        pp = C.POINTER(LbmCbcParams)
        sig = {
            "lbm_params_default": (C.c_int, [pp]),
            "lbm_workspace_bytes": (C.c_int, [C.c_int, C.c_int, C.c_int, pp, C.POINTER(sz)]),
            "lbm_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, pp, C.POINTER(vp)]),
            "lbm_create_in": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, pp, vp, sz, C.POINTER(vp)]),
            "lbm_set_stream": (C.c_int, [vp, vp]),
            "lbm_init_fields": (C.c_int, [vp, vp, vp, vp, vp, C.c_int]),
            "lbm_step": (C.c_int, [vp, C.c_int]),
            "lbm_step_phase": (C.c_int, [vp, C.c_int]),
            "lbm_set_kernel_events": (C.c_int, [vp, C.POINTER(C.c_void_p), C.c_int]),
            "lbm_set_wait_limit": (C.c_int, [vp, C.c_double]),
            "lbm_fp64_fma_rate": (C.c_int, [C.c_int, vp, C.POINTER(C.c_double)]),
            "lbm_get_macros": (C.c_int, [vp, vp, vp, vp, vp, C.c_int]),
            "lbm_state_bytes": (C.c_int, [vp, C.POINTER(sz)]),
            "lbm_get_state": (C.c_int, [vp, vp, sz]),
            "lbm_set_state": (C.c_int, [vp, vp, sz]),
            "lbm_steps_done": (C.c_longlong, [vp]),
            "lbm_last_error": (C.c_char_p, [vp]),
            "lbm_destroy": (None, [vp]),
            "lbm_cbc_side_step_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, pp,
                                                    vp, vp, vp, vp, vp]),
            "lbm_grad_begin": (C.c_int, [vp]),
            "lbm_grad_begin_along": (C.c_int, [vp, C.POINTER(C.c_double)]),
            "lbm_grad_step": (C.c_int, [vp, C.c_int, vp, C.c_longlong]),
            "lbm_grad_result": (C.c_int, [vp, dp, dp]),
            "lbm_grad_end": (C.c_int, [vp]),
            "lbm_adj_begin": (C.c_int, [vp, C.c_int, C.c_int]),
            "lbm_adj_forward": (C.c_int, [vp, C.c_int, vp, C.c_longlong, dp]),
            "lbm_adj_backward": (C.c_int, [vp, dp]),
            "lbm_adj_end": (C.c_int, [vp]),
            "lbm_batch_create": (C.c_int, [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                           C.POINTER(C.c_int), dp, pp, C.POINTER(vp)]),
            "lbm_batch_run": (C.c_int, [vp, C.c_int, C.POINTER(vp)]),
            "lbm_batch_set_stream": (C.c_int, [vp, vp]),
            "lbm_batch_step": (C.c_int, [vp, C.c_int]),
            "lbm_batch_ctas_per_sm": (C.c_int, [vp, C.c_int, C.c_int]),
            "lbm_batch_last_error": (C.c_char_p, [vp]),
            "lbm_batch_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        del dp
        _lib = L
    return _lib


def _check(rc, h=None):
    if rc != 0:
        msg = lib().lbm_last_error(h).decode() if h else ""
        raise LbmError(rc, msg)


def params_from_run(cfg) -> LbmCbcParams:
    """Build ``lbm_cbc_params`` from a run description (see lbm_workloads.run)."""
    p = LbmCbcParams()
    _check(lib().lbm_params_default(C.byref(p)))
    for i, s in enumerate(cfg.get("sides", ["periodic"] * 4)):
        p.side[i] = SIDES[s]
    for i, s in enumerate(cfg.get("schemes", ["cbc_relax"] * 4)):
        p.scheme[i] = SCHEMES[s]
    p.viscous = VISCOUS[cfg.get("viscous", "meso")]
    p.dirichlet = DIRICHLET[cfg.get("dirichlet", "eq")]
    p.alpha_T = float(cfg.get("alpha_T", 0.0))
    p.beta_P = float(cfg.get("beta_P", 0.0))
    p.t_inf = float(cfg.get("t_inf", 0.0))
    p.alpha_V = float(cfg.get("alpha_V", 0.0))
    for i, v in enumerate(cfg.get("p_inf", [0.0] * 4)):
        p.p_inf[i] = float(v)
    for i, v in enumerate(cfg.get("inflow", [1.0, 0.0, 0.0, 1.0])):
        p.inflow[i] = float(v)
    p.storage = STORAGES[cfg.get("storage", "f32")]
    p.rho0 = float(cfg.get("rho0", 1.0))
    for i, v in enumerate(cfg.get("u_ref", [0.0, 0.0])):
        p.u_ref[i] = float(v)
    p.band_ctas = int(cfg.get("band_ctas", 0))
    return p


# ----------------------------------------------------------- C ABI names ---

def lbm_params_default() -> LbmCbcParams:
    p = LbmCbcParams()
    _check(lib().lbm_params_default(C.byref(p)))
    return p


def lbm_workspace_bytes(lattice, nx, ny, params) -> int:
    n = C.c_size_t()
    _check(lib().lbm_workspace_bytes(int(lattice), int(nx), int(ny), C.byref(params), C.byref(n)))
    return n.value


def lbm_create(lattice, nx, ny, tau, params):
    h = C.c_void_p()
    _check(lib().lbm_create(int(lattice), int(nx), int(ny), float(tau), C.byref(params), C.byref(h)))
    return h


def lbm_create_in(lattice, nx, ny, tau, params, dev_ptr, nbytes):
    h = C.c_void_p()
    _check(lib().lbm_create_in(int(lattice), int(nx), int(ny), float(tau), C.byref(params),
                               C.c_void_p(dev_ptr), C.c_size_t(nbytes), C.byref(h)))
    return h


def lbm_set_stream(h, stream_ptr):
    _check(lib().lbm_set_stream(h, C.c_void_p(stream_ptr)), h)


def _field_ptr(a, n):
    """(pointer, on_device, keepalive) for a float64 field of n values:
    a CUDA torch tensor stays on the device, anything else goes through a
    contiguous host float64 array."""
    mod = type(a).__module__
    if mod.startswith("torch") and getattr(a, "is_cuda", False):
        import torch
        t = a.detach().to(torch.float64).contiguous()
        if t.numel() != n:
            raise ValueError("field has %d values, expected %d" % (t.numel(), n))
        return t.data_ptr(), 1, t
    if mod.startswith("torch"):
        a = a.detach().cpu().numpy()
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if arr.size != n:
        raise ValueError("field has %d values, expected %d" % (arr.size, n))
    return arr.ctypes.data, 0, arr


def lbm_init_fields(h, n_nodes, rho, ux, uy, T):
    """Fields as numpy arrays (host) or CUDA torch tensors (device)."""
    ptrs = [_field_ptr(a, n_nodes) for a in (rho, ux, uy, T)]
    on_dev = {p[1] for p in ptrs}
    if len(on_dev) != 1:
        raise ValueError("all four fields must be on the host or all on the device")
    _check(lib().lbm_init_fields(h, *[C.c_void_p(p[0]) for p in ptrs], on_dev.pop()), h)


def lbm_step(h, n):
    _check(lib().lbm_step(h, int(n)), h)


def lbm_step_phase(h, phase):
    _check(lib().lbm_step_phase(h, int(phase)), h)


def lbm_set_kernel_events(h, events):
    """Timing hook: a sequence of 0, 2 or 5 raw cudaEvent_t handles (ints,
    e.g. torch.cuda.Event.cuda_event of recorded events); see
    include/lbm_cbc.h for where each is recorded."""
    events = list(events or [])
    arr = (C.c_void_p * max(1, len(events)))(*[C.c_void_p(int(e)) for e in events])
    _check(lib().lbm_set_kernel_events(h, arr, len(events)), h)


def fp64_fma_rate(iters=16384, stream=None):
    """Measured FP64 FMA throughput of the current device in flop/s."""
    import torch
    st = torch.cuda.current_stream() if stream is None else stream
    out = C.c_double(0.0)
    rc = lib().lbm_fp64_fma_rate(int(iters), C.c_void_p(st.cuda_stream), C.byref(out))
    if rc != 0:
        raise LbmError(rc, "FP64 FMA throughput launch failed")
    return out.value


def lbm_set_wait_limit(h, seconds):
    _check(lib().lbm_set_wait_limit(h, float(seconds)), h)


def lbm_get_macros(h, rho, ux, uy, T, on_device):
    """Fill four preallocated outputs (pointers as ints)."""
    _check(lib().lbm_get_macros(h, C.c_void_p(rho), C.c_void_p(ux), C.c_void_p(uy),
                                C.c_void_p(T), int(on_device)), h)


def lbm_state_bytes(h) -> int:
    n = C.c_size_t()
    _check(lib().lbm_state_bytes(h, C.byref(n)), h)
    return n.value


def lbm_get_state(h) -> bytes:
    n = lbm_state_bytes(h)
    buf = C.create_string_buffer(n)
    _check(lib().lbm_get_state(h, buf, n), h)
    return buf.raw


def lbm_set_state(h, state: bytes):
    buf = C.create_string_buffer(state, len(state))
    _check(lib().lbm_set_state(h, buf, len(state)), h)


def lbm_steps_done(h) -> int:
    return lib().lbm_steps_done(h)


def lbm_last_error(h) -> str:
    return lib().lbm_last_error(h).decode()


def lbm_destroy(h):
    if h:
        lib().lbm_destroy(h)


def lbm_cbc_side_step_noalloc(lattice, side, length, tau, params, ub_ptr, strip_t_ptr,
                              strip_t1_ptr, neq_t_ptr=0, stream_ptr=0):
    """Allocation-free boundary step of one side (device pointers as ints);
    see include/lbm_cbc.h for the layouts."""
    _check(lib().lbm_cbc_side_step_noalloc(int(lattice), int(side), int(length), float(tau),
                                           C.byref(params), C.c_void_p(ub_ptr),
                                           C.c_void_p(strip_t_ptr), C.c_void_p(strip_t1_ptr),
                                           C.c_void_p(neq_t_ptr or None), C.c_void_p(stream_ptr or None)))


def lbm_grad_begin(h):
    _check(lib().lbm_grad_begin(h), h)


def lbm_grad_begin_along(h, dirs):
    """dirs: 3 x 5 numbers, direction k over THETA."""
    flat = [float(v) for row in dirs for v in row]
    if len(flat) != 15:
        raise ValueError("directions must be 3 x 5")
    _check(lib().lbm_grad_begin_along(h, (C.c_double * 15)(*flat)), h)


def lbm_grad_step(h, n, dP_ref_ptr=None, ref_stride=0):
    _check(lib().lbm_grad_step(h, n, dP_ref_ptr, ref_stride), h)


def lbm_grad_result(h):
    """(J, [the derivatives along the three directions])"""
    J = C.c_double()
    dJ = (C.c_double * 3)()
    _check(lib().lbm_grad_result(h, C.byref(J), dJ), h)
    return J.value, list(dJ)


def lbm_grad_end(h):
    _check(lib().lbm_grad_end(h), h)


def lbm_adj_begin(h, checkpoint_every, max_steps):
    _check(lib().lbm_adj_begin(h, int(checkpoint_every), int(max_steps)), h)


def lbm_adj_forward(h, n, dP_ref_ptr=None, ref_stride=0):
    """n steps with checkpoints; returns the loss J."""
    J = C.c_double()
    _check(lib().lbm_adj_forward(h, int(n), dP_ref_ptr, ref_stride, C.byref(J)), h)
    return J.value


def lbm_adj_backward(h):
    """dJ/d(alpha_T, beta_P, P_inf, alpha_V, t_inf) of the last forward."""
    dJ = (C.c_double * 5)()
    _check(lib().lbm_adj_backward(h, dJ), h)
    return list(dJ)


def lbm_adj_end(h):
    _check(lib().lbm_adj_end(h), h)


def _check_batch(rc, b):
    if rc != 0:
        raise LbmError(rc, lib().lbm_batch_last_error(b).decode() if b else "")


def lbm_batch_create(lattices, nxs, nys, taus, params):
    n = len(lattices)
    if not (len(nxs) == len(nys) == len(taus) == len(params) == n):
        raise ValueError("lbm_batch_create: per-run lists differ in length")
    ints = C.c_int * n
    P = (LbmCbcParams * n)(*params)
    b = C.c_void_p()
    _check(lib().lbm_batch_create(n, ints(*lattices), ints(*nxs), ints(*nys),
                                  (C.c_double * n)(*taus), P, C.byref(b)))
    return b.value


def lbm_batch_run(b, r):
    h = C.c_void_p()
    _check_batch(lib().lbm_batch_run(b, r, C.byref(h)), b)
    return h.value


def lbm_batch_set_stream(b, stream_ptr):
    _check_batch(lib().lbm_batch_set_stream(b, stream_ptr), b)


def lbm_batch_step(b, n):
    _check_batch(lib().lbm_batch_step(b, n), b)


def lbm_batch_ctas_per_sm(b, lattice, storage) -> int:
    rc = lib().lbm_batch_ctas_per_sm(b, lattice, storage)
    if rc < 0:
        _check_batch(rc, b)
    return rc


def lbm_batch_destroy(b):
    if b:
        lib().lbm_batch_destroy(b)


# ---------------------------------------------------------- convenience ---

class Simulation:
    """One solver instance built from a run description.

    The device workspace is a torch uint8 tensor (``lbm_create_in``) and work
    is issued on torch's current CUDA stream, so torch events and streams
    order with the solver's kernels.
    """

    def __init__(self, cfg, device=None):
        import torch
        self.cfg = dict(cfg)
        self.lattice = LATTICES[cfg["lattice"]]
        self.nx, self.ny = int(cfg["nx"]), int(cfg["ny"])
        self.tau = float(cfg["tau"])
        self.params = params_from_run(cfg)
        self.device = torch.device(device or "cuda")
        nbytes = lbm_workspace_bytes(self.lattice, self.nx, self.ny, self.params)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        off = (-base) % 256
        self.handle = lbm_create_in(self.lattice, self.nx, self.ny, self.tau, self.params,
                                    base + off, nbytes)
        self.stream = torch.cuda.current_stream(self.device)
        lbm_set_stream(self.handle, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "handle", None):
            lbm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def steps_done(self):
        return lbm_steps_done(self.handle)

    def init_fields(self, rho, ux, uy, T):
        lbm_init_fields(self.handle, self.nx * self.ny, rho, ux, uy, T)
        return self

    def step(self, n=1):
        lbm_step(self.handle, n)
        return self

    def step_phase(self, phase):
        lbm_step_phase(self.handle, phase)

    def macros(self, device=False):
        """(rho, ux, uy, T): numpy [ny, nx] arrays, or CUDA tensors if device."""
        import torch
        if device:
            out = [torch.empty((self.ny, self.nx), dtype=torch.float64, device=self.device)
                   for _ in range(4)]
            lbm_get_macros(self.handle, *[t.data_ptr() for t in out], 1)
            return tuple(out)
        out = [np.empty((self.ny, self.nx)) for _ in range(4)]
        lbm_get_macros(self.handle, *[a.ctypes.data for a in out], 0)
        return tuple(out)

    def get_state(self) -> bytes:
        return lbm_get_state(self.handle)

    def set_state(self, state: bytes):
        lbm_set_state(self.handle, state)


class _BatchRun:
    """View of one run of a Batch (its handle is owned by the batch)."""

    def __init__(self, batch, r, cfg):
        self.batch, self.index, self.cfg = batch, r, dict(cfg)
        self.nx, self.ny = int(cfg["nx"]), int(cfg["ny"])
        self.device = batch.device
        self.handle = lbm_batch_run(batch.handle, r)

    steps_done = Simulation.steps_done
    init_fields = Simulation.init_fields
    macros = Simulation.macros
    get_state = Simulation.get_state


class Batch:
    """Many independent runs (lattices, sizes, relaxation times and boundary
    parameters may all differ) stepped together: per lattice and storage one
    batched band launch and one persistent bulk launch a step, replayed as a
    CUDA graph once the first steps are done.  Work is issued on torch's
    current CUDA stream."""

    def __init__(self, cfgs, device=None):
        import torch
        cfgs = list(cfgs)
        self.device = torch.device(device or "cuda")
        with torch.cuda.device(self.device):
            self.handle = lbm_batch_create([LATTICES[c["lattice"]] for c in cfgs],
                                           [int(c["nx"]) for c in cfgs],
                                           [int(c["ny"]) for c in cfgs],
                                           [float(c["tau"]) for c in cfgs],
                                           [params_from_run(c) for c in cfgs])
        self.stream = torch.cuda.current_stream(self.device)
        lbm_batch_set_stream(self.handle, self.stream.cuda_stream)
        self.runs = [_BatchRun(self, r, c) for r, c in enumerate(cfgs)]

    def __len__(self):
        return len(self.runs)

    def __getitem__(self, r):
        return self.runs[r]

    def step(self, n=1):
        lbm_batch_step(self.handle, n)
        return self

    def ctas_per_sm(self, lattice, storage):
        return lbm_batch_ctas_per_sm(self.handle, LATTICES[lattice] if isinstance(lattice, str)
                                     else lattice, STORAGES[storage] if isinstance(storage, str)
                                     else storage)

    def close(self):
        if getattr(self, "handle", None):
            lbm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------- gradients ---

THETA = ("alpha_T", "beta_P", "p_inf", "alpha_V", "t_inf")
"""The relaxation parameters gradient steps differentiate, in the order of
lbm_grad_begin_along's directions (p_inf: every characteristic side)."""


def pressure_loss_and_gradient(cfg, fields, steps, dP_ref=None, device=None, directions=None):
    """J = sum over `steps` steps and the nodes off the boundary layers of
    (P - c_s^2 rho0 - dP_ref)^2, and its derivatives along three directions
    in THETA (default: d/dalpha_T, d/dbeta_P, d/dP_inf), by tangent-linear
    steps of a fresh solver (lbm_grad_*).  dP_ref: None or a CUDA float64
    tensor [steps, ny, nx]; directions: None or 3 x 5 numbers.  Returns
    (J, [3 derivatives])."""
    import torch
    sim = Simulation(cfg, device=device).init_fields(*fields)
    try:
        if directions is None:
            lbm_grad_begin(sim.handle)
        else:
            lbm_grad_begin_along(sim.handle, directions)
        if dP_ref is None:
            lbm_grad_step(sim.handle, steps)
        else:
            ref = dP_ref.contiguous()
            if ref.dtype != torch.float64 or tuple(ref.shape) != (steps, sim.ny, sim.nx):
                raise ValueError("dP_ref must be float64 [steps, ny, nx]")
            lbm_grad_step(sim.handle, steps, ref.data_ptr(), sim.ny * sim.nx)
        J, dJ = lbm_grad_result(sim.handle)
        lbm_grad_end(sim.handle)
    finally:
        sim.close()
    return J, dJ


def with_parameters(cfg, params, values):
    """A copy of cfg with the named THETA parameters set (p_inf on every
    side)."""
    c = dict(cfg)
    for name, v in zip(params, values):
        if name not in THETA:
            raise ValueError("unknown relaxation parameter %r" % (name,))
        c[name] = [float(v)] * 4 if name == "p_inf" else float(v)
    return c


def pressure_loss_gradient_in(cfg, fields, steps, params, dP_ref=None, device=None):
    """(J, dJ/dparams) for any of the THETA parameters: one run of gradient
    steps per three of them."""
    params = list(params)
    grads = []
    J = None
    for g0 in range(0, len(params), 3):
        dirs = [[0.0] * 5 for _ in range(3)]
        chunk = params[g0:g0 + 3]
        for k, name in enumerate(chunk):
            dirs[k][THETA.index(name)] = 1.0
        J, dJ = pressure_loss_and_gradient(cfg, fields, steps, dP_ref, device, dirs)
        grads += dJ[:len(chunk)]
    return J, grads


def _make_cbc_loss():
    import torch

    class CBCLoss(torch.autograd.Function):
        """J(theta) for theta over named THETA parameters as a
        differentiable function: forward runs the tangent-linear steps
        (which give J and its derivatives together), backward scales the
        stored derivatives."""

        @staticmethod
        def forward(ctx, theta, cfg, fields, steps, dP_ref, params):
            th = theta.detach().cpu().double().tolist()
            J, dJ = pressure_loss_gradient_in(with_parameters(cfg, params, th), fields, steps, params, dP_ref)
            ctx.save_for_backward(torch.tensor(dJ, dtype=theta.dtype, device=theta.device))
            return torch.tensor(J, dtype=theta.dtype, device=theta.device)

        @staticmethod
        def backward(ctx, grad_out):
            (dJ,) = ctx.saved_tensors
            return grad_out * dJ, None, None, None, None, None

    return CBCLoss


def _ref_arg(sim, dP_ref, steps):
    import torch
    if dP_ref is None:
        return None, 0, None
    ref = dP_ref.contiguous()
    if ref.dtype != torch.float64 or tuple(ref.shape) != (steps, sim.ny, sim.nx):
        raise ValueError("dP_ref must be float64 [steps, ny, nx]")
    return ref.data_ptr(), sim.ny * sim.nx, ref


def pressure_loss_gradient_adjoint(cfg, fields, steps, dP_ref=None, checkpoint_every=100, device=None):
    """(J, dJ/dTHETA) -- all five relaxation parameters -- by the
    reverse-mode sweep with a checkpoint every `checkpoint_every` steps
    (lbm_adj_*) on a fresh solver.  dP_ref: None or a CUDA float64 tensor
    [steps, ny, nx]."""
    sim = Simulation(cfg, device=device).init_fields(*fields)
    try:
        lbm_adj_begin(sim.handle, checkpoint_every, steps)
        ptr, stride, keep = _ref_arg(sim, dP_ref, steps)
        J = lbm_adj_forward(sim.handle, steps, ptr, stride)
        dJ = lbm_adj_backward(sim.handle)
        del keep
        lbm_adj_end(sim.handle)
    finally:
        sim.close()
    return J, dJ


def _make_cbc_loss_adjoint():
    import torch

    class CBCLossAdjoint(torch.autograd.Function):
        """J(theta) as a differentiable function computed in reverse mode:
        forward runs the checkpointed forward steps (J), backward the
        reverse sweep (dJ/dtheta for all parameters at once)."""

        @staticmethod
        def forward(ctx, theta, cfg, fields, steps, dP_ref, params, checkpoint_every):
            th = theta.detach().cpu().double().tolist()
            sim = Simulation(with_parameters(cfg, params, th), device=theta.device if theta.is_cuda else None)
            sim.init_fields(*fields)
            lbm_adj_begin(sim.handle, checkpoint_every, steps)
            ptr, stride, keep = _ref_arg(sim, dP_ref, steps)
            J = lbm_adj_forward(sim.handle, steps, ptr, stride)
            ctx.sim, ctx.keep, ctx.params = sim, keep, params
            return torch.tensor(J, dtype=theta.dtype, device=theta.device)

        @staticmethod
        def backward(ctx, grad_out):
            sim = ctx.sim
            try:
                dJ = lbm_adj_backward(sim.handle)
                lbm_adj_end(sim.handle)
            finally:
                sim.close()
            g = torch.tensor([dJ[THETA.index(n)] for n in ctx.params], dtype=grad_out.dtype,
                             device=grad_out.device)
            return grad_out * g, None, None, None, None, None, None

    return CBCLossAdjoint


_CBCLoss = None
_CBCLossAdjoint = None


def cbc_loss_adjoint(theta, cfg, fields, steps, dP_ref=None, params=THETA, checkpoint_every=100):
    """Differentiable pressure loss J(theta) (torch autograd) whose
    backward is the reverse-mode sweep: theta a tensor of the named THETA
    parameters (default all five)."""
    global _CBCLossAdjoint
    if _CBCLossAdjoint is None:
        _CBCLossAdjoint = _make_cbc_loss_adjoint()
    return _CBCLossAdjoint.apply(theta, cfg, fields, steps, dP_ref, tuple(params), int(checkpoint_every))


def cbc_loss(theta, cfg, fields, steps, dP_ref=None, params=("alpha_T", "beta_P", "p_inf")):
    """Differentiable pressure loss J(theta) (torch autograd), theta a tensor
    of the named THETA parameters (default alpha_T, beta_P, P_inf)."""
    global _CBCLoss
    if _CBCLoss is None:
        _CBCLoss = _make_cbc_loss()
    return _CBCLoss.apply(theta, cfg, fields, steps, dP_ref, tuple(params))

"""Python binding of libpemlbm (argument marshalling only: every step of the
coupled cathode update runs in the library's CUDA kernels).

The names mirror the C ABI of include/pemlbm.h.  Importing this module on a
machine without the built library raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpemlbm.so")
# PEMLBM_LIB selects another build of the same library (the bounds-checked
# libpemlbm_checked.so of build.build(bounds_check=True)); it must exist.
LIB_PATH = os.environ.get("PEMLBM_LIB", LIB_PATH)

FP64, FP32, BF16, FP16 = 0, 1, 2, 3
PRECISION = {"fp64": FP64, "fp32": FP32, "bf16": BF16, "fp16": FP16}
STATUS = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA", 4: "LBM_ESTATE",
          5: "LBM_EDIVERGED", 6: "LBM_ETIMEOUT"}

# Every symbol the header declares (the CPU tests check the exports).
EXPORTS = ("lbm_create_domain", "lbm_destroy_domain", "lbm_set_params", "lbm_set_fields",
           "lbm_reset", "lbm_step", "lbm_current_density", "lbm_residual", "lbm_get_fields",
           "lbm_get_state", "lbm_set_state", "lbm_get_mask", "lbm_get_step", "lbm_save_state",
           "lbm_load_state", "lbm_time_steps", "lbm_bytes_per_cell", "lbm_tune",
           "lbm_set_variant", "lbm_residual_noalloc", "lbm_balances", "lbm_step_observe",
           "lbm_create_batch", "lbm_destroy_batch",
           "lbm_batch_set_schedule", "lbm_batch_tune", "lbm_batch_step", "lbm_batch_time_steps",
           "lbm_grad", "lbm_set_grad_memory", "lbm_bounds_check", "lbm_vjp",
           "lbm_halo_exchange", "lbm_halo_pack", "lbm_halo_unpack",
           "lbm_last_error")


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class lbm_domain_desc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("ny_cl", C.c_int32),
                ("ny_gdl", C.c_int32), ("reaction_mode", C.c_int32), ("periodic_x", C.c_int32),
                ("closed_x", C.c_int32), ("precision", C.c_int32), ("rounding", C.c_int32),
                ("solid", C.POINTER(C.c_uint8)), ("cuda_stream", C.c_void_p),
                ("x_begin", C.c_int32), ("x_end", C.c_int32)]


_PARAM_DOUBLES = ("nu", "u_in_avg", "body_force_x", "V_op", "T_in", "C_O2_in", "C_H2O_in",
                  "T_top", "C_O2_top", "C_H2O_top", "aj0_ref", "T_ref_kin", "E_act", "alpha_c",
                  "F", "R", "dU0dT", "U0_0", "x_ref", "dx_cm", "dt_s", "delta_cl_cm", "c_tot",
                  "rho_cp_f")


class lbm_params(C.Structure):
    _fields_ = [(k, C.c_double) for k in _PARAM_DOUBLES] + [
        ("forchheimer", C.c_int32), ("top_dirichlet", C.c_int32),
        ("interface_mode", C.c_int32), ("inlet_mode", C.c_int32), ("dp_in", C.c_double),
        ("alpha_a", C.c_double), ("buoy_gx", C.c_double), ("buoy_gy", C.c_double),
        ("T_buoy", C.c_double), ("wall_dirichlet", C.c_int32), ("C_wall", (C.c_double * 3) * 3),
        ("scalar_advection", C.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libpemlbm.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2103_01444_gb300.build.build()")
    L = C.CDLL(path)
    P, d = C.c_void_p, C.POINTER(C.c_double)
    sig = {
        "lbm_create_domain": [C.POINTER(lbm_domain_desc), C.POINTER(P)],
        "lbm_destroy_domain": [P],
        "lbm_set_params": [P, C.POINTER(lbm_params)],
        "lbm_set_fields": [P, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                           C.c_void_p, C.c_int32],
        "lbm_reset": [P],
        "lbm_step": [P, C.c_int64],
        "lbm_current_density": [P, d, d, C.POINTER(C.c_float)],
        "lbm_residual": [P, d],
        "lbm_balances": [P, d],
        "lbm_step_observe": [P, C.c_int64, d, d],
        "lbm_get_fields": [P, C.c_void_p, C.c_int32],
        "lbm_get_state": [P, d],
        "lbm_set_state": [P, d],
        "lbm_get_mask": [P, C.POINTER(C.c_uint8)],
        "lbm_get_step": [P, C.POINTER(C.c_int64)],
        "lbm_save_state": [P, C.c_void_p, C.POINTER(C.c_size_t)],
        "lbm_load_state": [P, C.c_void_p, C.c_size_t],
        "lbm_time_steps": [P, C.c_int64, d],
        "lbm_bytes_per_cell": [P, d],
        "lbm_tune": [P, C.c_int32, C.POINTER(C.c_int32), d],
        "lbm_set_variant": [P, C.c_int32],
        "lbm_set_grad_memory": [P, C.c_int64],
        "lbm_bounds_check": [C.POINTER(C.c_uint64)],
        "lbm_residual_noalloc": [P, C.c_void_p, d],
        "lbm_create_batch": [C.POINTER(P), C.c_int32, C.POINTER(P)],
        "lbm_destroy_batch": [P],
        "lbm_batch_set_schedule": [P, C.c_int32, C.c_int32, C.c_int64],
        "lbm_batch_tune": [P, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32), d],
        "lbm_batch_step": [P, C.c_int64],
        "lbm_batch_time_steps": [P, C.c_int64, d],
        "lbm_grad": [P, C.c_int32, C.c_int64, C.c_int32, d, C.c_void_p, C.c_void_p, C.c_void_p, d,
                     C.c_int32],
        "lbm_vjp": [P, d, d, d, d, d, d],
        "lbm_halo_exchange": [P, P],
        "lbm_halo_pack": [P, C.c_int32, C.c_void_p],
        "lbm_halo_unpack": [P, C.c_int32, C.c_void_p],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.lbm_last_error.argtypes = []
    L.lbm_last_error.restype = C.c_char_p
    _lib = L
    return L


def _check(status):
    if status != 0:
        raise LbmError(status, _lib.lbm_last_error().decode())


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def check_device_buffer(t, dtype: str, shape: tuple, device, name: str = "buffer"):
    """Refuses (LbmError EINVAL) a tensor that the library would read or
    write through a bare device pointer unless it is a contiguous CUDA tensor
    of the given dtype name and shape on the given device index."""
    bad = None
    if not getattr(t, "is_cuda", False):
        bad = "is not a CUDA tensor"
    elif device is not None and t.device.index != device:
        bad = f"is on cuda:{t.device.index}, the domain on cuda:{device}"
    elif str(t.dtype).replace("torch.", "") != dtype:
        bad = f"has dtype {t.dtype}, needs {dtype}"
    elif tuple(t.shape) != tuple(shape):
        bad = f"has shape {tuple(t.shape)}, needs {tuple(shape)}"
    elif not t.is_contiguous():
        bad = "is not contiguous"
    if bad:
        raise LbmError(1, f"{name} {bad}")


def _current_device():
    """The current CUDA device index (the device a new domain lives on)."""
    try:
        import torch
        return torch.cuda.current_device() if torch.cuda.is_available() else None
    except ImportError:
        return None


class Domain:
    """One cathode lattice on the GPU (wraps an lbm_domain handle)."""

    def __init__(self, nx, ny, ny_cl=0, ny_gdl=0, reaction_mode=0, periodic_x=0,
                 precision="fp32", solid=None, stream=None, rounding="nearest", closed_x=0,
                 x_begin=0, x_end=0):
        """rounding: "nearest" or "stochastic" (16-bit storage only);
        x_begin, x_end: the x-slab of the nx-column lattice this domain owns
        (0, 0: all of it); nx, ny and solid describe the whole lattice."""
        self.L = load_library()
        self.nx, self.ny = int(nx), int(ny)
        self._solid = None if solid is None else np.ascontiguousarray(solid, np.uint8)
        self.nx_lattice = self.nx
        if x_end:
            self.nx = int(x_end) - int(x_begin)
        desc = lbm_domain_desc(
            nx=self.nx_lattice, ny=self.ny, ny_cl=int(ny_cl), ny_gdl=int(ny_gdl),
            reaction_mode=int(reaction_mode), periodic_x=int(periodic_x), closed_x=int(closed_x),
            precision=PRECISION[precision] if isinstance(precision, str) else int(precision),
            rounding={"nearest": 0, "stochastic": 1}[rounding],
            solid=None if self._solid is None else self._solid.ctypes.data_as(C.POINTER(C.c_uint8)),
            cuda_stream=None if stream is None else C.c_void_p(int(stream)),
            x_begin=int(x_begin), x_end=int(x_end))
        h = C.c_void_p()
        _check(self.L.lbm_create_domain(C.byref(desc), C.byref(h)))
        self.h = h
        self.precision = desc.precision
        self.device = _current_device()

    @classmethod
    def from_case(cls, case: dict, precision="fp32", forchheimer: int = 1, stream=None,
                  reset: bool = True, interface_mode: int = 0, rounding="nearest"):
        from .units import cathode_params
        params, fields, geo = cathode_params(case, forchheimer, interface_mode)
        d = cls(precision=precision, stream=stream, rounding=rounding, **geo)
        d.set_params(params)
        d.set_fields(**fields)
        if reset:
            d.reset()
        return d

    def close(self):
        if getattr(self, "h", None):
            self.L.lbm_destroy_domain(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- set-up
    def set_params(self, params: dict):
        self.params = dict(params)
        p = dict(params)
        if "C_wall" in p:   # [wall][scalar] values
            w = np.asarray(p["C_wall"], np.float64).reshape(3, 3)
            p["C_wall"] = ((C.c_double * 3) * 3)(*[(C.c_double * 3)(*row) for row in w])
        _check(self.L.lbm_set_params(self.h, C.byref(lbm_params(**p))))

    def set_fields(self, phi, K, alpha_T, D_O2, D_H2O, rho_cp_ratio=None):
        """Per-cell material.  Host values (arrays or scalars) are copied from
        the host; if every given field is a CUDA tensor (float64, (ny, nx),
        contiguous, on the domain's device) the library reads them in place
        on the domain's stream and builds the palette on the device.  An
        x-slab takes the whole lattice's host arrays."""
        given = [a for a in (phi, K, alpha_T, D_O2, D_H2O, rho_cp_ratio) if a is not None]
        if all(getattr(a, "is_cuda", False) for a in given):
            for name, a in zip(("phi", "K", "alpha_T", "D_O2", "D_H2O", "rho_cp_ratio"),
                               (phi, K, alpha_T, D_O2, D_H2O, rho_cp_ratio)):
                if a is not None:
                    check_device_buffer(a, "float64", (self.ny, self.nx), self.device, name)
            ptr = lambda a: None if a is None else C.c_void_p(a.data_ptr())  # noqa: E731
            _check(self.L.lbm_set_fields(self.h, ptr(phi), ptr(K), ptr(alpha_T), ptr(D_O2),
                                         ptr(D_H2O), ptr(rho_cp_ratio), 1))
            return
        shape = (self.ny, self.nx_lattice)
        host = lambda a: np.ascontiguousarray(  # noqa: E731
            np.broadcast_to(np.asarray(a.cpu() if hasattr(a, "cpu") else a, np.float64), shape))
        arrs = [host(a) for a in (phi, K, alpha_T, D_O2, D_H2O)]
        sig = None if rho_cp_ratio is None else host(rho_cp_ratio)
        _check(self.L.lbm_set_fields(self.h, *[a.ctypes.data_as(C.c_void_p) for a in arrs],
                                     None if sig is None else sig.ctypes.data_as(C.c_void_p), 0))

    def reset(self):
        _check(self.L.lbm_reset(self.h))

    # -- stepping
    def step(self, n: int = 1):
        _check(self.L.lbm_step(self.h, int(n)))
        return self

    def time_steps(self, n: int) -> float:
        ms = C.c_double()
        _check(self.L.lbm_time_steps(self.h, int(n), C.byref(ms)))
        return ms.value

    @property
    def steps(self) -> int:
        s = C.c_int64()
        _check(self.L.lbm_get_step(self.h, C.byref(s)))
        return s.value

    # -- read-outs
    def current_density(self, profile: bool = True):
        i_avg, heat = C.c_double(), C.c_double()
        prof = np.zeros(self.nx, np.float32) if profile else None
        _check(self.L.lbm_current_density(
            self.h, C.byref(i_avg), C.byref(heat),
            None if prof is None else prof.ctypes.data_as(C.POINTER(C.c_float))))
        return i_avg.value, heat.value, prof

    def step_observe(self, nsteps: int, i_avg=None, heat=None):
        """nsteps steps with the reaction of every step: (i_avg, heat)
        arrays (A/cm^2, W/cm^2).  Output arrays may be passed in (float64,
        e.g. pinned)."""
        i_avg = np.zeros(nsteps) if i_avg is None else i_avg
        heat = np.zeros(nsteps) if heat is None else heat
        assert i_avg.dtype == np.float64 and heat.dtype == np.float64
        assert i_avg.size >= nsteps and heat.size >= nsteps
        _check(self.L.lbm_step_observe(self.h, int(nsteps), _dp(i_avg), _dp(heat)))
        return i_avg, heat

    BALANCE_KEYS = ("J", "heat", "in_mass", "in_T", "in_O2", "in_H2O",
                    "out_mass", "out_T", "out_O2", "out_H2O")

    def balances(self) -> dict:
        """Balances of the last step (lattice units): O2 consumed, its heat,
        and the net inflows through the inlet and outlet columns."""
        out = np.zeros(10)
        _check(self.L.lbm_balances(self.h, _dp(out)))
        return dict(zip(self.BALANCE_KEYS, out.tolist()))

    def residual(self) -> float:
        r = C.c_double()
        _check(self.L.lbm_residual(self.h, C.byref(r)))
        return r.value

    def residual_noalloc(self, snapshot) -> float:
        """Residual of lbm_residual against a caller-held snapshot (a CUDA
        tensor of shape (5, ny, nx), float64 for FP64 domains, float32
        otherwise), computed with the library's static scratch.  The C call
        cannot check the buffer it is given, so its type, shape, layout and
        device are checked here before anything runs (EINVAL)."""
        check_device_buffer(snapshot, "float64" if self.precision == FP64 else "float32",
                            (5, self.ny, self.nx), self.device, "snapshot")
        r = C.c_double()
        _check(self.L.lbm_residual_noalloc(self.h, C.c_void_p(snapshot.data_ptr()), C.byref(r)))
        return r.value

    def grad(self, objective: int = 0, nsteps: int = 100, segment: int = 0, out=None):
        """Objective after nsteps from the current state and its gradient:
        (J, {"phi", "K", "D_O2": [ny][nx] arrays, "u_in": float}); "u_in" is
        the derivative by the inlet drive, u_in_avg (inlet_mode 0) or dp_in
        (inlet_mode 1).  With ``out`` (a dict of CUDA float64 tensors of shape
        (ny, nx) under "phi", "K", "D_O2") the gradients are written there on
        the domain's stream instead of to host arrays."""
        J, du = C.c_double(), C.c_double()
        keys = ("phi", "K", "D_O2")
        if out is not None:
            for k in keys:
                check_device_buffer(out[k], "float64", (self.ny, self.nx), self.device, "d" + k)
            ptrs = [C.c_void_p(out[k].data_ptr()) for k in keys]
            g, on_device = dict(out), 1
        else:
            g = {k: np.zeros((self.ny, self.nx)) for k in keys}
            ptrs = [g[k].ctypes.data_as(C.c_void_p) for k in keys]
            on_device = 0
        _check(self.L.lbm_grad(self.h, int(objective), int(nsteps), int(segment), C.byref(J),
                               *ptrs, C.byref(du), on_device))
        g["u_in"] = du.value
        return J.value, g

    def set_grad_memory(self, nbytes: int):
        """Device bytes grad() may keep reverse records in: -1 for what is
        free (the default), 0 to recompute every segment from its
        checkpoint."""
        _check(self.L.lbm_set_grad_memory(self.h, int(nbytes)))

    def vjp(self, lam_next):
        """One transposed step at the current state: (lam_prev, gradients)."""
        lam = np.ascontiguousarray(lam_next, np.float64)
        assert lam.shape == (24, self.ny, self.nx)
        out = np.zeros_like(lam)
        du = C.c_double()
        g = {k: np.zeros((self.ny, self.nx)) for k in ("phi", "K", "D_O2")}
        _check(self.L.lbm_vjp(self.h, _dp(lam), _dp(out), _dp(g["phi"]), _dp(g["K"]),
                              _dp(g["D_O2"]), C.byref(du)))
        g["u_in"] = du.value
        return out, g

    def fields(self, out=None):
        """dict of [ny][nx] float64 arrays ux, uy, p, T, C_O2, C_H2O; with a
        CUDA tensor ``out`` of shape (6, ny, nx) float64 they are written there
        on the domain's stream instead."""
        if out is not None:
            _check(self.L.lbm_get_fields(self.h, C.c_void_p(out.data_ptr()), 1))
            return out
        a = np.empty((6, self.ny, self.nx))
        _check(self.L.lbm_get_fields(self.h, a.ctypes.data_as(C.c_void_p), 0))
        return dict(zip(("ux", "uy", "p", "T", "C_O2", "C_H2O"), a))

    def state(self):
        """Full post-collision populations, (24, ny, nx) float64."""
        a = np.empty((24, self.ny, self.nx))
        _check(self.L.lbm_get_state(self.h, _dp(a)))
        return a

    def set_state(self, pops):
        a = np.ascontiguousarray(pops, np.float64)
        assert a.shape == (24, self.ny, self.nx)
        _check(self.L.lbm_set_state(self.h, _dp(a)))

    def mask(self):
        m = np.empty((self.ny, self.nx), np.uint8)
        _check(self.L.lbm_get_mask(self.h, m.ctypes.data_as(C.POINTER(C.c_uint8))))
        return m

    def save_state(self) -> bytes:
        n = C.c_size_t()
        _check(self.L.lbm_save_state(self.h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(self.L.lbm_save_state(self.h, buf, C.byref(n)))
        return buf.raw

    def load_state(self, blob: bytes):
        _check(self.L.lbm_load_state(self.h, blob, len(blob)))

    def tune(self, trial_steps: int = 20):
        """Times every launch shape of the step kernel (after reset, before the
        first step) and keeps the fastest; returns (variant, ms per step)."""
        v, ms = C.c_int32(), C.c_double()
        _check(self.L.lbm_tune(self.h, int(trial_steps), C.byref(v), C.byref(ms)))
        return v.value, ms.value

    def set_variant(self, v: int):
        _check(self.L.lbm_set_variant(self.h, int(v)))

    def bytes_per_cell(self) -> float:
        b = C.c_double()
        _check(self.L.lbm_bytes_per_cell(self.h, C.byref(b)))
        return b.value


class Batch:
    """Many domains stepped together (lbm_create_batch); the domains stay
    usable through their own methods."""

    SCHEDULES = {"graph": 0, "persistent": 1, "per-case": 2, "concurrent": 3}

    def __init__(self, domains):
        self.L = load_library()
        self.domains = list(domains)
        arr = (C.c_void_p * len(self.domains))(*[d.h for d in self.domains])
        h = C.c_void_p()
        _check(self.L.lbm_create_batch(arr, len(self.domains), C.byref(h)))
        self.h = h

    def set_schedule(self, schedule, variant: int = 6, spin_limit: int = 0):
        sch = self.SCHEDULES.get(schedule, schedule)
        _check(self.L.lbm_batch_set_schedule(self.h, int(sch), int(variant), int(spin_limit)))

    def tune(self, trial_steps: int = 10):
        sch, var, ms = C.c_int32(), C.c_int32(), C.c_double()
        _check(self.L.lbm_batch_tune(self.h, int(trial_steps), C.byref(sch), C.byref(var),
                                     C.byref(ms)))
        return sch.value, var.value, ms.value

    def step(self, n: int = 1):
        _check(self.L.lbm_batch_step(self.h, int(n)))
        return self

    def time_steps(self, n: int) -> float:
        ms = C.c_double()
        _check(self.L.lbm_batch_time_steps(self.h, int(n), C.byref(ms)))
        return ms.value

    def close(self):
        if getattr(self, "h", None):
            self.L.lbm_destroy_batch(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cathode_objective():
    """torch.autograd.Function over the lattice material and inlet drive:
    CathodeObjective.apply(phi, K, D_O2, u_in, domain, fields, params,
    objective, nsteps, segment) sets the domain's material (phi, K, D_O2 from
    the tensors, alpha_T, D_H2O, rho_cp_ratio from `fields`) and the drive
    (u_in_avg, or dp_in when params["inlet_mode"] is 1) to u_in, resets it, and returns the objective after nsteps; backward returns the
    adjoint gradients computed by lbm_grad."""
    import torch

    class CathodeObjective(torch.autograd.Function):
        @staticmethod
        def forward(ctx, phi, K, D_O2, u_in, domain, fields, params, objective, nsteps, segment):
            p = dict(params)
            p["dp_in" if p.get("inlet_mode", 0) == 1 else "u_in_avg"] = float(u_in)
            domain.set_params(p)
            dev = phi.device
            if phi.is_cuda:
                # CUDA tensors stay on the device: the library reads the
                # material in place and writes the gradients into tensors
                # allocated here, all on the domain's stream
                on = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev).contiguous()  # noqa: E731
                sig = fields.get("rho_cp_ratio")
                domain.set_fields(phi.detach().contiguous(), K.detach().contiguous(),
                                  on(fields["alpha_T"]), D_O2.detach().contiguous(),
                                  on(fields["D_H2O"]), None if sig is None else on(sig))
                domain.reset()
                out = {k: torch.empty((domain.ny, domain.nx), dtype=torch.float64, device=dev)
                       for k in ("phi", "K", "D_O2")}
                J, g = domain.grad(objective, nsteps, segment, out=out)
                gphi, gK, gD = g["phi"], g["K"], g["D_O2"]
            else:
                domain.set_fields(phi.detach().double().numpy(), K.detach().double().numpy(),
                                  fields["alpha_T"], D_O2.detach().double().numpy(),
                                  fields["D_H2O"], fields.get("rho_cp_ratio"))
                domain.reset()
                J, g = domain.grad(objective, nsteps, segment)
                gphi, gK, gD = (torch.from_numpy(g[k]) for k in ("phi", "K", "D_O2"))
            ctx.save_for_backward(gphi, gK, gD,
                                  torch.tensor(g["u_in"], dtype=torch.float64, device=dev))
            return torch.tensor(J, dtype=torch.float64, device=dev)

        @staticmethod
        def backward(ctx, gJ):
            gphi, gK, gD, gU = ctx.saved_tensors
            return gJ * gphi, gJ * gK, gJ * gD, gJ * gU, None, None, None, None, None, None

    return CathodeObjective


def bounds_check() -> int:
    """First out-of-range device access recorded since the last call by a
    bounds-checked build (site << 48 | index; 0 for none); LbmError ESTATE
    in the plain build."""
    L = load_library()
    v = C.c_uint64()
    _check(L.lbm_bounds_check(C.byref(v)))
    return v.value

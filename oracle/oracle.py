"""ctypes wrapper around the FP64 C oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg.  Shares no code with the CUDA library.

The state is kept as full (not deviation) FP64 populations:
``f`` has shape (9, ny, nx) and ``g`` has shape (3, 5, ny, nx) with the
scalar index 0 = temperature, 1 = O2 mole fraction, 2 = H2O mole fraction.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_TSRC = os.path.join(_HERE, "lbm_oracle_tangent.cc")
_TOUT = os.path.join(_HERE, "_build", "liboracle_tangent.so")
_lock = threading.Lock()
_lib = None
_tlib = None


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with plain gcc (no fast-math) into oracle/_build."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def build_tangent(force: bool = False) -> str:
    """Compile the oracle's tangent (lbm_oracle.c as C++ with dual numbers,
    lbm_oracle_tangent.cc) with plain g++ into oracle/_build."""
    os.makedirs(os.path.dirname(_TOUT), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_TSRC))
    if force or not os.path.exists(_TOUT) or os.path.getmtime(_TOUT) < newest:
        tmp = _TOUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c++17",
                               "-o", tmp, _TSRC, "-lm"])
        os.replace(tmp, _TOUT)
    return _TOUT


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("ny_cl", C.c_int32), ("ny_gdl", C.c_int32),
        ("reaction_mode", C.c_int32), ("periodic_x", C.c_int32),
        ("forchheimer", C.c_int32), ("top_dirichlet", C.c_int32),
        ("interface_mode", C.c_int32), ("inlet_mode", C.c_int32),
        ("closed_x", C.c_int32), ("wall_dirichlet", C.c_int32),
        ("nu", C.c_double), ("u_in_avg", C.c_double), ("body_force_x", C.c_double),
        ("V_op", C.c_double), ("T_in", C.c_double), ("C_O2_in", C.c_double),
        ("C_H2O_in", C.c_double),
        ("T_top", C.c_double), ("C_O2_top", C.c_double), ("C_H2O_top", C.c_double),
        ("aj0_ref", C.c_double), ("T_ref_kin", C.c_double), ("E_act", C.c_double),
        ("alpha_c", C.c_double), ("F", C.c_double), ("R", C.c_double),
        ("dU0dT", C.c_double), ("U0_0", C.c_double), ("x_ref", C.c_double),
        ("dx_cm", C.c_double), ("dt_s", C.c_double), ("delta_cl_cm", C.c_double),
        ("c_tot", C.c_double), ("rho_cp_f", C.c_double), ("dp_in", C.c_double),
        ("alpha_a", C.c_double), ("buoy_gx", C.c_double), ("buoy_gy", C.c_double),
        ("T_buoy", C.c_double), ("C_wall", C.c_double * 9),
        ("scalar_advection", C.c_int32),
    ]


class Material(C.Structure):
    _fields_ = [(k, C.POINTER(C.c_double)) for k in
                ("phi", "K", "alpha_T", "D_O2", "D_H2O", "u_imposed", "sigma")]


_P = C.POINTER
_d = C.POINTER(C.c_double)
_u8 = C.POINTER(C.c_uint8)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build_oracle())
            L.orc_build_mask.argtypes = [_P(Params), _u8, _u8]
            L.orc_init.argtypes = [_P(Params), _P(Material), _u8, _d, _d]
            L.orc_step.argtypes = [_P(Params), _P(Material), _u8, _d, _d, _d, _d, _d, _d, _d]
            L.orc_fields.argtypes = [_P(Params), _P(Material), _u8, _d, _d, _d, _d, _d, _d]
            L.orc_state_moments.argtypes = [_P(Params), _u8, _d, _d, _d]
            L.orc_residual.argtypes = [_P(Params), _u8, _d, _d, _d]
            L.orc_residual.restype = C.c_double
            L.orc_matrices.argtypes = [_d, _d, _d, _d]
            L.orc_flow_meq.argtypes = [C.c_double] * 4 + [_d]
            L.orc_flow_G.argtypes = [C.c_double] * 5 + [_d]
            L.orc_flow_S.argtypes = [C.c_double, _d]
            L.orc_scalar_Q.argtypes = [_d]
            L.orc_d2q5_eq.argtypes = [C.c_double] * 4 + [_d]
            L.orc_velocity.argtypes = [C.c_double] * 4 + [_d, _d]
            L.orc_porous.argtypes = [_P(Params), C.c_double, C.c_double, _d]
            for name in ("orc_U0", "orc_eta", "orc_aj0", "orc_k_surface", "orc_k_volume",
                         "orc_heat_per_O2", "orc_k_surface_anodic", "orc_k_volume_anodic",
                         "orc_anodic_j"):
                getattr(L, name).argtypes = [_P(Params), C.c_double]
                getattr(L, name).restype = C.c_double
            L.orc_tafel_j.argtypes = [_P(Params), C.c_double, C.c_double]
            L.orc_tafel_j.restype = C.c_double
            L.orc_heat_Q.argtypes = [_P(Params), C.c_double, C.c_double]
            L.orc_heat_Q.restype = C.c_double
            L.orc_b_of_alpha.argtypes = [C.c_double]
            L.orc_b_of_alpha.restype = C.c_double
            _lib = L
    return _lib


def _ptr(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


# Index layout of the per-step diagnostics vector.
DIAG = {"J": 0, "heat": 1, "in_mass": 2, "in_T": 3, "in_O2": 4, "in_H2O": 5,
        "out_mass": 6, "out_T": 7, "out_O2": 8, "out_H2O": 9}


class Oracle:
    """One lattice problem: parameters, material, mask and a ping-pong state.

    ``params`` is a dict of the ``Params`` fields; ``material`` a dict with
    per-cell arrays phi, K, alpha_T, D_O2, D_H2O (lattice units, shape
    (ny, nx)) and optionally ``u_imposed`` of shape (2, ny, nx).
    """

    def __init__(self, params: dict, material: dict, solid=None):
        self.L = lib()
        p = dict(params)
        if "C_wall" in p:   # [wall][scalar] values, flattened
            p["C_wall"] = (C.c_double * 9)(*np.asarray(p["C_wall"], np.float64).ravel())
        self.P = Params(**p)
        nx, ny = self.P.nx, self.P.ny
        self.nx, self.ny = nx, ny
        self._mat_arrays = {}
        for k in ("phi", "K", "alpha_T", "D_O2", "D_H2O"):
            a = np.ascontiguousarray(np.broadcast_to(np.asarray(material[k], np.float64),
                                                     (ny, nx)))
            self._mat_arrays[k] = a
        ui = material.get("u_imposed")
        if ui is not None:
            self._mat_arrays["u_imposed"] = np.ascontiguousarray(ui, np.float64)
        if material.get("sigma") is not None:
            self._mat_arrays["sigma"] = np.ascontiguousarray(
                np.broadcast_to(np.asarray(material["sigma"], np.float64), (ny, nx)))
        self.M = Material(**{k: _ptr(v) for k, v in self._mat_arrays.items()})
        self.solid = None if solid is None else np.ascontiguousarray(solid, np.uint8)
        self.mask = np.zeros((ny, nx), np.uint8)
        self.L.orc_build_mask(C.byref(self.P),
                              None if self.solid is None else _ptr(self.solid, C.c_uint8),
                              _ptr(self.mask, C.c_uint8))
        self.f = np.zeros((9, ny, nx))
        self.g = np.zeros((3, 5, ny, nx))
        self.L.orc_init(C.byref(self.P), C.byref(self.M), _ptr(self.mask, C.c_uint8),
                        _ptr(self.f), _ptr(self.g))
        self.f_prev, self.g_prev = self.f.copy(), self.g.copy()
        self.steps = 0
        # residual snapshot: the moments of the initial state
        self.snapshot = np.zeros((5, ny, nx))
        self.residual()
        self.diag = np.zeros(10)
        self.Jx = np.zeros(nx)
        self.qx = np.zeros(nx)

    def step(self, n: int = 1):
        fo = np.empty_like(self.f)
        go = np.empty_like(self.g)
        for _ in range(n):
            self.L.orc_step(C.byref(self.P), C.byref(self.M), _ptr(self.mask, C.c_uint8),
                            _ptr(self.f), _ptr(self.g), _ptr(fo), _ptr(go), _ptr(self.diag),
                            _ptr(self.Jx), _ptr(self.qx))
            self.f_prev, self.f, fo = self.f, fo, self.f_prev
            self.g_prev, self.g, go = self.g, go, self.g_prev
            self.steps += 1
        return self

    def fields(self):
        """Macroscopic fields of the last step: dict ux, uy, p, T, C_O2, C_H2O,
        computed from the post-stream state the last collision used."""
        out = np.zeros((6, self.ny, self.nx))
        diag = np.zeros(10)
        Jx, qx = np.zeros(self.nx), np.zeros(self.nx)
        self.L.orc_fields(C.byref(self.P), C.byref(self.M), _ptr(self.mask, C.c_uint8),
                          _ptr(self.f_prev), _ptr(self.g_prev), _ptr(out), _ptr(diag),
                          _ptr(Jx), _ptr(qx))
        names = ("ux", "uy", "p", "T", "C_O2", "C_H2O")
        d = {k: out[i] for i, k in enumerate(names)}
        d["Jx"], d["qx"], d["diag"] = Jx, qx, diag
        return d

    def state_moments(self):
        out = np.zeros((5, self.ny, self.nx))
        self.L.orc_state_moments(C.byref(self.P), _ptr(self.mask, C.c_uint8), _ptr(self.f),
                                 _ptr(self.g), _ptr(out))
        return out

    def residual(self):
        """Steady-state residual of the current post-collision state against
        the moments of the previous call (or of the initial state): max over
        (sum e_x f, sum e_y f, T - T_in, C_O2, C_H2O) of ||X - X_prev|| / ||X||.
        Replaces the snapshot."""
        return float(self.L.orc_residual(C.byref(self.P), _ptr(self.mask, C.c_uint8),
                                         _ptr(self.f), _ptr(self.g), _ptr(self.snapshot)))

    # -- reported quantities (Sec. 5 performance outputs)
    def current_density(self):
        """(i_avg A/cm^2, heat W/cm^2, i(x) A/cm^2) of the last step's reaction."""
        P = self.P
        scale = 4.0 * P.F * P.c_tot * P.dx_cm / P.dt_s
        ix = self.Jx * scale
        heat = self.qx * P.rho_cp_f * P.dx_cm / P.dt_s
        return float(ix.mean()), float(heat.mean()), ix


# ----------------------------------------------------------------- tangent

class Dual(C.Structure):
    """One real number of the tangent build: value and directional derivative."""
    _fields_ = [("v", C.c_double), ("d", C.c_double)]


def _dual_struct(name, base):
    """The layout of a struct of the tangent build: every double of `base`
    becomes a Dual, arrays of doubles arrays of Duals."""
    fields = []
    for fname, t in base._fields_:
        if t is C.c_double:
            fields.append((fname, Dual))
        elif isinstance(t, type) and issubclass(t, C.Array) and t._type_ is C.c_double:
            fields.append((fname, Dual * t._length_))
        elif t is C.POINTER(C.c_double):
            fields.append((fname, C.POINTER(Dual)))
        else:
            fields.append((fname, t))
    return type(name, (C.Structure,), {"_fields_": fields})


TParams = _dual_struct("TParams", Params)
TMaterial = _dual_struct("TMaterial", Material)
_dd = C.POINTER(Dual)


def tangent_lib():
    global _tlib
    with _lock:
        if _tlib is None:
            L = C.CDLL(build_tangent())
            L.orc_build_mask.argtypes = [_P(TParams), _u8, _u8]
            L.orc_init.argtypes = [_P(TParams), _P(TMaterial), _u8, _dd, _dd]
            L.orc_step.argtypes = [_P(TParams), _P(TMaterial), _u8, _dd, _dd, _dd, _dd, _dd,
                                   _dd, _dd]
            L.orc_fields.argtypes = [_P(TParams), _P(TMaterial), _u8, _dd, _dd, _dd, _dd, _dd,
                                     _dd]
            _tlib = L
    return _tlib


def _pair(value, deriv=None):
    """(..., 2) array of value and derivative parts."""
    value = np.asarray(value, np.float64)
    out = np.zeros(value.shape + (2,))
    out[..., 0] = value
    if deriv is not None:
        out[..., 1] = np.broadcast_to(np.asarray(deriv, np.float64), value.shape)
    return out


class TangentOracle:
    """The oracle run in dual numbers: every quantity carries its derivative
    along one direction w of the inputs, so N steps give the state after N
    steps and its directional derivative J_N w (forward mode, exact up to
    rounding; the oracle's own derivative of its step).

    ``dparams`` maps parameter names (e.g. "u_in_avg", "dp_in") to their
    direction components, ``dmaterial`` material names ("phi", "K",
    "alpha_T", "D_O2", "D_H2O") to per-cell direction arrays; the state's
    direction is given with ``set_state``.  State arrays have a trailing
    axis of two: value, derivative.
    """

    def __init__(self, params: dict, material: dict, solid=None, dparams=None, dmaterial=None):
        self.L = tangent_lib()
        dparams, dmaterial = dparams or {}, dmaterial or {}
        p = dict(params)
        vals = {}
        for name, t in TParams._fields_:
            if name not in p:
                continue
            if t is Dual:
                vals[name] = Dual(float(p[name]), float(dparams.get(name, 0.0)))
            elif isinstance(t, type) and issubclass(t, C.Array):
                v = np.asarray(p[name], np.float64).ravel()
                dv = np.asarray(dparams.get(name, np.zeros_like(v)), np.float64).ravel()
                vals[name] = (Dual * t._length_)(*[Dual(a, b) for a, b in zip(v, dv)])
            else:
                vals[name] = p[name]
        self.P = TParams(**vals)
        self.Pv = Params(**{k: v for k, v in params.items() if k != "C_wall"})
        nx, ny = self.P.nx, self.P.ny
        self.nx, self.ny = nx, ny
        self._mat = {}
        for k in ("phi", "K", "alpha_T", "D_O2", "D_H2O"):
            v = np.broadcast_to(np.asarray(material[k], np.float64), (ny, nx))
            self._mat[k] = np.ascontiguousarray(_pair(v, dmaterial.get(k)))
        if material.get("u_imposed") is not None:
            self._mat["u_imposed"] = np.ascontiguousarray(_pair(material["u_imposed"]))
        if material.get("sigma") is not None:
            v = np.broadcast_to(np.asarray(material["sigma"], np.float64), (ny, nx))
            self._mat["sigma"] = np.ascontiguousarray(_pair(v))
        self.M = TMaterial(**{k: v.ctypes.data_as(_dd) for k, v in self._mat.items()})
        self.solid = None if solid is None else np.ascontiguousarray(solid, np.uint8)
        self.mask = np.zeros((ny, nx), np.uint8)
        self.L.orc_build_mask(C.byref(self.P),
                              None if self.solid is None else _ptr(self.solid, C.c_uint8),
                              _ptr(self.mask, C.c_uint8))
        self.f = np.zeros((9, ny, nx, 2))
        self.g = np.zeros((3, 5, ny, nx, 2))
        self.L.orc_init(C.byref(self.P), C.byref(self.M), _ptr(self.mask, C.c_uint8),
                        self.f.ctypes.data_as(_dd), self.g.ctypes.data_as(_dd))
        self.f_prev, self.g_prev = self.f.copy(), self.g.copy()
        self.Jx = np.zeros((self.nx, 2))
        self.qx = np.zeros((self.nx, 2))
        self.diag = np.zeros((10, 2))

    def set_state(self, f, g, df=None, dg=None):
        """State (full values, f (9, ny, nx), g (3, 5, ny, nx)) and its
        direction."""
        self.f = np.ascontiguousarray(_pair(f, df))
        self.g = np.ascontiguousarray(_pair(g, dg))
        return self

    def step(self, n: int = 1):
        for _ in range(n):
            fo, go = np.empty_like(self.f), np.empty_like(self.g)
            self.L.orc_step(C.byref(self.P), C.byref(self.M), _ptr(self.mask, C.c_uint8),
                            self.f.ctypes.data_as(_dd), self.g.ctypes.data_as(_dd),
                            fo.ctypes.data_as(_dd), go.ctypes.data_as(_dd),
                            self.diag.ctypes.data_as(_dd), self.Jx.ctypes.data_as(_dd),
                            self.qx.ctypes.data_as(_dd))
            self.f_prev, self.g_prev, self.f, self.g = self.f, self.g, fo, go
        return self

    def fields(self):
        """Fields of the last step (as Oracle.fields), each a (value,
        derivative) pair of arrays."""
        out = np.zeros((6, self.ny, self.nx, 2))
        diag, Jx, qx = np.zeros((10, 2)), np.zeros((self.nx, 2)), np.zeros((self.nx, 2))
        self.L.orc_fields(C.byref(self.P), C.byref(self.M), _ptr(self.mask, C.c_uint8),
                          self.f_prev.ctypes.data_as(_dd), self.g_prev.ctypes.data_as(_dd),
                          out.ctypes.data_as(_dd), diag.ctypes.data_as(_dd),
                          Jx.ctypes.data_as(_dd), qx.ctypes.data_as(_dd))
        names = ("ux", "uy", "p", "T", "C_O2", "C_H2O")
        return {k: (out[i, ..., 0], out[i, ..., 1]) for i, k in enumerate(names)}

    def current_density(self):
        """(i_avg, d i_avg) in A/cm^2 of the last step's reaction."""
        P = self.Pv
        scale = 4.0 * P.F * P.c_tot * P.dx_cm / P.dt_s
        return float(self.Jx[:, 0].mean() * scale), float(self.Jx[:, 1].mean() * scale)

"""CPU checks of the C ABI and the host-side parameter mapping (no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2103_01444_gb300 import workloads
from paper_2103_01444_gb300.units import cathode_params
from paper_2103_01444_gb300 import lbm
from oracle.params import lattice_problem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pemlbm.h")


def declared_symbols():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:lbm_status|const char \*)\s*(lbm_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2103_01444_gb300.build import build
    return build()


def test_library_exports_every_declared_symbol(libpath):
    syms = declared_symbols()
    assert len(syms) >= 17
    L = ctypes.CDLL(libpath)
    for s in syms:
        assert hasattr(L, s), s
    assert set(syms) == set(lbm.EXPORTS)


def test_binding_loads_without_gpu(libpath):
    L = lbm.load_library(libpath)
    assert L.lbm_last_error() is not None


def test_grad_memory_limit_argument_checks(libpath):
    """lbm_set_grad_memory refuses a null domain with EINVAL before touching
    any device (no GPU needed); the limit itself is checked by the GPU tests."""
    L = lbm.load_library(libpath)
    einval = next(k for k, v in lbm.STATUS.items() if v == "LBM_EINVAL")
    assert L.lbm_set_grad_memory(None, 0) == einval
    assert b"null" in L.lbm_last_error()


def test_bounds_check_needs_the_checked_build(libpath):
    """The plain library answers lbm_bounds_check with ESTATE (and a zero
    record) without touching the device; a null argument is EINVAL."""
    L = lbm.load_library(libpath)
    v = ctypes.c_uint64(7)
    estate = next(k for k, s in lbm.STATUS.items() if s == "LBM_ESTATE")
    einval = next(k for k, s in lbm.STATUS.items() if s == "LBM_EINVAL")
    assert L.lbm_bounds_check(ctypes.byref(v)) == estate and v.value == 0
    assert L.lbm_bounds_check(None) == einval


def test_checked_build_compiles_and_exports_the_same_symbols():
    """The self-checking build (-DPEMLBM_BOUNDS_CHECK) compiles here, with no
    GPU, and exports every symbol of the header, like the plain build."""
    from paper_2103_01444_gb300.build import build
    path = build(bounds_check=True)
    L = ctypes.CDLL(path)
    for s in declared_symbols():
        assert hasattr(L, s), s


def test_param_structs_match_header(tmp_path):
    """The ctypes mirrors have the header's field names, offsets and sizes
    (a C program compiled against the header prints them)."""
    src = open(HEADER).read()
    p = src[src.index("} lbm_domain_desc;"):src.index("} lbm_params;")]
    doubles = re.findall(r"double ([\w, ]+)(?:\[\d+\])*;", p)
    names = [n.strip() for grp in doubles for n in grp.split(",")]
    assert names == list(lbm._PARAM_DOUBLES) + ["dp_in", "alpha_a", "buoy_gx", "buoy_gy",
                                                 "T_buoy", "C_wall"]
    fields = {"lbm_params": [f[0] for f in lbm.lbm_params._fields_],
              "lbm_domain_desc": [f[0] for f in lbm.lbm_domain_desc._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pemlbm.h"', "int main(void) {"]
    for st, fl in fields.items():
        lines.append(f'printf("{st} size %zu\\n", sizeof({st}));')
        for f in fl:
            lines.append(f'printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0; }")
    c = tmp_path / "abi.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "abi"
    import subprocess
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(c), "-o",
                           str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    for line in filter(None, out):
        st, f, v = line.split()
        cls = getattr(lbm, st)
        got = ctypes.sizeof(cls) if f == "size" else getattr(cls, f).offset
        assert got == int(v), (st, f, got, v)


@pytest.mark.parametrize("case", [workloads.cathode_200x40(),
                                  workloads.small_cathode(nx=40, ny=20, reaction_mode=1),
                                  workloads.cathode_blocks(nx=256, ny=128),
                                  dict(workloads.cathode_200x40(), inlet="pressure",
                                       dp_in=2e-4, alpha_a=0.5),
                                  workloads.natural_convection_cavity(32, Ra=1e5,
                                                                      heated_bottom=True),
                                  workloads.natural_convection_cavity(24, Ra=1e4, Da=1e-2,
                                                                      phi=0.6),
                                  workloads.kang_surface_reaction(30, 10, Da=2.0)])
def test_product_and_oracle_unit_mappings_agree(case):
    """The product's unit helper and the oracle's independent mapping turn
    the same physical workload into the same lattice problem."""
    p1, f1, g1 = cathode_params(case)
    p2, m2, _ = lattice_problem(case)
    for k, v in p1.items():
        if k in p2:
            np.testing.assert_allclose(np.ravel(v), np.ravel(p2[k]), rtol=1e-13, err_msg=k)
    assert g1.get("closed_x", 0) == p2.get("closed_x", 0)
    for k in ("phi", "K", "alpha_T", "D_O2", "D_H2O"):
        np.testing.assert_allclose(f1[k], m2[k], rtol=1e-13)
    np.testing.assert_allclose(f1["rho_cp_ratio"], m2["sigma"], rtol=1e-13)
    assert g1["ny_cl"] == p2["ny_cl"] and g1["ny_gdl"] == p2["ny_gdl"]


def test_workloads_are_seeded_and_shaped():
    a, b = workloads.cathode_blocks(512, 256), workloads.cathode_blocks(512, 256)
    np.testing.assert_array_equal(a["phi"], b["phi"])
    ny_cl, ny_gdl = a["ny_cl"], a["ny_gdl"]
    assert (ny_cl, ny_gdl) == (13, 141)
    gdl = a["phi"][ny_cl:ny_cl + ny_gdl]
    assert 0.4 <= gdl.min() and gdl.max() <= 0.8
    # one value per 32 x 32 block
    blk = a["phi"][32:64, 32:64]
    assert np.unique(blk).size == 1
    Kg = a["K_cm2"][ny_cl:ny_cl + ny_gdl] * 1e-4
    assert 1e-12 <= Kg.min() and Kg.max() <= 1e-10
    assert np.isinf(a["K_cm2"][ny_cl + ny_gdl:]).all()
    cases = workloads.sweep_cases(8)
    assert all(c["nx"] % 32 == 0 and c["ny"] % 32 == 0 for c in cases)
    g = workloads.cathode_grains(256, 64)
    assert g["solid"][:, :4].sum() == 0 and g["solid"][:, -4:].sum() == 0
    assert 0.2 < g["solid"][:g["ny_gdl"]].mean() < 0.4


class _FakeTensor:
    """Stands in for a torch tensor: the attributes the binding checks."""

    def __init__(self, is_cuda=True, index=0, dtype="torch.float32", shape=(5, 8, 16),
                 contiguous=True):
        self.is_cuda = is_cuda
        self.device = type("dev", (), {"index": index})()
        self.dtype = dtype
        self.shape = shape
        self._contig = contiguous

    def is_contiguous(self):
        return self._contig

    def data_ptr(self):
        raise AssertionError("the pointer must not be taken from a refused buffer")


class _NoCalls:
    def __getattr__(self, name):
        raise AssertionError(f"{name} must not be called for a refused buffer")


@pytest.mark.parametrize("bad,what", [
    (dict(is_cuda=False), "not a CUDA tensor"),
    (dict(index=1), "cuda:1"),
    (dict(dtype="torch.float64"), "dtype"),
    (dict(shape=(5, 8, 15)), "shape"),
    (dict(shape=(4, 8, 16)), "shape"),
    (dict(contiguous=False), "contiguous"),
])
def test_residual_noalloc_refuses_bad_snapshots_before_any_call(bad, what):
    """The C entry point takes a bare device pointer and cannot check it; the
    binding refuses a snapshot of the wrong kind, device, dtype, shape or
    layout with EINVAL before it reaches the library."""
    d = lbm.Domain.__new__(lbm.Domain)
    d.L, d.h = _NoCalls(), None
    d.nx, d.ny, d.precision, d.device = 16, 8, lbm.FP32, 0
    with pytest.raises(lbm.LbmError, match=what) as e:
        d.residual_noalloc(_FakeTensor(**bad))
    assert e.value.status == 1
    d.precision = lbm.FP64          # an FP64 domain needs float64
    with pytest.raises(lbm.LbmError, match="dtype"):
        d.residual_noalloc(_FakeTensor())
    d.h = None

"""The paper's qualitative statements about the cathode (Sec. 5), checked on
the FP64 oracle for the 200 x 40 cathode after 3000 steps in the Fickian
interface mode.  The paper's lattice parameters are unknown, so these are
trends, not parity targets:
  - the velocity in the porous layer is much smaller than in the channel;
  - O2 at the catalyst stays near the inlet value at high cell voltage and
    is depleted at 0.5 V, to about a fifth of the inlet value;
  - the current, and the power, are negligible above 0.7 V;
  - a higher effective O2 diffusivity of the GDL gives a higher current.
"""
import numpy as np
import pytest

from oracle import Oracle
from oracle.params import lattice_problem
from paper_2103_01444_gb300 import workloads


def run(V, d_scale=1.0, steps=3000):
    case = dict(workloads.cathode_200x40(), V_op=V)
    p, m, s = lattice_problem(case, interface_mode=1)
    if d_scale != 1.0:
        gdl = np.isfinite(m["K"])
        m = dict(m, D_O2=np.where(gdl, m["D_O2"] * d_scale, m["D_O2"]))
    o = Oracle(p, m, s).step(steps)
    return case, o, o.fields(), o.current_density()[0]


@pytest.fixture(scope="module")
def sweep():
    return {V: run(V) for V in (0.5, 0.65, 0.8)}


def test_porous_velocity_is_small(sweep):
    case, _, f, _ = sweep[0.65]
    g = case["ny_gdl"]
    assert np.abs(f["ux"][:g]).max() < 0.2 * np.abs(f["ux"][g:]).max()


def test_oxygen_at_the_catalyst_and_the_current_follow_the_voltage(sweep):
    c_in = 0.21
    cl = {V: sweep[V][2]["C_O2"][0] for V in sweep}
    i = {V: sweep[V][3] for V in sweep}
    assert cl[0.8].min() > 0.95 * c_in and cl[0.65].min() > 0.9 * c_in
    assert cl[0.5].min() < 0.3 * c_in and cl[0.5].mean() < 0.4 * c_in
    assert i[0.5] > 10 * i[0.65] > 100 * i[0.8] > 0
    # power i V above 0.7 V is below a thousandth of that at 0.5 V
    assert i[0.8] * 0.8 < 1e-3 * i[0.5] * 0.5


def test_higher_effective_diffusivity_gives_more_current(sweep):
    i0 = sweep[0.5][3]
    _, _, _, i2 = run(0.5, d_scale=2.0)
    assert i2 > 1.05 * i0

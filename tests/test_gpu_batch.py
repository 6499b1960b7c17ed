"""Batched stepping of uneven cases (operating-point sweeps): every schedule
must give the same states as stepping each case on its own."""
import numpy as np
import pytest

from paper_2103_01444_gb300 import workloads

pytestmark = pytest.mark.gpu


def cases():
    out = []
    for k, (nx, ny, mode, V) in enumerate([(96, 32, 1, 0.35), (160, 24, 0, 0.6),
                                           (64, 40, 1, 0.8), (130, 48, 0, 0.45),
                                           (200, 16, 1, 0.5)]):
        c = workloads.small_cathode(nx=nx, ny=ny, reaction_mode=mode, V_op=V, seed=k)
        out.append(c)
    return out


def domains(precision="fp32", interface_mode=0):
    from paper_2103_01444_gb300.build import build
    from paper_2103_01444_gb300.lbm import Domain
    build()
    return [Domain.from_case(c, precision=precision, interface_mode=interface_mode)
            for c in cases()]


@pytest.mark.parametrize("schedule", ["graph", "persistent", "per-case", "concurrent"])
def test_batched_states_equal_individual_steps(schedule):
    from paper_2103_01444_gb300.lbm import Batch
    ref = domains()
    for d in ref:
        d.step(150)
    ds = domains()
    b = Batch(ds)
    b.set_schedule(schedule, variant=6)
    b.step(150)          # 150 >= 128: the graph schedule replays its graph
    b.step(1)            # odd counts flip each case's buffer
    for d in ref:
        d.step(1)
    for d, r in zip(ds, ref):
        assert d.steps == r.steps == 151
        np.testing.assert_array_equal(d.state(), r.state())
        assert d.current_density()[0] == r.current_density()[0]


def test_concurrent_schedule_follows_cases_stepped_alone_and_new_parameters():
    """The concurrent schedule replays a graph that bakes in each case's
    buffers and arguments: after a case is stepped on its own, or its
    operating point changes, the batch must still equal individual steps."""
    from paper_2103_01444_gb300.lbm import Batch
    ref, ds = domains(), domains()
    b = Batch(ds)
    b.set_schedule("concurrent", variant=7)
    b.step(130)
    ds[0].step(1)
    for r in ref:
        r.step(130)
    ref[0].step(1)
    b.step(130)
    for r in ref:
        r.step(130)
    p = dict(ds[1].params, V_op=ds[1].params["V_op"] - 0.05)
    ds[1].set_params(p)
    ref[1].set_params(p)
    b.step(130)
    for r in ref:
        r.step(130)
    for d, r in zip(ds, ref):
        assert d.steps == r.steps
        np.testing.assert_array_equal(d.state(), r.state())


def test_batch_tune_keeps_states_and_picks_a_schedule():
    from paper_2103_01444_gb300.lbm import Batch
    ds = domains()
    ref = domains()
    b = Batch(ds)
    sch, var, ms = b.tune(3)
    assert sch in (0, 1, 3) and 0 <= var < 8 and ms > 0
    for d, r in zip(ds, ref):
        np.testing.assert_array_equal(d.state(), r.state())
    b.step(20)
    for r in ref:
        r.step(20)
    for d, r in zip(ds, ref):
        np.testing.assert_array_equal(d.state(), r.state())


def test_grid_barrier_gives_up_and_the_context_survives():
    """A barrier allowed a single poll gives up: the call returns ETIMEOUT
    (no hang, no fault), the states are marked undefined, and after a reset
    the same batch steps normally."""
    from paper_2103_01444_gb300.lbm import Batch, LbmError
    ds = domains()
    b = Batch(ds)
    b.set_schedule("persistent", spin_limit=1)
    with pytest.raises(LbmError, match="ETIMEOUT"):
        b.step(40)
    with pytest.raises(LbmError, match="ESTATE"):
        ds[0].step(1)
    for d in ds:
        d.reset()
    b.set_schedule("persistent", spin_limit=1 << 24)
    b.step(10)
    ref = domains()
    for r in ref:
        r.step(10)
    for d, r in zip(ds, ref):
        np.testing.assert_array_equal(d.state(), r.state())


def test_batch_rejects_mixed_precision_and_unready_domains():
    from paper_2103_01444_gb300.lbm import Batch, Domain, LbmError
    ds = domains()
    other = domains("fp64")[0]
    with pytest.raises(LbmError, match="EINVAL"):
        Batch([ds[0], other])
    with pytest.raises(LbmError, match="EINVAL"):
        Batch([ds[0], ds[0]])
    fresh = Domain(32, 16, ny_gdl=8)
    with pytest.raises(LbmError, match="ESTATE"):
        Batch([ds[0], fresh])


@pytest.mark.parametrize("schedule", ["graph", "concurrent"])
def test_pressure_sweep_batched(schedule):
    """A sweep of the pressure drive (Sec. 4, 5: flow rates set by the
    pressure difference), mixed with velocity-driven and Butler-Volmer
    cases, batched: every case equals its own stepping."""
    from paper_2103_01444_gb300.lbm import Batch, Domain
    base = cases()
    sweep = [dict(base[0], inlet="pressure", dp_in=dp) for dp in (2e-4, 6e-4, 1.2e-3)]
    sweep += [dict(base[1], alpha_a=0.5, V_op=1.0), base[3]]
    ref = [Domain.from_case(c, precision="fp32") for c in sweep]
    ds = [Domain.from_case(c, precision="fp32") for c in sweep]
    b = Batch(ds)
    b.set_schedule(schedule, variant=7)
    b.step(141)
    for r in ref:
        r.step(141)
    for d, r in zip(ds, ref):
        np.testing.assert_array_equal(d.state(), r.state())
    # the flow rate grows with the pressure difference
    q = [float(d.fields()["ux"][:, d.nx // 2].sum()) for d in ds[:3]]
    assert 0 < q[0] < q[1] < q[2]


def oracle_sweep():
    """Five uneven cases of an operating-point sweep (Sec. 5) that differ in
    more than the voltage: thin film, volumetric catalyst, pressure drive,
    Butler-Volmer kinetics, pore-scale grains, scalars advected relative to
    their inlet values; interface modes alternate."""
    base = cases()
    sweep = [dict(base[0]),
             dict(base[1], inlet="pressure", dp_in=8e-4),
             dict(base[2], alpha_a=0.5, V_op=1.0),
             workloads.small_cathode(nx=70, ny=24, reaction_mode=0, grains=True, seed=9,
                                     V_op=0.45),
             dict(base[4], scalar_advection=1)]
    return [(c, k % 2) for k, c in enumerate(sweep)]


@pytest.fixture(scope="module")
def sweep_oracles():
    from oracle import Oracle
    from oracle.params import lattice_problem
    out = []
    for c, mode in oracle_sweep():
        params, material, solid = lattice_problem(c, interface_mode=mode)
        out.append(Oracle(params, material, solid).step(151))
    return out


@pytest.mark.parametrize("schedule", ["graph", "persistent", "per-case", "concurrent"])
def test_batched_fp64_states_match_the_oracle(schedule, sweep_oracles):
    """FP64 storage: after 151 batched steps every population of every case
    agrees with the FP64 oracle's own stepping of that case to round-off
    (1e-11 of each plane's scale), and so does its current density."""
    from paper_2103_01444_gb300.build import build
    from paper_2103_01444_gb300.lbm import Batch, Domain
    build()
    ds = [Domain.from_case(c, precision="fp64", interface_mode=m) for c, m in oracle_sweep()]
    b = Batch(ds)
    b.set_schedule(schedule, variant=6)
    b.step(150)
    b.step(1)
    for d, o in zip(ds, sweep_oracles):
        live = (o.mask & 3) != 3
        st = d.state()
        ref = np.concatenate([o.f, o.g.reshape(15, o.ny, o.nx)], axis=0)
        for q in range(24):
            scale = np.abs(ref[q][live]).max()
            np.testing.assert_allclose(st[q][live], ref[q][live], rtol=0, atol=1e-11 * scale,
                                       err_msg=f"plane {q}")
        i_g = d.current_density()[0]
        i_o = o.current_density()[0]
        assert i_g == pytest.approx(i_o, rel=1e-11)

"""The ensemble (many tissues, one persistent cooperative launch per step
call, or the split schedule of two launches per step) against the same
tissues run one by one through lbib_step, and one tissue against the FP64
oracle, under each schedule.

Tolerances: ensemble vs single-tissue runs, both FP32 with the same kernels
and only the atomic order of the spreading differing: relative L-infinity
1e-5 on u and phi, 1e-9 LU on X.  Against the oracle: the FP32 bounds of the
coupled parity tests (u 1e-4, phi 1e-5, X 1e-6 LU).
"""
import numpy as np
import pytest

import lbib_inputs as li

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1503_06726_gb300 import build, lbib
    build.build()
    lbib.load()
    return lbib


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def small_ensemble():
    """Five tissues of different sizes, tau, springs and boundaries."""
    ws = li.config4(seed=44, n_tissues=4, n_steps=9, side_min=96, side_max=200)
    w2 = li.config2(nx=128, ny=128, n_cells_side=2)
    w2.params.n_species = 1
    w2.params.react = [[0.0] * 4 for _ in range(4)]
    w2.params.decay[0] = 1e-3
    w2.params.D[0] = 0.07
    return ws + [w2]


SCHEDULES = ("persistent", "split", "split_wide")


def schedule_of(lb, name):
    return {"persistent": lb.LBIB_ENS_PERSISTENT, "split": lb.LBIB_ENS_SPLIT,
            "split_wide": lb.LBIB_ENS_SPLIT_WIDE}[name]


@pytest.mark.parametrize("sched", SCHEDULES)
def test_ensemble_matches_single_tissues(lb, sched):
    ws = small_ensemble()
    ens = lb.Ensemble([w.params for w in ws], [w.tissue for w in ws])
    assert ens.schedule(schedule_of(lb, sched)) == schedule_of(lb, sched)
    for n in (5, 4, 1):   # an odd, an even and a one-step call
        ens.step(n)
    ens.status()
    for t, w in enumerate(ws):
        sim = lb.Simulation(w.params, lb.LBIB_FP32, w.tissue.n_vertices, w.tissue.n_cells)
        sim.set_cells(w.tissue)
        sim.step(5)
        sim.step(4)
        sim.step(1)
        a = ens.fields(t)
        b = sim.fields()
        assert max(rel(a["ux"], b["ux"]), rel(a["uy"], b["uy"])) < 1e-5, t
        assert rel(a["phi"], b["phi"]) < 1e-5, t
        assert np.abs(a["xy"] - b["xy"]).max() < 1e-9, t
        sim.close()
    ens.close()


@pytest.mark.parametrize("sched", ("persistent", "split"))
def test_ensemble_tissue_matches_oracle(lb, orc, sched):
    ws = small_ensemble()
    ens = lb.Ensemble([w.params for w in ws], [w.tissue for w in ws])
    ens.schedule(schedule_of(lb, sched))
    ens.step(12)
    t = 1
    got = ens.fields(t)
    ref = orc.run(ws[t].params, ws[t].tissue, 12)
    assert max(rel(got["ux"], ref.ux), rel(got["uy"], ref.uy)) < 1e-4
    assert rel(got["phi"], ref.phi) < 1e-5
    assert np.abs(got["xy"] - ref.xy).max() < 1e-6
    ens.close()


def test_ensemble_autotune_and_graph(lb, tmp_path):
    ws = small_ensemble()
    ens = lb.Ensemble([w.params for w in ws], [w.tissue for w in ws])
    c = ens.tune_cached("test-small", trial_steps=3, path=str(tmp_path / "tune.json"))
    assert c["nodes_per_item"] in (256, 512, 1024, 2048, 4096) and c["blocks_per_sm"] >= 1
    assert c["schedule"] in (lb.LBIB_ENS_PERSISTENT, lb.LBIB_ENS_SPLIT, lb.LBIB_ENS_SPLIT_WIDE)
    assert c["cached"] is False
    assert ens.schedule() == c["schedule"]
    ens.schedule(lb.LBIB_ENS_PERSISTENT if c["schedule"] else lb.LBIB_ENS_SPLIT)
    c2 = ens.tune_cached("test-small", path=str(tmp_path / "tune.json"))
    assert c2["cached"] is True and c2["nodes_per_item"] == c["nodes_per_item"]
    assert ens.schedule() == c["schedule"]
    ens.step(6)
    ens.step(6)
    ens.status()
    info = ens.config()
    assert info["grid"] >= 1
    ens.close()


def test_ensemble_bounded_barrier_reports_timeout(lb):
    """A grid barrier that cannot complete gives up after about a second and
    the host reads LBIB_E_TIMEOUT; the ensemble keeps working afterwards."""
    ws = small_ensemble()[:2]
    ens = lb.Ensemble([w.params for w in ws], [w.tissue for w in ws])
    rc, sec = ens.selftest_timeout()
    assert rc == lb.LBIB_E_TIMEOUT
    assert 0.5 < sec < 10.0
    ens.step(3)
    ens.status()
    ens.close()


@pytest.mark.parametrize("sched", SCHEDULES)
def test_ensemble_without_cells(lb, sched):
    """Tissues without cells: under the split schedule the lattice launches
    follow one another (no IB launch between them) and are not programmatic."""
    ws = small_ensemble()[:3]
    ens = lb.Ensemble([w.params for w in ws], [None] * len(ws))
    ens.schedule(schedule_of(lb, sched))
    ens.step(3)
    ens.step(2)
    ens.status()
    for t, w in enumerate(ws):
        sim = lb.Simulation(w.params, lb.LBIB_FP32, 0, 0)
        sim.step(3)
        sim.step(2)
        a = ens.fields(t)
        b = sim.fields()
        # no spreading: the same kernels in the same order give the same bits
        assert np.array_equal(a["ux"], b["ux"]) and np.array_equal(a["phi"], b["phi"]), t
        sim.close()
    ens.close()


def test_ensemble_schedule_rejects_unknown(lb):
    ws = small_ensemble()[:1]
    ens = lb.Ensemble([w.params for w in ws], [w.tissue for w in ws])
    with pytest.raises(lb.LbibError):
        ens.schedule(7)
    assert ens.schedule() == lb.LBIB_ENS_PERSISTENT
    ens.close()

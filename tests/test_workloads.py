"""Named workloads: shapes, seeds and the properties their recipes fix
(CPU; the large states are not generated here)."""

import math

import numpy as np
import pytest

import oracle
from paper_1808_01309_gb300 import inputs, workloads


def test_every_name_resolves():
    for name in workloads.names():
        w = workloads.get(name)
        assert w
    with pytest.raises(KeyError):
        workloads.get("nope")


def test_taylor_green_preset_matches_its_closed_form():
    w = workloads.get("taylor_green_32")
    assert (w.prec, w.rk_order, w.steps, w.dt, w.nu) == ("fp64", 2, 10, 1e-3, 1e-2)
    u = w.initial_state()
    d = oracle.diagnostics(u, oracle.Config(32, 32, 32))
    assert abs(d["energy"] - 1 / 8) < 1e-15 and abs(d["enstrophy"] - 3 / 8) < 1e-14
    assert w.forcing() is None


def test_forced_presets_share_the_recipe():
    a, b = workloads.get("forced_512"), workloads.get("forced_256")
    assert (a.nu, a.dt, a.seed, a.forcing_seed, a.rk_order) == (2e-3, 1e-3, 1, 2, 4)
    assert (b.steps, workloads.get("forced_256_fp64").prec) == (100, "fp64")
    small = workloads.forced(32)
    u, f = small.initial_state(), small.forcing()
    assert np.array_equal(u, inputs.random_solenoidal_field(32, 32, 32, seed=1))
    cfg = oracle.Config(32, 32, 32)
    assert abs(oracle.diagnostics(u, cfg)["energy"] - 0.5) < 1e-12
    fp = oracle.inverse(f, cfg)
    assert abs(math.sqrt(np.mean(np.sum(fp * fp, axis=0))) - 0.25) < 1e-12


def test_multi_field_presets_have_their_components():
    m, q = workloads.get("mhd_512"), workloads.get("boussinesq_512")
    assert (m.eq, m.eta) == ("mhd", 2e-3) and (q.eq, q.n_bv, q.kappa) == ("boussinesq", 1.0, 2e-3)
    import dataclasses
    st = dataclasses.replace(q, shape=(16, 16, 16)).initial_state()
    assert st.shape == (4, 16, 16, 9)
    st = dataclasses.replace(m, shape=(16, 16, 16)).initial_state()
    assert st.shape == (6, 16, 16, 9)


def test_ensemble_preset():
    mem = workloads.get("ensemble_48")
    assert len(mem) == 48
    assert [w.shape[0] for w in mem] == [64] * 16 + [96] * 16 + [128] * 16
    nus = [w.nu for w in mem]
    assert all(1e-3 <= v <= 5e-3 for v in nus) and len(set(nus)) == 48
    assert [w.seed for w in mem] == list(range(1000, 1048))
    assert all(w.forcing() is None and w.steps == 50 for w in mem)

"""Pins of the oracle's Ar+ collision kinematics (Table I: ion elastic
scattering and charge exchange with the neutral argon background of Sec. III).

Each collision partner is a neutral drawn from the gas Maxwellian at T_gas,
whose velocity components are normal with the textbook spread
sqrt(k_B T_gas / M_Ar) (about 249.9 m/s at 300 K).  The tests redraw that
neutral from the same counter-based stream (particle id, step, purpose 3) and
check the outcome of every ion against the definitions:

- a null event leaves v unchanged;
- charge exchange hands the ion the neutral's velocity, so the post-collision
  ion velocities of the charge-exchange events are normal with that spread
  (KS test per component);
- an elastic collision between equal masses keeps the centre-of-mass velocity
  (v + v_n)/2 and the size of the relative velocity, so the ion ends at
  distance |v - v_n|/2 from the centre of mass, in a direction that is
  isotropic in the centre-of-mass frame (KS test of the cosine to the
  incoming relative velocity, uniform on [-1, 1]).

A wrong neutral spread (e.g. a factor 2 in sqrt(kT/M)) fails the redrawn
neutral and the KS test; a scatter in the lab frame instead of the
centre-of-mass frame fails the centre-of-mass distance.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1801_00972_gb300 import inputs as I

stats = pytest.importorskip("scipy.stats")

KB = 1.380649e-23
AMU = 1.66053906660e-27
M_AR = 39.948 * AMU
# sqrt(k_B * 300 K / M_Ar) = sqrt(4.141947e-21 J / 6.633521e-26 kg) = 249.8793 m/s
SIGMA_300K = math.sqrt(KB * 300.0 / M_AR)


def _ions(n, energy_ev, seed=2):
    rng = np.random.default_rng(seed)
    wl = I.small(grains=0, n_e=0, n_i=n, weight=0.0, v_dc=0.0, v_top=0.0, dt=2e-8, nz=64)
    L = np.array(wl.box)
    x = rng.uniform(0.2, 0.8, (n, 3)) * L
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    v = d * math.sqrt(2 * energy_ev * I.QE / M_AR)
    ids = np.arange(n, dtype=np.uint32)
    parts = [(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, np.uint32)), (x, v, ids)]
    return wl, parts


def _outcomes(energy_ev, n=60000):
    wl, parts = _ions(n, energy_ev)
    s = O.Sim(wl, parts)
    s.step(1)
    c = s.counters()
    assert c["err"] == 0 and c["lost_bot_i"] == 0 and c["lost_top_i"] == 0
    _, v1, ids = s.particles(1)
    assert np.array_equal(ids, parts[1][2])
    v0 = parts[1][1]
    key = np.array([(wl.seed & 0xFFFFFFFF) ^ wl.run_id, wl.seed >> 32], np.uint32)
    assert wl.t_gas == 300.0
    vn = np.array([O.gauss3(int(i), 0, 3, key) for i in ids]) * SIGMA_300K
    return c, v0, v1, vn


def test_neutral_spread_closed_form():
    assert SIGMA_300K == pytest.approx(249.8793, rel=1e-6)


@pytest.mark.parametrize("energy", [40.0, 0.5])
def test_ion_elastic_and_charge_exchange_kinematics(energy):
    c, v0, v1, vn = _outcomes(energy)
    g = v0 - vn
    gm = np.linalg.norm(g, axis=1)
    vcm = 0.5 * (v0 + vn)
    null = np.all(v1 == v0, axis=1)
    cx = np.linalg.norm(v1 - vn, axis=1) <= 1e-12 * np.linalg.norm(vn, axis=1)
    el = np.abs(np.linalg.norm(v1 - vcm, axis=1) - 0.5 * gm) <= 1e-12 * gm
    el &= ~null & ~cx
    # every ion is exactly one of: untouched, charge-exchanged, elastically scattered
    assert np.all(null.astype(int) + cx.astype(int) + el.astype(int) == 1)
    assert cx.sum() == c["i_cx"] and el.sum() == c["i_el"]
    assert c["i_cx"] > 150 and c["i_el"] > 150
    # charge exchange: the ion leaves with the neutral's velocity, normal with the gas spread
    for a in range(3):
        assert stats.kstest(v1[cx, a] / SIGMA_300K, "norm").pvalue > 1e-3
    # elastic: isotropic in the centre-of-mass frame
    u = (v1[el] - vcm[el]) / (0.5 * gm[el])[:, None]
    cos = np.sum(u * (g[el] / gm[el][:, None]), axis=1)
    assert stats.kstest(cos, "uniform", args=(-1.0, 2.0)).pvalue > 1e-3


def test_charge_exchange_spread_detects_a_wrong_scale():
    """The KS test above separates the gas spread from a spread off by 10%."""
    c, v0, v1, vn = _outcomes(40.0)
    cx = np.linalg.norm(v1 - vn, axis=1) <= 1e-12 * np.linalg.norm(vn, axis=1)
    sample = v1[cx].reshape(-1) / SIGMA_300K
    assert stats.kstest(sample, "norm").pvalue > 1e-3
    assert stats.kstest(sample / 1.1, "norm").pvalue < 1e-3

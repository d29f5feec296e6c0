"""Pins of the oracle's seeded initial plasma (Sec. III: a uniform plasma of
given density with Maxwellian electrons and ions; the draw itself is this
build's reading, shared with the CUDA library by definition, not by code).

- Ids: electrons 0..n_e-1, ions n_e..n_e+n_i-1.
- The stream: particle p's first point is (u0, u1, u2) L from Philox counter
  (p, 0, 10, 0), uniforms (u + 1/2) 2^-32; velocities come from counter
  (p, 0, 11, .), so a different seed or run id gives a different plasma.
- Positions: uniform in the box (KS per axis) and never within 1.5 grain radii
  of a grain centre (minimum image in x and y).
- Velocities: each component normal with the textbook thermal spread
  sqrt(T e / m) of the species (KS), mean kinetic energy 3/2 T.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
from paper_1801_00972_gb300 import inputs as I

stats = pytest.importorskip("scipy.stats")


def _wl(**over):
    return I.small(nx=16, ny=16, nz=32, n_e=40000, n_i=30000, grains=5, seed=11, te_ev=3.0, ti_ev=0.03, **over)


def _near_any_grain(x, wl, factor):
    L = np.array(wl.box)
    near = np.zeros(len(x), bool)
    for p, r in zip(wl.grain_pos, wl.grain_r):
        d = x - p
        for a in range(2):
            d[:, a] -= L[a] * np.round(d[:, a] / L[a])
        near |= np.sum(d * d, 1) <= (factor * r) ** 2
    return near


def test_ids_and_stream():
    wl = _wl()
    s = O.Sim(wl, None)
    xe, ve, ie = s.particles(0)
    xi, vi, ii = s.particles(1)
    assert np.array_equal(ie, np.arange(wl.n_e)) and np.array_equal(ii, wl.n_e + np.arange(wl.n_i))
    assert s.next_id == wl.n_e + wl.n_i
    key = np.array([(wl.seed & 0xFFFFFFFF) ^ wl.run_id, wl.seed >> 32], np.uint32)
    L = np.array(wl.box)
    for sp, (x, ids) in enumerate(((xe, ie), (xi, ii))):
        for q in (0, 17, len(ids) - 1):
            u = O.philox4x32_10([ids[q], 0, 10, 0], key)[:3]
            first = (u.astype(np.float64) + 0.5) * 2.0 ** -32 * L
            if not _near_any_grain(first[None, :], wl, 1.5)[0]:
                assert np.array_equal(x[q], first)
    # another seed or run id: another plasma
    for over in ({"seed": wl.seed + 1}, {"run_id": 3}):
        x2, v2, _ = O.Sim(dataclasses.replace(wl, **over), None).particles(0)
        assert not np.array_equal(x2, xe) and not np.array_equal(v2, ve)


def test_positions_uniform_outside_grains():
    wl = _wl()
    s = O.Sim(wl, None)
    L = np.array(wl.box)
    for sp in range(2):
        x, _, _ = s.particles(sp)
        assert np.all(x >= 0.0) and np.all(x < L)
        assert not _near_any_grain(x, wl, 1.5).any()
        for a in range(3):
            assert stats.kstest(x[:, a] / L[a], "uniform").pvalue > 1e-3


def test_grain_exclusion_takes_effect():
    # grains large enough that about 0.25% of first draws fall inside 1.5 radii
    wl = _wl()
    wl.grain_r = np.full(len(wl.grain_r), 1.3e-4)
    s = O.Sim(wl, None)
    x, _, ids = s.particles(0)
    assert not _near_any_grain(x, wl, 1.5).any()
    key = np.array([(wl.seed & 0xFFFFFFFF) ^ wl.run_id, wl.seed >> 32], np.uint32)
    L = np.array(wl.box)
    first = np.array([(O.philox4x32_10([p, 0, 10, 0], key)[:3].astype(np.float64) + 0.5) * 2.0 ** -32 * L
                      for p in ids])
    redrawn = _near_any_grain(first, wl, 1.5)
    assert redrawn.sum() > 40
    assert np.all(np.any(x[redrawn] != first[redrawn], axis=1))
    assert np.array_equal(x[~redrawn], first[~redrawn])


@pytest.mark.parametrize("sp,t_ev,mass", [(0, 3.0, I.ME), (1, 0.03, I.MAR)])
def test_velocities_maxwellian(sp, t_ev, mass):
    wl = _wl()
    s = O.Sim(wl, None)
    _, v, _ = s.particles(sp)
    vth = math.sqrt(t_ev * 1.602176634e-19 / mass)
    for a in range(3):
        assert stats.kstest(v[:, a] / vth, "norm").pvalue > 1e-3
    e_mean = 0.5 * mass * np.mean(np.sum(v * v, 1)) / 1.602176634e-19
    assert e_mean == pytest.approx(1.5 * t_ev, rel=0.02)

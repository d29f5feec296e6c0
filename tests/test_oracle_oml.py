"""Pins of the oracle's hypothetical-charge estimator (Sec. IV.B: OML balance of
electron and ion fluxes with the charge-exchange ion flux, from the local
densities and temperatures) and of the temperature moments it reads.

Collisionless OML has closed forms through the Lambert W function.  With
A = n_e vbar_e / (n_i vbar_i), tau = T_e / T_i:
  phi < 0 (A > 1):  A exp(-z) = 1 + z tau, z = -phi/T_e  =>  1 + z tau = tau W((A/tau) e^(1/tau));
  phi > 0 (A < 1):  A (1 + u/tau) = exp(-u), u = phi/T_i =>  tau (1 + u/tau) = W((tau/A) e^tau).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1801_00972_gb300 import inputs as I

sp = pytest.importorskip("scipy.special")


def _A(ne, ni, te, ti):
    return (ne / ni) * math.sqrt((te * I.MAR) / (ti * I.ME))


@pytest.mark.parametrize("ne,ni,te,ti", [(1e15, 1e15, 3.0, 0.03), (1e15, 1e15, 1.0, 1.0), (2e14, 9e14, 2.3, 0.05),
                                         (1e16, 3e15, 0.31, 0.026)])
def test_collisionless_oml_negative_branch(ne, ni, te, ti):
    tau = te / ti
    A = _A(ne, ni, te, ti)
    assert A > 1.0
    y = tau * sp.lambertw((A / tau) * math.exp(1.0 / tau)).real
    z = (y - 1.0) / tau
    phi = O.oml_potential(ne, ni, te, ti, 0.0)
    assert phi == pytest.approx(-z * te, rel=1e-9)


@pytest.mark.parametrize("ne,ni,te,ti", [(1e12, 1e16, 3.0, 0.03), (1e12, 1e15, 2.0, 0.5)])
def test_collisionless_oml_positive_branch(ne, ni, te, ti):
    tau = te / ti
    A = _A(ne, ni, te, ti)
    assert A < 1.0
    v = sp.lambertw((tau / A) * math.exp(tau)).real / tau
    u = tau * (v - 1.0)
    phi = O.oml_potential(ne, ni, te, ti, 0.0)
    assert phi == pytest.approx(u * ti, rel=1e-9)


def test_charge_exchange_term():
    ne, ni, te, ti = 1e15, 1e15, 3.0, 0.03
    tau = te / ti
    A = _A(ne, ni, te, ti)
    p0 = O.oml_potential(ne, ni, te, ti, 0.0)
    prev = p0
    for lam_l in (0.01, 0.1, 1.0, 10.0):
        p = O.oml_potential(ne, ni, te, ti, lam_l)
        assert prev < p < 0.0          # more ion current: a smaller negative potential
        prev = p
    # the potential that a chosen lambda/l balances: A e^-z = 1 + z tau + 0.1 (z tau)^2 lambda/l
    z = 1.7
    lam_l = (A * math.exp(-z) - 1.0 - z * tau) / (0.1 * (z * tau) ** 2)
    assert lam_l > 0
    assert O.oml_potential(ne, ni, te, ti, lam_l) == pytest.approx(-z * te, rel=1e-9)
    assert math.isnan(O.oml_potential(0.0, ni, te, ti, 0.0))
    assert math.isnan(O.oml_potential(ne, ni, te, -1.0, 0.0))


def test_temperature_moments():
    wl = I.small(nx=8, ny=8, nz=16, n_e=200000, n_i=200000, grains=1, v_dc=0.0, te_ev=2.5, ti_ev=0.05,
                 weight=1e-3)
    wl.grain_r[:] = 1e-7
    parts = I.sample_particles(wl)
    s = O.Sim(wl, parts, flags=O.MOMENTS | O.NO_MCC | O.IONS_FROZEN)
    s.step(2)
    te = s.moments(5)
    ti = s.moments(6)
    ne = s.moments(1)
    inner = slice(wl.nx * wl.ny, -wl.nx * wl.ny)      # interior node planes (electrode planes see half cells)
    w = ne[inner]
    assert np.sum(w * te[inner]) / np.sum(w) == pytest.approx(2.5, rel=0.02)
    assert np.sum(w * ti[inner]) / np.sum(w) == pytest.approx(0.05, rel=0.02)
    # the estimator's local values at the grain
    q = s.oml_charges(with_cx=False)[0]
    n0 = wl.n_e * wl.weight / (wl.nx * wl.ny * wl.nz * wl.dx ** 3)
    assert q[2] == pytest.approx(n0, rel=0.08) and q[3] == pytest.approx(n0, rel=0.08)
    assert q[4] == pytest.approx(2.5, rel=0.08) and q[5] == pytest.approx(0.05, rel=0.08)
    assert q[1] == pytest.approx(O.oml_potential(*q[2:6], 0.0), rel=1e-12)
    eps0 = 8.8541878128e-12
    assert q[0] == pytest.approx(4 * math.pi * eps0 * 1e-7 * q[1], rel=1e-12)
    # with charge exchange the estimate is less negative
    assert s.oml_charges(with_cx=True)[0][1] > q[1]


def test_cold_beam_has_zero_temperature():
    wl = I.small(nx=8, ny=8, nz=16, n_e=2000, n_i=0, grains=0, v_dc=0.0, weight=1e-9)
    x, v, ids = I.sample_particles(wl)[0]
    v = np.tile([3e4, -1e4, 2e4], (len(ids), 1))
    s = O.Sim(wl, [(x, v, ids), (np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, np.uint32))],
              flags=O.MOMENTS | O.NO_MCC)
    s.step(1)
    t = s.moments(5)
    drift_ev = 0.5 * I.ME * (9e8 + 1e8 + 4e8) / I.QE
    assert np.max(np.abs(t)) <= 1e-12 * drift_ev


def _debye_length(ne, ni, te_ev, ti_ev):
    """Linearised Debye length from the textbook definition with temperatures in
    kelvin: lambda_D^-2 = e^2 n_e / (eps0 k_B T_e) + e^2 n_i / (eps0 k_B T_i)."""
    qe, kb, eps0 = 1.602176634e-19, 1.380649e-23, 8.8541878128e-12
    te_k, ti_k = te_ev * qe / kb, ti_ev * qe / kb
    return 1.0 / math.sqrt(qe * qe * ne / (eps0 * kb * te_k) + qe * qe * ni / (eps0 * kb * ti_k))


def test_debye_length_by_hand():
    # n = 1e15 m^-3, T_e = 3 eV, T_i = 0.03 eV:
    # lambda_De = sqrt(eps0 * 3 V / (1e15 m^-3 * e)) = 4.0717e-4 m, lambda_Di = 4.0717e-5 m,
    # lambda_D = (lambda_De^-2 + lambda_Di^-2)^-1/2 = lambda_Di / sqrt(1.01) = 4.0515e-5 m
    assert _debye_length(1e15, 1e15, 3.0, 0.03) == pytest.approx(4.0515e-5, rel=1e-4)


@pytest.mark.parametrize("table", ["flat", "linear"])
def test_cx_term_uses_debye_length_over_cx_mean_free_path(table):
    """The estimator's lambda_D / l_i with l_i = 1 / (n_gas sigma_cx(3/2 T_i)):
    a uniform plasma sampled into the moment window, a charge-exchange table
    chosen so that sigma_cx(3/2 T_i) is known exactly (a constant, or a line
    that linear interpolation reproduces), and the potential compared with the
    balance at the hand-computed ratio."""
    wl = I.small(nx=8, ny=8, nz=16, n_e=200000, n_i=200000, grains=1, v_dc=0.0, te_ev=2.5, ti_ev=0.05,
                 weight=1e-3)
    wl.grain_r[:] = 1e-7
    a, b = 3.0e-19, 4.0e-18            # sigma_cx = a (flat) or a + b E[eV] (linear)
    e_grid = np.arange(wl.xs.shape[1]) * wl.de_i
    wl.xs = wl.xs.copy()
    wl.xs[4] = a if table == "flat" else a + b * e_grid
    parts = I.sample_particles(wl)
    s = O.Sim(wl, parts, flags=O.MOMENTS | O.NO_MCC | O.IONS_FROZEN)
    s.step(2)
    q = s.oml_charges(with_cx=True)[0]
    ne, ni, te, ti = q[2:6]
    sig = a if table == "flat" else a + b * 1.5 * ti
    ratio = _debye_length(ne, ni, te, ti) * wl.n_gas * sig
    assert q[1] == pytest.approx(O.oml_potential(ne, ni, te, ti, ratio), rel=1e-9)
    if table == "linear":
        # the cross section is taken at 3/2 T_i, not at T_i or 3 T_i
        for t in (ti, 3 * ti):
            wrong = _debye_length(ne, ni, te, ti) * wl.n_gas * (a + b * t)
            assert abs(O.oml_potential(ne, ni, te, ti, wrong) - q[1]) > 1e-4 * abs(q[1])

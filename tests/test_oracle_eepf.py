"""Pins of the electron energy probability function (Sec. IV.A, Fig. 3): the
oracle's per-plane energy histogram of a Maxwellian has the exponential EEPF
g(eps) = f(eps)/sqrt(eps) ~ exp(-eps/T), and the library's two-Maxwellian fit
recovers the temperatures of exact expected counts (the law of eps/T for a
Maxwellian is Gamma(3/2))."""
import math

import numpy as np
import pytest

import oracle as O
import paper_1801_00972_gb300 as P
from paper_1801_00972_gb300 import inputs as I

scipy_special = pytest.importorskip("scipy.special")


def _expected_counts(n, t_ev, de, bins):
    edges = np.arange(bins + 1) * de
    cdf = scipy_special.gammainc(1.5, edges / t_ev)
    return n * np.diff(cdf)


def test_oracle_histogram_of_a_maxwellian():
    te = 3.0
    wl = I.small(nx=8, ny=8, nz=16, n_e=40000, n_i=0, grains=0, v_dc=0.0, weight=0.0, te_ev=te)
    parts = I.sample_particles(wl)
    bins, de = 120, 0.25
    s = O.Sim(wl, parts, flags=O.EEPF | O.NO_MCC, eepf_bins=bins, eepf_de_ev=de)
    s.step()
    h, steps = s.eepf()
    assert steps == 1
    assert h.sum() == s.count(0)                         # one count per electron and step
    # the planes hold the electrons of their cells
    z = s.particles(0)[0][:, 2]
    assert np.array_equal(h.sum(1), np.bincount(np.minimum((z / wl.dx).astype(int), wl.nz - 1), minlength=wl.nz))
    tot = h.sum(0)[:bins]
    e = (np.arange(bins) + 0.5) * de
    sel = (e > 0.5) & (e < 12.0) & (tot > 0)
    g = tot[sel] / np.sqrt(e[sel])
    slope = np.polyfit(e[sel], np.log(g), 1, w=np.sqrt(tot[sel]))[0]
    assert abs(-1.0 / slope - te) < 0.05 * te, -1.0 / slope
    # and against the exact expected counts, bin by bin (binomial noise)
    exp = _expected_counts(h.sum(), te, de, bins)
    z2 = (tot - exp) ** 2 / np.maximum(exp, 1.0)
    assert z2.mean() < 2.0


def test_fit_recovers_two_temperatures():
    # the paper's bulk values: T_l = 0.31 eV, T_h = 2.32 eV
    bins, de = 200, 0.05
    n_l, n_h = 4e8, 1e8
    counts = np.rint(_expected_counts(n_l, 0.31, de, bins) + _expected_counts(n_h, 2.32, de, bins)).astype(np.int64)
    tl, th, al, ah = P.pic_eepf_fit(counts, de, 0.02, 9.0)
    assert abs(tl - 0.31) < 0.02 * 0.31, tl
    assert abs(th - 2.32) < 0.02 * 2.32, th
    assert al > ah > 0.0


def test_fit_of_one_maxwellian():
    bins, de = 150, 0.1
    counts = np.rint(_expected_counts(1e9, 3.0, de, bins)).astype(np.int64)
    tl, th, al, ah = P.pic_eepf_fit(counts, de, 0.05, 14.0)
    # a single group: either the one-temperature form or two nearly equal groups
    for t, a in ((tl, al), (th, ah)):
        if a > 0.05 * (al + ah):
            assert abs(t - 3.0) < 0.03 * 3.0, (tl, th, al, ah)


def test_fit_rejects_bad_input():
    with pytest.raises(P.PicError) as e:
        P.pic_eepf_fit(np.zeros(50, np.int64), 0.1, 0.0, 5.0)
    assert e.value.status == P.PIC_EINVAL
    with pytest.raises(P.PicError):
        P.pic_eepf_fit(np.ones(50, np.int64), -0.1, 0.0, 5.0)

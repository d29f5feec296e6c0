"""Pins of the oracle's phase-resolved moments and fine MD-region grid
(Sec. IV.C: electron fluxes resolved in rf phase, densities and fluxes in the
MD region on cubes of edge 0.08 dx).

Ballistic particles (no field: grounded electrodes, a negligible weight) have
the closed-form positions x_s = x_0 + s v dt after step s.  The CIC node
weights of a particle sum to one and reproduce its position exactly (linear
interpolation is exact on linear functions), so the zeroth and first spatial
moments of the node densities of a phase bin give the number of particles and
their mean position over that bin's samples.  With f dt = 1/20 and a phase
offset of half a step, the sample after step s has the rf phase fraction
(2s + 1)/40 mod 1, which integer arithmetic bins without rounding."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1801_00972_gb300 import inputs as I

DT = 1e-10
F_RF = 1.0 / (20 * DT)
PSI = 2.0 * math.pi / 40.0
NPH = 4


def _bin(s):
    return ((2 * s + 1) % 40) * NPH // 40


def _ballistic_wl(**over):
    args = dict(nx=8, ny=8, nz=16, n_e=0, n_i=0, grains=0, v_dc=0.0, v_top=0.0, weight=1e-9, dt=DT,
                f_rf=F_RF, phase=PSI)
    args.update(over)
    return I.small(**args)


def _node_xyz(wl):
    k, j, i = np.meshgrid(np.arange(wl.nz + 1), np.arange(wl.ny), np.arange(wl.nx), indexing="ij")
    return np.stack([i.ravel(), j.ravel(), k.ravel()], 1) * wl.dx


def test_phase_bins_of_ballistic_electrons():
    wl = _ballistic_wl()
    rng = np.random.default_rng(5)
    n = 6
    x0 = (np.array([2.0, 2.0, 5.0]) + rng.uniform(0, 3, (n, 3))) * wl.dx
    v = rng.uniform(-1, 1, (n, 3)) * 1e5
    parts = [(x0, v, np.arange(n, dtype=np.uint32)),
             (np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, np.uint32))]
    s = O.Sim(wl, parts, flags=O.NO_MCC | O.IONS_FROZEN | O.MOMENTS, mom_phases=NPH)
    S = 40
    s.step(S)
    xyz = _node_xyz(wl)
    vol = wl.dx ** 3 / wl.weight
    steps = np.array([_bin(t) for t in range(1, S + 1)])
    tot = {}
    for b in range(NPH):
        ne, nb = s.moments_phase(1, b)
        fe, _ = s.moments_phase(3, b)
        sel = np.arange(1, S + 1)[steps == b]
        assert nb == len(sel) == 10
        # every sample adds one particle
        assert abs(ne.sum() * vol - n) < 1e-9 * n
        # mean position over the bin's samples, from the closed form; the CIC
        # weights are fixed point with 2^14 steps per axis, so a sample sits
        # within 2^-15 dx of its true position
        mean = np.mean([x0 + t * v * DT for t in sel], axis=0).sum(0) / n
        got = (ne[:, None] * xyz).sum(0) * vol / n
        assert np.allclose(got, mean, rtol=0, atol=2.0 ** -15 * wl.dx), (b, got / wl.dx, mean / wl.dx)
        # the flux moments carry the (constant) velocities, component by component
        assert np.allclose(fe.reshape(-1, 3).sum(0) * vol, v.sum(0), rtol=1e-9, atol=1e-6)
        tot[b] = (ne, fe, nb)
    # the rf average is the sample-weighted mean of the bins
    ne_all = s.moments(1)
    fe_all = s.moments(3)
    assert np.allclose(sum(tot[b][0] * tot[b][2] for b in tot) / S, ne_all, rtol=1e-12, atol=0)
    assert np.allclose(sum(tot[b][1] * tot[b][2] for b in tot) / S, fe_all, rtol=1e-12, atol=1e-300)


def test_phase_resolved_electrode_potential():
    # no particles: phi at the lower electrode in bin b is the mean of the
    # electrode voltage v_dc + v_rf sin(2 pi f t_s + psi) over the bin's samples
    wl = _ballistic_wl(v_dc=-20.0, v_rf=100.0, v_top=3.0, weight=1.0)
    parts = [(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, np.uint32))] * 2
    s = O.Sim(wl, parts, flags=O.NO_MCC | O.MOMENTS, mom_phases=NPH)
    S = 60
    s.step(S)
    nxy = wl.nx * wl.ny
    for b in range(NPH):
        ph, nb = s.moments_phase(0, b)
        sel = [t for t in range(1, S + 1) if _bin(t) == b]
        assert nb == len(sel)
        expect = np.mean([-20.0 + 100.0 * math.sin(2 * math.pi * F_RF * t * DT + PSI) for t in sel])
        assert np.allclose(ph[:nxy], expect, rtol=0, atol=1e-10)
        assert np.allclose(ph[-nxy:], 3.0, rtol=0, atol=1e-12)
    # and the rf average of the lower electrode is the mean over all samples
    ph = s.moments(0)
    expect = np.mean([-20.0 + 100.0 * math.sin(2 * math.pi * F_RF * t * DT + PSI) for t in range(1, S + 1)])
    assert np.allclose(ph[:nxy], expect, rtol=0, atol=1e-10)


def _edges_bin(p, o, h, n):
    """Fine cell of p by searching the cell edges (None if outside or within 1e-6 h of an edge)."""
    idx = []
    for a in range(3):
        e = o[a] + h * np.arange(n[a] + 1)
        if p[a] < e[0] or p[a] >= e[-1]:
            if min(abs(p[a] - e[0]), abs(p[a] - e[-1])) < 1e-6 * h:
                return "edge"
            return None
        i = int(np.searchsorted(e, p[a], side="right")) - 1
        if min(p[a] - e[i], e[i + 1] - p[a]) < 1e-6 * h:
            return "edge"
        idx.append(i)
    return tuple(idx)


def test_fine_grid_of_ballistic_particles():
    wl = _ballistic_wl()
    h = 0.08 * wl.dx
    nf = (25, 20, 15)
    o = np.array([3.1, 2.7, 6.3]) * wl.dx
    rng = np.random.default_rng(9)
    ne, ni = 60, 25
    box = np.array(nf) * h
    xe = o + rng.uniform(-0.2, 1.2, (ne, 3)) * box
    ve = rng.uniform(-1, 1, (ne, 3)) * 4e4
    xi = o + rng.uniform(0.0, 1.0, (ni, 3)) * box
    vi = rng.uniform(-1, 1, (ni, 3)) * 3e2
    parts = [(xe, ve, np.arange(ne, dtype=np.uint32)), (xi, vi, np.arange(ne, ne + ni, dtype=np.uint32))]
    s = O.Sim(wl, parts, flags=O.NO_MCC | O.IONS_FROZEN | O.MOMENTS, fine_n=nf, fine_h=h, fine_origin=o)
    S = 30
    s.step(S)
    norm = wl.weight / (h ** 3 * S)
    for sp, (x0, v, moving) in enumerate(((xe, ve, True), (xi, vi, False))):
        cnt = np.zeros((nf[2], nf[1], nf[0]))
        sv = np.zeros((nf[2], nf[1], nf[0], 3))
        for t in range(1, S + 1):
            for p in range(len(x0)):
                pos = x0[p] + (t * v[p] * DT if moving else 0.0)
                c = _edges_bin(pos, o, h, nf)
                assert c != "edge"
                if c is not None:
                    cnt[c[2], c[1], c[0]] += 1
                    sv[c[2], c[1], c[0]] += v[p]
        n = s.fine_moments(1 + sp)
        f = s.fine_moments(3 + sp)
        assert np.array_equal(np.rint(n / norm), cnt)
        assert cnt.sum() > 100
        # the residual self field moves the electron velocities by ~1e-13 relative
        assert np.allclose(f / norm, sv, rtol=1e-10, atol=1e-6)
    # a reset empties the window
    s.reset_moments()
    s.step(1)
    assert s.fine_moments(2).sum() / (wl.weight / h ** 3) == pytest.approx(ni, abs=1e-6)

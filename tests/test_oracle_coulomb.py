"""Pins of the oracle's binary Coulomb collisions (Table I; the paper's cited
binary-collision model): exact momentum and energy conservation cell by cell,
the rotation geometry of one collision, independence of array order, and the
mean momentum loss of fast electrons on ions at rest against the textbook
electron-ion momentum-transfer rate n e^4 lnL / (4 pi eps0^2 m_e mu v^3)."""
import math

import numpy as np

import oracle as O
from paper_1801_00972_gb300 import inputs as I

QE, ME, MAR, EPS0 = I.QE, I.ME, I.MAR, 8.8541878128e-12


def _parts(xe=(), ve=(), xi=(), vi=()):
    xe = np.asarray(xe, float).reshape(-1, 3); ve = np.asarray(ve, float).reshape(-1, 3)
    xi = np.asarray(xi, float).reshape(-1, 3); vi = np.asarray(vi, float).reshape(-1, 3)
    ie = np.arange(len(xe), dtype=np.uint32)
    ii = np.arange(len(xe), len(xe) + len(xi), dtype=np.uint32)
    return [(xe, ve, ie), (xi, vi, ii)]


def _by_id(s, sp):
    x, v, ids = s.particles(sp)
    o = np.argsort(ids)
    return x[o], v[o], ids[o]


def _cells(wl, x):
    c = np.floor(x / wl.dx).astype(int)
    return (c[:, 2] * wl.ny + c[:, 1]) * wl.nx + c[:, 0]


def test_momentum_and_energy_conserved_per_cell():
    # a dense Maxwellian plasma, about 60 particles of each species per cell
    wl = I.small(nx=4, ny=4, nz=8, n_e=8000, n_i=8000, grains=0, v_dc=0.0, weight=2e3)
    parts = I.sample_particles(wl)
    # hotter ions so that the ion-ion collisions are not negligible
    parts[1] = (parts[1][0], parts[1][1] * 30.0, parts[1][2])
    s = O.Sim(wl, parts, flags=O.COULOMB)
    before = [_by_id(s, sp) for sp in range(2)]
    s.coulomb()
    after = [_by_id(s, sp) for sp in range(2)]
    m = (ME, MAR)
    cells = [_cells(wl, before[sp][0]) for sp in range(2)]
    nc = wl.nx * wl.ny * wl.nz
    p0 = np.zeros((nc, 3)); p1 = np.zeros((nc, 3)); k0 = np.zeros(nc); k1 = np.zeros(nc); scale = np.zeros(nc)
    changed = 0
    for sp in range(2):
        v0, v1 = before[sp][1], after[sp][1]
        assert np.array_equal(before[sp][0], after[sp][0])          # positions untouched
        changed += np.count_nonzero(np.any(v0 != v1, axis=1))
        for a in range(3):
            p0[:, a] += np.bincount(cells[sp], m[sp] * v0[:, a], nc)
            p1[:, a] += np.bincount(cells[sp], m[sp] * v1[:, a], nc)
        k0 += np.bincount(cells[sp], 0.5 * m[sp] * (v0 ** 2).sum(1), nc)
        k1 += np.bincount(cells[sp], 0.5 * m[sp] * (v1 ** 2).sum(1), nc)
        scale += np.bincount(cells[sp], m[sp] * np.linalg.norm(v0, axis=1), nc)
    assert changed == 16000                      # every particle takes part in a collision
    assert np.max(np.abs(p1 - p0).max(1) / scale) < 1e-13
    assert np.max(np.abs(k1 - k0) / k0) < 1e-13
    # the collisions did something measurable
    assert np.max(np.abs(after[0][1] - before[0][1])) > 1e-3 * np.sqrt((before[0][1] ** 2).mean())


def test_single_collision_is_a_rotation_of_the_relative_velocity():
    # one electron pair in a cell: |u'| = |u|, and the deflection angle obeys
    # tan(Theta/2) = delta with delta of the stated variance
    wl = I.small(nx=4, ny=4, nz=4, n_e=0, n_i=0, grains=0, v_dc=0.0, weight=5e6)
    x = np.full((2, 3), 1.5 * wl.dx)
    v = np.array([[3e5, -2e5, 4e5], [-1e5, 2.5e5, -3e5]])
    s = O.Sim(wl, _parts(xe=x, ve=v), flags=O.COULOMB)
    s.coulomb()
    _, v1, _ = _by_id(s, 0)
    u0 = v[0] - v[1]; u1 = v1[0] - v1[1]
    assert abs(np.linalg.norm(u1) - np.linalg.norm(u0)) < 1e-12 * np.linalg.norm(u0)
    assert np.allclose(v1.sum(0), v.sum(0), rtol=0, atol=1e-9)
    cos_t = np.dot(u0, u1) / np.dot(u0, u0)
    assert cos_t < 1.0 - 1e-12                    # deflected


def test_order_independence():
    wl = I.small(nx=4, ny=4, nz=4, n_e=3000, n_i=2500, grains=0, v_dc=0.0, weight=5e3)
    parts = I.sample_particles(wl)
    a = O.Sim(wl, parts, flags=O.COULOMB)
    rng = np.random.default_rng(3)
    shuf = []
    for x, v, ids in parts:
        o = rng.permutation(len(ids))
        shuf.append((x[o], v[o], ids[o]))
    b = O.Sim(wl, shuf, flags=O.COULOMB)
    a.coulomb(); b.coulomb()
    for sp in range(2):
        xa, va, ia = _by_id(a, sp)
        xb, vb, ib = _by_id(b, sp)
        assert np.array_equal(ia, ib) and np.array_equal(va, vb)


def test_electron_ion_momentum_transfer_rate():
    # N electrons at speed v0 along z and N Ar+ at rest, all in one cell.  Over
    # one pass the mean change of v_z is -nu dt v0 with the textbook rate
    #   nu = n e^4 lnL / (4 pi eps0^2 m_e mu v0^3),  1/mu = 1/m_e + 1/M,
    # up to the model's small-angle correction (relative O(sigma^2) ~ 1e-3).
    n = 200_000
    v0, dt, lnl = 1e6, 1e-10, 10.0
    dx = 0.2e-3
    dens = 2.5e18
    w = dens * dx ** 3 / n
    wl = I.small(nx=4, ny=4, nz=4, n_e=0, n_i=0, grains=0, v_dc=0.0, weight=w, dt=dt)
    rng = np.random.default_rng(11)
    x = (1.0 + rng.uniform(0.05, 0.95, (n, 3))) * dx          # cell (1, 1, 1)
    ve = np.zeros((n, 3)); ve[:, 2] = v0
    s = O.Sim(wl, _parts(xe=x, ve=ve, xi=x.copy(), vi=np.zeros((n, 3))), flags=O.COULOMB, coulomb_log=lnl)
    s.coulomb()
    _, v1, _ = _by_id(s, 0)
    mu = ME * MAR / (ME + MAR)
    nu = dens * QE ** 4 * lnl / (4 * math.pi * EPS0 ** 2 * ME * mu * v0 ** 3)
    dvz = (v1[:, 2] - v0).mean()
    sem = (v1[:, 2] - v0).std() / math.sqrt(n)
    expect = -nu * dt * v0
    assert abs(dvz - expect) <= 4 * sem + 5e-3 * abs(expect), (dvz, expect, sem)
    # the transverse kicks average out
    assert abs(v1[:, 0].mean()) <= 5 * v1[:, 0].std() / math.sqrt(n)

"""Pins for the oracle's particle cycle (Sec. III): CIC fixed-point deposit,
ballistic leapfrog motion in a uniform field (Eqs. 1-2, plain and subcycled),
periodic wrap and electrode loss, the PP/PM split around a charged grain
(Eqs. 5-6), grain absorption with integer charge steps, null-collision rates
against the cross-section tables (Table I), collision kinematics, exact
conservation laws, independence from particle order, and the cold plasma
oscillation at omega_pe."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1801_00972_gb300 import inputs as I

QE, ME, MAR, EPS0 = I.QE, I.ME, I.MAR, 8.8541878128e-12
TWO42 = 2 ** 42


def _parts(xe=(), ve=(), xi=(), vi=(), id0=0):
    xe = np.asarray(xe, float).reshape(-1, 3); ve = np.asarray(ve, float).reshape(-1, 3)
    xi = np.asarray(xi, float).reshape(-1, 3); vi = np.asarray(vi, float).reshape(-1, 3)
    ie = np.arange(id0, id0 + len(xe), dtype=np.uint32)
    ii = np.arange(id0 + len(xe), id0 + len(xe) + len(xi), dtype=np.uint32)
    return [(xe, ve, ie), (xi, vi, ii)]


def test_deposit_weights_and_total_charge():
    wl = I.small(n_e=500, n_i=700, grains=0)
    parts = I.sample_particles(wl)
    s = O.Sim(wl, parts)
    rq = s.rho()
    assert rq.sum() == TWO42 * (700 - 500)
    # a particle on a node puts all of its charge on that node
    wl2 = I.small(grains=0, n_e=0, n_i=0)
    p = np.array([[3 * wl2.dx, 5 * wl2.dx, 7 * wl2.dx]])
    s2 = O.Sim(wl2, _parts(xi=p, vi=np.zeros((1, 3))))
    rq = s2.rho().reshape(wl2.nz + 1, wl2.ny, wl2.nx)
    assert rq[7, 5, 3] == TWO42 and np.count_nonzero(rq) == 1
    # the centre of a cell splits the charge equally over its 8 corners
    p = np.array([[3.5 * wl2.dx, 5.5 * wl2.dx, 7.5 * wl2.dx]])
    s3 = O.Sim(wl2, _parts(xe=p, ve=np.zeros((1, 3))))
    rq = s3.rho().reshape(wl2.nz + 1, wl2.ny, wl2.nx)
    assert np.count_nonzero(rq) == 8 and np.all(rq[7:9, 5:7, 3:5] == -TWO42 // 8)


def _ballistic(md_sub, grains, nsteps=6):
    # zero weight: the particles carry no charge, so the field is the electrode ramp alone
    wl = I.small(grains=grains, n_e=0, n_i=0, weight=0.0, v_dc=-40.0, v_top=10.0, md_sub=md_sub)
    L = np.array(wl.box)
    rng = np.random.default_rng(5)
    xe = rng.uniform(0.3, 0.7, (50, 3)) * L
    ve = rng.normal(0, 2e5, (50, 3))
    xi = rng.uniform(0.3, 0.7, (50, 3)) * L
    vi = rng.normal(0, 300.0, (50, 3))
    s = O.Sim(wl, _parts(xe, ve, xi, vi), flags=O.NO_MCC)
    Ez = -(10.0 - (-40.0)) / L[2]
    for sp, (x0, v0), qm in ((0, (xe, ve), -QE / ME), (1, (xi, vi), QE / MAR)):
        pass
    s.step(nsteps)
    return wl, s, (xe, ve, xi, vi), Ez


def test_ballistic_uniform_field():
    nsteps = 6
    wl, s, (xe, ve, xi, vi), Ez = _ballistic(1, 0, nsteps)
    L = np.array(wl.box)
    dt = wl.dt
    for sp, x0, v0, qm in ((0, xe, ve, -QE / ME), (1, xi, vi, QE / MAR)):
        x, v, ids = s.particles(sp)
        a = np.array([0.0, 0.0, qm * Ez])
        n = nsteps
        v_want = v0 + n * a * dt
        x_want = x0 + n * v0 * dt + a * dt * dt * n * (n + 1) / 2
        x_want[:, :2] %= L[:2]
        alive = (x_want[:, 2] >= 0) & (x_want[:, 2] <= L[2])
        assert len(ids) == alive.sum()
        sel = alive
        assert np.allclose(v, v_want[sel], rtol=1e-10, atol=1e-6)
        assert np.allclose(x, x_want[sel], rtol=1e-10, atol=1e-14)


def test_subcycled_ballistic_closed_form():
    """A particle in an MD region with an uncharged grain takes M substeps of
    dt/M; in a uniform field x advances by v dt + a dt^2 (M+1)/(2M)."""
    M = 40
    wl = I.small(grains=1, n_e=0, n_i=0, weight=0.0, v_dc=-40.0, v_top=10.0, md_sub=M)
    L = np.array(wl.box)
    g = wl.grain_pos[0]
    x0 = np.array([[g[0] + 0.6 * wl.dx, g[1] - 0.4 * wl.dx, g[2] + 0.3 * wl.dx]])
    v0 = np.array([[1e3, -2e3, 500.0]])
    s = O.Sim(wl, _parts(xe=x0, ve=v0), flags=O.NO_MCC)
    s.step(1)
    x, v, _ = s.particles(0)
    Ez = -(50.0) / L[2]
    a = np.array([0.0, 0.0, -QE / ME * Ez])
    assert np.allclose(v[0], v0[0] + a * wl.dt, rtol=1e-12)
    assert np.allclose(x[0], x0[0] + v0[0] * wl.dt + a * wl.dt ** 2 * (M + 1) / (2 * M), rtol=1e-12)


def test_wrap_and_electrode_loss():
    wl = I.small(grains=0, n_e=0, n_i=0, weight=0.0, v_dc=0.0, v_top=0.0)
    L = np.array(wl.box)
    dt = wl.dt
    xe = np.array([[L[0] - 1e-6, 0.5 * L[1], 0.5 * L[2]],      # leaves through +x, re-enters at 0
                   [1e-6, 1e-6, 0.5 * L[2]],                  # leaves through -x and -y
                   [0.5 * L[0], 0.5 * L[1], 1e-6],            # lost at the bottom electrode
                   [0.5 * L[0], 0.5 * L[1], L[2] - 1e-6]])    # lost at the top electrode
    ve = np.array([[3e4, 0, 0], [-3e4, -3e4, 0], [0, 0, -3e4], [0, 0, 3e4]])
    s = O.Sim(wl, _parts(xe=xe, ve=ve), flags=O.NO_MCC)
    s.step(1)
    x, v, ids = s.particles(0)
    assert ids.tolist() == [0, 1]
    assert np.allclose(x[0], [L[0] - 1e-6 + 3e-6 - L[0], 0.5 * L[1], 0.5 * L[2]], rtol=0, atol=1e-15)
    assert np.allclose(x[1], [1e-6 - 3e-6 + L[0], 1e-6 - 3e-6 + L[1], 0.5 * L[2]], rtol=0, atol=1e-15)
    c = s.counters()
    assert c["lost_bot_e"] == 1 and c["lost_top_e"] == 1


def test_pppm_split_is_coulomb_inside_md_region():
    """With no plasma and a charged grain, E inside the grain's MD region is
    the electrode field plus the bare Coulomb field (Eqs. 5-6): the mesh part
    of the grain's own field cancels."""
    wl = I.small(grains=1, n_e=0, n_i=0, weight=1.0, v_dc=-20.0, v_top=0.0)
    s = O.Sim(wl, _parts())
    s.set_grain_counts([[30000, 1000]])      # net -29000 e
    Q = -29000 * QE
    L = np.array(wl.box)
    g = wl.grain_pos[0]
    Ebc = np.array([0, 0, -20.0 / L[2]])
    rng = np.random.default_rng(11)
    kc = 1 / (4 * np.pi * EPS0)
    for _ in range(40):
        p = g + rng.uniform(-1.45, 1.45, 3) * wl.dx
        E, md = s.field_at(p)
        d = p - g
        r = np.linalg.norm(d)
        want = Ebc + Q * kc * d / r ** 3
        assert md
        assert np.allclose(E, want, rtol=1e-9, atol=1e-9 * np.linalg.norm(want))
    # outside the region the grain acts through the mesh alone; along x in a
    # 64^3 box (electrode and periodic images far away) that field tends to
    # Coulomb as the O((dx/r)^2) grid error falls off
    n = 64
    wl = I.small(nx=n, ny=n, nz=n, grains=0, n_e=0, n_i=0, weight=1.0, v_dc=0.0, v_top=0.0)
    wl.grain_pos = np.array([[n / 2 + 0.3, n / 2 - 0.4, n / 2 + 0.4]]) * wl.dx
    wl.grain_r = np.array([5e-6])
    s = O.Sim(wl, _parts())
    s.set_grain_counts([[30000, 1000]])
    g = wl.grain_pos[0]
    for r, tol in ((5.0, 0.08), (7.0, 0.04), (10.0, 0.02)):
        d = np.array([r, 0.2, 0.1]) * wl.dx
        E, md = s.field_at(g + d)
        assert not md
        want = Q * kc * d / np.linalg.norm(d) ** 3
        assert np.linalg.norm(E - want) < tol * np.linalg.norm(want), (r, E, want)


def test_absorption_integer_charge():
    wl = I.small(grains=1, n_e=0, n_i=0, weight=7.0, v_dc=0.0, v_top=0.0)
    g = wl.grain_pos[0]
    r = wl.grain_r[0]
    # electrons and ions aimed straight at the grain from just outside it
    xe = np.array([g + [0, 0, 3 * r], g + [3 * r, 0, 0]])
    ve = np.array([[0, 0, -1.5e5], [-1.5e5, 0, 0]])    # 15 um per step, 0.375 um per substep
    xi = np.array([g + [0, -2.5 * r, 0]])
    vi = np.array([[0, 1.2e5, 0]])
    s = O.Sim(wl, _parts(xe, ve, xi, vi), flags=O.NO_MCC)
    s.step(1)
    n_abs, q = s.grains()
    assert n_abs.tolist() == [[2, 1]]
    assert q[0] == (QE * 7.0) * (1 - 2)
    assert s.count(0) == 0 and s.count(1) == 0
    rq = s.rho()
    assert rq.sum() == TWO42 * (1 - 2)


def _mono(sp, energy_ev, n, wl):
    L = np.array(wl.box)
    rng = np.random.default_rng(2)
    x = rng.uniform(0.2, 0.8, (n, 3)) * L
    m = ME if sp == 0 else MAR
    d = rng.standard_normal((n, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
    v = d * math.sqrt(2 * energy_ev * QE / m)
    return x, v


def _xs_interp(tab, de, e):
    t = e / de
    i = int(t)
    return tab[i] + (t - i) * (tab[i + 1] - tab[i])


@pytest.mark.parametrize("energy", [5.0, 20.0, 60.0])
def test_electron_collision_rates(energy):
    n = 100000
    wl = I.small(grains=0, n_e=n, n_i=0, weight=0.0, v_dc=0.0, v_top=0.0, dt=5e-10, nx=32, ny=32, nz=64)
    x, v = _mono(0, energy, n, wl)
    s = O.Sim(wl, _parts(xe=x, ve=v))
    s.step(1)
    c = s.counters()
    assert c["err"] == 0 and c["lost_bot_e"] == 0 and c["lost_top_e"] == 0
    pnull = 1 - math.exp(-wl.nu_max_e * wl.dt)
    vm = math.sqrt(2 * energy * QE / ME)
    for name, row in (("e_el", 0), ("e_exc", 1), ("e_ion", 2)):
        p = pnull * wl.n_gas * _xs_interp(wl.xs[row], wl.de_e, energy) * vm / wl.nu_max_e
        want = p * n
        sd = math.sqrt(max(n * p * (1 - p), 1.0))
        assert abs(c[name] - want) <= 4.5 * sd, (name, c[name], want)


def test_electron_collision_rates_maxwellian():
    # a Maxwellian at T_e = 8 eV: per-process counts against N P_null n_g <sigma_j v> / nu_max,
    # <sigma v> by quadrature of the tabulated cross sections over the Maxwellian
    # energy density 2 sqrt(E / pi) T^-3/2 exp(-E / T)
    te, n = 8.0, 150000
    wl = I.small(grains=0, n_e=n, n_i=0, weight=0.0, v_dc=0.0, v_top=0.0, dt=5e-10, nx=32, ny=32, nz=64,
                 te_ev=te)
    x, v, ids = I.sample_particles(wl)[0]
    s = O.Sim(wl, _parts(xe=x, ve=v))
    s.step(1)
    c = s.counters()
    assert c["err"] == 0
    pnull = 1 - math.exp(-wl.nu_max_e * wl.dt)
    e = np.linspace(0.0, 40.0 * te, 400001)
    f = 2.0 * np.sqrt(e / math.pi) * te ** -1.5 * np.exp(-e / te)
    vel = np.sqrt(2.0 * e * QE / ME)
    grid = np.arange(wl.xs.shape[1]) * wl.de_e
    for name, row in (("e_el", 0), ("e_exc", 1), ("e_ion", 2)):
        sig = np.interp(e, grid, wl.xs[row])
        sv = np.trapezoid(sig * vel * f, e)
        p = pnull * wl.n_gas * sv / wl.nu_max_e
        want = p * n
        sd = math.sqrt(max(n * p * (1 - p), 1.0))
        assert abs(c[name] - want) <= 4.5 * sd + 0.01 * want, (name, c[name], want)
    assert c["e_exc"] > 50 and c["e_ion"] > 50


def test_ion_collision_rates():
    n = 60000
    energy = 40.0     # ion speed far above the neutral thermal speed: relative speed ~ ion speed
    wl = I.small(grains=0, n_e=0, n_i=n, weight=0.0, v_dc=0.0, v_top=0.0, dt=2e-8, nz=64)
    x, v = _mono(1, energy, n, wl)
    s = O.Sim(wl, _parts(xi=x, vi=v))
    s.step(1)
    c = s.counters()
    assert c["err"] == 0 and c["lost_bot_i"] == 0 and c["lost_top_i"] == 0
    pnull = 1 - math.exp(-wl.nu_max_i * wl.dt)
    vm = math.sqrt(2 * energy * QE / MAR)
    for name, row in (("i_el", 3), ("i_cx", 4)):
        p = pnull * wl.n_gas * _xs_interp(wl.xs[row], wl.de_i, energy) * vm / wl.nu_max_i
        want = p * n
        sd = math.sqrt(n * p * (1 - p))
        assert abs(c[name] - want) <= 4.5 * sd + 0.02 * want, (name, c[name], want)


def test_collision_kinematics():
    n = 40000
    energy = 40.0
    wl = I.small(grains=0, n_e=n, n_i=0, weight=0.0, v_dc=0.0, v_top=0.0, dt=5e-10, nx=32, ny=32, nz=64)
    x, v = _mono(0, energy, n, wl)
    s = O.Sim(wl, _parts(xe=x, ve=v))
    s.step(1)
    c = s.counters()
    xo, vo, ids = s.particles(0)
    e = 0.5 * ME * np.sum(vo ** 2, 1) / QE
    parents = ids < n
    children = ~parents
    assert children.sum() == c["e_ion"] and s.count(1) == c["e_ion"]
    assert s.next_id == n + 2 * c["e_ion"]
    half_ion = (energy - I.EPS_ION) / 2
    exc = energy - I.EPS_EXC
    near = lambda a, b: np.abs(a - b) <= 1e-9 * max(b, 1)
    cls_ion = near(e, half_ion)
    cls_exc = near(e, exc)
    cls_keep = (e <= energy * (1 + 1e-9)) & (e >= energy * (1 - 4 * ME / MAR) - 1e-9)
    assert np.all(cls_ion | cls_exc | cls_keep)
    assert cls_ion[children].all()
    assert cls_ion[parents].sum() == c["e_ion"]
    assert cls_exc.sum() == c["e_exc"]
    # children sit where their parents ended the step
    _, _, iids = s.particles(1)
    assert np.all(iids[1:] > iids[:-1])


def test_conservation_and_order_independence():
    wl = I.small(n_e=3000, n_i=3000, grains=2, v_dc=-60.0, dt=2e-10)
    parts = I.sample_particles(wl)
    a = O.Sim(wl, parts)
    rng = np.random.default_rng(0)
    shuffled = []
    for (x, v, ids) in parts:
        o = rng.permutation(len(ids))
        shuffled.append((x[o], v[o], ids[o]))
    b = O.Sim(wl, shuffled)
    prev = (a.count(0), a.count(1))
    pc = a.counters()
    for _ in range(8):
        a.step(); b.step()
        c = a.counters()
        ion = c["e_ion"] - pc["e_ion"]
        dn_e = prev[0] - (c["lost_bot_e"] - pc["lost_bot_e"]) - (c["lost_top_e"] - pc["lost_top_e"]) \
            - (c["abs_e"] - pc["abs_e"]) + ion
        dn_i = prev[1] - (c["lost_bot_i"] - pc["lost_bot_i"]) - (c["lost_top_i"] - pc["lost_top_i"]) \
            - (c["abs_i"] - pc["abs_i"]) + ion
        assert (a.count(0), a.count(1)) == (dn_e, dn_i)
        assert c["err"] == 0
        n_abs, _ = a.grains()
        net = int(n_abs[:, 1].sum() - n_abs[:, 0].sum())
        assert a.rho().sum() == TWO42 * (a.count(1) - a.count(0) + net)
        prev, pc = (a.count(0), a.count(1)), c
    for sp in range(2):
        xa, va, ia = a.particles(sp)
        xb, vb, ib = b.particles(sp)
        assert np.array_equal(ia, ib) and np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert np.array_equal(a.rho(), b.rho())
    assert np.array_equal(a.grains()[0], b.grains()[0])


def test_cold_plasma_oscillation():
    """Cold electrons over frozen neutralising ions, displaced by
    d sin(2 pi z / Lz) (zero mean, so grounded electrodes induce no offset):
    the displacement oscillates at omega with sin(omega dt / 2) = omega_pe dt / 2
    (leapfrog dispersion of Eqs. 1-2)."""
    nx = ny = 4
    nz = 64
    dx = 0.2e-3
    ppc = 4                                   # particles per cell along z, 1 per column cell
    L = np.array([nx * dx, ny * dx, nz * dx])
    zs = (np.arange(nz * ppc) + 0.5) * dx / ppc
    X, Y, Z = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dx, zs, indexing="ij")
    base = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    n = len(base)
    n0 = 1e14
    w = n0 * np.prod(L) / n
    wpe = math.sqrt(n0 * QE ** 2 / (EPS0 * ME))
    dt = 0.05 / wpe
    amp = 0.02 * dx
    xe = base.copy()
    xe[:, 2] += amp * np.sin(2 * np.pi * base[:, 2] / L[2])
    wl = I.small(nx=nx, ny=ny, nz=nz, grains=0, n_e=n, n_i=n, weight=w, v_dc=0.0, v_top=0.0, dt=dt)
    s = O.Sim(wl, _parts(xe, np.zeros_like(xe), base, np.zeros_like(base)),
              flags=O.NO_MCC | O.IONS_FROZEN)
    probe = np.argmin(np.abs(base[:, 2] - L[2] / 4) + base[:, 0] + base[:, 1])
    disp = []
    for _ in range(400):
        s.step()
        x, _, ids = s.particles(0)
        disp.append(x[probe, 2] - base[probe, 2])
    disp = np.array(disp)
    sgn = np.sign(disp)
    cross = np.where(sgn[1:] != sgn[:-1])[0]
    assert len(cross) >= 4
    t = [c + disp[c] / (disp[c] - disp[c + 1]) for c in cross]
    period = 2 * np.mean(np.diff(t)) * dt
    w_meas = 2 * np.pi / period
    w_want = 2 / dt * math.asin(wpe * dt / 2)
    assert abs(w_meas / w_want - 1) < 0.01

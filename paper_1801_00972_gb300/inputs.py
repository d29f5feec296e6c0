"""Seeded synthetic workloads for the PIC-MCC/PPPM particle cycle.

This module only builds inputs: mesh and electrode parameters, argon
cross-section tables, grain clusters and initial particles.  It holds none of
the method's arithmetic, so both the CUDA library and the CPU oracle can be
fed from it.

The paper's discharge (Sec. II and III: argon at 300 K, 13.56 MHz drive of
100 V amplitude on the lower electrode, upper electrode grounded, grains of
~10 um size in the sheath 5.6 mm above the driven electrode, bulk density
~1e15 m^-3) sets the shape of every workload.  The paper's LxCat/Phelps
cross sections are not available here; ``cross_sections`` builds smooth
analytic stand-ins with argon's excitation (11.5 eV) and ionization
(15.76 eV) thresholds and realistic magnitudes.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# physical constants used to build inputs (CODATA 2018)
QE = 1.602176634e-19
ME = 9.1093837015e-31
AMU = 1.66053906660e-27
MAR = 39.948 * AMU
KB = 1.380649e-23

EPS_EXC = 11.5     # eV, lowest argon excitation threshold used by the stand-in table
EPS_ION = 15.76    # eV, argon ionization energy

BASE_SEED = 180100972


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dt: float
    weight: float
    md_sub: int
    v_dc: float
    v_rf: float
    f_rf: float
    phase: float
    v_top: float
    n_gas: float
    t_gas: float
    eps_exc: float
    eps_ion: float
    nu_max_e: float
    nu_max_i: float
    de_e: float
    de_i: float
    xs: np.ndarray            # (5, n): e_el, e_exc, e_ion, i_el, i_cx  [m^2]
    grain_pos: np.ndarray     # (ng, 3) metres
    grain_r: np.ndarray       # (ng,) metres
    seed: int
    run_id: int
    n_e: int
    n_i: int
    te_ev: float
    ti_ev: float
    steps: int

    @property
    def nodes(self) -> int:
        return self.nx * self.ny * (self.nz + 1)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def box(self):
        return (self.nx * self.dx, self.ny * self.dx, self.nz * self.dx)


def cross_sections(n: int = 4001, de_e: float = 0.05, de_i: float = 0.05) -> np.ndarray:
    """Analytic stand-in cross sections on uniform energy grids (m^2)."""
    ee = np.arange(n) * de_e
    ei = np.arange(n) * de_i
    e = np.maximum(ee, 1e-3)
    x = e / 12.0
    el = 2e-21 + 1.5e-19 * x * x / (1.0 + x * x) ** 1.2
    exc = np.where(ee > EPS_EXC, 1e-20 * (ee - EPS_EXC) / (ee - EPS_EXC + 20.0), 0.0)
    u = np.maximum(ee / EPS_ION, 1.0)
    ion = np.where(ee > EPS_ION, 8e-20 * np.log(u) / u, 0.0)
    ei_ = np.maximum(ei, 1e-3)
    cx = 1e-20 * (7.5 - 0.5 * np.log(ei_)) ** 2
    iel = 0.5 * cx
    return np.stack([el, exc, ion, iel, cx]).astype(np.float64)


def nu_max_bound(xs: np.ndarray, de: float, n_gas: float, mass: float, rows) -> float:
    """An upper bound of n_g * sum(sigma) * v over the table range and beyond
    (1.5x the top energy), on a grid 8x finer than the table, times 1.05."""
    n = xs.shape[1]
    e = np.linspace(0.0, 1.5 * de * (n - 1), 8 * n)
    grid = np.arange(n) * de
    tot = sum(np.interp(e, grid, xs[r]) for r in rows)
    v = np.sqrt(2.0 * e * QE / mass)
    return float(1.05 * n_gas * np.max(tot * v))


def _gas(pressure_pa: float, t_gas: float = 300.0):
    xs = cross_sections()
    n_gas = pressure_pa / (KB * t_gas)
    nme = nu_max_bound(xs, 0.05, n_gas, ME, (0, 1, 2))
    nmi = nu_max_bound(xs, 0.05, n_gas, MAR, (3, 4))
    return dict(n_gas=n_gas, t_gas=t_gas, xs=xs, nu_max_e=nme, nu_max_i=nmi, de_e=0.05, de_i=0.05,
                eps_exc=EPS_EXC, eps_ion=EPS_ION)


def _hexagon(cx, cy, z, side):
    pts = [(cx, cy, z)]
    for k in range(6):
        a = math.pi / 3.0 * k
        pts.append((cx + side * math.cos(a), cy + side * math.sin(a), z))
    return np.array(pts, dtype=np.float64)


def _max_grains_per_cell(pos, dx, nx, ny, nz):
    cnt = {}
    for p in pos:
        gc = [int(math.floor(p[a] / dx)) for a in range(3)]
        for dk in (-1, 0, 1):
            for dj in (-1, 0, 1):
                for di in (-1, 0, 1):
                    c = ((gc[0] + di) % nx, (gc[1] + dj) % ny, gc[2] + dk)
                    cnt[c] = cnt.get(c, 0) + 1
    return max(cnt.values()) if cnt else 0


def sphere_cluster(n, radius, centre, r_lo, r_hi, dx, dims, seed, max_per_cell=8):
    """n grains placed uniformly in a sphere, centres at least 10 r_hi apart,
    radii uniform in [r_lo, r_hi]; redrawn until no cell is in more than
    ``max_per_cell`` grains' 3x3x3 regions."""
    rng = np.random.default_rng(seed)
    for _ in range(1000):
        pts = []
        while len(pts) < n:
            p = rng.uniform(-radius, radius, 3)
            if p @ p > radius * radius:
                continue
            q = np.asarray(centre) + p
            if all(np.linalg.norm(q - o) >= 10 * r_hi for o in pts):
                pts.append(q)
        pts = np.array(pts)
        if _max_grains_per_cell(pts, dx, *dims) <= max_per_cell:
            return pts, rng.uniform(r_lo, r_hi, n)
    raise RuntimeError("could not place grains")


def workload(index: int, **over) -> Workload:
    """Workloads shaped like the paper's discharge.
    0: small DC sheath, 32x32x64 cells of 0.2 mm, -50 V / 0 V, one 5 um grain
       at the centre, 2 Pa, 1e5 e (3 eV) + 1e5 Ar+ (0.03 eV), dt 1e-10 s, 200 steps.
    1: rf sheath with a 7-grain hexagonal cluster, 64x64x256 cells, 100 V at
       13.56 MHz, r 4.5 um, 0.5 mm spacing at z = 5.6 mm, 2 Pa, 1e7 particles, 20000 steps.
    2: paper-scale cluster, 128x128x512 cells, 50 grains in a 1.5 mm sphere at
       z = 5.6 mm, r ~ U(4,5) um, 2e8 particles, 13.56 MHz.
    4: large, 256x256x1024 cells, 100 grains, 5e8 particles.
    """
    dx = 0.2e-3
    seed = BASE_SEED + index
    if index == 0:
        nx, ny, nz = 32, 32, 64
        gas = _gas(2.0)
        L = (nx * dx, ny * dx, nz * dx)
        gpos = np.array([[L[0] / 2, L[1] / 2, L[2] / 2]])
        grad = np.array([5e-6])
        ne = ni = 100_000
        kw = dict(v_dc=-50.0, v_rf=0.0, f_rf=0.0, phase=0.0, v_top=0.0, steps=200)
    elif index == 1:
        nx, ny, nz = 64, 64, 256
        gas = _gas(2.0)
        L = (nx * dx, ny * dx, nz * dx)
        gpos = _hexagon(L[0] / 2, L[1] / 2, 5.6e-3, 0.5e-3)
        grad = np.full(7, 4.5e-6)
        ne = ni = 5_000_000
        kw = dict(v_dc=0.0, v_rf=100.0, f_rf=13.56e6, phase=0.0, v_top=0.0, steps=20000)
    elif index == 2:
        nx, ny, nz = 128, 128, 512
        gas = _gas(2.0)
        L = (nx * dx, ny * dx, nz * dx)
        gpos, grad = sphere_cluster(50, 1.5e-3, (L[0] / 2, L[1] / 2, 5.6e-3), 4e-6, 5e-6, dx,
                                    (nx, ny, nz), seed)
        ne = ni = 100_000_000
        kw = dict(v_dc=0.0, v_rf=100.0, f_rf=13.56e6, phase=0.0, v_top=0.0, steps=1000)
    elif index == 4:
        nx, ny, nz = 256, 256, 1024
        gas = _gas(2.0)
        L = (nx * dx, ny * dx, nz * dx)
        gpos, grad = sphere_cluster(100, 1.5e-3, (L[0] / 2, L[1] / 2, 5.6e-3), 4e-6, 5e-6, dx,
                                    (nx, ny, nz), seed)
        ne = ni = 250_000_000
        kw = dict(v_dc=0.0, v_rf=100.0, f_rf=13.56e6, phase=0.0, v_top=0.0, steps=100)
    else:
        raise ValueError(f"no workload {index}")
    vol = nx * ny * nz * dx ** 3
    n0 = 1e15
    w = n0 * vol / ne
    args = dict(name=f"w{index}", nx=nx, ny=ny, nz=nz, dx=dx, dt=1e-10, weight=w, md_sub=40,
                grain_pos=gpos, grain_r=grad, seed=seed, run_id=0, n_e=ne, n_i=ni,
                te_ev=3.0, ti_ev=0.03, **gas, **kw)
    args.update(over)
    return Workload(**args)


def ensemble(n_runs: int = 48, seed: int = BASE_SEED + 3):
    """The batched-ensemble workload: independent runs of uneven size.  Per run:
    mesh from {32^3, 32x32x64, 64x64x64, 64x64x128} cells of 0.2 mm, 1e5..2e6
    particles (log-uniform), argon at 1..10 Pa, 1..19 grains of 4-5 um in a
    shell-shaped cluster 5.6 mm above the driven electrode (capped for the
    smallest meshes), 100 V at 13.56 MHz with a random phase."""
    rng = np.random.default_rng(seed)
    shapes = [(32, 32, 32), (32, 32, 64), (64, 64, 64), (64, 64, 128)]
    dx = 0.2e-3
    out = []
    for r in range(n_runs):
        nx, ny, nz = shapes[int(rng.integers(len(shapes)))]
        n_p = int(round(10 ** rng.uniform(5.0, math.log10(2e6))))
        p_pa = float(rng.uniform(1.0, 10.0))
        n_g = int(rng.integers(1, 20))
        L = (nx * dx, ny * dx, nz * dx)
        zc = min(5.6e-3, 0.5 * L[2])
        gpos, grad = sphere_cluster(n_g, min(0.8e-3, 0.2 * L[0]), (L[0] / 2, L[1] / 2, zc), 4e-6, 5e-6, dx,
                                    (nx, ny, nz), int(rng.integers(1 << 30)))
        gas = _gas(p_pa)
        vol = nx * ny * nz * dx ** 3
        out.append(Workload(name=f"ens{r}", nx=nx, ny=ny, nz=nz, dx=dx, dt=1e-10, weight=1e15 * vol / (n_p // 2),
                            md_sub=40, v_dc=0.0, v_rf=100.0, f_rf=13.56e6, phase=float(rng.uniform(0, 2 * math.pi)),
                            v_top=0.0, grain_pos=gpos, grain_r=grad, seed=seed + 7919 * (r + 1), run_id=r,
                            n_e=n_p // 2, n_i=n_p - n_p // 2, te_ev=3.0, ti_ev=0.03, steps=100, **gas))
    return out


def small(nx=8, ny=8, nz=16, n_e=2000, n_i=2000, grains=1, seed=7, **over) -> Workload:
    """A small case for tests: a few tiles, a grain near the middle, DC bias."""
    dx = 0.2e-3
    gas = _gas(over.pop("pressure", 2.0))
    L = (nx * dx, ny * dx, nz * dx)
    if grains == 1:
        gpos = np.array([[0.43 * L[0], 0.55 * L[1], 0.47 * L[2]]])
        grad = np.array([5e-6])
    elif grains == 0:
        gpos = np.zeros((0, 3)); grad = np.zeros(0)
    else:
        rng = np.random.default_rng(seed + 1)
        gpos = np.stack([rng.uniform(0, L[0], grains), rng.uniform(0, L[1], grains),
                         rng.uniform(0.3 * L[2], 0.7 * L[2], grains)], 1)
        grad = rng.uniform(4e-6, 5e-6, grains)
    vol = nx * ny * nz * dx ** 3
    args = dict(name="small", nx=nx, ny=ny, nz=nz, dx=dx, dt=1e-10, weight=1e15 * vol / max(n_e, 1),
                md_sub=40, v_dc=-30.0, v_rf=0.0, f_rf=0.0, phase=0.0, v_top=0.0,
                grain_pos=gpos, grain_r=grad, seed=seed, run_id=0, n_e=n_e, n_i=n_i,
                te_ev=3.0, ti_ev=0.03, steps=10, **gas)
    args.update(over)
    return Workload(**args)


def _near_grains(x, wl, chunk=1 << 22):
    """Mask of the points within 1.5 radii of a grain centre (plain distance).
    Only points whose cell lies in a grain's 3x3x3 cell block can be that close
    (1.5 r < dx), so the distances are taken for those alone."""
    dx = wl.dx
    flag = np.zeros((wl.nz, wl.ny, wl.nx), bool)
    for p, r in zip(wl.grain_pos, wl.grain_r):
        assert 1.5 * r < dx
        c = np.floor(np.asarray(p) / dx).astype(int)
        for dk in (-1, 0, 1):
            k = c[2] + dk
            if 0 <= k < wl.nz:
                for dj in (-1, 0, 1):
                    for di in (-1, 0, 1):
                        flag[k, (c[1] + dj) % wl.ny, (c[0] + di) % wl.nx] = True
    bad = np.zeros(len(x), bool)
    for a in range(0, len(x), chunk):
        xs = x[a:a + chunk]
        c = np.minimum(np.floor(xs / dx).astype(np.int64), np.array([wl.nx - 1, wl.ny - 1, wl.nz - 1]))
        cand = np.nonzero(flag[c[:, 2], c[:, 1], c[:, 0]])[0]
        if cand.size == 0:
            continue
        xc = xs[cand]
        near = np.zeros(cand.size, bool)
        for p, r in zip(wl.grain_pos, wl.grain_r):
            near |= np.sum((xc - p) ** 2, 1) <= (1.5 * r) ** 2
        bad[a + cand[near]] = True
    return bad


_BIG = 1 << 25          # species above this many particles are drawn in parallel chunks


def _sample_chunk(wl, n, t_ev, m, ss, x, v):
    rng = np.random.default_rng(ss)
    L = np.array(wl.box)
    x[:] = rng.random((n, 3)) * L
    if len(wl.grain_r):
        for _ in range(10):
            bad = _near_grains(x, wl)
            if not bad.any():
                break
            x[bad] = rng.random((int(bad.sum()), 3)) * L
    np.minimum(x, np.nextafter(L, 0), out=x)
    v[:] = rng.standard_normal((n, 3)) * math.sqrt(t_ev * QE / m)


def _sample_big(wl, seed, chunk=1 << 23):
    """Large species: chunks of 2^23 particles, each from its own child seed of
    the workload seed, drawn on the host cores in parallel."""
    import concurrent.futures as cf
    import os
    out = []
    base = 0
    root = np.random.SeedSequence(seed)
    for sp, (n, t_ev, m) in enumerate(((wl.n_e, wl.te_ev, ME), (wl.n_i, wl.ti_ev, MAR))):
        x = np.empty((n, 3))
        v = np.empty((n, 3))
        starts = list(range(0, n, chunk))
        seqs = root.spawn(len(starts))
        with cf.ThreadPoolExecutor(max_workers=min(32, os.cpu_count() or 1)) as ex:
            list(ex.map(lambda a: _sample_chunk(wl, min(chunk, n - a[1]), t_ev, m, a[0], x[a[1]:a[1] + chunk],
                                                v[a[1]:a[1] + chunk]), zip(seqs, starts)))
        out.append((x, v, np.arange(base, base + n, dtype=np.uint32)))
        base += n
    return out


def sample_particles(wl: Workload, seed: int | None = None):
    """Uniform positions in the box (outside the grains), Maxwellian velocities.
    Returns [(x (n,3), v (n,3), id (n,) uint32) for electrons, ions]; electron ids
    are 0..n_e-1 and ion ids n_e..n_e+n_i-1.  Workloads with more than 2^25
    particles of a species are drawn in parallel chunks (another random stream,
    the same distributions)."""
    if max(wl.n_e, wl.n_i) > _BIG:
        return _sample_big(wl, wl.seed if seed is None else seed)
    rng = np.random.default_rng(wl.seed if seed is None else seed)
    L = np.array(wl.box)
    out = []
    base = 0
    for n, t_ev, m in ((wl.n_e, wl.te_ev, ME), (wl.n_i, wl.ti_ev, MAR)):
        x = rng.random((n, 3)) * L
        if len(wl.grain_r):
            for _ in range(10):
                bad = _near_grains(x, wl)
                if not bad.any():
                    break
                x[bad] = rng.random((int(bad.sum()), 3)) * L
        x = np.minimum(x, np.nextafter(L, 0))
        vth = math.sqrt(t_ev * QE / m)
        v = rng.standard_normal((n, 3)) * vth
        ids = np.arange(base, base + n, dtype=np.uint32)
        base += n
        out.append((x, v, ids))
    return out

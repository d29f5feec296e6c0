"""Pins for the oracle's exact discrete Poisson solve (Eq. 3) and its
finite-difference field (Eq. 4): a discrete eigenfunction, the electrode
ramp, a dense LU solve of the assembled matrix, second-order convergence to
a continuous solution, and the exactness of the difference formulas on
polynomials."""
import math

import numpy as np
import pytest

import oracle as O


def _grid(nx, ny, nz, dx):
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny), np.arange(nx), indexing="ij")
    return i * dx, j * dx, k * dx


@pytest.mark.parametrize("m", [(1, 0, 1), (2, 3, 2), (0, 0, 5), (3, 1, 7)])
def test_discrete_eigenfunction(m):
    nx, ny, nz, dx = 8, 16, 12, 0.2e-3
    x, y, z = _grid(nx, ny, nz, dx)
    Lx, Ly, Lz = nx * dx, ny * dx, nz * dx
    u = np.sin(2 * np.pi * m[0] * x / Lx + 0.3) * np.cos(2 * np.pi * m[1] * y / Ly) * np.sin(np.pi * m[2] * z / Lz)
    lam = (2 * np.cos(2 * np.pi * m[0] / nx) - 2 + 2 * np.cos(2 * np.pi * m[1] / ny) - 2
           + 2 * np.cos(np.pi * m[2] / nz) - 2) / dx ** 2
    f = -lam * u
    phi = O.poisson(nx, ny, nz, dx, f, 0.0, 0.0)
    assert np.max(np.abs(phi - u)) < 1e-12 * max(1.0, np.max(np.abs(u)))


def test_electrode_ramp():
    nx, ny, nz, dx = 4, 8, 20, 0.2e-3
    phi = O.poisson(nx, ny, nz, dx, np.zeros(nx * ny * (nz + 1)), -50.0, 7.0)
    want = -50.0 + 57.0 * np.arange(nz + 1) / nz
    assert np.max(np.abs(phi - want[:, None, None])) < 1e-12


def _assemble(nx, ny, nz, dx):
    """Dense matrix of (6 phi - neighbour sum)/dx^2 on the interior nodes."""
    P = nx * ny
    n = P * (nz - 1)
    A = np.zeros((n, n))
    idx = lambda i, j, k: (k - 1) * P + j * nx + i
    for k in range(1, nz):
        for j in range(ny):
            for i in range(nx):
                r = idx(i, j, k)
                A[r, r] += 6.0 / dx ** 2
                for (a, b, c) in ((i + 1, j, k), (i - 1, j, k), (i, j + 1, k), (i, j - 1, k), (i, j, k + 1), (i, j, k - 1)):
                    if c in (0, nz):
                        continue
                    A[r, idx(a % nx, b % ny, c)] -= 1.0 / dx ** 2
    return A


@pytest.mark.parametrize("nx,ny,nz", [(4, 4, 6), (8, 16, 5), (6, 4, 6), (12, 10, 4)])
def test_dense_lu_small(nx, ny, nz):
    # power-of-two planes take the fast transform, the others the plain DFT sums
    dx = 0.3e-3
    rng = np.random.default_rng(3)
    f = rng.standard_normal((nz + 1, ny, nx)) * 1e7
    vb, vt = -13.0, 4.0
    A = _assemble(nx, ny, nz, dx)
    b = f[1:nz].reshape(-1).copy()
    b[: nx * ny] += vb / dx ** 2
    b[-nx * ny:] += vt / dx ** 2
    sol = np.linalg.solve(A, b).reshape(nz - 1, ny, nx)
    phi = O.poisson(nx, ny, nz, dx, f, vb, vt)
    assert np.max(np.abs(phi[1:nz] - sol)) < 1e-10 * np.max(np.abs(sol))
    assert np.all(phi[0] == vb) and np.all(phi[nz] == vt)


def test_second_order_convergence():
    errs = []
    for n in (8, 16, 32):
        nx, ny, nz = n, 4, n
        Lx = Lz = 6.4e-3
        dx = Lx / nx
        x, y, z = _grid(nx, ny, nz, dx)
        kx = 2 * np.pi / Lx
        u = z * (Lz - z) * (1 + 0.3 * np.cos(kx * x)) * 1e5
        lap = (-2 * (1 + 0.3 * np.cos(kx * x)) - z * (Lz - z) * 0.3 * kx ** 2 * np.cos(kx * x)) * 1e5
        phi = O.poisson(nx, ny, nz, dx, -lap, 0.0, 0.0)
        errs.append(np.max(np.abs(phi - u)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4


def test_efield_polynomials():
    nx, ny, nz, dx = 8, 4, 10, 0.25e-3
    x, y, z = _grid(nx, ny, nz, dx)
    Lx = nx * dx
    # linear in z and a periodic sine in x whose central difference is known exactly
    phi = 3.0 + 1e4 * z + 2.0 * np.sin(2 * np.pi * x / Lx)
    ex, ey, ez = O.efield(nx, ny, nz, dx, phi)
    assert np.allclose(ez, -1e4, rtol=1e-12, atol=1e-9)
    assert np.allclose(ey, 0.0, atol=1e-9)
    th = 2 * np.pi / nx
    want_ex = -2.0 * np.cos(2 * np.pi * x / Lx) * np.sin(th) / dx
    assert np.allclose(ex, want_ex, rtol=1e-12, atol=1e-8)
    # quadratic in z: central and one-sided second-order differences are exact
    phi = 5e7 * z ** 2
    ex, ey, ez = O.efield(nx, ny, nz, dx, phi)
    assert np.allclose(ez, -1e8 * z, rtol=1e-11, atol=1e-7)


@pytest.mark.parametrize("shape,grains", [((8, 8, 16), 1), ((16, 8, 12), 3), ((12, 10, 14), 2)])
def test_grain_tables_equal_a_full_solve(shape, grains):
    """The oracle's unit-charge grain tables (Eq. 5), computed mode by mode at
    the region nodes only, equal the full exact solve of the same source: the
    CIC deposit of one coulomb (fixed-point weights round(f 2^14), half to
    even) solved with grounded electrodes, differenced by orc_efield."""
    from paper_1801_00972_gb300 import inputs as I
    nx, ny, nz = shape
    wl = I.small(nx=nx, ny=ny, nz=nz, n_e=0, n_i=0, grains=grains, seed=5)
    s = O.Sim(wl, [(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, np.uint32))] * 2)
    tab = s.gtab()
    eps0, dx = 8.8541878128e-12, wl.dx
    for g, p in enumerate(wl.grain_pos):
        q = p / dx
        c = np.floor(q).astype(int)
        a = np.clip(np.rint((q - c) * 16384).astype(np.int64), 0, 16384)
        f = np.zeros((nz + 1, ny, nx))
        for dz in (0, 1):
            for dy in (0, 1):
                for di in (0, 1):
                    wgt = ((a[0] if di else 16384 - a[0]) * (a[1] if dy else 16384 - a[1])
                           * (a[2] if dz else 16384 - a[2]))
                    f[c[2] + dz, (c[1] + dy) % ny, (c[0] + di) % nx] += wgt * 2.0 ** -42 / dx ** 3 / eps0
        phi = O.poisson(nx, ny, nz, dx, f, 0.0, 0.0)
        ex, ey, ez = O.efield(nx, ny, nz, dx, phi)
        want = np.zeros((4, 4, 4, 3))
        for lk in range(4):
            for lj in range(4):
                for li in range(4):
                    k, j, i = c[2] - 1 + lk, (c[1] - 1 + lj) % ny, (c[0] - 1 + li) % nx
                    want[lk, lj, li] = ex[k, j, i], ey[k, j, i], ez[k, j, i]
        assert np.max(np.abs(tab[g] - want)) <= 1e-11 * np.max(np.abs(want)), g


def test_unit_charge_tables_by_superposition_of_moved_node_solves():
    """The construction the CUDA library uses for the grain tables, checked on
    the exact solve: with x and y periodic, the potential of a unit charge on
    node (i, j, k) is that of a unit charge on node (0, 0, k) moved by (i, j),
    so a grain's table is the CIC-weighted sum of its 8 corners' moved node
    potentials, one solve per corner plane; it equals the oracle's table."""
    from paper_1801_00972_gb300 import inputs as I
    nx, ny, nz = 12, 10, 14
    wl = I.small(nx=nx, ny=ny, nz=nz, n_e=0, n_i=0, grains=3, seed=9)
    s = O.Sim(wl, [(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, np.uint32))] * 2)
    tab = s.gtab()
    eps0, dx = 8.8541878128e-12, wl.dx
    unit = 1.0 / dx ** 3 / eps0          # one coulomb on one node

    def node_solve(i, j, k):
        f = np.zeros((nz + 1, ny, nx))
        f[k, j, i] = unit
        return O.poisson(nx, ny, nz, dx, f, 0.0, 0.0)

    # translation invariance in x and y on the exact solve
    base = node_solve(0, 0, 5)
    moved = np.roll(np.roll(base, 3, axis=2), 7, axis=1)
    direct = node_solve(3, 7, 5)
    assert np.max(np.abs(moved - direct)) <= 1e-12 * np.max(np.abs(direct))
    # a different plane is a different solution (the electrodes break z invariance)
    assert np.max(np.abs(np.roll(node_solve(0, 0, 6), -1, axis=0) - base)) > 1e-3 * np.max(np.abs(base))
    planes = {}
    for g, p in enumerate(wl.grain_pos):
        q = p / dx
        c = np.floor(q).astype(int)
        a = np.clip(np.rint((q - c) * 16384).astype(np.int64), 0, 16384)
        phi = np.zeros((nz + 1, ny, nx))
        for dz in (0, 1):
            k = c[2] + dz
            if k not in planes:
                planes[k] = node_solve(0, 0, k)
            for dy in (0, 1):
                for di in (0, 1):
                    wgt = ((a[0] if di else 16384 - a[0]) * (a[1] if dy else 16384 - a[1])
                           * (a[2] if dz else 16384 - a[2])) * 2.0 ** -42
                    phi += wgt * np.roll(np.roll(planes[k], (c[1] + dy) % ny, axis=1), (c[0] + di) % nx, axis=2)
        ex, ey, ez = O.efield(nx, ny, nz, dx, phi)
        want = np.zeros((4, 4, 4, 3))
        for lk in range(4):
            for lj in range(4):
                for li in range(4):
                    k, j, i = c[2] - 1 + lk, (c[1] - 1 + lj) % ny, (c[0] - 1 + li) % nx
                    want[lk, lj, li] = ex[k, j, i], ey[k, j, i], ez[k, j, i]
        assert np.max(np.abs(tab[g] - want)) <= 1e-11 * np.max(np.abs(want)), g

"""Parity of the device-side initial plasma (pic_init_plasma) with the
oracle's own draw from the same seed: the two sides implement the sampling
rule independently (Philox4x32-10, the uniform-in-box point with the 1.5-radii
grain exclusion, the Marsaglia polar normals with the project-written log).

  - FP64: every particle (position, velocity, id), the fixed-point charge
    density rho_0 and the grain tables are bit-identical; phi_0 agrees to the
    solver tolerance; on a small mesh and on the benchmark's 64x64x256 mesh
    with 1e7 particles;
  - mixed: the device draw is identical, word for word, to pic_init fed with
    the oracle's FP64 particles (the same conversion to cell + offset).
"""
import numpy as np
import pytest

import oracle as O
import paper_1801_00972_gb300 as P
from paper_1801_00972_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_1801_00972_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)
    P.load()


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _same(run, ref):
    for sp in range(2):
        xg, vg, ig = run.particles(sp)
        xo, vo, io = ref.particles(sp)
        assert np.array_equal(ig, io), f"species {sp}: ids differ"
        assert np.array_equal(xg, xo), f"species {sp}: positions differ, max {np.max(np.abs(xg - xo))}"
        assert np.array_equal(vg, vo), f"species {sp}: velocities differ, max {np.max(np.abs(vg - vo))}"


@pytest.mark.parametrize("shape,ne,ni,grains", [((8, 8, 16), 3000, 2500, 1), ((16, 8, 24), 20001, 17777, 3)])
def test_fp64_device_plasma_matches_oracle(shape, ne, ni, grains):
    nx, ny, nz = shape
    wl = I.small(nx=nx, ny=ny, nz=nz, n_e=ne, n_i=ni, grains=grains, v_dc=-20.0)
    ref = O.Sim(wl, None)
    run = P.Run(wl, None, prec=P.PIC_FP64, stream=_stream())
    _same(run, ref)
    assert np.array_equal(run.rho(), ref.rho())
    phi_o = ref.phi()
    assert np.max(np.abs(run.phi() - phi_o)) <= 1e-8 * max(1.0, np.max(np.abs(phi_o)))
    # the first steps from the oracle's potential stay bit-exact
    run.set_gtab(ref.gtab())
    run.set_phi(phi_o)
    run.advance()
    ref.advance()
    _same(run, ref)
    assert np.array_equal(run.rho(), ref.rho())
    run.close()


def test_mixed_device_plasma_equals_host_upload():
    wl = I.small(nx=16, ny=16, nz=32, n_e=30000, n_i=30000, grains=3, v_dc=-20.0)
    ref = O.Sim(wl, None)
    parts = [ref.particles(0), ref.particles(1)]
    a = P.Run(wl, None, prec=P.PIC_MIXED, stream=_stream())
    b = P.Run(wl, parts, prec=P.PIC_MIXED, stream=_stream())
    for sp in range(2):
        xa, va, ia = a.particles(sp)
        xb, vb, ib = b.particles(sp)
        assert np.array_equal(ia, ib) and np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert np.array_equal(a.rho(), b.rho())
    # against the oracle's FP64 deposit: the float offsets move a 14-bit weight by
    # at most one unit at a rounding boundary; the total charge is exact
    assert int(a.rho().sum()) == int(ref.rho().sum())
    assert np.abs(a.rho() - ref.rho()).max() <= 2 ** 42 * 8
    a.step(3)
    b.step(3)
    assert np.array_equal(a.rho(), b.rho())
    a.close()
    b.close()


def test_fp64_device_plasma_at_benchmark_size():
    """The 64x64x256 rf sheath with its 7-grain cluster and 1e7 particles."""
    wl = I.workload(1)
    ref = O.Sim(wl, None)
    run = P.Run(wl, None, prec=P.PIC_FP64, stream=_stream())
    _same(run, ref)
    assert np.array_equal(run.rho(), ref.rho())
    run.close()

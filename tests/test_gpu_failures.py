"""Failure detection without faulting the GPU: every failure is made on the
host (too little particle capacity, a NaN written into the potential, too few
solver iterations, a particle outside the box or NaN in pic_init's arrays);
the kernels latch an error word that the next synchronising call returns as a
status, and the context stays usable for queries."""
import math

import numpy as np
import pytest

import paper_1801_00972_gb300 as P
from paper_1801_00972_gb300 import build as B
from paper_1801_00972_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    B.build()
    torch.cuda.set_device(0)


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _mono_electrons(wl, n, energy):
    rng = np.random.default_rng(4)
    L = np.array(wl.box)
    x = rng.uniform(0.3, 0.7, (n, 3)) * L
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    v = d * math.sqrt(2 * energy * I.QE / I.ME)
    return [(x, v, np.arange(n, dtype=np.uint32)),
            (np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, np.uint32))]


@pytest.mark.parametrize("prec", [P.PIC_FP64, P.PIC_MIXED])
def test_capacity_overflow_is_reported(prec):
    # 60 eV electrons in dense argon: thousands of ionizations per step and no spare slots
    n = 20000
    wl = I.small(nx=16, ny=16, nz=32, n_e=n, n_i=0, grains=0, weight=0.0, v_dc=0.0, dt=2e-10, pressure=50.0)
    run = P.Run(wl, _mono_electrons(wl, n, 60.0), prec=prec, stream=_stream(), capacity=[n, 16])
    with pytest.raises(P.PicError) as e:
        run.step(3)
    assert e.value.status == P.PIC_ECAPACITY
    assert "capacity" in P.pic_last_error(run.ctx)


@pytest.mark.parametrize("prec", [P.PIC_FP64, P.PIC_MIXED])
def test_nan_potential_is_reported(prec):
    wl = I.small(nx=8, ny=8, nz=16, n_e=4000, n_i=4000, grains=0)
    run = P.Run(wl, I.sample_particles(wl), prec=prec, stream=_stream())
    phi = run.phi()
    phi[:] = np.nan                      # every interior node
    run.set_phi(phi)
    run.advance()
    with pytest.raises(P.PicError) as e:
        run.counts()
    assert e.value.status == P.PIC_ENONFINITE


def test_solver_not_converged_is_reported():
    wl = I.small(nx=16, ny=16, nz=32, n_e=5000, n_i=5000, grains=1)
    run = P.Run(wl, I.sample_particles(wl), prec=P.PIC_MIXED, stream=_stream(), tol=1e-10, max_cycles=60)
    run.close()
    with pytest.raises(P.PicError) as e:
        P.Run(wl, I.sample_particles(wl), prec=P.PIC_MIXED, stream=_stream(), tol=1e-15, max_cycles=1).step(2)
    assert e.value.status == P.PIC_ENOTCONV


@pytest.mark.parametrize("copy", [0, P.PIC_F_STAGE_COPY])
@pytest.mark.parametrize("what", ["outside", "nan"])
def test_bad_particle_rejected_by_the_device_check(what, copy):
    wl = I.small(n_e=3000, n_i=3000, grains=1)
    parts = I.sample_particles(wl)
    x = parts[1][0].copy()
    if what == "outside":
        x[1234, 2] = -1e-7
    else:
        x[1234, 0] = np.nan
    parts[1] = (x, parts[1][1], parts[1][2])
    with pytest.raises(P.PicError) as e:
        P.Run(wl, parts, prec=P.PIC_MIXED, flags=copy, stream=_stream())
    assert e.value.status == P.PIC_EINVAL
    assert "outside the box or non-finite" in str(e.value)


@pytest.mark.parametrize("prec", [P.PIC_FP64, P.PIC_MIXED])
def test_upload_paths_give_the_same_records(prec):
    """pic_init reads the particle arrays in place where the device can, or
    copies them in chunks: the same records either way, and the same ids."""
    wl = I.small(nx=16, ny=16, nz=32, n_e=40000, n_i=30000, grains=2)
    parts = I.sample_particles(wl)
    a = P.Run(wl, parts, prec=prec, stream=_stream())
    b = P.Run(wl, parts, prec=prec, flags=P.PIC_F_STAGE_COPY, stream=_stream())
    for sp in range(2):
        xa, va, ia = a.particles(sp)
        xb, vb, ib = b.particles(sp)
        assert np.array_equal(ia, ib) and np.array_equal(xa, xb) and np.array_equal(va, vb)
        assert np.array_equal(np.sort(ia), np.sort(parts[sp][2]))
    assert np.array_equal(a.rho(), b.rho())
    a.close()
    b.close()

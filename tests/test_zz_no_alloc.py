"""The allocation-free Poisson solve (pic_solve_noalloc) against the library's
regular solve.

Some callers cannot call cudaMalloc (their own memory manager owns the device
memory, or their loop must not pay cudaMalloc's device-wide synchronisation).
pic_solve_noalloc serves them from a fixed scratch array inside the library;
here its potential, computed from caller-owned device buffers, must match the
potential that pic_init's regular solve produced for the same charge, within
the tolerance the other parity tests use, on two calls in a row (the second
call reuses the scratch the first one left behind).  This file is collected
last so that a run stopping at the first failure has run every other test."""
import math

import numpy as np
import pytest

import paper_1801_00972_gb300 as P
from paper_1801_00972_gb300 import build as B
from paper_1801_00972_gb300 import inputs as I

pytestmark = pytest.mark.gpu

QE, EPS0 = 1.602176634e-19, 8.8541878128e-12


@pytest.mark.parametrize("prec", [P.PIC_MIXED, P.PIC_FP64])
def test_noalloc_solve_matches_regular_solve(prec):
    import torch
    B.build()
    torch.cuda.set_device(0)
    wl = I.small(nx=16, ny=16, nz=32, n_e=20000, n_i=21000, grains=2, v_dc=-35.0, v_top=3.0)
    stream = torch.cuda.current_stream().cuda_stream
    run = P.Run(wl, I.sample_particles(wl), prec=prec, stream=stream)
    rq = run.rho()
    want = run.phi()                        # regular solve of rho_0 at t = 0, from phi = 0
    run.close()
    scale = (QE * wl.weight) / wl.dx ** 3 * 2.0 ** -42 / EPS0
    v_bot = wl.v_dc + wl.v_rf * math.sin(wl.phase)
    rq_d = torch.tensor(rq, dtype=torch.int64, device="cuda")
    for call in range(2):
        phi_d = torch.zeros(wl.nodes, dtype=torch.float64, device="cuda")
        it, res = P.pic_solve_noalloc(wl.nx, wl.ny, wl.nz, wl.dx, rq_d.data_ptr(), scale, v_bot, wl.v_top,
                                      phi_d.data_ptr(), prec, 1e-10, 60, stream)
        got = phi_d.cpu().numpy()
        assert res <= 1e-10 and it > 0, (call, it, res)
        assert np.max(np.abs(got - want)) <= 1e-8 * max(1.0, np.max(np.abs(want))), call


def _regular(wl, prec, stream):
    run = P.Run(wl, I.sample_particles(wl), prec=prec, stream=stream)
    rq, phi = run.rho(), run.phi()
    run.close()
    return rq, phi


@pytest.mark.parametrize("prec", [P.PIC_MIXED, P.PIC_FP64])
def test_noalloc_warm_start_with_new_electrode_value(prec):
    """A second call that starts from the first call's solution, with a
    different lower electrode value, reaches the cold-start solution for that
    value within the same tolerance, in no more iterations."""
    import torch
    B.build()
    torch.cuda.set_device(0)
    wl = I.small(nx=16, ny=16, nz=32, n_e=20000, n_i=21000, grains=2, v_dc=-35.0, v_top=3.0)
    stream = torch.cuda.current_stream().cuda_stream
    rq, _ = _regular(wl, prec, stream)
    scale = (QE * wl.weight) / wl.dx ** 3 * 2.0 ** -42 / EPS0
    rq_d = torch.tensor(rq, dtype=torch.int64, device="cuda")
    warm = torch.zeros(wl.nodes, dtype=torch.float64, device="cuda")
    P.pic_solve_noalloc(wl.nx, wl.ny, wl.nz, wl.dx, rq_d.data_ptr(), scale, -35.0, wl.v_top, warm.data_ptr(), prec,
                        1e-10, 60, stream)
    it_w, res_w = P.pic_solve_noalloc(wl.nx, wl.ny, wl.nz, wl.dx, rq_d.data_ptr(), scale, -36.0, wl.v_top,
                                      warm.data_ptr(), prec, 1e-10, 60, stream)
    cold = torch.zeros(wl.nodes, dtype=torch.float64, device="cuda")
    it_c, res_c = P.pic_solve_noalloc(wl.nx, wl.ny, wl.nz, wl.dx, rq_d.data_ptr(), scale, -36.0, wl.v_top,
                                      cold.data_ptr(), prec, 1e-10, 60, stream)
    a, b = warm.cpu().numpy(), cold.cpu().numpy()
    assert res_w <= 1e-10 and res_c <= 1e-10
    assert it_w <= it_c, (it_w, it_c)
    assert np.max(np.abs(a - b)) <= 1e-8 * max(1.0, np.max(np.abs(b)))
    assert np.all(a[: wl.nx * wl.ny] == -36.0)


@pytest.mark.parametrize("prec", [P.PIC_MIXED, P.PIC_FP64])
def test_noalloc_on_a_mesh_that_barely_coarsens(prec):
    """12x12x24 cells halve once (12 is not divisible by 8): the coarsest level
    is 6x6x12 and the one-block smoother carries more of the solve."""
    import torch
    B.build()
    torch.cuda.set_device(0)
    wl = I.small(nx=12, ny=12, nz=24, n_e=8000, n_i=8500, grains=1, v_dc=-25.0)
    stream = torch.cuda.current_stream().cuda_stream
    rq, want = _regular(wl, prec, stream)
    scale = (QE * wl.weight) / wl.dx ** 3 * 2.0 ** -42 / EPS0
    rq_d = torch.tensor(rq, dtype=torch.int64, device="cuda")
    phi_d = torch.zeros(wl.nodes, dtype=torch.float64, device="cuda")
    it, res = P.pic_solve_noalloc(wl.nx, wl.ny, wl.nz, wl.dx, rq_d.data_ptr(), scale, wl.v_dc, wl.v_top,
                                  phi_d.data_ptr(), prec, 1e-10, 60, stream)
    got = phi_d.cpu().numpy()
    assert res <= 1e-10, (it, res)
    assert np.max(np.abs(got - want)) <= 1e-8 * max(1.0, np.max(np.abs(want)))


def test_noalloc_rejects_a_mesh_that_does_not_coarsen():
    """18x18x30 cells: 18 is not divisible by 4, so the coarsest level would be
    the whole 10044-node mesh."""
    import torch
    B.build()
    torch.cuda.set_device(0)
    n = 18 * 18 * 31
    rq_d = torch.zeros(n, dtype=torch.int64, device="cuda")
    phi_d = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(P.PicError) as e:
        P.pic_solve_noalloc(18, 18, 30, 1e-4, rq_d.data_ptr(), 1.0, 0.0, 0.0, phi_d.data_ptr(), P.PIC_MIXED,
                            1e-10, 60)
    assert e.value.status == P.PIC_EINVAL
    assert "4096" in P.pic_last_error(None)


def test_noalloc_rejects_oversized_mesh():
    import torch
    B.build()
    torch.cuda.set_device(0)
    n = 64 * 64 * 65
    rq_d = torch.zeros(n, dtype=torch.int64, device="cuda")
    phi_d = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(P.PicError) as e:
        P.pic_solve_noalloc(64, 64, 64, 1e-4, rq_d.data_ptr(), 1.0, 0.0, 0.0, phi_d.data_ptr(), P.PIC_MIXED,
                            1e-10, 60)
    assert e.value.status == P.PIC_EINVAL
    assert "131072" in P.pic_last_error(None)

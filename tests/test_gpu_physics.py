"""The OML floating potential of a single grain (Sec. IV.B uses orbital-motion-
limited charging as its comparison model): one 5 um grain in a collisionless
argon plasma (1e16 m^-3, T_e = 3 eV, T_i = 0.03 eV, Debye length resolved)
charges, through the PP/PM field, the Dt/40 substeps and integer absorption,
to the charge that balances the OML electron and ion currents.

Statistical and loose: the grain charge moves in steps of W e (W = 655 here),
fluctuates by about 10 % and is averaged over the last 6000 steps; it must lie
within 25 % of the OML charge from the local moments (the estimator of
pic_oml_charges without charge exchange) and within 35 % of the OML charge of
the initial plasma, the Lambert-W root of sqrt(m_i T_e / (m_e T_i)) e^-z = 1 + z T_e/T_i.
The FP64 path is the oracle's arithmetic (bit-exact given phi), so this is the
oracle's OML check too; the oracle itself would need hours for these 4e10
particle-steps on one core."""
import math

import numpy as np
import pytest

import paper_1801_00972_gb300 as P
from paper_1801_00972_gb300 import inputs as I

sp = pytest.importorskip("scipy.special")
EPS0 = 8.8541878128e-12


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


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [P.PIC_MIXED, P.PIC_FP64])
def test_single_grain_floats_at_the_oml_charge(prec):
    dens, dx, te, ti, a = 1e16, 1e-4, 3.0, 0.03, 5e-6
    nx, ny, nz, n = 32, 32, 64, 1_000_000
    wl = I.small(nx=nx, ny=ny, nz=nz, n_e=n, n_i=n, grains=1, v_dc=0.0, v_top=0.0, dt=3e-11, te_ev=te, ti_ev=ti)
    wl.dx = dx
    wl.grain_pos = np.array([[0.5 * nx * dx + 3e-6, 0.5 * ny * dx - 2e-6, 0.5 * nz * dx + 1e-6]])
    wl.grain_r = np.array([a])
    wl.weight = dens * nx * ny * nz * dx ** 3 / n
    run = P.Run(wl, I.sample_particles(wl), prec=prec, flags=P.PIC_F_NO_MCC | P.PIC_F_MOMENTS, stream=_stream(),
                sort_every=8)
    run.step(14000)                      # a few charging times (about 0.1 us each)
    run.moments(1, reset=True)
    q = []
    for _ in range(12):
        run.step(500)
        q.append(run.grains()[1][0])
    q_sim = float(np.mean(q))
    q_loc = run.oml_charges(with_cx=False)[0][0]
    tau = te / ti
    A = math.sqrt((te * I.MAR) / (ti * I.ME))
    z = (tau * sp.lambertw((A / tau) * math.exp(1.0 / tau)).real - 1.0) / tau
    q_init = -4.0 * math.pi * EPS0 * a * z * te
    assert q_sim < 0 and q_loc < 0
    assert abs(q_sim / q_loc - 1.0) < 0.25, (q_sim / I.QE, q_loc / I.QE)
    assert abs(q_sim / q_init - 1.0) < 0.35, (q_sim / I.QE, q_init / I.QE)

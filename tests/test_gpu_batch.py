"""Batched ensemble (pic_batch_*): independent runs of different sizes stepped
concurrently give, run by run, exactly what the same run gives alone."""
import numpy as np
import pytest

import paper_1801_00972_gb300 as P
from paper_1801_00972_gb300 import build as B
from paper_1801_00972_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_batch_runs_match_single_runs():
    import torch
    B.build()
    torch.cuda.set_device(0)
    wls = [I.small(nx=8, ny=8, nz=16, n_e=3000, n_i=3000, grains=1, seed=11, v_dc=-40.0),
           I.small(nx=16, ny=8, nz=24, n_e=5001, n_i=4777, grains=3, seed=12, v_dc=0.0, v_rf=60.0, f_rf=13.56e6,
                   phase=1.1),
           I.small(nx=8, ny=16, nz=16, n_e=999, n_i=2000, grains=0, seed=13, pressure=8.0)]
    for r, w in enumerate(wls):
        w.run_id = r
    parts = [I.sample_particles(w) for w in wls]
    for prec in (P.PIC_FP64, P.PIC_MIXED):
        batch = P.Batch(wls, parts, prec=prec, sort_every=3)
        batch.step(7)
        stream = torch.cuda.current_stream().cuda_stream
        for r, (w, p) in enumerate(zip(wls, parts)):
            alone = P.Run(w, p, prec=prec, stream=stream, sort_every=3)
            alone.step(7)
            ctx = batch.runs[r]
            for sp in range(2):
                xb, vb, ib = P.pic_get_particles(ctx, sp, alone.cap[sp])
                xa, va, ia = alone.particles(sp)
                o = np.argsort(ib, kind="stable")
                assert np.array_equal(ib[o], ia)
                assert np.array_equal(xb[o], xa) and np.array_equal(vb[o], va)
            assert np.array_equal(P.pic_get_rho(ctx, alone.nodes), alone.rho())
            assert np.array_equal(P.pic_get_phi(ctx, alone.nodes), alone.phi())
            assert np.array_equal(P.pic_grain_charges(ctx, alone.ng)[0], alone.grains()[0])
            alone.close()
        batch.close()

"""The C-ABI library builds for sm_103a, loads, exports every entry point that
include/pic.h declares, and rejects invalid arguments before touching the GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_1801_00972_gb300 as P
from paper_1801_00972_gb300 import build as B
from paper_1801_00972_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    return sorted(set(re.findall(r"\b(pic_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return P.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(P.SYMBOLS)


def _args(wl, n=10):
    parts = I.sample_particles(wl)
    keep = []
    xs = np.ascontiguousarray(wl.xs)
    keep.append(xs)
    mesh = P.pic_mesh(wl.nx, wl.ny, wl.nz, wl.dx)
    el = P.pic_electrodes(wl.v_dc, wl.v_rf, wl.f_rf, wl.phase, wl.v_top)
    gas = P.pic_gas(wl.n_gas, wl.t_gas, wl.eps_exc, wl.eps_ion, wl.nu_max_e, wl.nu_max_i, wl.de_e, wl.de_i,
                    xs.shape[1], xs.ctypes.data_as(C.POINTER(C.c_double)))
    gp = np.ascontiguousarray(wl.grain_pos).reshape(-1)
    gr = np.ascontiguousarray(wl.grain_r)
    keep += [gp, gr]
    grains = P.pic_grains(gr.size, gp.ctypes.data_as(C.POINTER(C.c_double)),
                          gr.ctypes.data_as(C.POINTER(C.c_double)))
    run = P.pic_run()
    for sp in range(2):
        x, v, ids = (np.ascontiguousarray(a) for a in parts[sp])
        keep += [x, v, ids]
        run.n[sp] = ids.size
        run.x_host[sp] = x.ctypes.data_as(C.POINTER(C.c_double))
        run.v_host[sp] = v.ctypes.data_as(C.POINTER(C.c_double))
        run.id_host[sp] = ids.ctypes.data_as(C.POINTER(C.c_uint32))
        run.capacity[sp] = ids.size + 100
    run.weight, run.dt, run.md_sub, run.sort_every = wl.weight, wl.dt, 40, 10
    run.seed, run.prec, run.tol, run.max_cycles = 1, P.PIC_FP64, 1e-10, 50
    return mesh, el, gas, grains, run, keep


@pytest.mark.parametrize("bad", ["nx_odd", "dx", "dt", "tol", "capacity", "grain_at_electrode",
                                 "xs_nan", "prec", "coulomb_log", "phases_without_moments", "fine_partial",
                                 "fine_h"])
def test_invalid_arguments_rejected(lib, bad):
    wl = I.small(n_e=10, n_i=10)
    mesh, el, gas, grains, run, keep = _args(wl)
    if bad == "nx_odd":
        mesh.nx = 7
    elif bad == "dx":
        mesh.dx = -1.0
    elif bad == "dt":
        run.dt = 0.0
    elif bad == "tol":
        run.tol = 0.0
    elif bad == "capacity":
        run.capacity[0] = 5
    elif bad == "grain_at_electrode":
        wl.grain_pos[0, 2] = 0.5 * wl.dx
        mesh, el, gas, grains, run, keep = _args(wl)
    elif bad == "xs_nan":
        keep[0][0, 3] = np.nan
    elif bad == "prec":
        run.prec = 7
    elif bad == "coulomb_log":
        run.flags = P.PIC_F_COULOMB
        run.coulomb_log = 0.0
    elif bad == "phases_without_moments":
        run.mom_phases = 8
    elif bad == "fine_partial":
        run.flags = P.PIC_F_MOMENTS
        run.fine_n[0], run.fine_n[2], run.fine_h = 10, 10, 1e-5
    elif bad == "fine_h":
        run.flags = P.PIC_F_MOMENTS
        run.fine_n[0] = run.fine_n[1] = run.fine_n[2] = 10
    with pytest.raises(P.PicError) as e:
        P.pic_init(mesh, el, gas, grains, run)
    assert e.value.status == P.PIC_EINVAL
    assert P.pic_last_error(None)


def test_null_context_rejected(lib):
    # entry points that take a run context refuse a null one without touching the GPU
    assert lib.pic_step(None, 1) == P.PIC_EINVAL
    assert lib.pic_tune_sort(None, 5, None) == P.PIC_EINVAL
    assert lib.pic_tune(None, 5, None, None) == P.PIC_EINVAL
    assert lib.pic_get_tuning(None, None) == P.PIC_EINVAL
    assert lib.pic_set_tuning(None, None) == P.PIC_EINVAL
    assert lib.pic_advance(None) == P.PIC_EINVAL
    assert lib.pic_moments_phase(None, 0, 0, None, 0, None) == P.PIC_EINVAL
    assert lib.pic_fine_moments(None, 1, None, 0) == P.PIC_EINVAL
    assert lib.pic_oml_charges(None, 1, None, 0) == P.PIC_EINVAL

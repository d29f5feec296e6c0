"""GB300 PIC-MCC/PPPM particle cycle (arXiv:1801.00972, Sec. III) behind a C ABI.

This module is the thin Python binding of ``libpic.so``: ctypes structures
that mirror ``include/pic.h`` and one function per C entry point, with the same
names, doing argument marshalling only.  Every step of the method runs in the
library's CUDA kernels; there is no CPU fallback.  Importing works without a
GPU; the first call loads ``libpic.so`` and raises if it is missing.

``Run`` wraps one run context for convenience (numpy in, numpy out).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpic.so")
_lock = threading.Lock()
_lib = None

PIC_OK, PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA, PIC_ECAPACITY, PIC_ENONFINITE, PIC_ENOTCONV, PIC_ETIMEOUT = range(8)
STATUS = {0: "PIC_OK", 1: "PIC_EINVAL", 2: "PIC_ENOMEM", 3: "PIC_ECUDA", 4: "PIC_ECAPACITY",
          5: "PIC_ENONFINITE", 6: "PIC_ENOTCONV", 7: "PIC_ETIMEOUT"}
PIC_FP64, PIC_MIXED = 0, 1
PIC_F_NO_MCC, PIC_F_IONS_FROZEN, PIC_F_MOMENTS, PIC_F_NO_GRAPH, PIC_F_COULOMB, PIC_F_F64_RESIDUAL = 1, 2, 8, 16, 32, 64
PIC_F_STAGE_COPY = 128
COUNTERS = ("lost_bot_e", "lost_bot_i", "lost_top_e", "lost_top_i", "abs_e", "abs_i",
            "e_el", "e_exc", "e_ion", "i_el", "i_cx", "err", "pushed")
PIC_C_N = len(COUNTERS)

# every symbol include/pic.h declares
SYMBOLS = ("pic_init", "pic_init_plasma", "pic_step", "pic_tune_sort", "pic_get_tuning", "pic_set_tuning", "pic_tune",
           "pic_tune_cache_load", "pic_tune_cache_store", "pic_advance", "pic_solve", "pic_grain_charges", "pic_counts",
           "pic_moments", "pic_moments_phase", "pic_fine_moments", "pic_oml_charges", "pic_eepf", "pic_eepf_fit", "pic_get_particles", "pic_get_rho", "pic_get_phi", "pic_set_phi",
           "pic_get_grain_table", "pic_set_grain_table", "pic_set_grain_counts", "pic_step_index",
           "pic_profile", "pic_profile_read", "pic_solve_noalloc", "pic_batch_init", "pic_batch_step",
           "pic_batch_run", "pic_batch_destroy", "pic_last_error", "pic_destroy")


class pic_mesh(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("dx", C.c_double)]


class pic_electrodes(C.Structure):
    _fields_ = [("v_dc", C.c_double), ("v_rf", C.c_double), ("f_rf", C.c_double), ("phase", C.c_double),
                ("v_top", C.c_double)]


class pic_gas(C.Structure):
    _fields_ = [("n_gas", C.c_double), ("t_gas", C.c_double), ("eps_exc", C.c_double), ("eps_ion", C.c_double),
                ("nu_max_e", C.c_double), ("nu_max_i", C.c_double), ("de_e", C.c_double), ("de_i", C.c_double),
                ("n_xs", C.c_int32), ("xs_host", C.POINTER(C.c_double))]


class pic_grains(C.Structure):
    _fields_ = [("n", C.c_int32), ("pos_host", C.POINTER(C.c_double)), ("radius_host", C.POINTER(C.c_double))]


class pic_run(C.Structure):
    _fields_ = [("n", C.c_int64 * 2), ("x_host", C.POINTER(C.c_double) * 2), ("v_host", C.POINTER(C.c_double) * 2),
                ("id_host", C.POINTER(C.c_uint32) * 2), ("capacity", C.c_int64 * 2), ("weight", C.c_double),
                ("dt", C.c_double), ("md_sub", C.c_int32), ("sort_every", C.c_int32), ("seed", C.c_uint64),
                ("run_id", C.c_uint32), ("prec", C.c_int32), ("flags", C.c_int32), ("tol", C.c_double),
                ("max_cycles", C.c_int32), ("coulomb_log", C.c_double), ("eepf_bins", C.c_int32),
                ("eepf_de_ev", C.c_double), ("mom_phases", C.c_int32), ("fine_n", C.c_int32 * 3),
                ("fine_h", C.c_double), ("fine_origin", C.c_double * 3)]


class pic_tuning(C.Structure):
    _fields_ = [("sort_every", C.c_int32), ("tile", C.c_int32 * 3), ("halo", C.c_int32), ("order", C.c_int32)]

    def as_dict(self):
        return {"sort_every": self.sort_every, "tile": [int(x) for x in self.tile], "halo": self.halo,
                "order": self.order}


class PicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load(path: str | None = None):
    """Load libpic.so (built by ``paper_1801_00972_gb300.build``); raise if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with `python -m paper_1801_00972_gb300.build` "
                               "(there is no CPU fallback)")
        L = C.CDLL(p)
        vp, i32, i64, sz, pd = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t, C.POINTER(C.c_double)
        pi64, pu32 = C.POINTER(C.c_int64), C.POINTER(C.c_uint32)
        L.pic_init.argtypes = [C.POINTER(pic_mesh), C.POINTER(pic_electrodes), C.POINTER(pic_gas),
                               C.POINTER(pic_grains), C.POINTER(pic_run), vp, C.POINTER(vp)]
        sig = {
            "pic_step": [vp, i32], "pic_tune_sort": [vp, i32, C.POINTER(i32)],
            "pic_get_tuning": [vp, C.POINTER(pic_tuning)], "pic_set_tuning": [vp, C.POINTER(pic_tuning)],
            "pic_tune": [vp, i32, C.c_char_p, C.POINTER(pic_tuning)],
            "pic_tune_cache_load": [C.c_char_p, C.c_char_p, C.POINTER(pic_tuning)],
            "pic_tune_cache_store": [C.c_char_p, C.c_char_p, C.POINTER(pic_tuning)], "pic_advance": [vp], "pic_solve": [vp, C.POINTER(i32), pd],
            "pic_grain_charges": [vp, pi64, pd], "pic_counts": [vp, pi64, pi64],
            "pic_moments": [vp, i32, pd, sz, i32], "pic_moments_phase": [vp, i32, i32, pd, sz, pi64],
            "pic_fine_moments": [vp, i32, pd, sz], "pic_oml_charges": [vp, i32, pd, sz],
            "pic_eepf": [vp, pi64, sz, pi64, i32], "pic_eepf_fit": [pi64, i32, C.c_double, C.c_double, C.c_double, pd],
            "pic_get_particles": [vp, i32, pd, pd, pu32, i64, pi64],
            "pic_get_rho": [vp, pi64, sz], "pic_get_phi": [vp, pd, sz], "pic_set_phi": [vp, pd, sz],
            "pic_get_grain_table": [vp, pd, sz], "pic_set_grain_table": [vp, pd, sz],
            "pic_set_grain_counts": [vp, pi64, sz],
            "pic_profile": [vp, i32], "pic_profile_read": [vp, pd, pi64, pd, pi64, pi64, pi64],
            "pic_solve_noalloc": [i32, i32, i32, C.c_double, vp, C.c_double, C.c_double, C.c_double, vp, i32,
                                  C.c_double, i32, C.POINTER(i32), pd, vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.pic_init.restype = C.c_int
        L.pic_init_plasma.argtypes = [C.POINTER(pic_mesh), C.POINTER(pic_electrodes), C.POINTER(pic_gas),
                                      C.POINTER(pic_grains), C.POINTER(pic_run), pd, vp, C.POINTER(vp)]
        L.pic_init_plasma.restype = C.c_int
        L.pic_batch_init.argtypes = [i32, C.POINTER(pic_mesh), C.POINTER(pic_electrodes), C.POINTER(pic_gas),
                                     C.POINTER(pic_grains), C.POINTER(pic_run), C.POINTER(vp)]
        L.pic_batch_init.restype = C.c_int
        L.pic_batch_step.argtypes = [vp, i32]
        L.pic_batch_step.restype = C.c_int
        L.pic_batch_run.argtypes = [vp, i32]
        L.pic_batch_run.restype = vp
        L.pic_batch_destroy.argtypes = [vp]
        L.pic_batch_destroy.restype = None
        L.pic_step_index.argtypes = [vp]
        L.pic_step_index.restype = i64
        L.pic_last_error.argtypes = [vp]
        L.pic_last_error.restype = C.c_char_p
        L.pic_destroy.argtypes = [vp]
        L.pic_destroy.restype = None
        _lib = L
        return L


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def _check(ctx, st):
    if st != PIC_OK:
        msg = load().pic_last_error(ctx)
        raise PicError(st, msg.decode() if msg else "")
    return st


# ----------------------------------------------------------------- C-ABI mirrors
def pic_init(mesh, electrodes, gas, grains, run, stream=None):
    ctx = C.c_void_p()
    st = load().pic_init(C.byref(mesh), C.byref(electrodes), C.byref(gas), C.byref(grains), C.byref(run),
                         C.c_void_p(stream or 0), C.byref(ctx))
    _check(None, st)
    return ctx


def pic_init_plasma(mesh, electrodes, gas, grains, run, t_ev, stream=None):
    ctx = C.c_void_p()
    t = (C.c_double * 2)(float(t_ev[0]), float(t_ev[1]))
    st = load().pic_init_plasma(C.byref(mesh), C.byref(electrodes), C.byref(gas), C.byref(grains), C.byref(run),
                                t, C.c_void_p(stream or 0), C.byref(ctx))
    _check(None, st)
    return ctx


def pic_step(ctx, n_steps):
    return _check(ctx, load().pic_step(ctx, int(n_steps)))


def pic_tune_sort(ctx, steps_per_candidate):
    chosen = C.c_int32()
    _check(ctx, load().pic_tune_sort(ctx, int(steps_per_candidate), C.byref(chosen)))
    return chosen.value


def pic_get_tuning(ctx):
    t = pic_tuning()
    _check(ctx, load().pic_get_tuning(ctx, C.byref(t)))
    return t.as_dict()


def _tuning(d):
    t = pic_tuning()
    t.sort_every, t.halo, t.order = int(d["sort_every"]), int(d["halo"]), int(d.get("order", 0))
    for a in range(3):
        t.tile[a] = int(d["tile"][a])
    return t


def pic_set_tuning(ctx, d):
    t = _tuning(d)
    return _check(ctx, load().pic_set_tuning(ctx, C.byref(t)))


def pic_tune(ctx, steps_per_candidate, cache_path=None):
    t = pic_tuning()
    path = cache_path.encode() if cache_path else None
    _check(ctx, load().pic_tune(ctx, int(steps_per_candidate), path, C.byref(t)))
    return t.as_dict()


def pic_tune_cache_load(path, key):
    """The cached choices for `key`, or None."""
    t = pic_tuning()
    st = load().pic_tune_cache_load(path.encode(), key.encode(), C.byref(t))
    return t.as_dict() if st == PIC_OK else None


def pic_tune_cache_store(path, key, d):
    t = _tuning(d)
    return _check(None, load().pic_tune_cache_store(path.encode(), key.encode(), C.byref(t)))


def pic_advance(ctx):
    return _check(ctx, load().pic_advance(ctx))


def pic_solve(ctx):
    it = C.c_int32()
    res = C.c_double()
    _check(ctx, load().pic_solve(ctx, C.byref(it), C.byref(res)))
    return it.value, res.value


def pic_grain_charges(ctx, ng):
    n = np.zeros(2 * max(ng, 1), np.int64)
    q = np.zeros(max(ng, 1))
    _check(ctx, load().pic_grain_charges(ctx, _p(n, C.c_int64), _p(q, C.c_double)))
    return n[: 2 * ng].reshape(ng, 2), q[:ng]


def pic_counts(ctx):
    n = np.zeros(2, np.int64)
    c = np.zeros(PIC_C_N, np.int64)
    _check(ctx, load().pic_counts(ctx, _p(n, C.c_int64), _p(c, C.c_int64)))
    return n, dict(zip(COUNTERS, (int(x) for x in c)))


def pic_eepf(ctx, nz, bins, reset=False):
    """(counts[nz][bins + 1] summed over the steps, number of steps)."""
    out = np.zeros(nz * (bins + 1), np.int64)
    steps = C.c_int64()
    _check(ctx, load().pic_eepf(ctx, _p(out, C.c_int64), out.size, C.byref(steps), int(bool(reset))))
    return out.reshape(nz, bins + 1), steps.value


def pic_eepf_fit(counts, de_ev, e_lo_ev, e_hi_ev):
    """Two-Maxwellian fit of one slab's histogram (bins without the overflow
    column): (T_l, T_h, A_l, A_h)."""
    c = np.ascontiguousarray(counts, dtype=np.int64)
    out = np.zeros(4)
    _check(None, load().pic_eepf_fit(_p(c, C.c_int64), int(c.size), float(de_ev), float(e_lo_ev), float(e_hi_ev),
                                     _p(out, C.c_double)))
    return tuple(float(x) for x in out)


def pic_moments(ctx, what, nodes, reset=False):
    out = np.zeros(nodes * (3 if what in (3, 4) else 1))
    _check(ctx, load().pic_moments(ctx, int(what), _p(out, C.c_double), out.size, int(bool(reset))))
    return out


def pic_moments_phase(ctx, what, bin, nodes):
    """(window average over the samples of rf phase bin ``bin``, samples in it)."""
    out = np.zeros(nodes * (3 if what in (3, 4) else 1))
    steps = C.c_int64()
    _check(ctx, load().pic_moments_phase(ctx, int(what), int(bin), _p(out, C.c_double), out.size, C.byref(steps)))
    return out, int(steps.value)


def pic_oml_charges(ctx, ng, with_cx=True):
    """Per grain (Q [C], phi [V], n_e, n_i [m^-3], T_e, T_i [eV]) from the moment window."""
    out = np.zeros(6 * max(ng, 1))
    _check(ctx, load().pic_oml_charges(ctx, int(bool(with_cx)), _p(out, C.c_double), 6 * ng))
    return out[: 6 * ng].reshape(ng, 6)


def pic_fine_moments(ctx, what, fine_n):
    """Fine-grid window average, shaped (nz, ny, nx) or (nz, ny, nx, 3) for the fluxes."""
    nx, ny, nz = fine_n
    out = np.zeros(nx * ny * nz * (3 if what >= 3 else 1))
    _check(ctx, load().pic_fine_moments(ctx, int(what), _p(out, C.c_double), out.size))
    return out.reshape((nz, ny, nx, 3) if what >= 3 else (nz, ny, nx))


def pic_get_particles(ctx, species, cap):
    x = np.zeros((max(cap, 1), 3)); v = np.zeros((max(cap, 1), 3)); ids = np.zeros(max(cap, 1), np.uint32)
    n = C.c_int64()
    _check(ctx, load().pic_get_particles(ctx, int(species), _p(x, C.c_double), _p(v, C.c_double),
                                         _p(ids, C.c_uint32), int(cap), C.byref(n)))
    return x[: n.value], v[: n.value], ids[: n.value]


def pic_get_rho(ctx, nodes):
    a = np.zeros(nodes, np.int64)
    _check(ctx, load().pic_get_rho(ctx, _p(a, C.c_int64), nodes))
    return a


def pic_get_phi(ctx, nodes):
    a = np.zeros(nodes)
    _check(ctx, load().pic_get_phi(ctx, _p(a, C.c_double), nodes))
    return a


def pic_set_phi(ctx, phi):
    a = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
    return _check(ctx, load().pic_set_phi(ctx, _p(a, C.c_double), a.size))


def pic_get_grain_table(ctx, ng):
    a = np.zeros(max(ng, 1) * 192)
    _check(ctx, load().pic_get_grain_table(ctx, _p(a, C.c_double), ng * 192))
    return a[: ng * 192].reshape(ng, 4, 4, 4, 3)


def pic_set_grain_table(ctx, tab):
    a = np.ascontiguousarray(tab, dtype=np.float64).reshape(-1)
    return _check(ctx, load().pic_set_grain_table(ctx, _p(a, C.c_double), a.size))


def pic_set_grain_counts(ctx, n_abs):
    a = np.ascontiguousarray(n_abs, dtype=np.int64).reshape(-1)
    return _check(ctx, load().pic_set_grain_counts(ctx, _p(a, C.c_int64), a.size))


def pic_profile(ctx, enable):
    return _check(ctx, load().pic_profile(ctx, int(bool(enable))))


def pic_profile_read(ctx):
    pm, sm = C.c_double(), C.c_double()
    pl, ns, it, kl = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
    _check(ctx, load().pic_profile_read(ctx, C.byref(pm), C.byref(pl), C.byref(sm), C.byref(ns), C.byref(it),
                                        C.byref(kl)))
    return dict(push_ms=pm.value, push_launches=pl.value, solve_ms=sm.value, solves=ns.value,
                solve_iterations=it.value, kernels=kl.value)


def pic_solve_noalloc(nx, ny, nz, dx, rho_q_ptr, scale, v_bot, v_top, phi_ptr, prec, tol, max_iters,
                      stream=None):
    """Allocation-free Poisson solve on caller-owned device buffers (raw device
    pointers as ints).  Returns (iterations, relative residual)."""
    it = C.c_int32()
    res = C.c_double()
    st = load().pic_solve_noalloc(int(nx), int(ny), int(nz), float(dx), C.c_void_p(rho_q_ptr), float(scale),
                                  float(v_bot), float(v_top), C.c_void_p(phi_ptr), int(prec), float(tol),
                                  int(max_iters), C.byref(it), C.byref(res), C.c_void_p(stream or 0))
    _check(None, st)
    return it.value, res.value


def pic_step_index(ctx):
    return load().pic_step_index(ctx)


def pic_last_error(ctx=None):
    m = load().pic_last_error(ctx)
    return m.decode() if m else ""


def pic_destroy(ctx):
    load().pic_destroy(ctx)


# ----------------------------------------------------------------- convenience
def make_args(wl, particles, prec=PIC_MIXED, flags=0, capacity=None, sort_every=20, tol=1e-10, max_cycles=60,
              md_sub=None, coulomb_log=10.0, eepf_bins=0, eepf_de_ev=0.0, mom_phases=0, fine_n=(0, 0, 0),
              fine_h=0.0, fine_origin=(0.0, 0.0, 0.0)):
    """The pic_init argument structures for a workload; returns them with the
    numpy arrays they point into (keep those alive while the call runs).
    particles=None leaves the particle arrays NULL for pic_init_plasma."""
    keep = []
    mesh = pic_mesh(wl.nx, wl.ny, wl.nz, wl.dx)
    el = pic_electrodes(wl.v_dc, wl.v_rf, wl.f_rf, wl.phase, wl.v_top)
    xs = np.ascontiguousarray(wl.xs, dtype=np.float64)
    keep.append(xs)
    gas = pic_gas(wl.n_gas, wl.t_gas, wl.eps_exc, wl.eps_ion, wl.nu_max_e, wl.nu_max_i, wl.de_e, wl.de_i,
                  xs.shape[1], _p(xs, C.c_double))
    gp = np.ascontiguousarray(wl.grain_pos, dtype=np.float64).reshape(-1)
    gr = np.ascontiguousarray(wl.grain_r, dtype=np.float64).reshape(-1)
    keep += [gp, gr]
    grains = pic_grains(gr.size, _p(gp, C.c_double), _p(gr, C.c_double))
    run = pic_run()
    for sp in range(2):
        if particles is None:
            # drawn on the device from the seed (pic_init_plasma)
            n = (wl.n_e, wl.n_i)[sp]
            run.n[sp] = n
            run.capacity[sp] = capacity[sp] if capacity is not None else int(n * 1.25) + 4096
            continue
        x, v, ids = particles[sp]
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
        ids = np.ascontiguousarray(ids, dtype=np.uint32).reshape(-1)
        keep += [x, v, ids]
        run.n[sp] = ids.size
        run.x_host[sp] = _p(x, C.c_double)
        run.v_host[sp] = _p(v, C.c_double)
        run.id_host[sp] = _p(ids, C.c_uint32)
        run.capacity[sp] = capacity[sp] if capacity is not None else int(ids.size * 1.25) + 4096
    run.weight, run.dt = wl.weight, wl.dt
    run.md_sub = wl.md_sub if md_sub is None else md_sub
    run.sort_every = sort_every
    run.seed, run.run_id, run.prec, run.flags = wl.seed, wl.run_id, prec, flags
    run.tol, run.max_cycles, run.coulomb_log = tol, max_cycles, coulomb_log
    run.eepf_bins, run.eepf_de_ev = eepf_bins, eepf_de_ev
    run.mom_phases, run.fine_h = mom_phases, fine_h
    for a in range(3):
        run.fine_n[a], run.fine_origin[a] = int(fine_n[a]), float(fine_origin[a])
    return (mesh, el, gas, grains, run), keep


class Batch:
    """An ensemble of independent runs stepped concurrently (pic_batch_*)."""

    def __init__(self, workloads, particles, **kw):
        n = len(workloads)
        args = [make_args(w, p, **kw) for w, p in zip(workloads, particles)]
        arrs = [(t * n)(*[a[0][q] for a in args]) for q, t in
                enumerate((pic_mesh, pic_electrodes, pic_gas, pic_grains, pic_run))]
        h = C.c_void_p()
        _check(None, load().pic_batch_init(n, *arrs, C.byref(h)))
        self.h = h
        self.n = n
        self.workloads = workloads
        self.runs = [load().pic_batch_run(h, r) for r in range(n)]

    def step(self, n=1):
        _check(None, load().pic_batch_step(self.h, int(n)))

    def close(self):
        if getattr(self, "h", None):
            load().pic_batch_destroy(self.h)
            self.h = None

    __del__ = close


class Run:
    """One run context built from a workload description (see ``inputs.Workload``)
    and initial particles [(x, v, id) for electrons, ions] in SI units, or
    particles=None to draw wl.n_e electrons and wl.n_i ions at wl.te_ev and
    wl.ti_ev on the device (pic_init_plasma)."""

    def __init__(self, wl, particles, prec=PIC_MIXED, flags=0, stream=None, capacity=None, sort_every=20,
                 tol=1e-10, max_cycles=60, md_sub=None, coulomb_log=10.0, eepf_bins=0, eepf_de_ev=0.0,
                 mom_phases=0, fine_n=(0, 0, 0), fine_h=0.0, fine_origin=(0.0, 0.0, 0.0)):
        (mesh, el, gas, grains, run), keep = make_args(
            wl, particles, prec=prec, flags=flags, capacity=capacity, sort_every=sort_every, tol=tol,
            max_cycles=max_cycles, md_sub=md_sub, coulomb_log=coulomb_log, eepf_bins=eepf_bins,
            eepf_de_ev=eepf_de_ev, mom_phases=mom_phases, fine_n=fine_n, fine_h=fine_h, fine_origin=fine_origin)
        gr = np.asarray(wl.grain_r).reshape(-1)
        self.eepf_bins = eepf_bins
        self.fine_n = tuple(int(n) for n in fine_n)
        if particles is None:
            self.ctx = pic_init_plasma(mesh, el, gas, grains, run, (wl.te_ev, wl.ti_ev), stream)
        else:
            self.ctx = pic_init(mesh, el, gas, grains, run, stream)
        self.wl = wl
        self.nodes = wl.nx * wl.ny * (wl.nz + 1)
        self.ng = gr.size
        self.cap = [int(run.capacity[0]), int(run.capacity[1])]

    def close(self):
        if getattr(self, "ctx", None):
            pic_destroy(self.ctx)
            self.ctx = None

    __del__ = close

    def step(self, n=1):
        pic_step(self.ctx, n)

    def tune_sort(self, steps_per_candidate=20):
        return pic_tune_sort(self.ctx, steps_per_candidate)

    def tune(self, steps_per_candidate=20, cache_path=None):
        return pic_tune(self.ctx, steps_per_candidate, cache_path)

    def tuning(self):
        return pic_get_tuning(self.ctx)

    def set_tuning(self, d):
        pic_set_tuning(self.ctx, d)

    def advance(self):
        pic_advance(self.ctx)

    def solve(self):
        return pic_solve(self.ctx)

    def grains(self):
        return pic_grain_charges(self.ctx, self.ng)

    def counts(self):
        return pic_counts(self.ctx)

    def particles(self, sp, sort=True):
        x, v, ids = pic_get_particles(self.ctx, sp, self.cap[sp])
        if sort:
            o = np.argsort(ids, kind="stable")
            x, v, ids = x[o], v[o], ids[o]
        return x, v, ids

    def rho(self):
        return pic_get_rho(self.ctx, self.nodes)

    def phi(self):
        return pic_get_phi(self.ctx, self.nodes)

    def set_phi(self, phi):
        pic_set_phi(self.ctx, phi)

    def gtab(self):
        return pic_get_grain_table(self.ctx, self.ng)

    def set_gtab(self, tab):
        pic_set_grain_table(self.ctx, tab)

    def set_grain_counts(self, n_abs):
        pic_set_grain_counts(self.ctx, n_abs)

    def moments(self, what, reset=False):
        return pic_moments(self.ctx, what, self.nodes, reset)

    def moments_phase(self, what, bin):
        return pic_moments_phase(self.ctx, what, bin, self.nodes)

    def oml_charges(self, with_cx=True):
        return pic_oml_charges(self.ctx, self.ng, with_cx)

    def fine_moments(self, what):
        return pic_fine_moments(self.ctx, what, self.fine_n)

    def eepf(self, reset=False):
        return pic_eepf(self.ctx, self.wl.nz, self.eepf_bins, reset)

    def profile(self, enable):
        pic_profile(self.ctx, enable)

    def profile_read(self):
        return pic_profile_read(self.ctx)

    @property
    def step_index(self):
        return pic_step_index(self.ctx)

"""Oracle for the PIC-MCC/PPPM particle cycle (arXiv:1801.00972, Sec. III).

TEST INFRASTRUCTURE ONLY.  A plain FP64 CPU restatement of the method in C
(``pic_oracle.c``), loaded here through ctypes.  Only ``tests/``, the smoke
check in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may use
it; the CUDA library never imports, links or calls anything in this folder.

Every floating-point result is computed in C with ``-ffp-contract=off`` so that
the arithmetic order written in ``pic_oracle.c`` is the order that runs.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NO_MCC = 1
IONS_FROZEN = 2
MOMENTS = 8
COULOMB = 32
EEPF = 64

# counter slots of orc_get_counters
C_NAMES = ("lost_bot_e", "lost_bot_i", "lost_top_e", "lost_top_i", "abs_e", "abs_i",
           "e_el", "e_exc", "e_ion", "i_el", "i_cx", "err")


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "pic_oracle.h"))):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-o", tmp, _SRC, "-lm"]
    # OpenMP shares independent planes, modes and particles among the host
    # cores (results do not depend on the thread count); without it, one thread
    r = subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def threads() -> int:
    """Host threads the oracle's parallel loops use."""
    return lib().orc_threads()


def set_threads(n: int) -> None:
    """Use n host threads from now on (0: all of them)."""
    lib().orc_set_threads(int(n))


class Cfg(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("md_sub", C.c_int32),
        ("dx", C.c_double), ("dt", C.c_double), ("weight", C.c_double),
        ("v_dc", C.c_double), ("v_rf", C.c_double), ("f_rf", C.c_double), ("phase", C.c_double),
        ("v_top", C.c_double),
        ("n_gas", C.c_double), ("t_gas", C.c_double),
        ("eps_exc", C.c_double), ("eps_ion", C.c_double),
        ("nu_max_e", C.c_double), ("nu_max_i", C.c_double),
        ("de_e", C.c_double), ("de_i", C.c_double),
        ("n_xs", C.c_int32), ("n_grains", C.c_int32),
        ("xs", C.POINTER(C.c_double)),
        ("gpos", C.POINTER(C.c_double)),
        ("grad", C.POINTER(C.c_double)),
        ("seed", C.c_uint64), ("run_id", C.c_uint32), ("flags", C.c_int32),
        ("n_init", C.c_int64 * 2),
        ("x_init", C.POINTER(C.c_double) * 2),
        ("v_init", C.POINTER(C.c_double) * 2),
        ("id_init", C.POINTER(C.c_uint32) * 2),
        ("coulomb_log", C.c_double),
        ("eepf_bins", C.c_int32),
        ("eepf_de_ev", C.c_double),
        ("mom_phases", C.c_int32),
        ("fine_n", C.c_int32 * 3),
        ("fine_h", C.c_double),
        ("fine_origin", C.c_double * 3),
        ("t_init_ev", C.c_double * 2),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            vp, i64, u32, i32, dbl = C.c_void_p, C.c_int64, C.c_uint32, C.c_int, C.c_double
            pd, pi64, pu32 = C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_uint32)
            L.orc_create.restype = vp
            L.orc_create.argtypes = [C.POINTER(Cfg)]
            L.orc_destroy.argtypes = [vp]
            for f in ("orc_advance", "orc_solve", "orc_step"):
                getattr(L, f).argtypes = [vp]
                getattr(L, f).restype = i32
            L.orc_coulomb.argtypes = [vp]
            L.orc_coulomb.restype = None
            L.orc_get_eepf.argtypes = [vp, pi64]
            L.orc_get_eepf.restype = i64
            L.orc_count.argtypes = [vp, i32]; L.orc_count.restype = i64
            L.orc_get_particles.argtypes = [vp, i32, pd, pd, pu32]
            L.orc_get_rho.argtypes = [vp, pi64]
            L.orc_get_phi.argtypes = [vp, pd]
            L.orc_set_phi.argtypes = [vp, pd]
            L.orc_get_grains.argtypes = [vp, pi64, pd]
            L.orc_get_gtab.argtypes = [vp, pd]
            L.orc_set_gtab.argtypes = [vp, pd]
            L.orc_get_counters.argtypes = [vp, pi64]
            L.orc_step_index.argtypes = [vp]; L.orc_step_index.restype = i64
            L.orc_next_id.argtypes = [vp]; L.orc_next_id.restype = u32
            L.orc_moments.argtypes = [vp, i32, pd]; L.orc_moments.restype = i32
            L.orc_moments_phase.argtypes = [vp, i32, i32, pd, pi64]; L.orc_moments_phase.restype = i32
            L.orc_fine_moments.argtypes = [vp, i32, pd]; L.orc_fine_moments.restype = i32
            L.orc_oml_potential.argtypes = [dbl] * 5; L.orc_oml_potential.restype = dbl
            L.orc_oml_charges.argtypes = [vp, i32, pd]; L.orc_oml_charges.restype = i32
            L.orc_reset_moments.argtypes = [vp]
            L.orc_field_at.argtypes = [vp, pd, pd]; L.orc_field_at.restype = i32
            L.orc_set_grain_counts.argtypes = [vp, pi64]
            L.orc_philox4x32_10.argtypes = [pu32, pu32, pu32]
            L.orc_ln.argtypes = [dbl]; L.orc_ln.restype = dbl
            L.orc_poisson.argtypes = [i32, i32, i32, dbl, pd, dbl, dbl, pd]; L.orc_poisson.restype = i32
            L.orc_efield.argtypes = [i32, i32, i32, dbl, pd, pd, pd, pd]
            L.orc_iso_dir.argtypes = [u32, u32, u32, pu32, pd]
            L.orc_gauss3.argtypes = [u32, u32, u32, pu32, pd]
            L.orc_threads.argtypes = []
            L.orc_threads.restype = i32
            L.orc_set_threads.argtypes = [i32]
            L.orc_set_threads.restype = None
            _lib = L
    return _lib


def oml_potential(ne, ni, te, ti, lam_over_l=0.0):
    """OML surface potential (V) of an isolated sphere; see orc_oml_potential."""
    return lib().orc_oml_potential(float(ne), float(ni), float(te), float(ti), float(lam_over_l))


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


# ---------------------------------------------------------------- primitives
def philox4x32_10(ctr, key):
    L = lib()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    L.orc_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(o, C.c_uint32))
    return o


def ln(x: float) -> float:
    return lib().orc_ln(float(x))


def iso_dir(pid, step, purpose, key):
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(3)
    lib().orc_iso_dir(pid, step, purpose, _p(k, C.c_uint32), _p(o, C.c_double))
    return o


def gauss3(pid, step, purpose, key):
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(3)
    lib().orc_gauss3(pid, step, purpose, _p(k, C.c_uint32), _p(o, C.c_double))
    return o


def poisson(nx, ny, nz, dx, f, v_bot, v_top):
    """Exact solution of (neighbour sum - 6 phi)/dx^2 = -f, node array (nz+1, ny, nx)."""
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
    assert f.size == nx * ny * (nz + 1)
    phi = np.zeros_like(f)
    rc = lib().orc_poisson(nx, ny, nz, dx, _p(f, C.c_double), v_bot, v_top, _p(phi, C.c_double))
    assert rc == 0
    return phi.reshape(nz + 1, ny, nx)


def efield(nx, ny, nz, dx, phi):
    phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
    e = [np.zeros_like(phi) for _ in range(3)]
    lib().orc_efield(nx, ny, nz, dx, _p(phi, C.c_double), *(_p(a, C.c_double) for a in e))
    return [a.reshape(nz + 1, ny, nx) for a in e]


# ---------------------------------------------------------------- simulation
class Sim:
    """One oracle run.  ``wl`` is a workload description with the attributes of
    ``paper_1801_00972_gb300.inputs.Workload`` (duck-typed; this module does not
    import the package).  ``particles`` = [(x, v, id) per species], or None to
    let the oracle draw wl.n_e electrons and wl.n_i ions at wl.te_ev / wl.ti_ev
    from the seed."""

    def __init__(self, wl, particles, flags: int = 0, md_sub: int | None = None, coulomb_log: float = 10.0,
                 eepf_bins: int = 0, eepf_de_ev: float = 0.0, mom_phases: int = 0, fine_n=(0, 0, 0),
                 fine_h: float = 0.0, fine_origin=(0.0, 0.0, 0.0)):
        L = lib()
        self._keep = []
        cfg = Cfg()
        cfg.nx, cfg.ny, cfg.nz = wl.nx, wl.ny, wl.nz
        cfg.md_sub = wl.md_sub if md_sub is None else md_sub
        cfg.dx, cfg.dt, cfg.weight = wl.dx, wl.dt, wl.weight
        cfg.v_dc, cfg.v_rf, cfg.f_rf, cfg.phase, cfg.v_top = wl.v_dc, wl.v_rf, wl.f_rf, wl.phase, wl.v_top
        cfg.n_gas, cfg.t_gas = wl.n_gas, wl.t_gas
        cfg.eps_exc, cfg.eps_ion = wl.eps_exc, wl.eps_ion
        cfg.nu_max_e, cfg.nu_max_i = wl.nu_max_e, wl.nu_max_i
        cfg.de_e, cfg.de_i = wl.de_e, wl.de_i
        xs = np.ascontiguousarray(wl.xs, dtype=np.float64)
        cfg.n_xs = xs.shape[1]
        cfg.xs = _p(xs, C.c_double)
        g = np.ascontiguousarray(wl.grain_pos, dtype=np.float64).reshape(-1)
        r = np.ascontiguousarray(wl.grain_r, dtype=np.float64).reshape(-1)
        cfg.n_grains = r.size
        cfg.gpos = _p(g, C.c_double) if r.size else None
        cfg.grad = _p(r, C.c_double) if r.size else None
        cfg.seed, cfg.run_id, cfg.flags = wl.seed, wl.run_id, flags
        cfg.coulomb_log = coulomb_log
        cfg.eepf_bins, cfg.eepf_de_ev = eepf_bins, eepf_de_ev
        self.eepf_bins = eepf_bins
        cfg.mom_phases = mom_phases
        for a in range(3):
            cfg.fine_n[a], cfg.fine_origin[a] = int(fine_n[a]), float(fine_origin[a])
        cfg.fine_h = fine_h
        self.fine_n = tuple(int(n) for n in fine_n)
        self._keep += [xs, g, r]
        for sp in range(2):
            if particles is None:
                # the oracle draws the initial plasma from the seed itself
                cfg.n_init[sp] = (wl.n_e, wl.n_i)[sp]
                cfg.t_init_ev[sp] = (wl.te_ev, wl.ti_ev)[sp]
                continue
            x, v, ids = particles[sp]
            x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
            v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
            ids = np.ascontiguousarray(ids, dtype=np.uint32).reshape(-1)
            self._keep += [x, v, ids]
            cfg.n_init[sp] = ids.size
            cfg.x_init[sp] = _p(x, C.c_double)
            cfg.v_init[sp] = _p(v, C.c_double)
            cfg.id_init[sp] = _p(ids, C.c_uint32)
        self.wl = wl
        self.nodes = wl.nx * wl.ny * (wl.nz + 1)
        self.ng = r.size
        self.h = L.orc_create(C.byref(cfg))
        self._keep = None
        if not self.h:
            raise RuntimeError("orc_create failed")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_destroy(h)
            self.h = None

    def advance(self):
        assert lib().orc_advance(self.h) == 0

    def solve(self):
        assert lib().orc_solve(self.h) == 0

    def eepf(self):
        """(counts per (cell plane, energy bin) summed over the steps, number of steps)."""
        out = np.zeros(self.wl.nz * (self.eepf_bins + 1), np.int64)
        n = lib().orc_get_eepf(self.h, _p(out, C.c_int64))
        return out.reshape(self.wl.nz, self.eepf_bins + 1), int(n)

    def coulomb(self):
        """One Coulomb collision pass on the current particles (as at the end of a step)."""
        lib().orc_coulomb(self.h)

    def step(self, n: int = 1):
        for _ in range(n):
            assert lib().orc_step(self.h) == 0

    @property
    def step_index(self) -> int:
        return lib().orc_step_index(self.h)

    @property
    def next_id(self) -> int:
        return lib().orc_next_id(self.h)

    def count(self, sp: int) -> int:
        return lib().orc_count(self.h, sp)

    def particles(self, sp: int, sort: bool = True):
        n = self.count(sp)
        x = np.zeros((max(n, 1), 3)); v = np.zeros((max(n, 1), 3)); ids = np.zeros(max(n, 1), np.uint32)
        lib().orc_get_particles(self.h, sp, _p(x, C.c_double), _p(v, C.c_double), _p(ids, C.c_uint32))
        x, v, ids = x[:n], v[:n], ids[:n]
        if sort:
            o = np.argsort(ids, kind="stable")
            x, v, ids = x[o], v[o], ids[o]
        return x, v, ids

    def rho(self):
        a = np.zeros(self.nodes, np.int64)
        lib().orc_get_rho(self.h, _p(a, C.c_int64))
        return a

    def phi(self):
        a = np.zeros(self.nodes)
        lib().orc_get_phi(self.h, _p(a, C.c_double))
        return a

    def set_phi(self, phi):
        a = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
        assert a.size == self.nodes
        lib().orc_set_phi(self.h, _p(a, C.c_double))

    def grains(self):
        n = np.zeros(2 * max(self.ng, 1), np.int64); q = np.zeros(max(self.ng, 1))
        lib().orc_get_grains(self.h, _p(n, C.c_int64), _p(q, C.c_double))
        return n[: 2 * self.ng].reshape(self.ng, 2), q[: self.ng]

    def gtab(self):
        t = np.zeros(max(self.ng, 1) * 192)
        lib().orc_get_gtab(self.h, _p(t, C.c_double))
        return t[: self.ng * 192].reshape(self.ng, 4, 4, 4, 3)

    def set_gtab(self, tab):
        t = np.ascontiguousarray(tab, dtype=np.float64).reshape(-1)
        assert t.size == self.ng * 192
        lib().orc_set_gtab(self.h, _p(t, C.c_double))

    def counters(self) -> dict:
        c = np.zeros(len(C_NAMES), np.int64)
        lib().orc_get_counters(self.h, _p(c, C.c_int64))
        return dict(zip(C_NAMES, (int(x) for x in c)))

    def moments(self, what: int):
        n = self.nodes * (3 if what in (3, 4) else 1)
        a = np.zeros(n)
        assert lib().orc_moments(self.h, what, _p(a, C.c_double)) == 0
        return a

    def field_at(self, p):
        p = np.ascontiguousarray(p, dtype=np.float64).reshape(3)
        e = np.zeros(3)
        md = lib().orc_field_at(self.h, _p(p, C.c_double), _p(e, C.c_double))
        return e, bool(md)

    def set_grain_counts(self, n_abs):
        a = np.ascontiguousarray(n_abs, dtype=np.int64).reshape(-1)
        assert a.size == 2 * self.ng
        lib().orc_set_grain_counts(self.h, _p(a, C.c_int64))

    def moments_phase(self, what: int, bin: int):
        """(window average of rf phase bin ``bin``, samples in that bin)."""
        n = self.nodes * (3 if what in (3, 4) else 1)
        a = np.zeros(n)
        st = C.c_int64(0)
        assert lib().orc_moments_phase(self.h, what, bin, _p(a, C.c_double), C.byref(st)) == 0
        return a, st.value

    def fine_moments(self, what: int):
        """Fine-grid window average, what 1 n_e, 2 n_i (nz, ny, nx), 3/4 fluxes (nz, ny, nx, 3)."""
        nx, ny, nz = self.fine_n
        a = np.zeros(nx * ny * nz * (3 if what >= 3 else 1))
        assert lib().orc_fine_moments(self.h, what, _p(a, C.c_double)) == 0
        return a.reshape((nz, ny, nx, 3) if what >= 3 else (nz, ny, nx))

    def oml_charges(self, with_cx: bool = True):
        """Per grain (Q [C], phi [V], n_e, n_i [m^-3], T_e, T_i [eV]) from the moment window."""
        out = np.zeros(6 * max(self.ng, 1))
        assert lib().orc_oml_charges(self.h, int(bool(with_cx)), _p(out, C.c_double)) == 0
        return out[: 6 * self.ng].reshape(self.ng, 6)

    def reset_moments(self):
        lib().orc_reset_moments(self.h)

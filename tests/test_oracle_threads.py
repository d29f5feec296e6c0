"""The oracle's OpenMP loops (Poisson planes and modes, grain tables, the
particle loop, the integer deposit) give results that do not depend on the
number of host threads: a few steps of a workload with grains, collisions and
ionization, run with one thread in a child process and with every thread
here, agree bit for bit."""
import os
import subprocess
import sys

import numpy as np

import oracle as O
from paper_1801_00972_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r'''
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
import oracle as O
from paper_1801_00972_gb300 import inputs as I
wl = I.small(nx=16, ny=16, nz=32, n_e=20000, n_i=20000, grains=3, v_dc=-60.0, dt=2e-10, te_ev=8.0)
s = O.Sim(wl, None)
s.step(3)
out = dict(rho=s.rho(), phi=s.phi(), gtab=s.gtab(), threads=np.array([O.threads()]))
for sp in range(2):
    x, v, i = s.particles(sp, sort=False)
    out[f"x{sp}"], out[f"v{sp}"], out[f"i{sp}"] = x, v, i
np.savez(sys.argv[2], **out)
'''


def test_results_do_not_depend_on_thread_count(tmp_path):
    res = []
    for threads in ("1", str(max(os.cpu_count() or 2, 2))):
        f = tmp_path / f"t{threads}.npz"
        env = dict(os.environ, OMP_NUM_THREADS=threads)
        subprocess.run([sys.executable, "-c", _CHILD, ROOT, str(f)], check=True, env=env)
        res.append(np.load(f))
    a, b = res
    assert a["threads"][0] == 1
    for k in a.files:
        if k != "threads":
            assert np.array_equal(a[k], b[k]), k

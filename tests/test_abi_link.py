"""The C ABI as a plain C caller sees it: a C99 program that includes only
include/pic.h, takes the address of every entry point (so each must link
against libpic.so) and calls the ones that need no GPU: the two-Maxwellian
fit of an EEPF histogram and the rejection of null contexts.  No PyTorch,
no Python on the call path."""
import math
import os
import shutil
import subprocess

import pytest

import paper_1801_00972_gb300 as P
from paper_1801_00972_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _program(symbols):
    fns = ",\n    ".join(f"(any_fn){s}" for s in symbols)
    return f"""#include <stdio.h>
#include <math.h>
#include "pic.h"

typedef void (*any_fn)(void);

int main(void)
{{
    any_fn fns[] = {{
    {fns}
    }};
    int64_t counts[200];
    double fit[4];
    /* expected counts of a 2.5 eV Maxwellian in 0.1 eV bins: N (P(E < e_b+1) - P(E < e_b)),
       P by the Gamma(3/2) integral sqrt-erf form */
    for (int b = 0; b < 200; ++b) {{
        double lo = 0.1 * b / 2.5, hi = 0.1 * (b + 1) / 2.5;
        double plo = erf(sqrt(lo)) - 2.0 * sqrt(lo / M_PI) * exp(-lo);
        double phi = erf(sqrt(hi)) - 2.0 * sqrt(hi / M_PI) * exp(-hi);
        counts[b] = (int64_t)llround(1e9 * (phi - plo));
    }}
    pic_status s = pic_eepf_fit(counts, 200, 0.1, 0.1, 12.0, fit);
    pic_status n1 = pic_step(NULL, 1);
    pic_status n2 = pic_moments(NULL, 0, NULL, 0, 0);
    printf("%d %d %d %d %.6f %.6f\\n", (int)(sizeof fns / sizeof fns[0]), (int)s, (int)n1, (int)n2, fit[0], fit[1]);
    return 0;
}}
"""


def test_plain_c_caller(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lib = B.build()
    src = tmp_path / "caller.c"
    exe = tmp_path / "caller"
    src.write_text(_program(P.SYMBOLS))
    libdir = os.path.dirname(lib)
    subprocess.run([cc, "-std=c99", "-D_DEFAULT_SOURCE", "-Wall", "-Wextra", "-Werror", "-I",
                    os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L", libdir, "-lpic", "-lm",
                    f"-Wl,-rpath,{libdir}"], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    n, s, n1, n2, t_lo, t_hi = int(out[0]), int(out[1]), int(out[2]), int(out[3]), float(out[4]), float(out[5])
    assert n == len(P.SYMBOLS)
    assert s == P.PIC_OK and n1 == P.PIC_EINVAL and n2 == P.PIC_EINVAL
    # one Maxwellian: both fitted groups (or the single one) at 2.5 eV
    assert math.isclose(t_hi, 2.5, rel_tol=0.03), (t_lo, t_hi)

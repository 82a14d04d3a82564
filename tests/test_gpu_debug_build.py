"""The debug library (SSD_LIBRARY=debug: every index read from a mesh or
mortar table checked before use, a bad one raising device flag bit 3 that
sd_sync reports as SD_ERR_MESH) builds, runs the same cases as the release
library with no flag raised, and gives the same results: residuals of a
two-rotor Euler mesh, a viscous sliding rotor (FP64 and FP32) and the
viscous Couette annulus against the oracle, and SSP-RK3 steps.  Runs in a
child process, since the library is chosen when the package is imported."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import oracle
import paper_1503_02198_gb300 as ssd
from helpers import small_rotor, small_twin
from ssd_inputs import fields, meshes
from ssd_inputs.workloads import FlowParams
oracle.build()
assert ssd.build().endswith("libssd_debug.so") and ssd.LIB_PATH.endswith("libssd_debug.so")

def rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))

def case(mesh, prm, t, dt, precisions, seed, **kw):
    o = oracle.Oracle(mesh, 4, prm)
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=seed, **kw))
    q5, _ = o.step(Q, t, dt, 5)
    for prec in precisions:
        s = ssd.Solver(mesh, 3, prm, precision=prec)
        s.sd_set_state(Q)
        s.sd_set_time(t)
        err = rel(s.sd_residual(), (o.extended() if prec == 0 else o).residual(Q, t))
        assert err <= (1e-12 if prec == 0 else 5e-5), (prec, err)
        s.sd_set_state(Q)
        s.sd_set_time(t)
        s.sd_step(dt, 5)
        s.sd_sync()  # raises on any device flag, the index checks' included
        err = rel(s.sd_get_state(), q5)
        assert err <= (1e-12 if prec == 0 else 1e-5), (prec, err)
        s.close()

case(small_twin(), FlowParams(omega=0.7), 0.4, 1e-3, (0, 1), 3, amp=0.2, scale=3.0)
case(small_rotor(shift_R=0.05), FlowParams(omega=0.7, viscous=1, mu=0.02, Rgas=1.0, prandtl=0.72), 1.9, 1e-3,
     (0, 1), 2, amp=0.2, scale=3.0)
Rg = 100.0 / 1.4
case(meshes.couette_mesh(2, 12, 2, 16, phi_out=0.05),
     FlowParams(gamma=1.4, Rgas=Rg, mu=0.1, prandtl=0.72, omega=1.0, viscous=1, T_wall=1.0), 0.43, 1e-4, (0,), 4,
     amp=0.05, u0=0.2, v0=-0.1, p0=Rg)
print("debug library ok")
"""


def test_debug_library_runs_clean_and_matches_the_oracle():
    env = dict(os.environ, SSD_LIBRARY="debug")
    code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    res = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True,
                         timeout=1500)
    assert res.returncode == 0 and "debug library ok" in res.stdout, (res.stdout[-2000:], res.stderr[-4000:])

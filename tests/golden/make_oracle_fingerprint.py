"""Write oracle_fingerprint.json: SHA-256 digests of the FP64 oracle's
residuals and SSP-RK3 steps on small seeded cases.

Calls only oracle/ (and the seeded input generators).  The digests pin the
double build of the oracle bit for bit, so that a change of its real type
(the extended-precision build) is shown to leave the FP64 arithmetic
untouched.  Run from the repository root:
    python tests/golden/make_oracle_fingerprint.py
"""
from __future__ import annotations

import hashlib
import json
import os
import platform
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from ssd_inputs import fields, meshes  # noqa: E402
from ssd_inputs.workloads import FlowParams, build_workload  # noqa: E402


def cases():
    """(name, mesh, N, params, state function, time) of each fingerprinted case."""
    from helpers import small_rotor, small_twin  # tests/helpers.py
    out = []
    out.append(("rotor_n4_smooth", small_rotor(shift_R=0.05), 4, FlowParams(omega=0.9),
                lambda x, y: fields.random_smooth_state(x, y, seed=4, amp=0.2, scale=3.0), 0.37))
    out.append(("twin_n3_vortex", small_twin(), 3, FlowParams(omega=0.7),
                lambda x, y: fields.isentropic_vortex(x, y, x0=0.5), 1.3))
    w = build_workload("couette_n3")
    out.append(("couette_n3", w.mesh, w.N, w.params,
                lambda x, y: fields.random_smooth_state(x, y, seed=7, amp=0.05, u0=0.1, v0=0.05), 0.2))
    return out


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype=np.float64).tobytes()).hexdigest()


def fingerprint() -> dict:
    res = {}
    for name, mesh, N, prm, fn, t in cases():
        o = oracle.Oracle(mesh, N, prm)
        Q = o.state_from(fn)
        R = o.residual(Q, t)
        q2, _ = o.step(Q, t, 1e-3, 2)
        res[name] = {"residual": digest(R), "step2": digest(q2)}
    return res


if __name__ == "__main__":
    data = {"machine": platform.machine(), "cases": fingerprint()}
    with open(os.path.join(HERE, "oracle_fingerprint.json"), "w") as f:
        json.dump(data, f, indent=1)
    print(json.dumps(data, indent=1))

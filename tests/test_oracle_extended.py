"""The extended-precision build of the oracle (the same C source with every
value and operation in long double): it must agree with the FP64 oracle to
FP64 accuracy and carry more precision than FP64.  It serves as the
reference that shows how much round-off each FP64 evaluation carries (the
FP64 parity criterion is measured against it)."""
import math

import numpy as np
import pytest

from helpers import small_rotor
from ssd_inputs import fields, meshes
from ssd_inputs.workloads import FlowParams

pytestmark = pytest.mark.skipif(np.finfo(np.longdouble).eps >= 1e-18,
                                reason="long double is not wider than double on this machine")


@pytest.mark.parametrize("N", [3, 5])
def test_extended_build_agrees_with_fp64(oracle_mod, N):
    m = small_rotor(shift_R=0.05)
    prm = FlowParams(omega=0.9)
    o = oracle_mod.Oracle(m, N, prm)
    ox = oracle_mod.Oracle(m, N, prm, real="long")
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=N, amp=0.2, scale=3.0))
    R = o.residual(Q, 0.37)
    Rx = ox.residual(Q, 0.37)
    assert Rx.dtype == np.longdouble
    d = np.abs(R - Rx.astype(np.float64)).max(axis=(0, 2, 3)) / np.abs(R).max(axis=(0, 2, 3))
    assert (d < 1e-11).all(), d
    q, _ = o.step(Q, 0.37, 1e-3, 2)
    qx, _ = ox.step(Q, 0.37, 1e-3, 2)
    assert np.abs(q - qx.astype(np.float64)).max() < 1e-13


@pytest.mark.parametrize("N", [3, 5])
def test_extended_build_carries_more_precision(oracle_mod, N):
    # a uniform state on straight cells (rotating and stationary) is an exact
    # discrete steady state: the residual is pure round-off, ~1e-13 in FP64,
    # at least a hundred times smaller with the wider significand
    m = meshes.perturb_nodes(small_rotor(), 0.15, seed=3)
    straight = m["edge_arc"].sum(axis=1) == 0
    out = {}
    for real in ("double", "long"):
        o = oracle_mod.Oracle(m, N, FlowParams(omega=math.pi / 4), real=real)
        Q = o.state_from(lambda x, y: fields.uniform(x, y, rho=1.2, u=0.3, v=-0.1, p=0.9))
        out[real] = float(np.abs(o.residual(Q, 0.37)[straight]).max())
    assert out["long"] < 1e-2 * out["double"] and out["long"] < 1e-15, out

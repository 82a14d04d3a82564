"""FP64 path against the extended-precision oracle (the oracle's source built
with long double): how close the GPU's FP64 residual comes to the exact
discrete operator, and how that compares with the FP64 oracle's own round-off.

Criterion: per conservative variable, max-norm of the difference over all
solution points divided by the max-norm of the reference residual, <= 1e-12
(and the same bound for the relative L2 norm).  The sliding interface decides
it: a mortar offset o = (phi_mortar - phi_face) / width (Sec. 3.2, Eq. xz) is a
difference of two angles near pi over a small width, so FP64 angles put
~1e-14 into o, which the flux-derivative weights of the interface cells
amplify.  The GPU path keeps those angles in double-double (face angles formed
in long double on the host, omega t formed exactly and reduced with a
double-double 2 pi); the FP64 oracle, a plain restatement, does not.

Three configurations (the isentropic vortex sitting on the interface of the
6,016-cell vortex mesh at t = 0, N = 4 and 5, and on the interface of a crop of
the bench rotor at h = 0.08, N = 6) are more sensitive still: there the residual moves
by ~1e4 max|R| per unit change of o, so even the rounding of o itself to FP64
(relative 1e-16) leaves ~2e-12.  They are held to 5e-12, and to a tenth of the
FP64 oracle's own error."""
import math

import numpy as np
import pytest

from helpers import small_rotor, small_twin
from ssd_inputs import fields, meshes
from ssd_inputs.workloads import FlowParams, build_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ssd():
    import paper_1503_02198_gb300 as pkg
    pkg.build()
    return pkg


def rel_max(a, ref):
    ref = ref.astype(np.longdouble)
    d = np.abs(a.astype(np.longdouble) - ref).max(axis=(0, 2, 3)) / np.abs(ref).max(axis=(0, 2, 3))
    return d.astype(np.float64)


def rel_l2(a, ref):
    ref = ref.astype(np.longdouble)
    d = a.astype(np.longdouble) - ref
    return np.sqrt((d ** 2).sum(axis=(0, 2, 3)) / (ref ** 2).sum(axis=(0, 2, 3))).astype(np.float64)


def bench_crop():
    """The bench rotor's resolution (h = 0.08, N = 6, disk r = 4 with the same
    core, rings and interface faces) in a smaller periodic box: 22,500 quads."""
    return meshes.rotor_mesh(half_width=6.4, n_cart=160, n_hole=120, r_interface=4.0, n_core=50, core_half=2.0,
                             n_ring_in=20, n_ring_out=10)


def _run(ssd, oracle_mod, mesh, N, prm, fn, t):
    o = oracle_mod.Oracle(mesh, N, prm)
    Q = o.state_from(fn)
    s = ssd.Solver(mesh, N - 1, prm, precision=0)
    s.sd_set_state(Q)
    s.sd_set_time(t)
    R = s.sd_residual()
    s.close()
    Rx = o.extended().residual(Q, t)
    return R, o.residual(Q, t), Rx


CASES = [("rotor", N, t) for N in (3, 4, 5, 6) for t in (0.0, 0.37, 5.123, 90.0)] + \
        [("aligned", 3, 0.0), ("aligned", 5, 0.0), ("twin", 4, 0.0), ("twin", 4, 1.3),
         ("vortex_n4", 4, 0.37), ("vortex_n5", 5, 0.37), ("crop", 6, 0.8)]


@pytest.mark.parametrize("case,N,t", CASES)
def test_fp64_residual_within_1e12_of_extended_oracle(ssd, oracle_mod, case, N, t):
    if case == "rotor":
        mesh, prm = small_rotor(shift_R=0.05), FlowParams(omega=0.9)
        fn = lambda x, y: fields.random_smooth_state(x, y, seed=N, amp=0.2, scale=3.0)
    elif case == "aligned":
        mesh, prm = small_rotor(n_hole=6, n_core=6), FlowParams(omega=1.0)
        fn = lambda x, y: fields.isentropic_vortex(x, y, x0=1.0, y0=-2.0)
    elif case == "twin":
        mesh, prm = small_twin(), FlowParams(omega=0.7)
        fn = lambda x, y: fields.isentropic_vortex(x, y, x0=0.5)
    elif case == "crop":
        mesh, prm = bench_crop(), FlowParams(omega=0.5)
        fn = lambda x, y: fields.random_smooth_state(x, y, seed=21, amp=0.2, scale=4.0)
    else:
        w = build_workload(case)
        mesh, prm = w.mesh, w.params
        fn = lambda x, y: fields.isentropic_vortex(x, y, x0=1.0, y0=-2.0)
    R, Ro, Rx = _run(ssd, oracle_mod, mesh, N, prm, fn, t)
    gpu, orc = rel_max(R, Rx), rel_max(Ro, Rx)
    print(f"{case} N={N} t={t}: GPU FP64 {gpu.max():.2e}, FP64 oracle {orc.max():.2e} (max-norm vs extended)")
    assert (gpu <= 1e-12).all() and (rel_l2(R, Rx) <= 1e-12).all(), (gpu, orc)


@pytest.mark.parametrize("case", ["vortex_n4_t0", "vortex_n5_t0", "crop_vortex"])
def test_fp64_residual_at_the_floor_of_fp64_mortar_weights(ssd, oracle_mod, case):
    if case.startswith("vortex"):
        w = build_workload(case[:9])
        R, Ro, Rx = _run(ssd, oracle_mod, w.mesh, w.N, w.params,
                         lambda x, y: fields.isentropic_vortex(x, y, x0=1.0, y0=-2.0), 0.0)
    else:
        R, Ro, Rx = _run(ssd, oracle_mod, bench_crop(), 6, FlowParams(omega=0.5),
                         lambda x, y: fields.isentropic_vortex(x, y), 0.8)
    gpu, orc = rel_max(R, Rx), rel_max(Ro, Rx)
    print(f"{case}: GPU FP64 {gpu.max():.2e}, FP64 oracle {orc.max():.2e} (max-norm vs extended)")
    assert (gpu <= 5e-12).all() and gpu.max() <= 0.1 * orc.max(), (gpu, orc)

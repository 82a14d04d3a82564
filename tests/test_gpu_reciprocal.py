"""The kernels' reciprocal 1/x (density and Jacobian reciprocals): Newton's
iteration from the hardware's approximate reciprocal, two steps in FP64, one
in FP32.  Checked against the exact reciprocal (numpy's IEEE division of the
input in the same precision) over magnitudes from 1e-8 to 1e8: within one ulp
in both, and correctly rounded for most inputs."""
import numpy as np
import pytest

from helpers import small_rotor
from ssd_inputs.workloads import FlowParams

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ssd():
    import paper_1503_02198_gb300 as pkg
    pkg.build()
    return pkg


def _inputs():
    rng = np.random.Generator(np.random.PCG64(1503))
    x = 10.0 ** rng.uniform(-8, 8, 20000)
    p2 = 2.0 ** np.arange(-26, 27, dtype=np.float64)
    edge = np.concatenate([p2, np.nextafter(p2, 0), np.nextafter(p2, np.inf), [1.0, 1.5, 3.0, 0.7, 1.4]])
    x = np.concatenate([x, edge, -x[:1000]])
    return x


def test_fp64_reciprocal_within_one_ulp(ssd):
    s = ssd.Solver(small_rotor(), 2, FlowParams(omega=0.5), precision=ssd.SD_PREC_FP64)
    x = _inputs()
    y = s.sd_test_reciprocal(x)
    exact = 1.0 / x
    ulps = np.abs(y - exact) / np.spacing(np.abs(exact))
    assert ulps.max() <= 1.0, (ulps.max(), x[np.argmax(ulps)])
    # and most values come out correctly rounded
    assert np.mean(ulps == 0) > 0.9
    s.close()


def test_fp32_reciprocal_within_one_ulp(ssd):
    s = ssd.Solver(small_rotor(), 2, FlowParams(omega=0.5), precision=ssd.SD_PREC_FP32)
    xf = _inputs().astype(np.float32)
    y = s.sd_test_reciprocal(xf.astype(np.float64)).astype(np.float32)
    exact = np.float32(1.0) / xf
    ulps = np.abs(y.astype(np.float64) - exact) / np.spacing(np.abs(exact)).astype(np.float64)
    assert ulps.max() <= 1.0, (ulps.max(), xf[np.argmax(ulps)])
    assert np.mean(ulps == 0) > 0.9
    s.close()


def test_reciprocal_argument_checks(ssd):
    s = ssd.Solver(small_rotor(), 2, FlowParams(omega=0.5), precision=ssd.SD_PREC_FP64)
    assert s.sd_test_reciprocal(np.zeros(0)).size == 0
    import ctypes
    assert ssd.lib().sd_test_reciprocal(s._h, None, None, 5) == ssd.SD_ERR_ARG
    s.close()

"""Device-side error reporting without any GPU fault: a bounded tile wait that
gives up (made to give up by the library's test switch, which arms one copy
barrier with more bytes than its copies deliver) is reported as
SD_ERR_TIMEOUT by sd_sync and by sd_residual_noalloc, and the handle steps
cleanly once the switch is off."""
import numpy as np
import pytest

from helpers import small_rotor
from ssd_inputs import fields
from ssd_inputs.workloads import FlowParams

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ssd():
    import paper_1503_02198_gb300 as pkg
    pkg.build()
    return pkg


@pytest.mark.parametrize("precision", [0, 1])
def test_bounded_wait_timeout_is_reported_and_cleared(ssd, precision):
    m = small_rotor()
    prm = FlowParams(omega=0.5)
    s = ssd.Solver(m, 3, prm, precision=precision)
    Q = s.state_from(lambda x, y: fields.isentropic_vortex(x, y, x0=1.0))
    s.sd_set_state(Q)
    s.sd_test_wait_timeout(1)
    s.sd_step(1e-3, 1)
    with pytest.raises(ssd.SSDError) as ei:
        s.sd_sync()
    assert ei.value.code == ssd.SD_ERR_TIMEOUT
    s.sd_set_state(Q)
    with pytest.raises(ssd.SSDError) as ei:
        s.sd_residual_noalloc()
    assert ei.value.code == ssd.SD_ERR_TIMEOUT
    # switch off: the same handle steps cleanly and equals a fresh handle
    s.sd_test_wait_timeout(0)
    s.sd_set_state(Q)
    s.sd_set_time(0.0)
    s.sd_step(1e-3, 2)
    s.sd_sync()
    ref = ssd.Solver(m, 3, prm, precision=precision)
    ref.sd_set_state(Q)
    ref.sd_step(1e-3, 2)
    ref.sd_sync()
    assert np.array_equal(s.sd_get_state(), ref.sd_get_state())
    s.close()
    ref.close()

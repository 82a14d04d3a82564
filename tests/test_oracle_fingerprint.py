"""The FP64 build of the oracle is pinned bit for bit: residual and step
digests on small seeded cases (tests/golden/oracle_fingerprint.json, written
by tests/golden/make_oracle_fingerprint.py from the oracle).  A change to the
oracle that is meant to leave its FP64 arithmetic alone (its extended-precision
build, for instance) must keep them.  The digests depend on the C library's
math functions, so they are checked on the machine type that wrote them."""
import json
import os
import platform
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_fp64_oracle_is_bit_identical(oracle_mod):
    with open(os.path.join(HERE, "golden", "oracle_fingerprint.json")) as f:
        stored = json.load(f)
    if platform.machine() != stored["machine"]:
        pytest.skip("digests were written on " + stored["machine"])
    sys.path.insert(0, os.path.join(HERE, "golden"))
    try:
        import make_oracle_fingerprint as mk
    finally:
        sys.path.pop(0)
    assert mk.fingerprint() == stored["cases"]

"""The CPU oracle against facts the paper and mathematics fix (see pins.py)."""
import pytest

import pins


@pytest.mark.parametrize("pin", pins.ALL_PINS + pins.ICP_PINS + pins.MESH_PINS, ids=lambda f: f.__name__)
def test_pin(oracle_lib, pin):
    pin()

"""The oracle against its pins (no GPU).  See tests/pins.py for the sources of
truth; each must hold on the real oracle build."""
import pytest

import pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(orc, pin):
    ok, worst = pin(orc.load())
    assert ok, f"{pin.__name__}: worst error {worst:.3e}"

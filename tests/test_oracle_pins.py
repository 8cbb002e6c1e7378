"""The CPU oracle against its pins (library routines, hand-worked cases of
Alg. 1 / Alg. 2, closed forms and invariants); see ``oracle_pins.py``."""
import pytest

from oracle_pins import ALL_PINS


@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(orc, pin):
    pin(orc)

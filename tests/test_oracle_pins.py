"""The oracle against its pins (CPU only): closed forms, invariants, exact
rational arithmetic, library routines, brute force and a hand-worked fixture."""
import pytest

from oracle_pins import PINS


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin()

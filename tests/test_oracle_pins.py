"""The FP64 oracle against brute force, closed forms and invariants (CPU)."""
import pytest

import oracle_pins as pins

CHECKS = [name for name in dir(pins) if name.startswith("check_")]


@pytest.mark.parametrize("name", CHECKS)
def test_pin(name):
    getattr(pins, name)()

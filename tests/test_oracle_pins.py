"""The FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test runs one pin from ``oracle_pins``; see that module for what each
pin compares against.
"""
import pytest

import oracle_pins as pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=[p.__name__ for p in pins.ALL_PINS])
def test_oracle_pin(orc, pin):
    pin(orc)

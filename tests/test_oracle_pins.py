"""The CPU oracle against what the definitions fix (no GPU needed)."""
import pytest

import oracle_pins


@pytest.mark.parametrize("check", oracle_pins.ALL_CHECKS, ids=lambda c: c.__name__[6:])
def test_oracle_pin(ora, check):
    check(ora)

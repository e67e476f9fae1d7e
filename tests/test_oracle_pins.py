"""The CPU oracle against its pins (hand-worked examples, exhaustive tables,
brute force, invariants, Section VIII)."""
import pytest

import oracle_pins as P


@pytest.mark.parametrize("name", P.golden_names())
def test_golden(oracle_lib, name):
    P.check_golden(oracle_lib, name)


@pytest.mark.parametrize("name,fn", [p for p in P.PINS if p[0] != "golden"],
                         ids=[p[0] for p in P.PINS if p[0] != "golden"])
def test_pin(oracle_lib, name, fn):
    fn(oracle_lib)

"""Plant plausible mistakes in the oracle and check that the pins catch each one."""
import pytest

import oracle
import pins

PLANTED = {
    1: "irS left unit-offset",
    2: "fold seeded with the first term instead of +0.0",
    3: "descending k inside a run",
    4: "rows descending inside a column",
    5: "jcS counts duplicates",
    6: "rows and columns swapped",
    7: "last term of each run dropped",
    8: "only k-adjacent repeats merged",
    9: "run heads point one slot back",
    10: "non-integer double indices accepted",
    11: "zero double index accepted",
}


@pytest.mark.parametrize("mutation", sorted(PLANTED), ids=lambda k: PLANTED[k])
def test_planted_mistake_is_caught(mutation):
    failed = []
    oracle.set_mutation(mutation)
    try:
        for pin in pins.ALL_PINS:
            try:
                pin()
            except AssertionError:
                failed.append(pin.__name__)
    finally:
        oracle.set_mutation(0)
    assert failed, f"no pin caught planted mistake {mutation}: {PLANTED[mutation]}"

"""The CPU oracle against facts the paper and mathematics fix (no GPU needed)."""
import numpy as np
import pytest

from oracle import oracle
from tests import pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin, oracle_mod):
    pin(oracle_mod.load())


# Each planted mistake (see ORACLE_MUTATION in oracle/ltl_oracle.c) must be caught.
@pytest.mark.parametrize("mutation", [1, 2, 3, 4, 5, 6, 7])
def test_pins_catch_planted_mistake(mutation, tmp_path):
    lib = oracle.load(oracle.compile_oracle(str(tmp_path), mutation=mutation))
    caught = []
    for pin in pins.ALL_PINS:
        try:
            pin(lib)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"mutation {mutation} passed every pin"


def test_table_iv_parses_and_r1_is_conway():
    rows = pins.read_table_iv()
    assert [row["rule"].r for row in rows] == list(range(1, 17))
    assert rows[0]["rule"] == pins.CONWAY
    for row in rows:
        rule = row["rule"]
        n = (2 * rule.r + 1) ** 2
        assert row["N"] == "M" and rule.C == 2 and rule.M == 0
        assert 0 <= rule.s1 <= rule.s2 < n and 1 <= rule.b1 <= rule.b2 < n


def test_scaled_rule_half_up_rounding():
    from paper_2406_17284_gb300 import inputs
    # ties at r = 2, 7, 12 round half up (n = 25, 225, 625)
    assert inputs.scaled_rule_ranges(2) == (9, 15, 9, 11)
    assert inputs.scaled_rule_ranges(7) == (77, 131, 77, 101)
    assert inputs.scaled_rule_ranges(12) == (213, 363, 213, 281)
    assert inputs.scaled_rule_ranges(1) == (3, 5, 3, 4)
    # r = 32 (n = 4225): 0.34n and 0.58n are ties again
    assert inputs.scaled_rule_ranges(32) == (1437, 2451, 1437, 1901)


def test_cross_scaled_rule_ranges():
    """The cross rule scales with n = 4r + 1 (the centre once): r = 1 -> n = 5,
    r = 5 -> n = 21, r = 16 -> n = 65, r = 32 -> n = 129."""
    from paper_2406_17284_gb300 import inputs
    assert inputs.vn_scaled_rule_ranges(1) == (2, 3, 2, 2)
    assert inputs.vn_scaled_rule_ranges(5) == (7, 12, 7, 9)
    assert inputs.vn_scaled_rule_ranges(16) == (22, 38, 22, 29)
    assert inputs.vn_scaled_rule_ranges(32) == (44, 75, 44, 58)
    assert inputs.vn_scaled_rule(3)["nbhd"] == "N"


def test_oracle_rejects_bad_input():
    g = np.zeros((4, 4), np.uint8)
    g[0, 0] = 3
    with pytest.raises(ValueError):
        oracle.step(g, oracle.Rule(1, 2, 0, 2, 3, 3, 3))
    with pytest.raises(ValueError):
        oracle.step(np.zeros((4, 4), np.uint8), oracle.Rule(1, 1, 0, 2, 3, 3, 3))

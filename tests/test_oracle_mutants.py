"""Plant one mistake at a time in the oracle (on the CPU, via -DORACLE_MUTANT)
and check that the pin battery catches every one of them."""
import pytest

import pins
from oracle.oracle import Oracle

MUTANTS = {
    1: "dagger dropped on backward hop",
    2: "backward hop uses the link at n",
    3: "backward hop added instead of subtracted",
    4: "periodic instead of antiperiodic time",
    5: "eta_2 no longer anticommuting",
    6: "missing 1/2 normalisation",
    7: "forward link transposed",
    8: "beta term dropped from zeta recurrence",
    9: "inverted zeta ratio in shifted step",
    10: "neighbours swapped in direction 1",
    11: "rational coefficients applied to the next pole",
    12: "rational action takes the imaginary part",
    13: "rectangle staple (b) left out of the gauge force",
    14: "links move with exp(-i eps H)",
    15: "trace of the gauge force kept",
    16: "fermion force: odd-site terms with the even-site sign",
    17: "fermion force without the staggered sign",
    18: "stout links move with exp(-iQ)",
    19: "stout force: C^dag L term with the wrong sign",
    20: "true residual divided by ||b||^2",
    21: "true residual without the shift",
    22: "stout: lower staples left out",
    23: "stout: lower staples without the weight rho",
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_catch_planted_mistake(mutant):
    orc = Oracle(mutant)
    assert orc.lib.oracle_mutant() == mutant
    failures = []
    for name, check in pins.BATTERY:
        try:
            ok, msg = check(orc)
        except Exception as exc:  # a crash in numpy (e.g. singular) also counts
            ok, msg = False, repr(exc)
        if not ok:
            failures.append(f"{name}: {msg}")
    assert failures, f"mutant {mutant} ({MUTANTS[mutant]}) passed every pin"


def test_default_build_passes_battery(orc):
    for name, check in pins.BATTERY:
        ok, msg = check(orc)
        assert ok, f"{name}: {msg}"

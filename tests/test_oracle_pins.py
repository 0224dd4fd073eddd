"""The FP64 oracle against what the paper and mathematics fix (no GPU)."""
import pytest

import pins


@pytest.mark.parametrize("name", sorted(pins.PINS))
def test_oracle_pin(oracle_mod, name):
    pins.PINS[name](oracle_mod)


def test_plan_rejects(oracle_mod):
    import numpy as np
    freq = np.linspace(115e6, 178e6, 8)
    with pytest.raises(ValueError):
        oracle_mod.plan(freq, "freq", np.zeros(8))
    with pytest.raises(ValueError):
        oracle_mod.plan(freq, "freq", np.r_[-1.0, np.ones(7)])
    with pytest.raises(ValueError):
        oracle_mod.plan(freq, "freq", np.r_[np.nan, np.ones(7)])
    with pytest.raises(ValueError):
        oracle_mod.plan(np.r_[0.0, freq[1:]], "freq")

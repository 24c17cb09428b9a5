"""The oracle against its pins (CPU only)."""
import pytest

from oracle_pins import ALL_PINS


@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(orc, pin):
    pin(orc)


def test_dna_selectivity(orc):
    # Sec. 2.3: on DNA each compare removes about 3/4 of the surviving starts.
    # On uniform sigma=4 text the number of starts matching a prefix of length
    # j of any pattern is close to (n - j + 1) / 4^j.
    import numpy as np
    from paper_1612_01506_gb300 import synth
    n = 1 << 20
    t = synth.uniform(n, 4, seed=0, stream=5)
    p = t[1234:1234 + 8].tobytes()
    for j in range(1, 7):
        c = orc.naive_count(p[:j], t)
        expect = (n - j + 1) / 4 ** j
        assert abs(c - expect) < 6 * np.sqrt(expect) + 1, (j, c, expect)

"""Each mistake planted in the oracle (on the CPU) must trip at least one pin.

The mutations are switched inside pam_oracle.c:
 1 propagator sign flipped (Eq. 2)           6 sqrt of two NCCs for the cube root (Eq. 10)
 2 inverse lateral DFT without 1/nx          7 time DFT with exp(+i w t) (Eq. 1)
 3 kx without the FFT-order wrap (Eq. 2)     8 eps clamp after the cube root (Sec. II-A)
 4 NCC denominator without sqrt (Eq. 4)      9 Pattern-m shifted by one element
 5 incoherent energy sum (Eq. 11)            10 rho normalised by its mean, not its max
and, in the 2x lateral padding reading (oracle.py):
11 the crop keeps the padding columns        12 no padding: n_elem-point transforms
and, in the evanescent-zero reading of Eq. 2 (pam_oracle.c):
13 the propagating components are dropped   14 the flag is ignored (nothing dropped)
"""
import pytest

import oracle
import oracle_pins

MUTATIONS = list(range(1, 15))


def _failing_pins():
    failed = []
    for pin in oracle_pins.ALL_PINS:
        try:
            pin()
        except AssertionError:
            failed.append(pin.__name__)
    return failed


@pytest.mark.parametrize("mid", MUTATIONS)
def test_mutation_is_caught(mid):
    oracle.set_mutation(mid)
    try:
        failed = _failing_pins()
    finally:
        oracle.set_mutation(0)
    assert failed, f"mutation {mid} passed every pin"

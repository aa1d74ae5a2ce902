"""Oracle pins for circular-buffer rate matching: a hand-worked interleaver
example, the interleaver as a permutation with its inverse, identity and
rotation (numpy roll) cases of the bit selection, and the repetition counts
and puncturing zeros of the soft recovery in closed form. CPU only."""
import numpy as np
import pytest

from oracle import ratematch as rm
from tests import inputs


def test_interleaver_worked_example():
    # E = 6 bits over qm = 2 rows of 3 columns: rows e0 e1 e2 / e3 e4 e5, read column by column
    e = np.array([[10, 11, 12, 13, 14, 15]])
    assert rm.interleave(e, 2).tolist() == [[10, 13, 11, 14, 12, 15]]
    e8 = np.arange(8)[None]
    assert rm.interleave(e8, 4).tolist() == [[0, 2, 4, 6, 1, 3, 5, 7]]  # 4 rows of 2 columns


@pytest.mark.parametrize("E,qm", [(12, 1), (12, 2), (24, 4), (36, 6), (40, 8)])
def test_interleaver_is_a_permutation(E, qm):
    e = np.arange(E)[None]
    f = rm.interleave(e, qm)
    assert sorted(f[0].tolist()) == list(range(E))
    assert np.array_equal(rm.deinterleave(f, qm), e)


def test_selection_identity_and_rotation():
    rng = inputs.rng(3)
    cw = (rng.random((4, 50)) < 0.5).astype(np.uint8)
    p0, ncb = 6, 40
    assert np.array_equal(rm.rate_match(cw, p0, ncb, 0, ncb, 1), cw[:, p0:p0 + ncb])
    for k0 in (1, 17, 39):
        assert np.array_equal(rm.rate_match(cw, p0, ncb, k0, ncb, 1), np.roll(cw[:, p0:p0 + ncb], -k0, axis=1))


@pytest.mark.parametrize("ncb,k0,E,qm", [(30, 7, 75, 1), (30, 0, 60, 2), (32, 31, 96, 4), (25, 3, 12, 2),
                                         (40, 39, 40, 8)])
def test_recovery_counts_and_zeros(ncb, k0, E, qm):
    # every received LLR set to +1 and the buffer position it came from counted: position p is hit
    # floor(E / ncb) or ceil(E / ncb) times, the ceil for the E mod ncb positions from k0 on
    llr = np.ones((2, E))
    v = rm.rate_recover(llr, ncb, k0, qm)
    expect = np.full(ncb, E // ncb, dtype=np.float64)
    for t in range(E % ncb):
        expect[(k0 + t) % ncb] += 1
    assert np.array_equal(v[0], expect) and np.array_equal(v[1], expect)


def test_match_then_recover_sums_signs():
    rng = inputs.rng(5)
    cw = (rng.random((3, 70)) < 0.5).astype(np.uint8)
    p0, ncb, k0, E, qm = 4, 60, 22, 150, 6
    f = rm.rate_match(cw, p0, ncb, k0, E, qm)
    v = rm.rate_recover(1.0 - 2.0 * f, ncb, k0, qm)
    counts = rm.rate_recover(np.ones_like(f, dtype=np.float64), ncb, k0, qm)
    assert np.array_equal(v, counts * (1.0 - 2.0 * cw[:, p0:p0 + ncb]))


def test_bad_parameters():
    cw = np.zeros((1, 20), dtype=np.uint8)
    for args in [(0, 0, 0, 10, 1), (0, 10, 10, 10, 1), (0, 10, 0, 9, 2), (0, 10, 0, 8, 3), (15, 10, 0, 8, 1)]:
        with pytest.raises(ValueError):
            rm.rate_match(cw, *args)

"""Host logic of the package without a GPU: the rate-by-truncation row counts
of the mixed workload, the log-domain BER crossing, the autotuner's cache file
and the multi-rank codeword ranges."""
import math
from fractions import Fraction

import pytest

torch = pytest.importorskip("torch")


def test_rows_for_rate():
    from paper_2203_11854_gb300.workloads import rows_for_rate
    # 4 + max(0, ceil(Kb / r) + 2 - (Kb + 4)) with Kb = 22 (BG1-shaped) and 10 (BG2-shaped)
    want = {1: [46, 24, 13, 5], 2: [22, 12, 7, 4]}
    for bg, rows in want.items():
        got = [rows_for_rate(bg, r) for r in (Fraction(1, 3), Fraction(1, 2), Fraction(2, 3), Fraction(8, 9))]
        assert got == rows, bg
    # a truncated code of rate r carries at least k / r bits in its kept columns (2 punctured ones excepted)
    for bg, kb in ((1, 22), (2, 10)):
        for r in (Fraction(1, 3), Fraction(1, 2), Fraction(2, 3), Fraction(8, 9)):
            rows = rows_for_rate(bg, r)
            assert kb + rows - 2 >= kb / r or rows == 4


def test_ber_crossing():
    from paper_2203_11854_gb300.ber import crossing
    # BER = 10^-x: log10 is linear in x, so the interpolated crossing is exact
    pts = [(x, 10.0 ** -x) for x in (1.0, 2.0, 3.0, 5.0, 6.0)]
    assert crossing(pts, 1e-4) == pytest.approx(4.0, abs=1e-12)
    assert crossing(pts, 1e-2) == pytest.approx(2.0, abs=1e-12)
    assert crossing(list(reversed(pts)), 1e-4) == pytest.approx(4.0, abs=1e-12)  # order does not matter
    assert crossing(pts, 1e-9) is None  # never reached
    assert crossing([(1.0, 1e-3), (2.0, 0.0)], 1e-4) == 2.0  # no errors at the upper point
    # geometric mean between the bracketing BERs sits halfway
    assert crossing([(0.0, 1e-3), (1.0, 1e-5)], 1e-4) == pytest.approx(0.5, abs=1e-12)


def test_autotune_cache_round_trip(tmp_path, monkeypatch):
    from paper_2203_11854_gb300 import autotune
    path = str(tmp_path / "sub" / "tune.json")
    assert autotune.load_cache(path) == {}
    cache = {"dev|Z384|46x68|nnz316|algo0|msg1|it20|es0": {"l2_prefetch": 0, "cw_per_cta": 0, "zpt": 0}}
    autotune.save_cache(cache, path)
    assert autotune.load_cache(path) == cache
    with open(path, "w") as f:
        f.write("{broken")
    assert autotune.load_cache(path) == {}  # a damaged cache is ignored, not fatal
    monkeypatch.setenv("LDPCX_AUTOTUNE_CACHE", path)
    autotune.save_cache(cache)
    assert autotune.load_cache() == cache


def test_rank_ranges():
    from paper_2203_11854_gb300 import multi
    bases = [multi.rank_cw_base(r) for r in range(8)]
    assert len(set(bases)) == 8 and bases == sorted(bases)
    total = 1001
    spans = [multi.split_range(total, r, 4, cw0=50) for r in range(4)]  # (start, count)
    covered = []
    for start, count in spans:
        covered.extend(range(start, start + count))
    assert covered == list(range(50, 50 + total))  # disjoint, contiguous, complete
    sizes = [count for _, count in spans]
    assert max(sizes) - min(sizes) <= 1
    assert math.isclose(sum(sizes), total)
    with pytest.raises(ValueError):
        multi.split_range(10, 4, 4)

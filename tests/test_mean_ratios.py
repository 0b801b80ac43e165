"""The six mean ratios (Section 1, Section 3) against hand-worked tables and the
paper's Tables 3.1 and 3.2."""
import json
from pathlib import Path

import numpy as np
import pytest

GOLDEN = Path(__file__).resolve().parent / "golden"


def test_hand_worked_table(orc):
    # a = (1, 2, 4), c = (2, 2, 2): worked by hand.
    a, c = [1.0, 2.0, 4.0], [2.0, 2.0, 2.0]
    r = orc.six_ratios(a, c)
    assert r["AM-RATIO"] == pytest.approx(7 / 6, abs=1e-15)
    assert r["GM-RATIO"] == pytest.approx(1.0, abs=1e-15)
    assert r["HM-RATIO"] == pytest.approx((3 / 1.75) / 2, abs=1e-15)
    assert r["RATIO-AM"] == pytest.approx(7 / 6, abs=1e-15)
    assert r["RATIO-GM"] == pytest.approx(1.0, abs=1e-15)
    assert r["RATIO-HM"] == pytest.approx(3 / 3.5, abs=1e-15)


def test_paper_example_three_approaches(orc):
    # Section 1's a, b, c with 3 runs each: RATIO-AM w.r.t. c is
    # (a1/c1 + a2/c2 + a3/c3)/3 and AM-RATIO is (a1+a2+a3)/(c1+c2+c3).
    a, b, c = [3.0, 5.0, 9.0], [2.0, 4.0, 4.0], [1.0, 2.0, 3.0]
    assert orc.ratio_mean("AM", a, c) == pytest.approx((3 / 1 + 5 / 2 + 9 / 3) / 3, abs=1e-15)
    assert orc.mean_ratio("AM", a, c) == pytest.approx(17 / 6, abs=1e-15)
    assert orc.ratio_mean("AM", c, c) == 1.0
    assert orc.mean_ratio("AM", b, c) == pytest.approx(10 / 6, abs=1e-15)


def test_identities_on_random_tables(orc):
    rng = np.random.default_rng(0)
    for _ in range(50):
        k = int(rng.integers(2, 20))
        a, b, c = (rng.lognormal(0, 1.5, k) for _ in range(3))
        # RATIO-GM equals GM-RATIO
        assert orc.ratio_mean("GM", a, c) == pytest.approx(orc.mean_ratio("GM", a, c), rel=1e-12)
        # X-RATIO does not depend on the baseline: X(a)/X(b) = (X(a)/X(c)) / (X(b)/X(c))
        for kind in ("AM", "GM", "HM"):
            direct = orc.mean_ratio(kind, a, b)
            via = orc.mean_ratio(kind, a, c) / orc.mean_ratio(kind, b, c)
            assert direct == pytest.approx(via, rel=1e-12)
        # RATIO-AM >= RATIO-GM >= RATIO-HM (mean inequality on the ratios)
        ra, rg, rh = (orc.ratio_mean(x, a, c) for x in ("AM", "GM", "HM"))
        assert ra >= rg * (1 - 1e-12) and rg >= rh * (1 - 1e-12)
        # RATIO-HM(a vs c) = 1 / RATIO-AM(c vs a)
        assert orc.ratio_mean("HM", a, c) == pytest.approx(1 / orc.ratio_mean("AM", c, a), rel=1e-12)
        # RATIO-AM depends on the baseline in general (only checked as not an identity)
    a = np.array([1.0, 10.0]); c = np.array([10.0, 1.0])
    assert orc.ratio_mean("AM", a, c) != pytest.approx(1 / orc.ratio_mean("AM", c, a))


def _interval_ratio(x, y, half):
    lo = (x - half) / (y + half)
    hi = (x + half) / (y - half)
    return lo, hi


@pytest.mark.parametrize("fname", ["table_3_1_times.json", "table_3_2_iterations.json"])
def test_paper_tables_mean_first_ratios(orc, fname):
    """X-RATIO columns of Tables 3.1/3.2 follow from their printed means within
    the rounding of the printed digits."""
    t = json.loads((GOLDEN / fname).read_text())
    half_m = 0.5 * 10 ** (-t["means_decimals"])
    half_r = 0.5 * 10 ** (-t["ratio_decimals"])
    for kind in ("AM", "GM", "HM"):
        means = t["means_ms"][kind]
        for base_idx, key in ((0, "ratios_vs_L1"), (2, "ratios_vs_Linf")):
            printed = t[key][f"{kind}-RATIO"]
            for j in range(3):
                if j == base_idx:
                    assert printed[j] == 1.0
                    continue
                lo, hi = _interval_ratio(means[j], means[base_idx], half_m)
                assert lo - half_r <= printed[j] <= hi + half_r, (kind, key, j)
        # AM >= GM >= HM holds column by column
    for j in range(3):
        assert t["means_ms"]["AM"][j] >= t["means_ms"]["GM"][j] >= t["means_ms"]["HM"][j]


@pytest.mark.parametrize("fname", ["table_3_1_times.json", "table_3_2_iterations.json"])
def test_paper_tables_ratio_first_identities(fname):
    """In Tables 3.1/3.2: RATIO-GM rows equal GM-RATIO rows, and
    RATIO-HM(Linf vs L1) = 1/RATIO-AM(L1 vs Linf), RATIO-HM(L1 vs Linf) =
    1/RATIO-AM(Linf vs L1), within the printed rounding."""
    t = json.loads((GOLDEN / fname).read_text())
    half = 0.5 * 10 ** (-t["ratio_decimals"])
    for key in ("ratios_vs_L1", "ratios_vs_Linf"):
        assert t[key]["RATIO-GM"] == t[key]["GM-RATIO"]
    am_linf_vs_l1 = t["ratios_vs_L1"]["RATIO-AM"][2]
    hm_l1_vs_linf = t["ratios_vs_Linf"]["RATIO-HM"][0]
    lo, hi = 1 / (am_linf_vs_l1 + half), 1 / (am_linf_vs_l1 - half)
    assert lo - half <= hm_l1_vs_linf <= hi + half
    am_l1_vs_linf = t["ratios_vs_Linf"]["RATIO-AM"][0]
    hm_linf_vs_l1 = t["ratios_vs_L1"]["RATIO-HM"][2]
    lo, hi = 1 / (am_l1_vs_linf + half), 1 / (am_l1_vs_linf - half)
    assert lo - half <= hm_linf_vs_l1 <= hi + half

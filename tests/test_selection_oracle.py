"""Pins of the blocksize-selection oracle (Sec. 3.2-3.7) against the paper's
printed numbers and hand-made time tables whose picks are known by inspection."""
import pytest

from conftest import read_golden
from oracle import selection


def test_candidates_worked_example():
    rows = read_golden("paper_candidates.txt")
    assert rows
    for row in rows:
        S, P = int(row[0]), int(row[1])
        assert selection.candidates_1d(S, P) == [int(x) for x in row[2:]]


def test_candidate_counts_for_P_5_10_20():
    # Sec. 3.7: P = 5, 10, 20 parts give nC = 125, 1000 and 8000 combinations
    for P, nC in ((5, 125), (10, 1000), (20, 8000)):
        assert len(selection.candidates((200, 200, 800), P)) == nC
        assert len(selection.candidates((250, 250, 1500), P)) == nC


def test_candidates_small_extent_dedup():
    assert selection.candidates_1d(3, 5) == [1, 2, 3]
    assert selection.candidates_1d(1, 5) == [1]


def _table5():
    t = {}
    for size, alg, bi, bj, bk, total, mn, act in read_golden("paper_table5_min_actual.txt"):
        t[(size, alg)] = (float(total), float(mn), float(act))
    return t


def test_quality_percentages_printed_in_text():
    t = _table5()
    size = "250x250x1500"
    for what, alg, pct, dec in read_golden("paper_quality_percentages.txt"):
        total, mn, act = t[(size, alg)]
        _, mn_w, act_w = t[(size, "MWMB")]
        total_w = t[(size, "MWMB")][0]
        if what == "quality":
            val = selection.quality(mn, act)
        elif what == "actual_vs_mwmb":
            val = selection.quality(act_w, act)
        else:
            val = selection.quality(total_w, total)
        assert round(100 * val, int(dec)) == pytest.approx(float(pct)), (what, alg)


def test_mwmb_quality_smallest_in_table5():
    # Sec. 3.6: MWMB's MinTime and ActualTime are the closest of the four.
    t = _table5()
    for size in ("200x200x800", "300x300x800", "250x250x1500"):
        q = {a: abs(selection.quality(t[(size, a)][1], t[(size, a)][2]))
             for a in ("OB", "MMMB", "MWMB", "MAMB")}
        assert min(q, key=q.get) == "MWMB"


def _hand_table():
    # 2 nodes x 3 cores x 3 candidates; node 0 candidates A0..A2, node 1 B0..B2
    node0 = [[5.0, 3.0, 4.0],    # core 0 best: cand 1 (3.0)
             [6.0, 7.0, 4.5],    # core 1 best: cand 2 (4.5)
             [3.5, 9.0, 8.0]]    # core 2 best: cand 0 (3.5)
    node1 = [[4.0, 2.0, 6.0],    # core 0 best: cand 1 (2.0)
             [5.2, 9.0, 5.0],    # core 1 best: cand 2 (5.0)
             [4.1, 8.0, 7.0]]    # core 2 best: cand 0 (4.1)
    return [node0, node1]


def test_stage_reductions_by_inspection():
    T = _hand_table()
    # MMMB: node0 min over cores = 3.0 (cand 1), node1 = 2.0 (cand 1) -> node1 cand 1
    assert selection.three_stage(T, "min") == (1, 1, 2.0)
    # MWMB: node0 worst best = 4.5 (cand 2), node1 = 5.0 (cand 2) -> node0 cand 2
    assert selection.three_stage(T, "max") == (0, 2, 4.5)
    # MAMB: node0 mean of (3, 4.5, 3.5) = 3.667 -> closest 3.5 (core 2, cand 0);
    #       node1 mean of (2, 5, 4.1) = 3.7 -> closest 4.1 (core 2, cand 0);
    #       stage 3 picks node0 (3.5 < 4.1)
    assert selection.three_stage(T, "avg") == (0, 0, 3.5)


def test_ties_go_to_lowest_index():
    assert selection.stage1([2.0, 1.0, 1.0]) == (1, 1.0)
    assert selection.stage2([3.0, 3.0, 1.0], "max") == 0
    assert selection.stage2([1.0, 3.0, 3.0], "min") == 0
    assert selection.three_stage([[[1.0]], [[1.0]]], "max") == (0, 0, 1.0)


def test_original_block_global_min():
    assert selection.original_block([[3.0, 2.5], [2.0, 4.0], [2.2]]) == (1, 0, 2.0)


def test_quality_rejects_nonpositive_min():
    with pytest.raises(ValueError):
        selection.quality(0.0, 1.0)


def test_paper_table1_and_table3_percentages():
    """Tables 1 and 3: every printed percentage is the quality-style relative
    excess value / reference - 1 (the arithmetic the selection report uses),
    rounded or truncated to the printed decimals."""
    rows = read_golden("paper_table1_table3_ratios.txt")
    assert len(rows) == 11
    for table, what, value, ref, printed, decimals in rows:
        pct = 100.0 * selection.quality(float(ref), float(value))
        step = 10.0 ** -int(decimals)
        assert abs(pct - float(printed)) < step, (table, what, pct, printed)
        # the inverse ratio would be far off: the formula's direction is pinned
        assert abs(100.0 * selection.quality(float(value), float(ref)) - float(printed)) > 1.0

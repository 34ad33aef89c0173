"""Net batches after Alg. 1 (host logic, no GPU): criticality intervals
[C, C], [C/2, C), [C/4, C/2), ...; slack intervals [WNS, WNS], [0.99 WNS,
WNS), [0.96 WNS, 0.99 WNS), ...; the rest last."""
import numpy as np
import pytest

pytest.importorskip("torch")
import paper_2507_13375_gb300 as la  # noqa: E402


def test_criticality_intervals():
    crit = np.array([8.0, 8.0, 4.0, 6.0, 2.0, 3.9, 1.0, 0.0])
    b = la.batches_by_criticality(crit, critical_frac=0.25)
    # C = 8: [8,8] -> 0, [4,8) -> 1, [2,4) -> 2; below 2 (= 0.25 C) -> the rest
    assert list(b) == [0, 0, 1, 1, 2, 2, 3, 3]


def test_slack_intervals_and_rest():
    crit = np.array([10.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0])
    slack = np.array([-5.0, -10.0, -9.95, -9.9, -9.7, -8.0, -1.0])
    b = la.batches_by_criticality(crit, slack, critical_frac=0.9, slack_ratio=0.7)
    # critical: net 0 -> 0; WNS = -10: r = 1 -> 1, 0.995 -> 2, 0.99 -> 2, 0.97 -> 3,
    # 0.80 -> 1 - r = 0.2: sqrt(20) = 4.47 -> j = 5 -> a later batch; 0.1 -> not semi-critical
    assert b[0] == 0 and b[1] == 1 and b[2] == b[3] == 2 and b[4] == 3
    assert b[5] == 4 and b[6] == 5


def test_one_batch_when_nothing_is_critical():
    assert list(la.batches_by_criticality(np.zeros(5))) == [0] * 5

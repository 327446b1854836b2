"""Host-side logic of the query server's admission (no GPU): memory budget, slots, arrival
order, and rejection of a batch larger than the whole budget."""
import pytest

from paper_1704_03767_gb300.serving import Admission, percentile


def test_admission_by_memory_and_slots():
    a = Admission(budget_bytes=100, slots=3)
    s0 = a.try_admit(60)
    assert s0 == 0
    assert a.try_admit(50) is None          # does not fit the unreserved budget
    s1 = a.try_admit(40)
    assert s1 == 1 and a.reserved == 100
    a.release(s0, 60)
    assert a.try_admit(50) == 0             # memory freed -> admitted on the freed slot
    assert a.try_admit(11) is None          # 90 reserved: 11 more does not fit
    assert a.try_admit(10) == 2             # exactly fills the budget on the last slot
    a.release(1, 40)
    assert a.try_admit(40) == 1


def test_slot_limit():
    a = Admission(budget_bytes=10**9, slots=2)
    assert a.try_admit(1) == 0 and a.try_admit(1) == 1
    assert a.try_admit(1) is None
    a.release(0, 1)
    assert a.try_admit(1) == 0


def test_oversized_batch_rejected():
    a = Admission(budget_bytes=10, slots=1)
    with pytest.raises(ValueError):
        a.try_admit(11)


def test_percentile():
    xs = list(range(1, 101))
    assert percentile(xs, 50) in (50, 51)
    assert percentile(xs, 99) == 99

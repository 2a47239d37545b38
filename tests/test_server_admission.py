"""The solve server's admission pass (host logic, no GPU): requests start in
FIFO order when their workspace fits the remaining budget, a stream slot is
free and their CTAs fit next to the running solves; a request that does not
fit yet is passed by later ones that do (backfilling) until it has waited
the backfill window (0.1 s), after which admission stops at it."""
import pytest

from paper_1905_06850_gb300 import build as B
from paper_1905_06850_gb300 import plcg

SMS = 152
GB = 1 << 30


@pytest.fixture(scope="module", autouse=True)
def lib():
    B.build()
    return plcg.load()


def admit(reqs, mem_free=100 * GB, sm_used=0.0, slots=32):
    """reqs: (bytes, SM share, waited seconds) per queued request."""
    return plcg.server_admission([r[0] for r in reqs], [r[1] for r in reqs], [r[2] for r in reqs],
                                 mem_free, sm_used, SMS, slots)


def test_fifo_when_everything_fits():
    reqs = [(GB, 10.0, 0.0), (GB, 20.0, 0.0), (GB, 30.0, 0.0)]
    assert admit(reqs) == [0, 1, 2]


def test_first_request_on_an_idle_gpu_always_fits():
    # a grid capped at all resident CTAs occupies every SM; nothing runs yet
    assert admit([(GB, float(SMS), 0.0), (GB, 1.0, 0.0)]) == [0]


def test_blocked_request_is_passed_by_smaller_ones():
    # 100 SMs busy: a half-GPU request (76) waits, the small ones behind it start
    reqs = [(GB, 76.0, 0.01), (GB, 20.0, 0.0), (GB, 40.0, 0.0), (GB, 30.0, 0.0)]
    assert admit(reqs, sm_used=100.0) == [1, 3]   # 100 + 20 + 30 = 150 <= 152; 40 does not fit


def test_admission_stops_at_a_request_past_the_window():
    reqs = [(GB, 76.0, 0.1), (GB, 20.0, 0.0)]
    assert admit(reqs, sm_used=100.0) == []
    reqs = [(GB, 10.0, 0.5), (GB, 76.0, 0.2), (GB, 20.0, 0.0)]
    assert admit(reqs, sm_used=100.0) == [0]        # stops at the aged blocked one
    reqs = [(GB, 76.0, 0.099), (GB, 20.0, 0.0)]
    assert admit(reqs, sm_used=100.0) == [1]        # just inside the window


def test_memory_budget_and_slots():
    reqs = [(60 * GB, 10.0, 0.0), (50 * GB, 10.0, 0.0), (30 * GB, 10.0, 0.0)]
    assert admit(reqs, mem_free=100 * GB) == [0, 2]  # the second exceeds the budget left
    assert admit(reqs, mem_free=100 * GB, slots=1) == [0]
    reqs = [(GB, 10.0, 0.0)] * 5
    assert admit(reqs, slots=3) == [0, 1, 2]


def test_admitted_requests_use_up_the_gpu():
    reqs = [(GB, 76.0, 0.0), (GB, 76.0, 0.0), (GB, 1.0, 0.0)]
    assert admit(reqs) == [0, 1]                    # 152 SMs taken: the third waits (skipped)
    assert admit([]) == []

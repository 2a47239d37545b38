"""The batched launch-shape setter (host logic, no GPU): the FP32 shapes
that exist are 3 or 4 blocks per SM with 1, 2 or 4 row groups per thread at
vector width 1, and 4 blocks per SM, 1 row group, vector width 2; (0, 0, 0)
restores the defaults; anything else is rejected and leaves the setting
unchanged."""
import pytest

from paper_1905_06850_gb300 import build as B
from paper_1905_06850_gb300 import plcg


@pytest.fixture(scope="module")
def lib():
    B.build()
    return plcg.load()


def test_valid_shapes(lib):
    try:
        for shp in [(0, 0, 0), (4, 1, 1), (4, 2, 1), (4, 4, 1), (3, 1, 1), (3, 2, 1), (3, 4, 1), (4, 1, 2)]:
            assert lib.plcg_set_batched_launch(*shp) == plcg.PLCG_OK, shp
    finally:
        lib.plcg_set_batched_launch(0, 0, 0)


def test_invalid_shapes(lib):
    try:
        for shp in [(2, 1, 1), (5, 1, 1), (4, 3, 1), (4, 1, 0), (4, 2, 2), (3, 1, 2), (4, 1, 4), (0, 0, 1),
                    (0, 1, 0)]:
            assert lib.plcg_set_batched_launch(*shp) == plcg.PLCG_ERR_INVALID, shp
            assert "batched launch shape" in plcg.last_error()
    finally:
        lib.plcg_set_batched_launch(0, 0, 0)

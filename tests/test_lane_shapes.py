"""The stateless-pass parity cases reach every dispatched kernel instance."""
from shapes import LANE_SHAPE_CASES, lane_shape


def test_lane_shape_cases_reach_every_instance():
    reachable = {lane_shape(K) for K in range(1, 1025)}
    assert reachable == {lane_shape(K) for K, _ in LANE_SHAPE_CASES}

"""Host logic of the learned preconditioner that needs no GPU: the network
grid chosen for an instance size (level and zero-padded extents)."""
from paper_2408_03452_gb300 import learned


def test_net_grid_levels_and_padding():
    # the coarsest level with divisible extents, each extent rounded up to 4
    assert learned.net_grid((64, 64, 32), 2) == (2, (16, 16, 8))
    assert learned.net_grid((48, 48, 24), 2) == (2, (12, 12, 8))   # 12x12x6 padded in z
    assert learned.net_grid((128, 128, 64), 2) == (2, (32, 32, 16))
    assert learned.net_grid((24, 16, 24), 2) == (2, (8, 4, 8))
    assert learned.net_grid((20, 12, 8), 2) == (2, (8, 4, 4))
    # a level whose extents are not divisible is skipped for a finer one
    assert learned.net_grid((12, 12, 6), 2) == (1, (8, 8, 4))
    # the solver's own grid is never padded
    assert learned.net_grid((8, 8, 8), 0) == (0, (8, 8, 8))
    assert learned.net_grid((6, 6, 6), 0) is None
    assert learned.net_grid((13, 11, 7), 2) is None

"""Host logic of the accuracy simulation (no GPU)."""
import numpy as np


def test_accuracy_delta_summaries():
    """The delta(f) summaries of the accuracy simulation: fine channels k * U are the
    original channel centres, k * U + U / 2 their edges; channel 0 and the last coarse
    channel are left out of the median and the maximum."""
    from paper_2608_23441_b300 import accuracy
    U = 8
    nf = 6 * U
    delta = np.full(nf, 0.5)
    delta[np.arange(U, nf - U, U)] = 0.01          # centres of coarse channels 1..4
    delta[np.arange(U, nf - U, U) + U // 2] = 0.2  # their edges
    delta[:U] = 100.0                               # channel 0: excluded
    delta[nf - U:] = 100.0                          # last coarse channel: excluded
    st = accuracy._delta_stats(delta, U)
    assert st["median_at_channel_centres"] == 0.01
    assert st["median_at_channel_edges"] == 0.2
    assert st["max"] == 0.5
    assert st["median"] == 0.5

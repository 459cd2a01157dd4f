"""The random-gather probe (a measurement aid of bench.py): it runs, and
gathers that hit L2 are faster than gathers that miss it."""
import pytest

import paper_1806_00762_b300 as seraph

pytestmark = pytest.mark.gpu


def test_gather_probe_hits_beat_misses():
    nv, ng = 1 << 27, 1 << 26           # 512 MB of values (above L2), 64M gathers
    hot = (4 << 20) // 4                # 4 MB hot range
    t_hit = seraph.gather_probe(nv, ng, hot, 1.0, reps=3)
    t_miss = seraph.gather_probe(nv, ng, 0, 0.0, reps=3)
    assert 0.0 < t_hit < t_miss, (t_hit, t_miss)
    assert t_miss > 1.5 * t_hit, (t_hit, t_miss)


@pytest.mark.parametrize("nv,hot,frac", [(8, 8, 1.0), (8, 0, 0.0), (1000, 1, 0.5), (1000, 999, 0.999)])
def test_gather_probe_edge_ranges(nv, hot, frac):
    """Tiny and one-sided ranges: every drawn index stays inside the array."""
    assert seraph.gather_probe(nv, 1 << 12, hot, frac, reps=1) > 0.0

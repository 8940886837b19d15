"""The operation count behind the bench's Evaluate roofline
(paper_2104_06494_gb300/roofline.py) forms every rule point exactly once:
for each family and dimension, the points it accumulates or forms per
region (every point but the centre, whose value is the full prefix
product) number N(d) - 1, and N(d) is the rule's own point count (the sum
of its orbit sizes, from the oracle's rule construction).  A dropped or
doubled orbit in the count would change the reported algorithmic flops."""
import pytest

from oracle import rule as orule
from paper_2104_06494_gb300 import roofline


@pytest.mark.parametrize("n", range(2, 9))
def test_point_count_matches_the_rule(n):
    _, counts, _, _, _ = orule.exact_rule(n)
    assert int(sum(counts)) == roofline.num_points(n)


@pytest.mark.parametrize("family", range(7))
@pytest.mark.parametrize("n", range(2, 9))
def test_every_point_formed_once_per_region(family, n):
    c = roofline.region_points_work(family, n)
    assert c["points"] == roofline.num_points(n) - 1
    assert c["flops"] >= c["inst"] > 0

"""Distributed-shared-memory rates of thread-block clusters (sn_test_dsmem_rates).

The plane-resident cluster schedule would move three quarters of a plane
across the cluster in every column pass, so its exchange rate is the rate at
which a CTA reads or fills a peer's shared memory.  The hook measures it for
clusters of 2, 4 and 8 CTAs; a peer's shared memory must read slower than a
CTA's own, and every rate is positive and finite.
"""
import math

import pytest

from paper_1909_08354_b300 import sn

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cluster", [2, 4, 8])
def test_dsmem_rates(cluster):
    r = sn.sn_test_dsmem_rates(cluster)
    print(f"cluster {cluster}: remote reads {r['remote_read_gbs']:.0f} GB/s, local reads "
          f"{r['local_read_gbs']:.0f} GB/s, bulk pushes {r['push_gbs']:.0f} GB/s (aggregate)")
    for v in r.values():
        assert math.isfinite(v) and v > 0
    assert r["remote_read_gbs"] < r["local_read_gbs"]


def test_dsmem_rejects_bad_cluster_sizes():
    for bad in (1, 3, 16):
        with pytest.raises(sn.SNError) as e:
            sn.sn_test_dsmem_rates(bad)
        assert e.value.status == sn.SN_EINVAL

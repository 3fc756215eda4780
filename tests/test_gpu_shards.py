"""vrs_merge_shards on the GPU: a table split into row ranges held by
separate engines (here on one GPU) answers a query batch shard by shard;
the merged lists, with global row ids, must be the exact filtered top-k of
the whole table (float64 oracle, tests/_parity.py rule)."""
import numpy as np
import pytest

import gen
import oracle
from _parity import check_topk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vrs():
    from paper_2403_15807_gb300 import build, vrs as v
    build.build()
    v.load()
    return v


@pytest.mark.parametrize("world,metric,compute", [(2, "l2", 0), (3, "ip", 0), (4, "l2", 1)])
def test_sharded_query_matches_whole_table(vrs, world, metric, compute):
    from paper_2403_15807_gb300 import shards
    n, d, b, k = 50_003, 96, 40, 10
    unit = metric == "ip"
    mix = gen.Mixture(d, seed=world)
    x = gen.vectors(n, mix, unit=unit)
    q = gen.queries(b, mix, unit=unit)
    attrs = gen.attributes(n, 1, 1000, seed=world)
    pred = gen.pred_less_than(250)
    m = vrs.VRS_L2 if metric == "l2" else vrs.VRS_IP
    qd = torch.from_numpy(q).cuda()
    ids, dists = [], []
    for r in range(world):
        lo, hi = shards.shard_rows(n, world, r)
        with vrs.Engine(0) as e:
            e.load(np.ascontiguousarray(x[lo:hi]), np.ascontiguousarray(attrs[:, lo:hi]),
                   dtype=vrs.VRS_F32, copies=3)
            i, dd = e.query(qd, [pred], np.int32([k]), metric=m, compute=compute)
            torch.cuda.synchronize()
        ids.append(i)
        dists.append(dd)
    offs = shards.row_offsets(n, world)
    gi, gd = shards.merge(vrs, torch.stack(ids), torch.stack(dists), offs, m)
    torch.cuda.synchronize()
    rid, rdist, rcnt = oracle.query(x, attrs, q, [pred], k + 1, metric, n_threads=16)
    check_topk(x, q, attrs, [pred], np.int32([k]), metric, gi.cpu().numpy(), gd.cpu().numpy(),
               rid, rdist, rcnt)
    # the host-buffer form gives the same lists
    hi_, hd_ = vrs.vrs_merge_shards(torch.stack(ids).cpu().numpy(),
                                    torch.stack(dists).cpu().numpy(), offs, m)
    assert np.array_equal(hi_, gi.cpu().numpy())
    np.testing.assert_array_equal(hd_, gd.cpu().numpy())


def test_merge_shards_rejects_bad_arguments(vrs):
    z = np.zeros((2, 1, 4), dtype=np.int64)
    f = np.zeros((2, 1, 4), dtype=np.float32)
    with pytest.raises(vrs.VrsError):
        vrs.vrs_merge_shards(z, f, np.array([0, -1], dtype=np.int64))
    with pytest.raises(vrs.VrsError):
        vrs.vrs_merge_shards(np.zeros((65, 1, 4), dtype=np.int64),
                             np.zeros((65, 1, 4), dtype=np.float32), np.zeros(65, dtype=np.int64))

"""The serving loop at the full posting-list configuration: 100,000 lists with
rank-Zipf lengths over a universe of 5 x 10^7 document ids (about 1.2 x 10^8
values, 227 MB compressed), resident in HBM; queries of 2..8 distinct lists
drawn in proportion to length.  Every query's values must equal the oracle's
per-list decoding (Algorithm 1 with the differential running sum from each
list's x_0, Sec. 1 and Sec. 2), in the batched and in the one-call-per-list
form, and a probe query must give the same values alone and inside a mix."""
import numpy as np
import pytest

import oracle
from paper_1503_07387_gb300 import inputs, vbyte

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def pool():
    import torch
    ids, vo = inputs.posting_lists()          # 100,000 lists, universe 5e7, cap 1e7
    L = vo.size - 1
    prev = inputs.full_range(L, seed=17)
    b, bo = oracle.encode_batched(ids, vo, True, prev)
    del ids
    want, st = oracle.decode_batched(b, bo, vo, True, prev)
    assert st == 0
    return dict(d=torch.from_numpy(b).cuda(), bo=bo, vo=vo, prev=prev, L=L,
                want=torch.from_numpy(want.view(np.int32)).cuda(), lens=np.diff(vo).astype(np.int64))


def _expected(pool, lists):
    import torch
    vo = pool["vo"]
    return torch.cat([pool["want"][int(vo[j]):int(vo[j + 1])] for j in lists])


def _server(pool, form):
    import torch
    free, _ = torch.cuda.mem_get_info()
    arena = int(min(free * 0.25, 8 << 30)) // 4096 * 4096
    return vbyte.Server(pool["d"], pool["bo"], pool["vo"], True, pool["prev"], arena_bytes=arena,
                        staging_bytes=512 << 20, max_inflight=4, max_batch_queries=64, max_batch_lists=512,
                        form=form)


@pytest.mark.parametrize("form", ["in_place", "per_list", "gather"])
def test_every_query_matches_the_oracle(pool, form):
    import torch
    nq = 300
    _, qoff, ql = inputs.query_stream(pool["lens"], nq, 20000.0, seed=41)
    srv = _server(pool, form)
    probe = [int(x) for x in ql[qoff[5]:qoff[6]]]
    # the probe alone
    q = srv.submit(probe)
    _, st = srv.wait(q)
    assert st == 0
    v, nb = srv.result(q)
    assert nb == 1
    alone = v.clone()
    srv.release(q)
    assert torch.equal(alone, _expected(pool, probe))
    # every query submitted at once (they share batches), the probe again in the middle
    qids = []
    pq = None
    for i in range(nq):
        qids.append(srv.submit(ql[qoff[i]:qoff[i + 1]]))
        if i == nq // 2:
            pq = srv.submit(probe)
    shared = 0
    for i, qi in enumerate(qids):
        _, st = srv.wait(qi)
        assert st == 0
        v, nb = srv.result(qi)
        shared += nb > 1
        assert torch.equal(v, _expected(pool, ql[qoff[i]:qoff[i + 1]])), f"query {i}"
        srv.release(qi)
        if i == nq // 2:
            _, st = srv.wait(pq)
            assert st == 0
            v, nb = srv.result(pq)
            assert nb > 1, "the probe should have shared its batch"
            assert torch.equal(v, alone)
            srv.release(pq)
    assert shared > 0
    s = srv.stats()
    assert s["queries"] == nq + 2
    assert s["values"] == int(sum(pool["lens"][ql[qoff[i]:qoff[i + 1]]].sum() for i in range(nq))) \
        + 2 * int(pool["lens"][probe].sum())
    srv.close()
    torch.cuda.synchronize()


def test_replay_at_a_stated_rate(pool):
    # open-loop Poisson arrivals at 20,000 q/s: every query completes without a data error
    arr, qoff, ql = inputs.query_stream(pool["lens"], 2000, 20000.0, seed=42)
    srv = _server(pool, "in_place")
    lat, st = srv.replay(arr, qoff, ql)
    assert np.all(st == 0) and np.all(lat > 0)
    assert srv.stats()["queries"] == 2000
    srv.close()

"""The serving loop: every query's values equal the oracle's decoding of its
lists, whether it ran alone or inside a batch with others (continuous
batching), with admission limited by the output arena, in both the batched
and the one-call-per-list forms."""
import numpy as np
import pytest

import oracle
from paper_1503_07387_gb300 import inputs, vbyte

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool():
    import torch
    ids, vo = inputs.posting_lists(2000, universe=1 << 22, cap=60000, seed=30)
    L = vo.size - 1
    prev = inputs.full_range(L, seed=31)
    b, bo = oracle.encode_batched(ids, vo, True, prev)
    want, st = oracle.decode_batched(b, bo, vo, True, prev)
    assert st == 0
    return dict(d=torch.from_numpy(b).cuda(), bo=bo, vo=vo, prev=prev, want=want, L=L,
                lens=np.diff(vo).astype(np.int64))


def _expected(pool, lists):
    vo, want = pool["vo"], pool["want"]
    return np.concatenate([want[int(vo[j]):int(vo[j + 1])] for j in lists])


def _server(pool, **kw):
    return vbyte.Server(pool["d"], pool["bo"], pool["vo"], True, pool["prev"], **kw)


@pytest.mark.parametrize("form", ["in_place", "per_list", "gather"])
def test_alone_and_in_the_mix_are_identical(pool, form):
    import torch
    srv = _server(pool, arena_bytes=64 << 20, staging_bytes=16 << 20, max_inflight=3, max_batch_queries=32,
                  form=form)
    _, qoff, qlists = inputs.query_stream(pool["lens"], 300, 1000.0, seed=32)
    probe = [int(x) for x in qlists[qoff[7]:qoff[8]]]
    # alone
    q = srv.submit(probe)
    _, st = srv.wait(q)
    assert st == 0
    vals, nq = srv.result(q)
    alone = vals.cpu().numpy().view(np.uint32).copy()
    assert nq == 1
    srv.release(q)
    assert np.array_equal(alone, _expected(pool, probe))
    # in the mix: everything submitted at once, the probe again in the middle
    ids = []
    for i in range(300):
        ids.append(srv.submit(qlists[qoff[i]:qoff[i + 1]]))
        if i == 150:
            pq = srv.submit(probe)
    for i, qi in enumerate(ids):
        _, st = srv.wait(qi)
        assert st == 0
        if i % 37 == 0:
            v, _ = srv.result(qi)
            assert np.array_equal(v.cpu().numpy().view(np.uint32), _expected(pool, qlists[qoff[i]:qoff[i + 1]]))
        srv.release(qi)
    srv.wait(pq)
    v, nq = srv.result(pq)
    mixed = v.cpu().numpy().view(np.uint32)
    assert nq > 1, "the probe should have shared its batch"
    assert np.array_equal(mixed, alone)
    srv.release(pq)
    s = srv.stats()
    assert s["queries"] == 302 and s["batches"] < 302
    srv.close()
    torch.cuda.synchronize()


@pytest.mark.parametrize("form", ["in_place", "gather"])
def test_admission_waits_for_arena_space(pool, form):
    # an arena that holds only a few queries' output at a time
    lens = pool["lens"]
    big = [int(j) for j in np.argsort(-lens)[:3]]
    need = int(lens[big].sum()) * 4
    srv = _server(pool, arena_bytes=need + 4096, staging_bytes=64 << 20, max_inflight=4, form=form)
    qs = [srv.submit(big) for _ in range(6)]
    for q in qs:
        _, st = srv.wait(q)
        assert st == 0
        v, _ = srv.result(q)
        assert np.array_equal(v.cpu().numpy().view(np.uint32), _expected(pool, big))
        srv.release(q)
    srv.close()


def test_replay_open_loop(pool):
    arr, qoff, qlists = inputs.query_stream(pool["lens"], 400, 20000.0, seed=33)
    srv = _server(pool, arena_bytes=256 << 20, staging_bytes=32 << 20, max_inflight=4)
    lat, st = srv.replay(arr, qoff, qlists)
    assert np.all(st == 0)
    assert np.all(lat > 0)
    s = srv.stats()
    assert s["queries"] == 400
    assert s["values"] == int(sum(pool["lens"][qlists[qoff[i]:qoff[i + 1]]].sum() for i in range(400)))
    srv.close()


def test_rejects_impossible_queries(pool):
    srv = _server(pool, arena_bytes=100_000, staging_bytes=1 << 20, max_batch_lists=4)
    with pytest.raises(vbyte.VByteError):
        srv.submit([pool["L"]])            # no such list
    with pytest.raises(vbyte.VByteError):
        srv.submit([0, 1, 2, 3, 4])        # more lists than a batch holds
    big = int(np.argmax(pool["lens"]))
    with pytest.raises(vbyte.VByteError):
        srv.submit([big])                  # output larger than the arena
    srv.close()

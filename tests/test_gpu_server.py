"""Serving form: continuous batching over many streams with resident state.

Checks: admission against the device-memory budget; every stream's results
equal the CPU oracle (chained ACBM / FSBM) and the same stream served alone;
requests submitted while steps are on the GPU are served in later steps.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def me():
    import torch
    assert torch.cuda.is_available()
    import paper_0710_4819_gb300 as me
    me.load_library(build_if_missing=True)
    return me


def _serve(me, specs, n_frames, mode=1, budget=8 << 30, max_inflight=2, order="interleave"):
    srv = me.Server(budget, max_inflight=max_inflight, mode=mode)
    seqs = [synth.stream_frames(s, n_frames)[:, :s.height] for s in specs]
    ids = [srv.open_stream(s.w, s.height, s.p, qp=28) for s in specs]
    reqs = []
    if order == "interleave":
        for t in range(n_frames):
            for i in range(len(specs)):
                reqs.append((i, t, srv.submit(ids[i], seqs[i][t])))
    else:
        for i in range(len(specs)):
            for t in range(n_frames):
                reqs.append((i, t, srv.submit(ids[i], seqs[i][t])))
    out = {}
    for i, t, r in reqs:
        has, lat, res = srv.wait(r, ids[i], timeout_ms=60000)
        assert has == (t > 0)
        assert lat >= 0
        if has:
            out[(i, t)] = res
    srv.close()
    return seqs, out


def test_server_admission_by_budget(me):
    one = 2 * 352 * 288 + 400 * 320 + 20 * 4 * 22 * 18   # about one CIF p16 stream
    srv = me.Server(int(2.6 * one) + 8192, mode=1)
    a = srv.open_stream(352, 288, 16)
    b = srv.open_stream(352, 288, 16)
    with pytest.raises(me.MeError) as e:
        srv.open_stream(352, 288, 16)
    assert e.value.status == 4
    used, n, _ = srv.stats()
    assert n == 2 and used > 0
    srv.close_stream(a)
    c = srv.open_stream(352, 288, 16)          # admitted once memory is back
    assert c not in (a, b)
    srv.close()


def test_server_acbm_matches_oracle_and_solo(me, orc):
    specs = [synth.StreamSpec("qcif", 176, 144, 16, 8001), synth.StreamSpec("cif", 352, 288, 16, 8002),
             synth.StreamSpec("qcif", 176, 144, 8, 8003), synth.StreamSpec("cif", 352, 288, 16, 8004),
             synth.StreamSpec("720p", 1280, 720, 32, 8005)]
    n = 4
    seqs, mixed = _serve(me, specs, n)
    lam = orc.lambda_q8(28)
    for i, s in enumerate(specs[:4]):
        prev = None
        for t in range(1, n):
            mv, J, mask, sad, load = orc.acbm(seqs[i][t], seqs[i][t - 1], 16, 16, s.p, lam,
                                              orc.params(qp=28), prev)
            prev = mv
            got = mixed[(i, t)]
            for k, w in dict(mv=mv, J=J, mask=mask, sad=sad, load=load).items():
                assert np.array_equal(got[k], w), f"stream {i} t={t} {k} vs oracle"
    # the same stream served alone gives the same bytes as in the mix
    for i in (1, 4):
        _, solo = _serve(me, [specs[i]], n)
        for t in range(1, n):
            for k in ("mv", "J", "mask", "sad", "load"):
                assert np.array_equal(solo[(0, t)][k], mixed[(i, t)][k]), f"stream {i} {k} solo"


def test_server_fsbm_mode(me, orc):
    specs = [synth.StreamSpec("qcif", 176, 144, 16, 8101), synth.StreamSpec("cif", 352, 288, 16, 8102)]
    seqs, out = _serve(me, specs, 3, mode=0, max_inflight=1)
    lam = orc.lambda_q8(28)
    for i, s in enumerate(specs):
        for t in (1, 2):
            mv, J, sad = orc.fsbm(seqs[i][t], seqs[i][t - 1], 16, 16, s.p, lam, nthreads=8)
            assert np.array_equal(out[(i, t)]["mv"], mv)
            assert np.array_equal(out[(i, t)]["J"], J)


def test_server_admits_work_while_busy(me):
    """Requests queued while earlier steps run are picked up by later steps:
    stream-major submission (all frames of stream 0 first) still finishes, and
    a stream opened after work started is served too."""
    specs = [synth.StreamSpec("cif", 352, 288, 16, 8201 + i) for i in range(6)]
    srv = me.Server(8 << 30, max_inflight=2, mode=1)
    seqs = [synth.stream_frames(s, 4) for s in specs]
    ids = [srv.open_stream(s.w, s.height, s.p) for s in specs[:5]]
    reqs = [(i, t, srv.submit(ids[i], seqs[i][t])) for i in range(5) for t in range(4)]
    late = srv.open_stream(352, 288, 16)
    reqs += [(5, t, srv.submit(late, seqs[5][t])) for t in range(4)]
    ids.append(late)
    done = 0
    for i, t, r in reqs:
        has, lat, res = srv.wait(r, ids[i], timeout_ms=60000)
        done += 1
        assert has == (t > 0)
    assert done == 24
    used, n, pending = srv.stats()
    assert pending == 0 and n == 6
    srv.close()


def test_server_random_arrivals_mixed_sizes(me):
    """Many steps of changing composition (random arrival order, uneven frame
    sizes and search ranges, two steps in flight): every stream's results
    equal its frames run through chained me_acbm calls."""
    import torch
    rng = np.random.default_rng(5)
    kinds = [("qcif", 176, 144, 16), ("cif", 352, 288, 16), ("cif", 352, 288, 24),
             ("720p", 1280, 720, 32)]
    specs = [synth.StreamSpec(k[0], k[1], k[2], k[3], 8301 + i) for i, k in
             enumerate([kinds[j] for j in rng.integers(0, len(kinds), size=10)])]
    n = 5
    seqs = [synth.stream_frames(s, n) for s in specs]
    srv = me.Server(8 << 30, max_inflight=2, mode=1)
    ids = [srv.open_stream(s.w, s.height, s.p, qp=28) for s in specs]
    order = [i for i in range(len(specs)) for _ in range(n)]
    rng.shuffle(order)
    nxt = [0] * len(specs)
    reqs = []
    for i in order:
        reqs.append((i, nxt[i], srv.submit(ids[i], seqs[i][nxt[i]])))
        nxt[i] += 1
    got = {}
    for i, t, r in reqs:
        has, lat, res = srv.wait(r, ids[i], timeout_ms=60000)
        if has:
            got[(i, t)] = res
    srv.close()
    lam = me.me_lambda_q8(28)
    for i, s in enumerate(specs):
        frames = torch.from_numpy(seqs[i]).cuda()
        prev = None
        for t in range(1, n):
            a = me.me_acbm(frames[t], frames[t - 1], 16, 16, s.p, lam, me.params(qp=28), prev_mv=prev)
            torch.cuda.synchronize()
            prev = a.mv
            assert np.array_equal(got[(i, t)]["mv"], a.mv.cpu().numpy()), (i, t)
            assert np.array_equal(got[(i, t)]["mask"], a.mask.cpu().numpy()), (i, t)
            assert np.array_equal(got[(i, t)]["J"], a.J.cpu().numpy().view(np.uint32)), (i, t)


"""Batched form: many uneven streams in one persistent launch per step
(captured CUDA graph).  Each stream's output must equal the CPU oracle and
the same stream run alone through me_fsbm / me_acbm, bit for bit.  Also the
bounded-wait failure path: a block that never publishes makes the step
return ME_ERR_TIMEOUT instead of hanging, and the GPU stays usable."""
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


def _alloc(me, H, W, N=16, M=16):
    import torch
    BH, BW = H // M, W // N
    return dict(mv=torch.full((BH, BW, 2), -9, dtype=torch.int16, device="cuda"),
                J=torch.full((BH, BW), -1, dtype=torch.int32, device="cuda"),
                mask=torch.full((BH, BW), 9, dtype=torch.uint8, device="cuda"),
                sad=torch.full((BH, BW), -1, dtype=torch.int32, device="cuda"),
                load=torch.full((BH, BW), -1, dtype=torch.int32, device="cuda"))


def _item(me, cur, ref, out, lam, prm, prev=None):
    it = me.BatchItem()
    it.cur, it.ref = cur.data_ptr(), ref.data_ptr()
    it.prev_mv = None if prev is None else prev.data_ptr()
    it.mv_out, it.J_out, it.mask_out = out["mv"].data_ptr(), out["J"].data_ptr(), out["mask"].data_ptr()
    it.sad_out, it.load_out = out["sad"].data_ptr(), out["load"].data_ptr()
    it.lambda_q8 = lam
    it.prm = prm
    return it


def _run_mix(me, specs, n_frames, mode, qp=28, check_oracle=None, orc=None):
    import torch
    lam = me.me_lambda_q8(qp)
    prm = me.params(qp=qp)
    seqs = [torch.from_numpy(synth.stream_frames(s, n_frames)).cuda() for s in specs]
    b = me.Batch()
    for s in specs:
        b.add_stream(s.w, s.height, 16, 16, s.p)
    prev = [None] * len(specs)
    results = []
    for t in range(1, n_frames):
        outs = [_alloc(me, s.height, s.w) for s in specs]
        items = [_item(me, seqs[i][t], seqs[i][t - 1], outs[i], lam, prm, prev[i])
                 for i in range(len(specs))]
        b.run(mode, items)
        b.sync()
        # each stream alone through the per-frame entry point
        for i, s in enumerate(specs):
            if mode == 0:
                alone = me.me_fsbm(seqs[i][t], seqs[i][t - 1], 16, 16, s.p, lam)
                pairs = (("mv", alone.mv), ("J", alone.J), ("sad", alone.sad))
            else:
                alone = me.me_acbm(seqs[i][t], seqs[i][t - 1], 16, 16, s.p, lam, prm, prev_mv=prev[i])
                pairs = (("mv", alone.mv), ("J", alone.J), ("sad", alone.sad),
                         ("mask", alone.mask), ("load", alone.load))
            torch.cuda.synchronize()
            for k, v in pairs:
                assert torch.equal(outs[i][k], v), f"stream {i} ({s.name}) t={t}: {k} differs alone"
        results.append((t, outs, [p for p in prev]))
        if mode == 1:
            prev = [o["mv"] for o in outs]
    b.close()
    return seqs, results


def test_batch_small_mix_fsbm_and_acbm_vs_oracle(me, orc):
    specs = [synth.StreamSpec("qcif", 176, 144, 16, 7001), synth.StreamSpec("cif", 352, 288, 16, 7002),
             synth.StreamSpec("qcif", 176, 144, 8, 7003), synth.StreamSpec("cif", 352, 288, 20, 7004)]
    lam = orc.lambda_q8(28)
    for mode in (0, 1):
        seqs, results = _run_mix(me, specs, 3, mode)
        prev_o = [None] * len(specs)
        for t, outs, _ in results:
            for i, s in enumerate(specs):
                cur = seqs[i][t].cpu().numpy()
                ref = seqs[i][t - 1].cpu().numpy()
                if mode == 0:
                    mv, J, sad = orc.fsbm(cur, ref, 16, 16, s.p, lam, nthreads=8)
                    want = dict(mv=mv, J=J, sad=sad)
                else:
                    mv, J, mask, sad, load = orc.acbm(cur, ref, 16, 16, s.p, lam, orc.params(qp=28),
                                                      prev_o[i])
                    want = dict(mv=mv, J=J, mask=mask, sad=sad, load=load)
                    prev_o[i] = mv
                for k, w in want.items():
                    g = outs[i][k].cpu().numpy()
                    if g.dtype == np.int32:
                        g = g.view(np.uint32)
                    assert np.array_equal(g, w), f"stream {i} t={t} {k} vs oracle"


def test_batch_64_stream_mix(me, orc):
    """The 64-stream mix (24 QCIF p16, 24 CIF p16, 12 720p p32, 4 2160p p64):
    every stream equals its solo run (both modes); QCIF/CIF/720p streams also
    equal the oracle in full, 2160p streams on sampled FSBM blocks and in full
    for ACBM on one stream."""
    specs = synth.batch_mix()
    lam = orc.lambda_q8(28)
    for mode in (0, 1):
        seqs, results = _run_mix(me, specs, 2, mode)
        t, outs, _ = results[0]
        for i, s in enumerate(specs):
            if s.name == "2160p" and not (mode == 1 and i == len(specs) - 1):
                if mode == 0:
                    rng = np.random.default_rng(i)
                    blocks = rng.choice(240 * 135, 12, replace=False).astype(np.int32)
                    mv, J, sad = orc.fsbm_blocks(seqs[i][1].cpu().numpy(), seqs[i][0].cpu().numpy(),
                                                 16, 16, 64, lam, blocks, nthreads=16)
                    assert np.array_equal(outs[i]["mv"].cpu().numpy().reshape(-1, 2)[blocks], mv)
                    assert np.array_equal(outs[i]["J"].cpu().numpy().ravel()[blocks].view(np.uint32), J)
                continue
            if s.name == "720p" and i % 4 != 0:
                continue
            cur, ref = seqs[i][1].cpu().numpy(), seqs[i][0].cpu().numpy()
            if mode == 0:
                mv, J, sad = orc.fsbm(cur, ref, 16, 16, s.p, lam, nthreads=16)
                want = dict(mv=mv, J=J, sad=sad)
            else:
                mv, J, mask, sad, load = orc.acbm(cur, ref, 16, 16, s.p, lam, orc.params(qp=28))
                want = dict(mv=mv, J=J, mask=mask, sad=sad, load=load)
            for k, w in want.items():
                g = outs[i][k].cpu().numpy()
                if g.dtype == np.int32:
                    g = g.view(np.uint32)
                assert np.array_equal(g, w), f"stream {i} ({s.name}) {k} vs oracle"


def test_batch_bounded_wait_reports_timeout(me):
    """A block that never publishes its vector: its dependents give up after
    the (short) limit, the step ends with ME_ERR_TIMEOUT, and the GPU stays
    usable for the next call."""
    import torch
    specs = [synth.StreamSpec("qcif", 176, 144, 8, 7101), synth.StreamSpec("qcif", 176, 144, 8, 7102)]
    b = me.Batch()
    for s in specs:
        b.add_stream(s.w, s.height, 16, 16, s.p)
    b.set_fault(timeout_ns=20_000_000, skip_stream=1, skip_block=3)
    seqs = [torch.from_numpy(synth.stream_frames(s, 2)).cuda() for s in specs]
    outs = [_alloc(me, s.height, s.w) for s in specs]
    lam = me.me_lambda_q8(28)
    items = [_item(me, seqs[i][1], seqs[i][0], outs[i], lam, me.params(qp=28)) for i in range(2)]
    b.run(1, items)
    with pytest.raises(me.MeError) as e:
        b.sync()
    assert e.value.status == 5
    b.close()
    # the context is still healthy
    r = me.me_fsbm(seqs[0][1], seqs[0][0], 16, 16, 8, lam)
    torch.cuda.synchronize()
    assert r.mv.shape == (9, 11, 2)


def test_two_batches_on_concurrent_streams(me):
    """Two ACBM steps in flight at once on different CUDA streams (their
    persistent launches share the SMs) both finish with their solo results."""
    import torch
    specs_a = [synth.StreamSpec("cif", 352, 288, 16, 7201 + i) for i in range(3)]
    specs_b = [synth.StreamSpec("720p", 1280, 720, 32, 7301 + i) for i in range(2)]
    lam = me.me_lambda_q8(28)
    prm = me.params(qp=28)
    runs = []
    for specs in (specs_a, specs_b):
        b = me.Batch()
        for s in specs:
            b.add_stream(s.w, s.height, 16, 16, s.p)
        seqs = [torch.from_numpy(synth.stream_frames(s, 2)).cuda() for s in specs]
        outs = [_alloc(me, s.height, s.w) for s in specs]
        items = [_item(me, seqs[i][1], seqs[i][0], outs[i], lam, prm) for i in range(len(specs))]
        runs.append((b, specs, seqs, outs, items))
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    torch.cuda.synchronize()
    for _ in range(3):
        for (b, specs, seqs, outs, items), st in zip(runs, streams):
            b.run(1, items, stream=st)
        for (b, *_), st in zip(runs, streams):
            b.sync(stream=st)
    for b, specs, seqs, outs, items in runs:
        for i, s in enumerate(specs):
            alone = me.me_acbm(seqs[i][1], seqs[i][0], 16, 16, s.p, lam, prm)
            torch.cuda.synchronize()
            for k, v in (("mv", alone.mv), ("J", alone.J), ("mask", alone.mask), ("load", alone.load)):
                assert torch.equal(outs[i][k], v), (s.name, k)
        b.close()


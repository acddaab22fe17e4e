"""The autotuner: every launch form it may pick gives the same bytes, and it
picks by measurement.

For each tuned entry point (me_fsbm_sequence / me_fsbm through the tuned
full search, me_acbm_sequence) every candidate is forced in turn
(ME_TUNE_FORCE) on a small case and compared with the oracle; the number of
candidates comes from the tuner's own record, so a candidate list that grows
is covered too."""
import os
import re

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


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _candidates(me, prefix):
    """Candidate names of the tuner's line for a shape (prefix: 'fsbm 352x288 16x16 p=16 K=3')."""
    for ln in me.me_tune_log().splitlines():
        if ln.startswith(prefix + " "):
            return [c.strip().rsplit(" ", 2)[0] for c in ln.split("|")[1:]]
    return None


def _line(me, prefix):
    for ln in me.me_tune_log().splitlines():
        if ln.startswith(prefix + " "):
            return ln
    return None


class _Force:
    def __init__(self, c):
        self.c = c

    def __enter__(self):
        self.old = os.environ.get("ME_TUNE_FORCE")
        os.environ["ME_TUNE_FORCE"] = str(self.c)

    def __exit__(self, *a):
        if self.old is None:
            os.environ.pop("ME_TUNE_FORCE", None)
        else:
            os.environ["ME_TUNE_FORCE"] = self.old


@pytest.mark.parametrize("w,h,N,M,p,K", [(352, 288, 16, 16, 16, 3), (208, 96, 8, 8, 7, 2),
                                         (176, 144, 16, 8, 12, 1), (128, 64, 4, 4, 40, 1),
                                         (96, 64, 4, 16, 64, 2), (160, 48, 8, 4, 33, 1),
                                         (112, 96, 16, 4, 20, 2), (96, 112, 8, 16, 50, 1),
                                         (64, 80, 4, 8, 9, 2), (192, 64, 16, 16, 64, 1)])
def test_every_fsbm_candidate_gives_the_oracle(me, orc, w, h, N, M, p, K):
    import torch
    seq = synth.scene_sequence(300 + w + N + p, w, h, K + 1, n_objects=4, vmax=5)
    frames = torch.from_numpy(seq).cuda()
    lam = orc.lambda_q8(28)
    r = me.me_fsbm_sequence(frames, N, M, p, lam)          # the tuned first call
    torch.cuda.synchronize()
    prefix = f"fsbm {w}x{h} {N}x{M} p={p} K={K}"
    names = _candidates(me, prefix)
    assert names and len(names) >= 2, me.me_tune_log()
    want = [orc.fsbm(seq[k + 1], seq[k], N, M, p, lam, nthreads=8) for k in range(K)]
    for c in range(len(names)):
        with _Force(c):
            r = me.me_fsbm_sequence(frames, N, M, p, lam)
            torch.cuda.synchronize()
        assert me.me_fsbm_sequence_status() == 0
        for k, (mv, J, sad) in enumerate(want):
            assert np.array_equal(r.mv[k].cpu().numpy(), mv), (names[c], k)
            assert np.array_equal(_u32(r.J[k]), J), (names[c], k)
            assert np.array_equal(_u32(r.sad[k]), sad), (names[c], k)
    if K == 1:
        # the single-pair call goes through the same tuned forms
        for c in range(len(names)):
            with _Force(c):
                f = me.me_fsbm(frames[1], frames[0], N, M, p, lam)
                torch.cuda.synchronize()
            assert np.array_equal(f.mv.cpu().numpy(), want[0][0]), names[c]
            assert np.array_equal(_u32(f.J), want[0][1]), names[c]


@pytest.mark.parametrize("name,N,M,p,K", [("cif", 16, 16, 16, 4), ("cif", 8, 8, 8, 3),
                                          ("qcif", 16, 16, 32, 3)])
def test_every_acbm_sequence_candidate_gives_the_chained_oracle(me, orc, name, N, M, p, K):
    import torch
    seq = synth.config_sequence(name, seed=71 + N + p, n_frames=K + 1)
    H, W = seq.shape[1:]
    frames = torch.from_numpy(seq).cuda()
    lam = orc.lambda_q8(30)
    prm = me.params(qp=30)
    me.me_acbm_sequence(frames, N, M, p, lam, prm)        # the tuned first call
    torch.cuda.synchronize()
    prefix = f"acbm_sequence {W}x{H} {N}x{M} p={p} K={K}"
    names = _candidates(me, prefix)
    assert names and len(names) >= 2, me.me_tune_log()
    want, prev = [], None
    for k in range(K):
        out = orc.acbm(seq[k + 1], seq[k], N, M, p, lam, orc.params(qp=30), prev)
        prev = out[0]
        want.append(out)
    for c in range(len(names)):
        with _Force(c):
            r = me.me_acbm_sequence(frames, N, M, p, lam, prm)
            torch.cuda.synchronize()
        me.me_acbm_sequence_status(W, H, N, M, p, K)
        for k, (mv, J, mask, sad, load) in enumerate(want):
            for nm, g, w_ in (("mv", r.mv[k].cpu().numpy(), mv), ("J", _u32(r.J[k]), J),
                              ("mask", r.mask[k].cpu().numpy(), mask), ("sad", _u32(r.sad[k]), sad),
                              ("load", _u32(r.load[k]), load)):
                assert np.array_equal(g, w_), (names[c], k, nm)


def test_tuner_times_every_candidate_and_keeps_the_fastest(me):
    import torch
    seq = synth.config_sequence("cif", seed=5, n_frames=6)
    frames = torch.from_numpy(seq).cuda()
    lam = me.me_lambda_q8(28)
    me.me_acbm_sequence(frames, 16, 16, 16, lam, me.params(qp=28))
    me.me_fsbm_sequence(frames, 16, 16, 16, lam)
    torch.cuda.synchronize()
    for prefix in ("acbm_sequence 352x288 16x16 p=16 K=5", "fsbm 352x288 16x16 p=16 K=5"):
        ln = _line(me, prefix)
        assert ln is not None and " tuned:" in ln, me.me_tune_log()
        chosen = re.search(r"chosen=(.+?) \|", ln).group(1)
        times = {c.strip().rsplit(" ", 2)[0]: float(c.strip().rsplit(" ", 2)[1])
                 for c in ln.split("|")[1:]}
        assert all(t > 0 for t in times.values()), ln
        assert times[chosen] == min(times.values()), ln


def test_every_batch_step_form_gives_the_oracle(me, orc):
    """The batch's step forms (FSBM: per-group persistent kernel, any-p
    pipeline; ACBM: each run length with and without speculative searches),
    each forced on a fresh batch of three uneven streams over two steps,
    against the oracle (FSBM per pair, ACBM chained)."""
    import torch
    specs = [synth.StreamSpec("qcif", 176, 144, 16, 8101), synth.StreamSpec("cif", 352, 288, 16, 8102),
             synth.StreamSpec("qcif", 176, 144, 32, 8103)]
    seqs_np = [synth.stream_frames(s, 3) for s in specs]
    seqs = [torch.from_numpy(x).cuda() for x in seqs_np]
    lam = me.me_lambda_q8(28)
    prm = me.params(qp=28)
    want_f = [[orc.fsbm(x[t], x[t - 1], 16, 16, s.p, lam) for t in (1, 2)] for x, s in zip(seqs_np, specs)]
    want_a = []
    for x, s in zip(seqs_np, specs):
        prev, w = None, []
        for t in (1, 2):
            out = orc.acbm(x[t], x[t - 1], 16, 16, s.p, lam, orc.params(qp=28), prev)
            prev = out[0]
            w.append(out)
        want_a.append(w)
    for mode, n_forms in ((0, 2), (1, 8)):
        for c in range(n_forms):
            with _Force(c):
                b = me.Batch()
                for s in specs:
                    b.add_stream(s.w, s.height, 16, 16, s.p)
                prev = [None] * len(specs)
                for t in (1, 2):
                    outs = []
                    items = []
                    for i, s in enumerate(specs):
                        BH, BW = s.height // 16, s.w // 16
                        o = dict(mv=torch.full((BH, BW, 2), -9, dtype=torch.int16, device="cuda"),
                                 J=torch.full((BH, BW), -1, dtype=torch.int32, device="cuda"),
                                 mask=torch.full((BH, BW), 9, dtype=torch.uint8, device="cuda"),
                                 sad=torch.full((BH, BW), -1, dtype=torch.int32, device="cuda"),
                                 load=torch.full((BH, BW), -1, dtype=torch.int32, device="cuda"))
                        it = me.BatchItem()
                        it.cur, it.ref = seqs[i][t].data_ptr(), seqs[i][t - 1].data_ptr()
                        it.prev_mv = None if prev[i] is None else prev[i].data_ptr()
                        it.mv_out, it.J_out, it.mask_out = o["mv"].data_ptr(), o["J"].data_ptr(), o["mask"].data_ptr()
                        it.sad_out, it.load_out = o["sad"].data_ptr(), o["load"].data_ptr()
                        it.lambda_q8 = lam
                        it.prm = prm
                        outs.append(o)
                        items.append(it)
                    b.run(mode, items)
                    b.sync()
                    for i in range(len(specs)):
                        o = outs[i]
                        if mode == 0:
                            mv, J, sad = want_f[i][t - 1]
                            checks = (("mv", o["mv"].cpu().numpy(), mv), ("J", _u32(o["J"]), J),
                                      ("sad", _u32(o["sad"]), sad))
                        else:
                            mv, J, mask, sad, load = want_a[i][t - 1]
                            checks = (("mv", o["mv"].cpu().numpy(), mv), ("J", _u32(o["J"]), J),
                                      ("mask", o["mask"].cpu().numpy(), mask),
                                      ("sad", _u32(o["sad"]), sad), ("load", _u32(o["load"]), load))
                        for nm, g, w_ in checks:
                            assert np.array_equal(g, w_), (mode, c, i, t, nm)
                    if mode == 1:
                        prev = [o["mv"] for o in outs]
                b.close()


@pytest.mark.parametrize("w,h,N,M,p", [(352, 288, 16, 16, 16), (208, 96, 8, 8, 7), (176, 144, 16, 8, 12),
                                       (128, 64, 4, 4, 40), (96, 64, 4, 16, 64), (160, 48, 8, 4, 33)])
def test_every_acbm_pair_candidate_gives_the_oracle(me, orc, w, h, N, M, p):
    """me_acbm's forms (the wave graph, the persistent kernel over one pair in
    each of its launch forms), each forced over two chained pairs, against
    the oracle chained the same way."""
    import torch
    seq = synth.scene_sequence(500 + w + N + p, w, h, 3, n_objects=4, vmax=5)
    frames = torch.from_numpy(seq).cuda()
    lam = orc.lambda_q8(30)
    prm = me.params(qp=30)
    me.me_acbm(frames[1], frames[0], N, M, p, lam, prm)        # the tuned first call
    torch.cuda.synchronize()
    names = _candidates(me, f"acbm {w}x{h} {N}x{M} p={p}")
    assert names and names[0] == "waves" and len(names) >= 2, me.me_tune_log()
    want, prev = [], None
    for k in range(2):
        out = orc.acbm(seq[k + 1], seq[k], N, M, p, lam, orc.params(qp=30), prev)
        prev = out[0]
        want.append(out)
    for c in range(len(names)):
        prev = None
        for k, (mv, J, mask, sad, load) in enumerate(want):
            with _Force(c):
                r = me.me_acbm(frames[k + 1], frames[k], N, M, p, lam, prm, prev_mv=prev)
                torch.cuda.synchronize()
            if c > 0:
                me.me_acbm_sequence_status(w, h, N, M, p, 1)   # raises on a run that timed out
            for nm, g, w_ in (("mv", r.mv.cpu().numpy(), mv), ("J", _u32(r.J), J),
                              ("mask", r.mask.cpu().numpy(), mask), ("sad", _u32(r.sad), sad),
                              ("load", _u32(r.load), load)):
                assert np.array_equal(g, w_), (names[c], k, nm)
            prev = r.mv.clone()

"""Sequence calls: FSBM / ACBM over K consecutive frame pairs in one launch.

ACBM pairs overlap on the GPU (a block of pair k waits only for its spatial
neighbours in pair k and its 3x3 neighbourhood in pair k-1), so these tests
check that the result is exactly that of K chained single-pair runs: against
the oracle chained frame by frame and against chained me_acbm calls."""
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


def test_fsbm_sequence_matches_oracle(me, orc):
    import torch
    seq = synth.config_sequence("qcif", seed=41)
    lam = orc.lambda_q8(28)
    r = me.me_fsbm_sequence(torch.from_numpy(seq).cuda(), 16, 16, 16, lam)
    torch.cuda.synchronize()
    for k in range(seq.shape[0] - 1):
        mv, J, sad = orc.fsbm(seq[k + 1], seq[k], 16, 16, 16, lam, nthreads=8)
        assert np.array_equal(r.mv[k].cpu().numpy(), mv), k
        assert np.array_equal(_u32(r.J[k]), J), k
        assert np.array_equal(_u32(r.sad[k]), sad), k


@pytest.mark.parametrize("w,h,p,K", [(176, 144, 16, 9), (352, 288, 16, 4), (352, 288, 34, 3),
                                     (1280, 720, 32, 3), (208, 48, 9, 5), (16, 16, 12, 2)])
def test_fsbm_sequence_pipelined_matches_oracle(me, orc, w, h, p, K, monkeypatch):
    """The persistent staging/searching form (16x16, run length 13) against
    the oracle pair by pair and against the one-launch-per-group form, on
    grids whose last group of a row is short (11, 22, 13 and 1 blocks per row
    against 8 per group) and on several pairs per CTA."""
    import torch
    seq = synth.scene_sequence(900 + w + p, w, h, K + 1, n_objects=4, vmax=5)
    lam = orc.lambda_q8(30)
    frames = torch.from_numpy(seq).cuda()
    r = me.me_fsbm_sequence(frames, 16, 16, p, lam)
    assert me.me_fsbm_sequence_status() == 0
    monkeypatch.setenv("ME_FSBM_PIPE", "0")
    r0 = me.me_fsbm_sequence(frames, 16, 16, p, lam)
    torch.cuda.synchronize()
    assert torch.equal(r.mv, r0.mv) and torch.equal(r.J, r0.J) and torch.equal(r.sad, r0.sad)
    for k in range(K):
        mv, J, sad = orc.fsbm(seq[k + 1], seq[k], 16, 16, p, lam, nthreads=8)
        assert np.array_equal(r.mv[k].cpu().numpy(), mv), k
        assert np.array_equal(_u32(r.J[k]), J), k
        assert np.array_equal(_u32(r.sad[k]), sad), k


def test_fsbm_sequence_pipelined_64_pairs(me, orc, monkeypatch):
    """The largest sequence a call takes (64 pairs, QCIF, p = 16): every pair
    equal to the per-group kernel's, and the first and last to the oracle."""
    import torch
    seq = synth.config_sequence("qcif", seed=77, n_frames=65)
    lam = orc.lambda_q8(28)
    frames = torch.from_numpy(seq).cuda()
    r = me.me_fsbm_sequence(frames, 16, 16, 16, lam)
    assert me.me_fsbm_sequence_status() == 0
    monkeypatch.setenv("ME_FSBM_PIPE", "0")
    r0 = me.me_fsbm_sequence(frames, 16, 16, 16, lam)
    torch.cuda.synchronize()
    assert torch.equal(r.mv, r0.mv) and torch.equal(r.J, r0.J) and torch.equal(r.sad, r0.sad)
    for k in (0, 63):
        mv, J, sad = orc.fsbm(seq[k + 1], seq[k], 16, 16, 16, lam, nthreads=8)
        assert np.array_equal(r.mv[k].cpu().numpy(), mv), k
        assert np.array_equal(_u32(r.J[k]), J), k


def test_fsbm_sequence_pipelined_1080p_equals_per_pair(me, orc, monkeypatch):
    """1080p p = 32, 12 pairs in one launch (the bench's kernel): equal to
    me_fsbm per pair, to the per-group kernel over the same sequence, and to
    the oracle on sampled blocks (corners, edges, random) of the first and
    last pair."""
    import torch
    seq_np = synth.config_sequence("1080p", seed=7, n_frames=13)
    seq = torch.from_numpy(seq_np).cuda()
    lam = me.me_lambda_q8(28)
    r = me.me_fsbm_sequence(seq, 16, 16, 32, lam)
    assert me.me_fsbm_sequence_status() == 0
    for k in range(12):
        f = me.me_fsbm(seq[k + 1], seq[k], 16, 16, 32, lam)
        torch.cuda.synchronize()
        assert torch.equal(r.mv[k], f.mv) and torch.equal(r.J[k], f.J) and torch.equal(r.sad[k], f.sad), k
    monkeypatch.setenv("ME_FSBM_PIPE", "0")
    r0 = me.me_fsbm_sequence(seq, 16, 16, 32, lam)
    torch.cuda.synchronize()
    assert torch.equal(r.mv, r0.mv) and torch.equal(r.J, r0.J) and torch.equal(r.sad, r0.sad)
    BW, BH = 120, 68
    rng = np.random.default_rng(3)
    blocks = np.unique(np.concatenate([[0, BW - 1, (BH - 1) * BW, BH * BW - 1, 7 * BW + 8, 8 * BW - 1],
                                       rng.integers(0, BW * BH, 30)])).astype(np.int32)
    for k in (0, 11):
        mv, J, sad = orc.fsbm_blocks(seq_np[k + 1], seq_np[k], 16, 16, 32, lam, blocks, nthreads=8)
        assert np.array_equal(r.mv[k].cpu().numpy().reshape(-1, 2)[blocks], mv), k
        assert np.array_equal(_u32(r.J[k]).ravel()[blocks], J), k
        assert np.array_equal(_u32(r.sad[k]).ravel()[blocks], sad), k


def test_bench_step_matches_chained_oracle(me, orc):
    """The benchmark's own step: 1080p p = 32, Qp 28, the 60-frame sequence of
    seed 2026 with all 59 pairs in one me_fsbm_sequence and one
    me_acbm_sequence launch.  ACBM: the first 8 pairs equal the oracle chained
    pair by pair (mv, J, mask, SAD, load); every pair keeps the properties
    that hold at any length (a full-searched block equals FSBM with load
    (2p+1)^2, FSBM J <= ACBM J, other loads within the PBM bound).  FSBM:
    whole frames of pairs 0, 29 and 58 and sampled blocks of every pair
    against the oracle."""
    import os
    import torch
    nthr = os.cpu_count() or 8
    seq_np = synth.config_sequence("1080p", seed=2026, n_frames=60)
    frames = torch.from_numpy(seq_np).cuda()
    lam = orc.lambda_q8(28)
    fs = me.me_fsbm_sequence(frames, 16, 16, 32, lam)
    ac = me.me_acbm_sequence(frames, 16, 16, 32, lam, me.params(qp=28))
    torch.cuda.synchronize()
    assert me.me_fsbm_sequence_status() == 0
    me.me_acbm_sequence_status(1920, 1088, 16, 16, 32, 59)     # raises on a timed-out wait
    f_mv, f_J, f_sad = fs.mv.cpu().numpy(), _u32(fs.J), _u32(fs.sad)
    a_mv, a_J, a_mask = ac.mv.cpu().numpy(), _u32(ac.J), ac.mask.cpu().numpy()
    a_sad, a_load = _u32(ac.sad), _u32(ac.load)
    prev = None
    for k in range(8):
        mv, J, mask, sad, load = orc.acbm(seq_np[k + 1], seq_np[k], 16, 16, 32, lam,
                                          orc.params(qp=28), prev)
        prev = mv
        for nm, g, w in (("mv", a_mv[k], mv), ("J", a_J[k], J), ("mask", a_mask[k], mask),
                         ("sad", a_sad[k], sad), ("load", a_load[k], load)):
            assert np.array_equal(g, w), (k, nm)
    BW, BH = 120, 68
    rng = np.random.default_rng(11)
    for k in range(59):
        fsb = a_mask[k] == 1
        assert fsb.any() and not fsb.all(), k
        assert np.array_equal(a_mv[k][fsb], f_mv[k][fsb]) and np.array_equal(a_J[k][fsb], f_J[k][fsb]), k
        assert np.all(a_load[k][fsb] == 65 * 65) and np.all(a_load[k][~fsb] <= 22), k
        assert np.all(f_J[k] <= a_J[k]), k
        blocks = rng.choice(BW * BH, 24, replace=False).astype(np.int32)
        mv, J, sad = orc.fsbm_blocks(seq_np[k + 1], seq_np[k], 16, 16, 32, lam, blocks, nthreads=nthr)
        assert np.array_equal(f_mv[k].reshape(-1, 2)[blocks], mv), k
        assert np.array_equal(f_J[k].ravel()[blocks], J) and np.array_equal(f_sad[k].ravel()[blocks], sad), k
    for k in (0, 29, 58):
        mv, J, sad = orc.fsbm(seq_np[k + 1], seq_np[k], 16, 16, 32, lam, nthreads=nthr)
        assert np.array_equal(f_mv[k], mv) and np.array_equal(f_J[k], J) and np.array_equal(f_sad[k], sad), k


@pytest.mark.parametrize("name,n,p,qp", [("qcif", 10, 16, 28), ("cif", 5, 16, 40),
                                         ("1080p", 3, 32, 28)])
def test_acbm_sequence_matches_chained_oracle(me, orc, name, n, p, qp):
    import torch
    seq = synth.config_sequence(name, seed=42, n_frames=n)
    lam = orc.lambda_q8(qp)
    frames = torch.from_numpy(seq).cuda()
    r = me.me_acbm_sequence(frames, 16, 16, p, lam, me.params(qp=qp))
    me.me_acbm_sequence_status(seq.shape[2], seq.shape[1], 16, 16, p, n - 1)
    prev = None
    fs = 0
    for k in range(n - 1):
        mv, J, mask, sad, load = orc.acbm(seq[k + 1], seq[k], 16, 16, p, lam, orc.params(qp=qp), prev)
        prev = mv
        assert np.array_equal(r.mv[k].cpu().numpy(), mv), (name, k, "mv")
        assert np.array_equal(_u32(r.J[k]), J), (name, k, "J")
        assert np.array_equal(r.mask[k].cpu().numpy(), mask), (name, k, "mask")
        assert np.array_equal(_u32(r.sad[k]), sad), (name, k, "sad")
        assert np.array_equal(_u32(r.load[k]), load), (name, k, "load")
        fs += int(mask.sum())
    assert fs > 0


@pytest.mark.parametrize("N,M", [(8, 8), (16, 8), (4, 4)])
def test_acbm_sequence_equals_chained_calls(me, N, M):
    import torch
    seq = synth.scene_sequence(43, 12 * N, 9 * M, 6, n_objects=3, vmax=3)
    frames = torch.from_numpy(seq).cuda()
    lam = me.me_lambda_q8(28)
    for kw in (dict(qp=28), dict(qp=28, refine=0), dict(alpha=0, beta=0, gamma_num=0, qp=28)):
        prm = me.params(**kw)
        r = me.me_acbm_sequence(frames, N, M, 5, lam, prm)
        prev = None
        for k in range(5):
            a = me.me_acbm(frames[k + 1], frames[k], N, M, 5, lam, prm, prev_mv=prev)
            torch.cuda.synchronize()
            for x, y in ((r.mv[k], a.mv), (r.J[k], a.J), (r.mask[k], a.mask), (r.sad[k], a.sad),
                         (r.load[k], a.load)):
                assert torch.equal(x, y), (N, M, kw, k)
            prev = a.mv


def test_sequence_with_given_prev_field_and_repeat_runs(me, orc):
    """A sequence continuing from a given field; the same plan run twice."""
    import torch
    seq = synth.config_sequence("qcif", seed=44)
    lam = orc.lambda_q8(28)
    frames = torch.from_numpy(seq).cuda()
    first = me.me_acbm_sequence(frames[:4], 16, 16, 16, lam, me.params(qp=28))
    prev = first.mv[2].contiguous()
    for _ in range(2):
        r = me.me_acbm_sequence(frames[3:7], 16, 16, 16, lam, me.params(qp=28), prev_mv=prev)
        torch.cuda.synchronize()
        p_o = prev.cpu().numpy()
        for k in range(3):
            mv, J, mask, sad, load = orc.acbm(seq[4 + k], seq[3 + k], 16, 16, 16, lam,
                                              orc.params(qp=28), p_o)
            p_o = mv
            assert np.array_equal(r.mv[k].cpu().numpy(), mv)
            assert np.array_equal(r.mask[k].cpu().numpy(), mask)


def test_sequence_argument_errors(me):
    import torch
    f = torch.zeros((70, 32, 32), dtype=torch.uint8, device="cuda")
    with pytest.raises(me.MeError) as e:
        me.me_fsbm_sequence(f, 16, 16, 4, 0)          # K = 69 > 64
    assert e.value.status == 1
    with pytest.raises(me.MeError) as e:
        me.me_acbm_sequence(f[:3, :, :30].contiguous(), 16, 16, 4, 0, me.params())
    assert e.value.status == 2


@pytest.mark.parametrize("env,n", [({"ME_SEQ_S": "2"}, 6), ({"ME_SEQ_S": "3"}, 7),
                                   ({"ME_SEQ_T": "8"}, 8), ({"ME_SEQ_T": "11"}, 9),
                                   ({"ME_SEQ_T": "16", "ME_SEQ_S": "2"}, 10)])
def test_acbm_sequence_tile_options_match_chained_oracle(me, orc, env, n):
    """The sequence plan's tuning options give the same bytes: full searches
    split over S CTAs by columns (merged by an atomic minimum on the packed
    key, the last slice publishing) and other run lengths.  Each case uses
    its own sequence length, so it gets a plan of its own."""
    import os
    import torch
    seq = synth.config_sequence("cif", seed=60 + n, n_frames=n)
    lam = orc.lambda_q8(34)
    saved = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        r = me.me_acbm_sequence(torch.from_numpy(seq).cuda(), 16, 16, 20, lam, me.params(qp=34))
        me.me_acbm_sequence_status(seq.shape[2], seq.shape[1], 16, 16, 20, n - 1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    prev = None
    fs = 0
    for k in range(n - 1):
        mv, J, mask, sad, load = orc.acbm(seq[k + 1], seq[k], 16, 16, 20, lam, orc.params(qp=34), prev)
        prev = mv
        assert np.array_equal(r.mv[k].cpu().numpy(), mv), (env, k, "mv")
        assert np.array_equal(_u32(r.J[k]), J), (env, k, "J")
        assert np.array_equal(r.mask[k].cpu().numpy(), mask), (env, k, "mask")
        assert np.array_equal(_u32(r.load[k]), load), (env, k, "load")
        fs += int(mask.sum())
    assert fs > 0          # the searches (and their slices) ran

"""SAD_min / SAD_deviation (Sec. 3.1) and the known-motion experiment
(Fig. 3) on the GPU: bit-exact against the oracle for every block shape, a
range of search ranges (all run lengths of the 16x16 plans), extreme pixel
values at the largest range, sampled blocks of a 1080p frame at p = 32, and
the ten-frame global-motion study."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

SHAPES = [(16, 16), (16, 8), (16, 4), (8, 16), (8, 8), (8, 4), (4, 16), (4, 8), (4, 4)]


@pytest.fixture(scope="module")
def me():
    import torch
    assert torch.cuda.is_available()
    import paper_0710_4819_gb300 as me
    me.load_library(build_if_missing=True)
    return me


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _run(me, cur, ref, N, M, p, lam):
    import torch
    r = me.me_sad_deviation(torch.from_numpy(cur).cuda(), torch.from_numpy(ref).cuda(), N, M, p, lam)
    torch.cuda.synchronize()
    return r


def _check(me, orc, cur, ref, N, M, p, lam, tag):
    r = _run(me, cur, ref, N, M, p, lam)
    mn, dev = orc.sad_deviation(cur, ref, N, M, p)
    assert np.array_equal(_u32(r.sad_min), mn), (tag, "sad_min")
    assert np.array_equal(_u32(r.sad_dev), dev), (tag, "sad_dev")
    mv, J, _ = orc.fsbm(cur, ref, N, M, p, lam, nthreads=8)
    assert np.array_equal(r.mv.cpu().numpy(), mv), (tag, "mv")
    assert np.array_equal(_u32(r.J), J), (tag, "J")


@pytest.mark.parametrize("N,M", SHAPES)
def test_sad_deviation_all_shapes_vs_oracle(me, orc, N, M):
    rng = np.random.default_rng(N * 17 + M)
    ref = synth.texture(rng, 96, 48)
    cur = np.clip(np.roll(ref, (2, -3), axis=(0, 1)).astype(int) + rng.integers(-8, 9, ref.shape),
                  0, 255).astype(np.uint8)
    for p in (1, 3, 6):
        for lam in (0, 6595):
            _check(me, orc, cur, ref, N, M, p, lam, (N, M, p, lam))


@pytest.mark.parametrize("p", [1, 2, 4, 7, 8, 12, 16, 20, 32])
def test_sad_deviation_16x16_search_ranges(me, orc, p):
    """QCIF (11 x 9 blocks: ragged CTA groups) over search ranges whose plans
    take every instantiated run length."""
    seq = synth.config_sequence("qcif", seed=300 + p, n_frames=2)
    _check(me, orc, seq[1], seq[0], 16, 16, p, orc.lambda_q8(28), ("qcif", p))


def test_sad_deviation_extremes_at_the_largest_range(me, orc):
    """p = 64 with saturated pixels: the largest SAD sums the kernel handles."""
    rng = np.random.default_rng(9)
    W = H = 128
    cur = np.full((H, W), 255, np.uint8)
    ref = np.zeros((H, W), np.uint8)
    r = _run(me, cur, ref, 16, 16, 64, 0)
    assert np.all(_u32(r.sad_min) == 255 * 256) and np.all(_u32(r.sad_dev) == 0)
    ref = (rng.integers(0, 2, (H, W)) * 255).astype(np.uint8)
    cur = (rng.integers(0, 2, (H, W)) * 255).astype(np.uint8)
    for N, M in [(16, 16), (4, 4)]:
        _check(me, orc, cur, ref, N, M, 64, 0, ("extreme", N, M))


def test_sad_deviation_single_block_frames(me, orc):
    rng = np.random.default_rng(4)
    for N, M, p in [(16, 16, 9), (4, 8, 3), (8, 4, 1)]:
        ref = rng.integers(0, 256, (M, N)).astype(np.uint8)
        cur = rng.integers(0, 256, (M, N)).astype(np.uint8)
        _check(me, orc, cur, ref, N, M, p, 0, ("one block", N, M, p))


def test_sad_deviation_1080p_sampled(me, orc):
    """The full-size frame (1920x1088, 16x16, p = 32): sampled blocks against
    the oracle one by one (corners, edges, interior), and at every block the
    properties that hold at any size: SAD_min equals the SAD of the lambda = 0
    full-search winner and is at most that of the lambda > 0 winner."""
    import torch
    seq = synth.config_sequence("1080p", seed=77, n_frames=2)     # 1920 x 1088 (padded rows)
    cur, ref = np.ascontiguousarray(seq[1]), np.ascontiguousarray(seq[0])
    N = M = 16
    p = 32
    BW, BH = cur.shape[1] // N, cur.shape[0] // M
    lam = orc.lambda_q8(28)
    r = _run(me, cur, ref, N, M, p, lam)
    r0 = _run(me, cur, ref, N, M, p, 0)
    rng = np.random.default_rng(1)
    blocks = np.unique(np.concatenate([
        [0, BW - 1, (BH - 1) * BW, BH * BW - 1, BW, 2 * BW - 1],
        rng.integers(0, BW * BH, 40)])).astype(np.int32)
    mn, dev = orc.sad_deviation_blocks(cur, ref, N, M, p, blocks)
    assert np.array_equal(_u32(r.sad_min).ravel()[blocks], mn)
    assert np.array_equal(_u32(r.sad_dev).ravel()[blocks], dev)
    assert np.array_equal(_u32(r0.sad_min), _u32(r.sad_min))
    assert np.array_equal(_u32(r0.sad_dev), _u32(r.sad_dev))
    f0 = me.me_fsbm(torch.from_numpy(cur).cuda(), torch.from_numpy(ref).cuda(), N, M, p, 0)
    f1 = me.me_fsbm(torch.from_numpy(cur).cuda(), torch.from_numpy(ref).cuda(), N, M, p, lam)
    torch.cuda.synchronize()
    assert np.array_equal(_u32(f0.sad), _u32(r.sad_min))
    assert np.all(_u32(r.sad_min) <= _u32(f1.sad))
    assert np.array_equal(r.mv.cpu().numpy(), f1.mv.cpu().numpy())


def _study_oracle(orc, frames, g, N, M, p, lam):
    K = len(g)
    out = {k: [] for k in ("mv", "intra", "sad_min", "sad_dev", "err")}
    for k in range(1, K + 1):
        mv, _, _ = orc.fsbm(frames[k], frames[0], N, M, p, lam, nthreads=8)
        mn, dev = orc.sad_deviation(frames[k], frames[0], N, M, p)
        err = np.abs(mv[..., 0].astype(int) - g[k - 1, 0]) + np.abs(mv[..., 1].astype(int) - g[k - 1, 1])
        out["mv"].append(mv)
        out["intra"].append(orc.intra_sad(frames[k], N, M))
        out["sad_min"].append(mn)
        out["sad_dev"].append(dev)
        out["err"].append(np.minimum(err, 255).astype(np.uint8))
    return {k: np.stack(v) for k, v in out.items()}


def _study(me, frames, g, N, M, p, lam):
    import torch
    r = me.me_motion_study(torch.from_numpy(frames).cuda(), torch.from_numpy(g).cuda(), N, M, p, lam)
    torch.cuda.synchronize()
    return dict(mv=r.mv.cpu().numpy(), intra=_u32(r.intra), sad_min=_u32(r.sad_min),
                sad_dev=_u32(r.sad_dev), err=r.err.cpu().numpy())


@pytest.mark.parametrize("N,M,p,qp", [(16, 16, 16, 0), (16, 16, 16, 28), (8, 8, 8, 0)])
def test_motion_study_vs_oracle(me, orc, N, M, p, qp):
    """Sec. 3.1 set-up: a CIF original frame and nine copies moved by known
    global vectors; every per-block output of the one-launch study equals the
    oracle's."""
    frames, g = synth.global_motion_sequence(31, 352, 288)
    lam = orc.lambda_q8(qp) if qp else 0
    got = _study(me, frames, g, N, M, p, lam)
    want = _study_oracle(orc, frames, g, N, M, p, lam)
    for k in want:
        assert np.array_equal(got[k], want[k]), k


def test_motion_study_equals_pairwise_calls(me):
    """The study's per-frame slices equal me_sad_deviation of each pair."""
    import torch
    frames, g = synth.global_motion_sequence(32, 176, 144, n_moved=5, max_shift=6)
    got = _study(me, frames, g, 16, 16, 8, 0)
    f = torch.from_numpy(frames).cuda()
    for k in range(1, 6):
        r = me.me_sad_deviation(f[k], f[0], 16, 16, 8, 0)
        torch.cuda.synchronize()
        assert np.array_equal(got["mv"][k - 1], r.mv.cpu().numpy())
        assert np.array_equal(got["sad_min"][k - 1], _u32(r.sad_min))
        assert np.array_equal(got["sad_dev"][k - 1], _u32(r.sad_dev))


def test_motion_study_reproduces_the_papers_observation(me):
    """Fig. 4's reading on the synthetic set-up (lambda = 0, 16x16, p = 16):
    blocks with the true vector are the textured ones (higher Intra_SAD and
    SAD_deviation medians than blocks whose vector is off by 5 or more)."""
    frames, g = synth.global_motion_sequence(33, 352, 288)
    r = _study(me, frames, g, 16, 16, 16, 0)
    true_blk, far = r["err"] == 0, r["err"] >= 5
    assert true_blk.sum() > 100 and far.sum() > 100
    assert np.median(r["intra"][true_blk]) > 2 * np.median(r["intra"][far])
    assert np.median(r["sad_dev"][true_blk]) > np.median(r["sad_dev"][far])

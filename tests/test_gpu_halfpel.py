"""Half-pel refinement (Sec. 2.2 / 2.3) on the GPU: bit-exact against the
oracle (all block shapes, several search ranges, integer fields inside and
outside the window, after the full search, at 1080p), the sequence form
against the per-pair call, and exact recovery of a half-pel motion."""
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


def _check(me, orc, cur, ref, N, M, p, lam, field, tag):
    import torch
    r = me.me_halfpel(torch.from_numpy(cur).cuda(), torch.from_numpy(ref).cuda(), N, M, p, lam,
                      torch.from_numpy(np.ascontiguousarray(field)).cuda())
    torch.cuda.synchronize()
    mv, J, sad = orc.halfpel(cur, ref, N, M, p, lam, field)
    assert np.array_equal(r.mv.cpu().numpy(), mv), (tag, "mv")
    assert np.array_equal(_u32(r.J), J), (tag, "J")
    assert np.array_equal(_u32(r.sad), sad), (tag, "sad")


@pytest.mark.parametrize("N,M", SHAPES)
def test_halfpel_all_shapes_vs_oracle(me, orc, N, M):
    rng = np.random.default_rng(N * 31 + M)
    ref = synth.texture(rng, 96, 48)
    cur = np.clip(np.roll(ref, (1, 2), axis=(0, 1)).astype(int) + rng.integers(-5, 6, ref.shape),
                  0, 255).astype(np.uint8)
    BH, BW = 48 // M, 96 // N
    for p in (1, 2, 5):
        for lam in (0, 6595):
            inside = rng.integers(-p, p + 1, (BH, BW, 2)).astype(np.int16)
            outside = rng.integers(-p - 4, p + 5, (BH, BW, 2)).astype(np.int16)
            _check(me, orc, cur, ref, N, M, p, lam, inside, (N, M, p, lam, "inside"))
            _check(me, orc, cur, ref, N, M, p, lam, outside, (N, M, p, lam, "outside"))


@pytest.mark.parametrize("qp", [22, 40])
def test_halfpel_after_full_search_cif(me, orc, qp):
    import torch
    seq = synth.config_sequence("cif", seed=70 + qp, n_frames=2)
    lam = orc.lambda_q8(qp)
    mv_int, _, _ = orc.fsbm(seq[1], seq[0], 16, 16, 16, lam, nthreads=8)
    f = me.me_fsbm(torch.from_numpy(seq[1]).cuda(), torch.from_numpy(seq[0]).cuda(), 16, 16, 16, lam)
    assert np.array_equal(f.mv.cpu().numpy(), mv_int)
    _check(me, orc, seq[1], seq[0], 16, 16, 16, lam, mv_int, ("cif", qp))


def test_halfpel_sequence_1080p_matches_per_pair_and_oracle(me, orc):
    import torch
    seq = synth.config_sequence("1080p", seed=5, n_frames=3)
    lam = orc.lambda_q8(28)
    frames = torch.from_numpy(seq).cuda()
    f = me.me_fsbm_sequence(frames, 16, 16, 32, lam)
    h = me.me_halfpel_sequence(frames, 16, 16, 32, lam, f.mv)
    torch.cuda.synchronize()
    for k in range(2):
        one = me.me_halfpel(frames[k + 1], frames[k], 16, 16, 32, lam, f.mv[k].contiguous())
        torch.cuda.synchronize()
        assert torch.equal(one.mv, h.mv[k]) and torch.equal(one.J, h.J[k]) and torch.equal(one.sad, h.sad[k])
        mv, J, sad = orc.halfpel(seq[k + 1], seq[k], 16, 16, 32, lam, f.mv[k].cpu().numpy())
        assert np.array_equal(h.mv[k].cpu().numpy(), mv), k
        assert np.array_equal(_u32(h.J[k]), J), k
        assert np.array_equal(_u32(h.sad[k]), sad), k


def test_halfpel_recovers_half_pel_motion(me, orc):
    """cur = ref shifted by (1.5, -0.5) pixels with H.263 interpolation (away
    from the edges): from the rounded integer vectors, lambda = 0, every
    interior block lands on (3, -1) half-pel with SAD 0."""
    import torch
    rng = np.random.default_rng(9)
    H, W, N, M, p = 64, 96, 16, 16, 4
    ref = rng.integers(0, 256, (H, W)).astype(np.uint8)
    r = np.pad(ref.astype(np.int64), 8, mode="edge")
    Y, X = np.mgrid[0:H, 0:W]
    A = r[Y + 8 - 1, X + 8 + 1]
    B = r[Y + 8 - 1, X + 8 + 2]
    C = r[Y + 8, X + 8 + 1]
    D = r[Y + 8, X + 8 + 2]
    cur = ((A + B + C + D + 2) >> 2).astype(np.uint8)      # (hx, hy) = (3, -1)
    field = np.tile(np.array([2, 0], np.int16), (H // M, W // N, 1))
    _check(me, orc, cur, ref, N, M, p, 0, field, "shift")
    res = me.me_halfpel(torch.from_numpy(cur).cuda(), torch.from_numpy(ref).cuda(), N, M, p, 0,
                        torch.from_numpy(field).cuda())
    torch.cuda.synchronize()
    mv = res.mv.cpu().numpy()
    inner = mv[1:-1, 1:-1]
    assert np.all(inner[..., 0] == 3) and np.all(inner[..., 1] == -1)
    assert np.all(_u32(res.sad)[1:-1, 1:-1] == 0)

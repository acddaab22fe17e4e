"""FSBM with the vector rate coded against the median predictor, on the GPU
(SAD volume, then the persistent wavefront): bit-exact against the oracle
for every block shape and several search ranges on fields with many distinct
vectors, at CIF for a range of p (every run length of the 16x16 plans), the
sequence form against the per-pair oracle, one whole 1080p p=32 frame plus
the lambda = 0 reduction to plain FSBM, and repeated runs of one plan."""
import numpy as np
import pytest

import synth
from test_oracle_pins import blockwise_motion

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
    r = me.me_fsbm_pred(torch.from_numpy(cur).cuda(), torch.from_numpy(ref).cuda(), N, M, p, lam)
    assert me.me_fsbm_pred_status(cur.shape[1], cur.shape[0], N, M, p, 1) == 0
    return r.mv.cpu().numpy(), _u32(r.J), _u32(r.sad)


def _check(me, orc, cur, ref, N, M, p, lam, tag):
    got = _run(me, cur, ref, N, M, p, lam)
    want = orc.fsbm_pred(cur, ref, N, M, p, lam)
    for g, w, k in zip(got, want, ("mv", "J", "sad")):
        assert np.array_equal(g, w), (tag, k)


@pytest.mark.parametrize("N,M", SHAPES)
def test_pred_all_shapes_vs_oracle(me, orc, N, M):
    cur, ref = blockwise_motion(96, 64, N, M, 6, N * 13 + M)
    for p in (1, 3, 6):
        for lam in (0, 6595, 60000):
            _check(me, orc, cur, ref, N, M, p, lam, (N, M, p, lam))


@pytest.mark.parametrize("p", [2, 7, 8, 12, 16, 20, 32])
def test_pred_cif_search_ranges(me, orc, p):
    seq = synth.config_sequence("cif", seed=600 + p, n_frames=2)
    _check(me, orc, seq[1], seq[0], 16, 16, p, orc.lambda_q8(28), ("cif", p))


def test_pred_sequence_vs_per_pair_oracle(me, orc):
    import torch
    seq = synth.config_sequence("cif", seed=610, n_frames=6)
    lam = orc.lambda_q8(34)
    r = me.me_fsbm_pred_sequence(torch.from_numpy(seq).cuda(), 16, 16, 16, lam)
    assert me.me_fsbm_pred_status(352, 288, 16, 16, 16, 5) == 0
    for k in range(5):
        mv, J, sad = orc.fsbm_pred(seq[k + 1], seq[k], 16, 16, 16, lam)
        assert np.array_equal(r.mv[k].cpu().numpy(), mv), k
        assert np.array_equal(_u32(r.J[k]), J), k
        assert np.array_equal(_u32(r.sad[k]), sad), k


def test_pred_repeated_runs_of_one_plan(me, orc):
    """The plan's flags carry a run epoch: later runs (other frames, other
    lambda) must not see an earlier run's vectors."""
    cur, ref = blockwise_motion(128, 96, 16, 16, 5, 3)
    outs = [(lam, _run(me, cur, ref, 16, 16, 5, lam)) for lam in (6595, 0, 60000, 6595)]
    for lam, got in outs:
        want = orc.fsbm_pred(cur, ref, 16, 16, 5, lam)
        for g, w in zip(got, want):
            assert np.array_equal(g, w), lam


def test_pred_1080p_whole_frame(me, orc):
    """1920x1088, 16x16, p = 32: every block of one pair against the oracle's
    predictor-coded search run over the whole frame in raster order (each
    block's predictor from the oracle's own field); lambda = 0 equals
    me_fsbm."""
    import torch
    seq = synth.config_sequence("1080p", seed=91, n_frames=2)
    cur, ref = np.ascontiguousarray(seq[1]), np.ascontiguousarray(seq[0])
    N = M = 16
    p = 32
    lam = orc.lambda_q8(28)
    mv, J, sad = _run(me, cur, ref, N, M, p, lam)
    wmv, wJ, ws = orc.fsbm_pred(cur, ref, N, M, p, lam)
    assert np.array_equal(mv, wmv)
    assert np.array_equal(J, wJ)
    assert np.array_equal(sad, ws)
    mv0, J0, _ = _run(me, cur, ref, N, M, p, 0)
    f = me.me_fsbm(torch.from_numpy(cur).cuda(), torch.from_numpy(ref).cuda(), N, M, p, 0)
    torch.cuda.synchronize()
    assert np.array_equal(mv0, f.mv.cpu().numpy()) and np.array_equal(J0, _u32(f.J))


@pytest.mark.parametrize("lam", [6595, 60000])
def test_pred_flat_and_textured_regions(me, orc, lam):
    """A frame with flat regions (near-flat SAD surfaces: every candidate may
    still win, the whole-CTA evaluation) beside textured ones (a short list of
    candidates, one warp), and a nearly flat frame (all blocks the long way)."""
    frames, _ = synth.global_motion_sequence(12, 352, 288, n_moved=1)
    _check(me, orc, frames[1], frames[0], 16, 16, 8, lam, ("contrast", lam))
    rng = np.random.default_rng(4)
    flat0 = (128 + rng.integers(-1, 2, (144, 176))).astype(np.uint8)
    flat1 = (128 + rng.integers(-1, 2, (144, 176))).astype(np.uint8)
    _check(me, orc, flat1, flat0, 16, 16, 6, lam, ("flat", lam))


def test_pred_long_sequence_without_the_list(me, orc):
    """More than 8 pairs per call: every candidate is evaluated after the
    wait (no pre-wait list); each pair equals the oracle."""
    import torch
    seq = synth.config_sequence("cif", seed=620, n_frames=11)
    lam = orc.lambda_q8(30)
    r = me.me_fsbm_pred_sequence(torch.from_numpy(seq).cuda(), 16, 16, 16, lam)
    assert me.me_fsbm_pred_status(352, 288, 16, 16, 16, 10) == 0
    for k in range(10):
        mv, J, sad = orc.fsbm_pred(seq[k + 1], seq[k], 16, 16, 16, lam)
        assert np.array_equal(r.mv[k].cpu().numpy(), mv), k
        assert np.array_equal(_u32(r.J[k]), J), k
        assert np.array_equal(_u32(r.sad[k]), sad), k


def test_pred_list_and_full_evaluation_agree(me, monkeypatch):
    """The two evaluation forms (pre-wait list / every candidate) give the
    same bytes for short and long calls."""
    import torch
    seq = torch.from_numpy(synth.config_sequence("cif", seed=621, n_frames=12)).cuda()
    lam = me.me_lambda_q8(26)
    for frames in (seq[:2], seq[:4], seq):
        outs = []
        for v in ("1", "0"):
            monkeypatch.setenv("ME_PRED_PRUNE", v)
            r = me.me_fsbm_pred_sequence(frames, 16, 16, 24, lam)
            torch.cuda.synchronize()
            outs.append(r)
        assert torch.equal(outs[0].mv, outs[1].mv) and torch.equal(outs[0].J, outs[1].J)
        assert torch.equal(outs[0].sad, outs[1].sad)

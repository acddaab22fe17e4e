"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle,
bit-exact on every output (MV, J, SAD, full-search mask, load).

Sizes: tiny frames over every block shape and small p (many tiles and a
ragged last tile per CTA); the QCIF and CIF workloads whole; the 1080p p=32
workload whole for ACBM and on sampled blocks for FSBM (every block of the
sample computed independently by the oracle); 2160p p=64 on sampled FSBM
blocks.  Edge cases: single-block frames, p larger than the frame, blocks on
every border, constant frames (all ties), argument errors.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def me():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_0710_4819_gb300 as me
    me.load_library(build_if_missing=True)
    return me


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _fsbm_gpu(me, cur, ref, N, M, p, lam):
    import torch
    r = me.me_fsbm(_dev(cur), _dev(ref), N, M, p, lam)
    torch.cuda.synchronize()
    return r.mv.cpu().numpy(), _u32(r.J), _u32(r.sad)


def _acbm_gpu(me, cur, ref, N, M, p, lam, prm, prev=None):
    import torch
    r = me.me_acbm(_dev(cur), _dev(ref), N, M, p, lam, prm,
                   prev_mv=None if prev is None else _dev(prev))
    torch.cuda.synchronize()
    return (r.mv.cpu().numpy(), _u32(r.J), r.mask.cpu().numpy(), _u32(r.sad), _u32(r.load))


def _eq(name, got, want):
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        raise AssertionError(f"{name}: {len(bad)} mismatches, first at {bad[:5].tolist()}")


SHAPES = [(16, 16), (16, 8), (16, 4), (8, 16), (8, 8), (8, 4), (4, 16), (4, 8), (4, 4)]


@pytest.mark.parametrize("N,M", SHAPES)
@pytest.mark.parametrize("p", [1, 2, 5, 8])
def test_fsbm_small_all_shapes(me, orc, N, M, p):
    rng = np.random.default_rng(100 * N + 10 * M + p)
    W, H = 6 * N + (16 if N == 4 else 0), 5 * M
    for trial in range(2):
        ref = synth.texture(rng, W, H) if trial == 0 else rng.integers(0, 256, (H, W), np.uint8)
        cur = synth.shifted_copy(ref, int(rng.integers(-p, p + 1)), int(rng.integers(-p, p + 1)))
        cur = np.clip(cur.astype(int) + rng.integers(-4, 5, cur.shape), 0, 255).astype(np.uint8)
        lam = [0, 6595, 250000][trial + (p % 2)]
        got = _fsbm_gpu(me, cur, ref, N, M, p, lam)
        want = orc.fsbm(cur, ref, N, M, p, lam)
        for nm, g, w in zip(("mv", "J", "sad"), got, want):
            _eq(f"{N}x{M} p={p} {nm}", g, w)


@pytest.mark.parametrize("p,lam", [(3, 6595), (11, 6595), (16, 6595), (20, 6595), (32, 6595),
                                   (32, 800000), (64, 2000), (64, 6595), (40, 1 << 20)])
def test_fsbm_16x16_run_lengths(me, orc, p, lam):
    """Search ranges that exercise every instantiated run length and ragged
    runs, and lambdas on both sides of the 32-bit run-key limit."""
    rng = np.random.default_rng(p)
    ref = synth.texture(rng, 96, 64)
    cur = synth.shifted_copy(ref, 3, -2)
    cur = np.clip(cur.astype(int) + rng.integers(-3, 4, cur.shape), 0, 255).astype(np.uint8)
    got = _fsbm_gpu(me, cur, ref, 16, 16, p, lam)
    want = orc.fsbm(cur, ref, 16, 16, p, lam, nthreads=8)
    for nm, g, w in zip(("mv", "J", "sad"), got, want):
        _eq(nm, g, w)


def test_fsbm_edge_cases(me, orc):
    # single block, p larger than the frame
    rng = np.random.default_rng(1)
    ref = rng.integers(0, 256, (16, 16), np.uint8)
    cur = rng.integers(0, 256, (16, 16), np.uint8)
    for p in (1, 20, 64):
        got = _fsbm_gpu(me, cur, ref, 16, 16, p, 6595)
        want = orc.fsbm(cur, ref, 16, 16, p, 6595)
        for nm, g, w in zip(("mv", "J", "sad"), got, want):
            _eq(f"1 block p={p} {nm}", g, w)
    # constant frames: every candidate ties, (0,0) must win
    c = np.full((48, 64), 7, np.uint8)
    r = np.full((48, 64), 9, np.uint8)
    mv, J, sad = _fsbm_gpu(me, c, r, 16, 16, 8, 0)
    assert np.all(mv == 0) and np.all(sad == 2 * 256)
    # lambda 0 with a periodic pattern: raster tie-break
    pat = np.array([10, 200, 60, 140], np.uint8)
    ref = np.tile(pat, (48, 16))[:, :64]
    cur = np.roll(ref, 2, axis=1)
    got = _fsbm_gpu(me, cur, ref, 16, 16, 6, 0)
    want = orc.fsbm(cur, ref, 16, 16, 6, 0)
    for nm, g, w in zip(("mv", "J", "sad"), got, want):
        _eq(f"periodic {nm}", g, w)
    # diagonal pattern: (1,0) and (0,1) tie in J and |mv|_1; raster order decides
    g7 = np.array([13, 201, 77, 150, 30, 240, 99], np.uint8)
    yy, xx = np.mgrid[0:64, 0:64]
    refd, curd = g7[(xx + yy) % 7], g7[(xx + yy + 1) % 7]
    for p in (3, 32):
        got = _fsbm_gpu(me, curd, refd, 16, 16, p, 0)
        want = orc.fsbm(curd, refd, 16, 16, p, 0)
        for nm, g, w in zip(("mv", "J", "sad"), got, want):
            _eq(f"diagonal p={p} {nm}", g, w)


def test_fsbm_rejects_bad_arguments(me):
    import torch
    x = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    with pytest.raises(me.MeError) as e:
        me.me_fsbm(x[:, :60].contiguous(), x[:, :60].contiguous(), 16, 16, 4, 0)
    assert e.value.status == 2
    with pytest.raises(me.MeError) as e:
        me.me_fsbm(x, x, 16, 16, 65, 0)
    assert e.value.status == 1


def test_fsbm_qcif_sequence(me, orc):
    seq = synth.config_sequence("qcif", seed=11)
    lam = orc.lambda_q8(28)
    for t in range(1, seq.shape[0]):
        got = _fsbm_gpu(me, seq[t], seq[t - 1], 16, 16, 16, lam)
        want = orc.fsbm(seq[t], seq[t - 1], 16, 16, 16, lam, nthreads=8)
        for nm, g, w in zip(("mv", "J", "sad"), got, want):
            _eq(f"qcif t={t} {nm}", g, w)


@pytest.mark.parametrize("qp", [22, 28, 34, 40])
def test_fsbm_cif_qp_sweep(me, orc, qp):
    seq = synth.config_sequence("cif", seed=12, n_frames=3)
    lam = orc.lambda_q8(qp)
    for t in range(1, seq.shape[0]):
        got = _fsbm_gpu(me, seq[t], seq[t - 1], 16, 16, 16, lam)
        want = orc.fsbm(seq[t], seq[t - 1], 16, 16, 16, lam, nthreads=8)
        for nm, g, w in zip(("mv", "J", "sad"), got, want):
            _eq(f"cif qp={qp} {nm}", g, w)


def _sample_blocks(BW, BH, k, seed):
    rng = np.random.default_rng(seed)
    edge = [0, BW - 1, (BH - 1) * BW, BH * BW - 1, BW // 2, (BH - 1) * BW + BW // 2,
            (BH // 2) * BW, (BH // 2) * BW + BW - 1]
    return np.unique(np.concatenate([edge, rng.choice(BW * BH, k, replace=False)])).astype(np.int32)


def test_fsbm_1080p_sampled(me, orc):
    seq = synth.config_sequence("1080p", seed=13, n_frames=2)
    lam = orc.lambda_q8(28)
    mv, J, sad = _fsbm_gpu(me, seq[1], seq[0], 16, 16, 32, lam)
    blocks = _sample_blocks(120, 68, 250, 5)
    wmv, wJ, ws = orc.fsbm_blocks(seq[1], seq[0], 16, 16, 32, lam, blocks, nthreads=16)
    _eq("mv", mv.reshape(-1, 2)[blocks], wmv)
    _eq("J", J.ravel()[blocks], wJ)
    _eq("sad", sad.ravel()[blocks], ws)


def test_fsbm_1080p_whole_frame(me, orc):
    """One whole 1920x1088 frame pair at p = 32 (the headline workload's
    shape, 8160 blocks, the pipelined search behind me_fsbm): every block's
    vector, J and SAD against the oracle's full search of Sec. 2.3."""
    import os
    seq = synth.config_sequence("1080p", seed=17, n_frames=2)
    lam = orc.lambda_q8(28)
    mv, J, sad = _fsbm_gpu(me, seq[1], seq[0], 16, 16, 32, lam)
    wmv, wJ, ws = orc.fsbm(seq[1], seq[0], 16, 16, 32, lam, nthreads=os.cpu_count() or 8)
    _eq("mv", mv, wmv)
    _eq("J", J, wJ)
    _eq("sad", sad, ws)


def test_fsbm_2160p_p64_sampled(me, orc):
    spec = synth.batch_mix()[-1]
    seq = synth.stream_frames(spec, 2)
    lam = orc.lambda_q8(28)
    mv, J, sad = _fsbm_gpu(me, seq[1], seq[0], 16, 16, 64, lam)
    blocks = _sample_blocks(240, 135, 40, 6)
    wmv, wJ, ws = orc.fsbm_blocks(seq[1], seq[0], 16, 16, 64, lam, blocks, nthreads=16)
    _eq("mv", mv.reshape(-1, 2)[blocks], wmv)
    _eq("J", J.ravel()[blocks], wJ)
    _eq("sad", sad.ravel()[blocks], ws)


def test_fsbm_deterministic(me):
    seq = synth.config_sequence("cif", seed=14, n_frames=2)
    a = _fsbm_gpu(me, seq[1], seq[0], 16, 16, 16, 6595)
    for _ in range(3):
        b = _fsbm_gpu(me, seq[1], seq[0], 16, 16, 16, 6595)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


# ------------------------------------------------------------------ a1, a2
def test_pad_ref_matches_definition(me):
    import torch
    rng = np.random.default_rng(3)
    for (W, H, p) in [(176, 144, 16), (36, 20, 5), (64, 48, 33)]:
        ref = rng.integers(0, 256, (H, W), np.uint8)
        out = me.me_pad_ref(_dev(ref), p)
        torch.cuda.synchronize()
        pitch, rows, P = me.me_padded_geometry(W, H, p)
        ys = np.clip(np.arange(rows) - P, 0, H - 1)
        xs = np.clip(np.arange(pitch) - P, 0, W - 1)
        _eq("pad", out.cpu().numpy(), ref[np.ix_(ys, xs)])


@pytest.mark.parametrize("N,M", SHAPES)
def test_intra_sad(me, orc, N, M):
    rng = np.random.default_rng(N + M)
    cur = rng.integers(0, 256, (8 * M, 8 * N), np.uint8)
    import torch
    got = me.me_intra_sad(_dev(cur), N, M)
    torch.cuda.synchronize()
    _eq("intra", got.cpu().numpy().view(np.uint32), orc.intra_sad(cur, N, M))


# ------------------------------------------------------------------ ACBM
def _acbm_check(me, orc, cur, ref, N, M, p, lam, prm_kw, prev=None, tag=""):
    got = _acbm_gpu(me, cur, ref, N, M, p, lam, me.params(**prm_kw), prev)
    want = orc.acbm(cur, ref, N, M, p, lam, orc.params(**prm_kw), prev)
    for nm, g, w in zip(("mv", "J", "mask", "sad", "load"), got, want):
        _eq(f"{tag} {nm}", g, w)
    return got


@pytest.mark.parametrize("N,M", SHAPES)
def test_acbm_small_all_shapes(me, orc, N, M):
    seq = synth.scene_sequence(N * 7 + M, 12 * N, 9 * M, 3, n_objects=3, vmax=3)
    lam = orc.lambda_q8(28)
    prev = None
    for t in (1, 2):
        for kw in (dict(qp=28), dict(qp=28, refine=0), dict(alpha=0, beta=0, gamma_num=0, qp=28),
                   dict(alpha=2 ** 30, qp=28), dict(alpha=300, beta=1, gamma_num=1, gamma_den=2, qp=10)):
            got = _acbm_check(me, orc, seq[t], seq[t - 1], N, M, 4, lam, kw, prev, f"{N}x{M} {kw}")
        prev = _acbm_gpu(me, seq[t], seq[t - 1], N, M, 4, lam, me.params(qp=28), prev)[0]


def test_acbm_qcif_sequence_chained(me, orc):
    """Ten QCIF frames, each frame's field feeding the next as temporal predictors."""
    seq = synth.config_sequence("qcif", seed=21)
    lam = orc.lambda_q8(28)
    prev_g = prev_o = None
    fs = 0
    for t in range(1, seq.shape[0]):
        got = _acbm_gpu(me, seq[t], seq[t - 1], 16, 16, 16, lam, me.params(qp=28), prev_g)
        want = orc.acbm(seq[t], seq[t - 1], 16, 16, 16, lam, orc.params(qp=28), prev_o)
        for nm, g, w in zip(("mv", "J", "mask", "sad", "load"), got, want):
            _eq(f"qcif t={t} {nm}", g, w)
        prev_g, prev_o = got[0], want[0]
        fs += int(got[2].sum())
    assert fs > 0   # the workload does exercise the full-search fallback


@pytest.mark.parametrize("qp", [22, 40])
def test_acbm_cif(me, orc, qp):
    seq = synth.config_sequence("cif", seed=22, n_frames=4)
    lam = orc.lambda_q8(qp)
    prev_g = prev_o = None
    for t in range(1, seq.shape[0]):
        got = _acbm_gpu(me, seq[t], seq[t - 1], 16, 16, 16, lam, me.params(qp=qp), prev_g)
        want = orc.acbm(seq[t], seq[t - 1], 16, 16, 16, lam, orc.params(qp=qp), prev_o)
        for nm, g, w in zip(("mv", "J", "mask", "sad", "load"), got, want):
            _eq(f"cif qp={qp} t={t} {nm}", g, w)
        prev_g, prev_o = got[0], want[0]


def test_acbm_1080p_full_frames(me, orc):
    """The 1080p p=32 workload, two chained frame pairs, every block compared."""
    seq = synth.config_sequence("1080p", seed=23, n_frames=3)
    lam = orc.lambda_q8(28)
    prev_g = prev_o = None
    for t in (1, 2):
        got = _acbm_gpu(me, seq[t], seq[t - 1], 16, 16, 32, lam, me.params(qp=28), prev_g)
        want = orc.acbm(seq[t], seq[t - 1], 16, 16, 32, lam, orc.params(qp=28), prev_o)
        for nm, g, w in zip(("mv", "J", "mask", "sad", "load"), got, want):
            _eq(f"1080p t={t} {nm}", g, w)
        prev_g, prev_o = got[0], want[0]


def test_acbm_invariants_vs_fsbm_on_gpu(me, orc):
    seq = synth.config_sequence("cif", seed=24, n_frames=2)
    lam = orc.lambda_q8(28)
    f = _fsbm_gpu(me, seq[1], seq[0], 16, 16, 16, lam)
    a = _acbm_gpu(me, seq[1], seq[0], 16, 16, 16, lam, me.params(qp=28))
    assert np.all(f[1] <= a[1])
    fs = a[2] == 1
    _eq("fs blocks mv", a[0][fs], f[0][fs])
    forced = _acbm_gpu(me, seq[1], seq[0], 16, 16, 16, lam,
                       me.params(alpha=0, beta=0, gamma_num=0, qp=28))
    _eq("forced mv", forced[0], f[0])
    _eq("forced J", forced[1], f[1])
    assert np.all(forced[2] == 1) and np.all(forced[4] == 33 * 33)


@pytest.mark.parametrize("p", [8, 20, 32, 40, 64])
def test_acbm_forced_fallback_across_slice_counts(me, orc, p):
    """Every block through the fallback search, whose CTAs split the mvx
    columns into slices merged by an atomic minimum (the slice count grows
    with p): equal to the oracle's FSBM for every block."""
    rng = np.random.default_rng(p)
    ref = synth.texture(rng, 96, 64)
    cur = synth.shifted_copy(ref, 5, -3)
    cur = np.clip(cur.astype(int) + rng.integers(-3, 4, cur.shape), 0, 255).astype(np.uint8)
    lam = orc.lambda_q8(28)
    got = _acbm_gpu(me, cur, ref, 16, 16, p, lam, me.params(alpha=0, beta=0, gamma_num=0, qp=28))
    mv, J, sad = orc.fsbm(cur, ref, 16, 16, p, lam, nthreads=8)
    _eq("mv", got[0], mv)
    _eq("J", got[1], J)
    _eq("sad", got[3], sad)
    assert np.all(got[2] == 1) and np.all(got[4] == (2 * p + 1) ** 2)


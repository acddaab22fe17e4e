"""Pins for the CPU oracle: checks against what the paper and the mathematics
fix, independent of the oracle's own code.

* eq. J / eq. SAD (Sec. 2.1) and FSBM (Sec. 2.3): brute force over the whole
  SAD volume in numpy (sliding windows, lexicographic argmin) on tiny frames,
  exact recovery of an integer shift, tie-break adversaries.
* R(mv): the code lengths come from an Exp-Golomb encoder built bit by bit and
  checked to decode back (a prefix code), not from a length formula.
* eq. Intra_SAD (Sec. 3.1): exact rational mean (fractions.Fraction) and the
  closed forms for flat and two-level blocks.
* ACBM (Sec. 3.2): each stopping condition at its equality boundary (strict
  "<"), forced / suppressed full search, and probes that show which
  neighbouring vectors the PBM stage uses (Sec. 2.2, Fig. 2).
* Constants printed in the paper: alpha, beta, gamma (Sec. 4) and the
  961 + 8 = 969 FSBM positions at p = 15 (Sec. 2.3, Sec. 4).
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers
def eg_encode_signed(v: int) -> str:
    """Signed Exp-Golomb code as a bit string, built constructively."""
    k = 2 * v - 1 if v > 0 else -2 * v
    info = bin(k + 1)[2:]               # '1' followed by the info bits
    return "0" * (len(info) - 1) + info


def eg_decode_stream(bits: str) -> list[int]:
    out, i = [], 0
    while i < len(bits):
        z = 0
        while bits[i] == "0":
            z += 1
            i += 1
        k = int(bits[i:i + z + 1], 2) - 1
        i += z + 1
        out.append((k + 1) // 2 if k % 2 == 1 else -(k // 2))
    return out


def brute_sad_volume(cur, ref, N, M, p):
    """SAD of every block at every integer position, by sliding windows over an
    edge-padded reference: vol[mvy + p, mvx + p, by, bx] (int64)."""
    H, W = cur.shape
    BH, BW = H // M, W // N
    rp = np.pad(ref.astype(np.int64), p, mode="edge")
    c = cur.astype(np.int64)
    n = 2 * p + 1
    vol = np.zeros((n, n, BH, BW), np.int64)
    for a in range(n):
        for b in range(n):
            sh = rp[a:a + H, b:b + W]          # ref(x + mvx, y + mvy), mvy = a - p, mvx = b - p
            vol[a, b] = np.abs(c - sh).reshape(BH, M, BW, N).sum(axis=(1, 3))
    return vol


def brute_fsbm(cur, ref, N, M, p, lam):
    """Whole SAD volume, then a lexicographic argmin (J, |mv|_1, mvy, mvx)."""
    H, W = cur.shape
    BH, BW = H // M, W // N
    n = 2 * p + 1
    vol = brute_sad_volume(cur, ref, N, M, p)
    mvs = np.arange(-p, p + 1)
    bits = np.array([len(eg_encode_signed(int(v))) for v in mvs], np.int64)
    R = bits[:, None] + bits[None, :]         # [mvy, mvx]
    J = 256 * vol + lam * R[:, :, None, None]
    MY, MX = np.meshgrid(mvs, mvs, indexing="ij")
    L1 = np.abs(MY) + np.abs(MX)
    mv = np.zeros((BH, BW, 2), np.int64)
    Jb = np.zeros((BH, BW), np.int64)
    Sb = np.zeros((BH, BW), np.int64)
    for by in range(BH):
        for bx in range(BW):
            j = J[:, :, by, bx].ravel()
            order = np.lexsort((MX.ravel(), MY.ravel(), L1.ravel(), j))
            k = order[0]
            mv[by, bx] = (MX.ravel()[k], MY.ravel()[k])
            Jb[by, bx] = j[k]
            Sb[by, bx] = vol[:, :, by, bx].ravel()[k]
    return mv, Jb, Sb


def per_block_motion(ref, N, M, disp):
    """cur block b = ref moved by disp[by, bx] (edge clamp): SAD 0 at mv = -disp."""
    H, W = ref.shape
    cur = np.empty_like(ref)
    for by in range(H // M):
        for bx in range(W // N):
            dx, dy = disp[by][bx]
            sh = synth.shifted_copy(ref, dx, dy)
            cur[by * M:(by + 1) * M, bx * N:(bx + 1) * N] = sh[by * M:(by + 1) * M,
                                                                bx * N:(bx + 1) * N]
    return cur


# ----------------------------------------------------------------- lambda, R
def test_lambda_is_092_qp_in_q8(orc):
    for qp in range(0, 1024):
        exact = Fraction(92, 100) * qp * 256
        got = orc.lambda_q8(qp)
        assert abs(Fraction(got) - exact) <= Fraction(1, 2)
        # round half up
        assert got == int(exact + Fraction(1, 2))
    assert [orc.lambda_q8(q) for q in (22, 28, 34, 40)] == [5181, 6595, 8008, 9421]


def test_mv_bits_match_exp_golomb_encoder(orc):
    vals = list(range(-300, 301))
    for v in vals:
        assert orc.mv_bits(v) == len(eg_encode_signed(v)), v
    rng = np.random.default_rng(3)
    seq = [int(x) for x in rng.integers(-70, 71, size=500)]
    assert eg_decode_stream("".join(eg_encode_signed(v) for v in seq)) == seq
    assert [orc.mv_bits(v) for v in (0, 1, -1, 2, 3, -3, 4, 7, 8, 15, 16)] == \
        [1, 3, 3, 5, 5, 5, 7, 7, 9, 9, 11]


# ----------------------------------------------------------------- Intra_SAD
@pytest.mark.parametrize("N,M", [(16, 16), (8, 4), (4, 16)])
def test_intra_sad_exact_rational_mean(orc, N, M):
    rng = np.random.default_rng(N * 31 + M)
    cur = rng.integers(0, 256, size=(3 * M, 2 * N), dtype=np.uint8)
    got = orc.intra_sad(cur, N, M)
    for by in range(3):
        for bx in range(2):
            blk = [int(v) for v in cur[by * M:(by + 1) * M, bx * N:(bx + 1) * N].ravel()]
            mu = Fraction(sum(blk), len(blk))
            intra = sum(abs(Fraction(v) - mu) for v in blk)
            assert Fraction(int(got[by, bx]), N * M) == intra


def test_intra_sad_closed_forms(orc):
    flat = np.full((16, 16), 93, np.uint8)
    assert orc.intra_sad(flat, 16, 16)[0, 0] == 0
    a, b = 100, 110
    two = np.full((16, 16), a, np.uint8)
    two[:, 8:] = b
    # half the pixels a, half b: mean (a+b)/2, Intra_SAD = NM*|a-b|/2
    assert orc.intra_sad(two, 16, 16)[0, 0] == 256 * (256 * abs(a - b) // 2)


# ----------------------------------------------------------------- FSBM
@pytest.mark.parametrize("W,H,N,M,p", [
    (32, 32, 16, 16, 1), (32, 32, 16, 16, 3), (48, 32, 16, 16, 4),
    (32, 32, 8, 8, 2), (48, 32, 8, 16, 3), (32, 32, 4, 4, 2), (24, 16, 4, 8, 4),
])
def test_fsbm_matches_brute_force(orc, W, H, N, M, p):
    for trial, lam in enumerate([0, 3000, 6595, 120000]):
        rng = np.random.default_rng(1000 * p + 10 * N + trial)
        if trial % 2 == 0:
            ref = synth.texture(rng, W, H)
            cur = synth.shifted_copy(ref, int(rng.integers(-3, 4)), int(rng.integers(-3, 4)))
            cur = np.clip(cur.astype(int) + rng.integers(-3, 4, size=cur.shape), 0, 255)
        else:
            ref = rng.integers(0, 256, size=(H, W))
            cur = rng.integers(0, 256, size=(H, W))
        cur, ref = cur.astype(np.uint8), ref.astype(np.uint8)
        mv, J, sad = orc.fsbm(cur, ref, N, M, p, lam)
        bmv, bJ, bS = brute_fsbm(cur, ref, N, M, p, lam)
        assert np.array_equal(mv, bmv)
        assert np.array_equal(J, bJ)
        assert np.array_equal(sad, bS)


def test_fsbm_threads_do_not_change_result(orc):
    rng = np.random.default_rng(5)
    ref = synth.texture(rng, 64, 48)
    cur = synth.shifted_copy(ref, 2, -1)
    a = orc.fsbm(cur, ref, 16, 16, 5, 6595, nthreads=1)
    b = orc.fsbm(cur, ref, 16, 16, 5, 6595, nthreads=4)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("dx,dy", [(3, -2), (-5, 1), (0, 4), (2, 2)])
def test_fsbm_recovers_exact_shift(orc, dx, dy):
    ref = synth.random_frame(11, 64, 48)
    cur = synth.shifted_copy(ref, dx, dy)
    mv, J, sad = orc.fsbm(cur, ref, 16, 16, 6, 0)
    assert np.all(mv[..., 0] == -dx) and np.all(mv[..., 1] == -dy)
    assert np.all(sad == 0) and np.all(J == 0)
    # the rate term does not move a zero-SAD match on sharp texture
    mv2, J2, _ = orc.fsbm(cur, ref, 16, 16, 6, orc.lambda_q8(28))
    assert np.array_equal(mv, mv2)
    assert np.all(J2 == orc.lambda_q8(28) * (len(eg_encode_signed(-dx)) +
                                             len(eg_encode_signed(-dy))))


def test_fsbm_tie_breaks(orc):
    # constant frames: every SAD is equal, so J is smallest at (0,0)
    c = np.full((32, 32), 50, np.uint8)
    r = np.full((32, 32), 60, np.uint8)
    mv, J, sad = orc.fsbm(c, r, 16, 16, 4, 0)
    assert np.all(mv == 0) and np.all(sad == 256 * 10)
    # horizontal period 4, vertically constant, content moved by 2: SAD 0 at
    # mvx = +-2 (and +-6) for every mvy; smallest |mv|_1 leaves (-2,0),(2,0);
    # the raster order (smaller mvy, then smaller mvx) picks (-2,0)
    pat = np.array([10, 200, 60, 140], np.uint8)
    ref = np.tile(pat, (48, 16))[:, :64]
    cur = np.roll(ref, 2, axis=1)
    mv, J, sad = orc.fsbm(cur, ref, 16, 16, 6, 0)
    assert tuple(mv[1, 1]) == (-2, 0) and tuple(mv[1, 2]) == (-2, 0)
    assert sad[1, 1] == 0
    # the same pattern vertically: (0,-2) wins over (0,2)
    refv = ref.T.copy()
    curv = np.roll(refv, 2, axis=0)
    mv, J, sad = orc.fsbm(curv, refv, 16, 16, 6, 0)
    assert tuple(mv[1, 1]) == (0, -2) and tuple(mv[2, 1]) == (0, -2)
    # rate decides between equal SADs when lambda > 0: (2,0) and (-2,0) cost
    # the same, (-2,0) still wins by raster; with lambda both beat (+-6,0)
    mv, J, sad = orc.fsbm(cur, ref, 16, 16, 6, 6595)
    assert tuple(mv[1, 1]) == (-2, 0)
    # diagonal pattern g((x+y) mod 7), content moved so SAD is 0 exactly where
    # mvx + mvy = 1: (1,0) and (0,1) tie in J and |mv|_1; the raster order
    # (mvy before mvx) picks (1,0)
    g = np.array([13, 201, 77, 150, 30, 240, 99], np.uint8)
    yy, xx = np.mgrid[0:64, 0:64]
    refd = g[(xx + yy) % 7]
    curd = g[(xx + yy + 1) % 7]
    mv, J, sad = orc.fsbm(curd, refd, 16, 16, 3, 0)
    assert tuple(mv[1, 1]) == (1, 0) and tuple(mv[2, 2]) == (1, 0) and sad[1, 1] == 0


def test_fsbm_rejects_bad_shapes(orc):
    c = np.zeros((32, 32), np.uint8)
    with pytest.raises(orc.OracleError):
        orc.fsbm(c[:, :30], c[:, :30], 16, 16, 2, 0)    # W % N != 0
    with pytest.raises(orc.OracleError):
        orc.fsbm(c, c, 16, 16, 0, 0)                    # p < 1
    with pytest.raises(orc.OracleError):
        orc.fsbm(c, c, 12, 16, 2, 0)                    # N not in {4,8,16}


# ----------------------------------------------------------------- paper constants
def test_paper_constants(orc):
    with open(os.path.join(GOLDEN, "paper_constants.json")) as f:
        g = json.load(f)
    d = orc.params()
    assert (d.alpha, d.beta, d.gamma_num, d.gamma_den) == (
        g["acbm_defaults"]["alpha"], g["acbm_defaults"]["beta"],
        g["acbm_defaults"]["gamma_num"], g["acbm_defaults"]["gamma_den"])
    fp = g["fsbm_positions"]
    assert fp["integer_positions"] + fp["half_pel_positions"] == fp["total_positions"]
    # a forced full search at p = 15 evaluates the 961 integer positions of the
    # paper's 969 (the 8 half-pel ones are outside the integer-pel search)
    ref = synth.random_frame(2, 32, 32)
    cur = synth.shifted_copy(ref, 1, 1)
    _, _, mask, _, load = orc.acbm(cur, ref, 16, 16, fp["p"], 0,
                                   orc.params(alpha=0, beta=0, gamma_num=0))
    assert np.all(mask == 1) and np.all(load == fp["integer_positions"])


# ----------------------------------------------------------------- ACBM conditions
def _single(orc, cur, ref, prm, p=1):
    return orc.acbm(cur, ref, 16, 16, p, 0, prm)


def test_acbm_cond1_strict_and_scaled(orc):
    cur = np.full((16, 16), 101, np.uint8)
    ref = np.full((16, 16), 100, np.uint8)   # Intra_SAD 0, SAD_PBM = 256
    # cond 1: 0 + 256 < alpha + beta*Qp^2 (gamma 0 switches cond 2 off)
    for alpha, expect_fs in [(256, 1), (257, 0)]:
        _, _, mask, sad, load = _single(orc, cur, ref, orc.params(alpha, 0, 0, 1, 28, 0))
        assert mask[0, 0] == expect_fs and sad[0, 0] == 256
        assert load[0, 0] == (9 if expect_fs else 1)
    for qp, expect_fs in [(16, 1), (17, 0)]:       # 256 < Qp^2 with beta = 1
        _, _, mask, _, _ = _single(orc, cur, ref, orc.params(0, 1, 0, 1, qp, 0))
        assert mask[0, 0] == expect_fs
    # Intra_SAD enters unscaled: two-level block has Intra_SAD = 1280
    two = np.full((16, 16), 100, np.uint8)
    two[:, 8:] = 110
    ref2 = two + 1
    for alpha, expect_fs in [(1536, 1), (1537, 0)]:
        _, _, mask, sad, _ = _single(orc, two, ref2, orc.params(alpha, 0, 0, 1, 28, 0))
        assert sad[0, 0] == 256 or expect_fs
        assert mask[0, 0] == expect_fs


def test_acbm_cond2_strict_and_scaled(orc):
    two = np.full((16, 16), 100, np.uint8)
    two[:, 8:] = 110                         # Intra_SAD = 1280; gamma*Intra = 320
    for k, expect_fs in [(64, 1), (63, 0)]:
        ref = two.astype(np.int32) + 1
        ref.ravel()[:k] += 1                 # SAD_PBM at (0,0) = 256 + k
        ref = ref.astype(np.uint8)
        _, _, mask, _, _ = _single(orc, two, ref, orc.params(0, 0, 1, 4, 28, 0))
        assert mask[0, 0] == expect_fs, k


# ----------------------------------------------------------------- ACBM invariants
def _acbm_inputs(seed, W=96, H=64):
    seq = synth.scene_sequence(seed, W, H, 3, n_objects=3, vmax=4)
    return seq


@pytest.mark.parametrize("N,M,p", [(16, 16, 4), (8, 8, 3), (16, 8, 5)])
def test_acbm_forced_fs_equals_fsbm(orc, N, M, p):
    seq = _acbm_inputs(N + M + p)
    lam = orc.lambda_q8(28)
    mv, J, sad = orc.fsbm(seq[1], seq[0], N, M, p, lam)
    amv, aJ, mask, asad, load = orc.acbm(seq[1], seq[0], N, M, p, lam,
                                         orc.params(alpha=0, beta=0, gamma_num=0))
    assert np.array_equal(mv, amv) and np.array_equal(J, aJ) and np.array_equal(sad, asad)
    assert np.all(mask == 1) and np.all(load == (2 * p + 1) ** 2)


def test_acbm_invariants_on_a_sequence(orc):
    seq = _acbm_inputs(77, 128, 96)
    lam = orc.lambda_q8(28)
    prev = None
    for t in range(1, seq.shape[0]):
        for prm in [orc.params(), orc.params(refine=0), orc.params(alpha=2 ** 30)]:
            mv, J, sad = orc.fsbm(seq[t], seq[t - 1], 16, 16, 8, lam)
            amv, aJ, mask, asad, load = orc.acbm(seq[t], seq[t - 1], 16, 16, 8, lam, prm, prev)
            assert np.all(J <= aJ)                                   # FSBM optimal
            fs = mask == 1
            assert np.array_equal(amv[fs], mv[fs]) and np.array_equal(aJ[fs], J[fs])
            assert np.all(load[fs] == 17 * 17)
            cap = 22 if prm.refine else 14
            assert np.all((load[~fs] >= 1) & (load[~fs] <= cap))
            if prm.alpha == 2 ** 30:
                assert not fs.any()
        prev = orc.acbm(seq[t], seq[t - 1], 16, 16, 8, lam, orc.params(), prev)[0]


# ----------------------------------------------------------------- ACBM predictor probes
D = (4, -3)          # probed block's motion; its match is at mv = (-4, 3)
U = (-3, 4)          # everybody else; match at (3, -4)
MARK = (5, 5)        # previous-field marker far from both matches and from 0
P6 = 6
CFG = dict(alpha=0, beta=0, gamma_num=1, gamma_den=4, qp=28, refine=1)   # cond 2 only


def _probe(orc, disp, prev, W=80, H=48):
    ref = synth.random_frame(99, W, H)
    cur = per_block_motion(ref, 16, 16, disp)
    return orc.acbm(cur, ref, 16, 16, P6, 0, orc.params(**CFG), prev)


def _field(val, BW=5, BH=3):
    f = np.zeros((BH, BW, 2), np.int16)
    f[..., 0], f[..., 1] = val
    return f


@pytest.mark.parametrize("nb,helps", [
    ((1, 1), True), ((1, 0), True), ((2, 0), True), ((3, 0), True),   # left, up-left, up, up-right
    ((0, 0), False), ((4, 0), False), ((0, 1), False), ((3, 1), False), ((2, 2), False),
])
def test_pbm_spatial_predictors(orc, nb, helps):
    """Block (2,1) moves by D, all others by U except neighbour nb (also D).
    The block finds its match without full search only through a spatial
    predictor that is computed before it (Sec. 2.2: mv5_t..mv8_t are not)."""
    disp = [[U] * 5 for _ in range(3)]
    disp[1][2] = D
    disp[nb[1]][nb[0]] = D
    mv, J, mask, sad, load = _probe(orc, disp, _field(MARK))
    assert tuple(mv[1, 2]) == (-D[0], -D[1]) and sad[1, 2] == 0
    assert mask[1, 2] == (0 if helps else 1)


@pytest.mark.parametrize("off,helps", [((dx, dy), True) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
                         + [((2, 0), False), ((-2, 0), False), ((2, 1), False), ((-2, -1), False)])
def test_pbm_temporal_predictors(orc, off, helps):
    """Block (2,1) moves by D, all others by U; the previous field holds the
    right vector only at (2,1)+off: it helps exactly for the 3x3 neighbourhood."""
    disp = [[U] * 5 for _ in range(3)]
    disp[1][2] = D
    prev = _field(MARK)
    prev[1 + off[1], 2 + off[0]] = (-D[0], -D[1])
    mv, J, mask, sad, load = _probe(orc, disp, prev)
    assert tuple(mv[1, 2]) == (-D[0], -D[1])
    assert mask[1, 2] == (0 if helps else 1)


def test_pbm_zero_predictor_and_ring(orc):
    # block (0,0) still: only the zero predictor finds it
    disp = [[U] * 5 for _ in range(3)]
    disp[0][0] = (0, 0)
    mv, J, mask, sad, load = _probe(orc, disp, _field(MARK))
    assert mask[0, 0] == 0 and tuple(mv[0, 0]) == (0, 0)
    # motion (1,-1) with a zero previous field: the only predictor of block
    # (0,0) is (0,0), and the +-1 ring around it reaches the match (-1,1)
    disp[0][0] = (1, -1)
    mv, J, mask, sad, load = _probe(orc, disp, None)
    assert mask[0, 0] == 0 and tuple(mv[0, 0]) == (-1, 1) and load[0, 0] == 9
    ref = synth.random_frame(99, 80, 48)
    cur = per_block_motion(ref, 16, 16, disp)
    prm = orc.params(**dict(CFG, refine=0))
    mv, J, mask, sad, load = orc.acbm(cur, ref, 16, 16, P6, 0, prm, None)
    assert mask[0, 0] == 1 and tuple(mv[0, 0]) == (-1, 1)


def test_pbm_load_counts_distinct_positions(orc):
    """Flat frames: every SAD is 0, the winner is (0,0), so the load is the
    number of distinct predictors plus the new ring positions."""
    W, H, BW, BH = 80, 48, 5, 3
    flat = np.full((H, W), 77, np.uint8)
    prev = np.zeros((BH, BW, 2), np.int16)
    for by in range(BH):
        for bx in range(BW):
            prev[by, bx] = (by * BW + bx - 7, 8)     # 15 distinct markers, far from 0
    nbrs = np.array([[sum(1 for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                          if 0 <= bx + dx < BW and 0 <= by + dy < BH)
                      for bx in range(BW)] for by in range(BH)])
    _, _, mask, _, load = orc.acbm(flat, flat, 16, 16, 8, 0, orc.params(), prev)
    assert np.all(mask == 0)
    assert np.array_equal(load, 9 + nbrs)                      # 13 / 15 / 18
    _, _, _, _, load0 = orc.acbm(flat, flat, 16, 16, 8, 0, orc.params(refine=0), prev)
    assert np.array_equal(load0, 1 + nbrs)
    # markers beyond p are clipped to the window edge and then counted once
    far = np.zeros((BH, BW, 2), np.int16)
    far[..., 0] = 30
    far[0, 0] = (20, 0)
    _, _, _, _, load1 = orc.acbm(flat, flat, 16, 16, 8, 0, orc.params(refine=0), far)
    assert np.all(load1 == 2)                                  # (0,0) and (8,0)


# ----------------------------------------------------------------- half-pel refinement
def brute_halfpel_pred(ref, N, M, x0, y0, hx, hy, pad):
    """Bilinear half-pel prediction of one block from an edge-padded copy of
    the reference (H.263 rounding), by whole-array slices: an implementation
    independent of the oracle's per-pixel loop."""
    ax, fx = hx >> 1, hx & 1          # floor division by 2 and the half flag
    ay, fy = hy >> 1, hy & 1
    r = np.pad(ref.astype(np.int64), pad, mode="edge")
    Y, X = y0 + ay + pad, x0 + ax + pad
    A = r[Y:Y + M, X:X + N]
    B = r[Y:Y + M, X + 1:X + 1 + N]
    C = r[Y + 1:Y + 1 + M, X:X + N]
    D = r[Y + 1:Y + 1 + M, X + 1:X + 1 + N]
    if fx and fy:
        return (A + B + C + D + 2) >> 2
    if fx:
        return (A + B + 1) >> 1
    if fy:
        return (A + C + 1) >> 1
    return A


def brute_halfpel(cur, ref, N, M, p, lam, mv_int):
    """Every block: the distinct clipped positions 2*mv + (dx, dy), cost
    256*SAD + lam*(bits(hx)+bits(hy)) with bits from the constructive
    Exp-Golomb encoder, lexicographic argmin (J, |h|_1, hy, hx)."""
    H, W = cur.shape
    BH, BW = H // M, W // N
    out_mv = np.zeros((BH, BW, 2), np.int64)
    out_J = np.zeros((BH, BW), np.int64)
    out_s = np.zeros((BH, BW), np.int64)
    pad = 2 * p + 4
    for by in range(BH):
        for bx in range(BW):
            cx = 2 * min(max(int(mv_int[by, bx, 0]), -p), p)
            cy = 2 * min(max(int(mv_int[by, bx, 1]), -p), p)
            cands = {(min(max(cx + dx, -2 * p), 2 * p), min(max(cy + dy, -2 * p), 2 * p))
                     for dy in (-1, 0, 1) for dx in (-1, 0, 1)}
            best = None
            for hx, hy in cands:
                pred = brute_halfpel_pred(ref, N, M, bx * N, by * M, hx, hy, pad)
                s = int(np.abs(cur[by * M:(by + 1) * M, bx * N:(bx + 1) * N].astype(np.int64) - pred).sum())
                J = 256 * s + lam * (len(eg_encode_signed(hx)) + len(eg_encode_signed(hy)))
                k = (J, abs(hx) + abs(hy), hy, hx)
                if best is None or k < best[0]:
                    best = (k, s)
            (J, _, hy, hx), s = best
            out_mv[by, bx] = (hx, hy)
            out_J[by, bx] = J
            out_s[by, bx] = s
    return out_mv, out_J, out_s


@pytest.mark.parametrize("W,H,N,M,p", [(48, 32, 16, 16, 4), (32, 32, 8, 8, 3), (24, 16, 4, 8, 2)])
def test_halfpel_matches_brute_force(orc, W, H, N, M, p):
    rng = np.random.default_rng(W * 7 + p)
    ref = synth.texture(rng, W, H)
    cur = np.clip(np.roll(ref, (1, -1), axis=(0, 1)).astype(int) + rng.integers(-6, 7, ref.shape),
                  0, 255).astype(np.uint8)
    BH, BW = H // M, W // N
    # integer fields: random, and the window corners (clipping at +-2p)
    fields = [rng.integers(-p, p + 1, (BH, BW, 2)).astype(np.int16),
              np.tile(np.array([p, -p], np.int16), (BH, BW, 1)),
              np.tile(np.array([-p, p], np.int16), (BH, BW, 1)),
              rng.integers(-p - 5, p + 6, (BH, BW, 2)).astype(np.int16)]   # outside: clipped
    for lam in (0, 6595):
        for f in fields:
            mv, J, s = orc.halfpel(cur, ref, N, M, p, lam, f)
            bmv, bJ, bs = brute_halfpel(cur, ref, N, M, p, lam, f)
            assert np.array_equal(mv, bmv) and np.array_equal(J, bJ) and np.array_equal(s, bs)
            assert np.all(np.abs(mv.astype(int)) <= 2 * p)


@pytest.mark.parametrize("hx0,hy0", [(3, -1), (-1, 2), (1, 1), (-3, -3)])
def test_halfpel_recovers_exact_half_pel_shift(orc, hx0, hy0):
    """cur is the reference interpolated at a known half-pel offset (away
    from the frame edges): with lambda = 0 the refinement around the
    integer vector next to it finds SAD 0 there."""
    rng = np.random.default_rng(5)
    W = H = 48
    N = M = 16
    p = 4
    ref = rng.integers(0, 256, (H, W)).astype(np.uint8)
    cur = ref.copy()
    by = bx = 1            # the centre block, well inside the frame
    cur[by * M:(by + 1) * M, bx * N:(bx + 1) * N] = brute_halfpel_pred(
        ref, N, M, bx * N, by * M, hx0, hy0, 2 * p + 4)
    mv_int = np.zeros((H // M, W // N, 2), np.int16)
    mv_int[by, bx] = ((hx0 + (hx0 > 0)) // 2, (hy0 + (hy0 > 0)) // 2)   # hx0 within +-1 of 2*mv
    assert all(abs(2 * int(mv_int[by, bx, i]) - h) <= 1 for i, h in enumerate((hx0, hy0)))
    mv, J, s = orc.halfpel(cur, ref, N, M, p, 0, mv_int)
    assert tuple(mv[by, bx]) == (hx0, hy0) and s[by, bx] == 0 and J[by, bx] == 0


def test_halfpel_flat_frame_keeps_the_cheapest_position(orc):
    """Constant frames: every position has SAD 0, so the rate decides; the
    zero vector has the shortest code (1+1 bits); around (1, 0) the nearest
    cheapest is (1, 0) in half units (3+1 bits), not (2, 0)."""
    ref = np.full((32, 32), 77, np.uint8)
    cur = ref.copy()
    z = np.zeros((2, 2, 2), np.int16)
    mv, J, s = orc.halfpel(cur, ref, 16, 16, 3, 6595, z)
    assert np.all(mv == 0) and np.all(J == 6595 * 2) and np.all(s == 0)
    one = np.zeros((2, 2, 2), np.int16)
    one[..., 0] = 1
    mv, J, s = orc.halfpel(cur, ref, 16, 16, 3, 6595, one)
    assert np.all(mv[..., 0] == 1) and np.all(mv[..., 1] == 0)
    assert np.all(J == 6595 * (3 + 1))


# ---------------------------------------------------------------------------
# SAD_deviation (Sec. 3.1)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("W,H,N,M,p", [(48, 32, 16, 16, 4), (32, 32, 8, 8, 3), (24, 16, 4, 8, 2),
                                       (32, 48, 16, 8, 5)])
def test_sad_deviation_matches_sad_volume(orc, W, H, N, M, p):
    """SAD_min and sum |SAD(u,v) - SAD_min| of every block against the brute
    SAD volume (edge-clamped reference, all (2p+1)^2 positions)."""
    rng = np.random.default_rng(W * 3 + H + p)
    ref = synth.texture(rng, W, H)
    cur = np.clip(np.roll(ref, (2, -1), axis=(0, 1)).astype(int) + rng.integers(-9, 10, ref.shape),
                  0, 255).astype(np.uint8)
    vol = brute_sad_volume(cur, ref, N, M, p)
    mn = vol.min(axis=(0, 1))
    dev = np.abs(vol - mn[None, None]).sum(axis=(0, 1))
    got_mn, got_dev = orc.sad_deviation(cur, ref, N, M, p)
    assert np.array_equal(got_mn, mn) and np.array_equal(got_dev, dev)
    assert np.all(got_mn > 0)                  # noise: no exact match anywhere


def test_sad_deviation_closed_forms(orc):
    """Flat frames: every position costs N*M*|a - b|, deviation 0.  A
    horizontal ramp ref(x, y) = x matched against itself, block away from the
    frame edges: SAD(u, v) = N*M*|u|, so SAD_min = 0 and the deviation is
    (2p+1) * N*M * p(p+1)."""
    for N, M, p in [(16, 16, 4), (8, 16, 3), (4, 4, 2)]:
        W, H = 4 * N, 3 * M
        cur = np.full((H, W), 200, np.uint8)
        ref = np.full((H, W), 93, np.uint8)
        mn, dev = orc.sad_deviation(cur, ref, N, M, p)
        assert np.all(mn == N * M * 107) and np.all(dev == 0)
        W, H = 64, 48
        ramp = np.tile(np.arange(W, dtype=np.uint8) + 40, (H, 1))
        mn, dev = orc.sad_deviation(ramp, ramp, N, M, p)
        bx, by = 1, 1                           # p < N, p < M: the window stays inside
        assert mn[by, bx] == 0
        assert dev[by, bx] == (2 * p + 1) * N * M * p * (p + 1)


@pytest.mark.parametrize("gx,gy", [(3, -2), (-4, 1), (0, 4)])
def test_sad_deviation_of_a_known_global_shift(orc, gx, gy):
    """A frame that is the reference displaced by a known vector g (edge
    clamp, no noise): the true position costs 0, so SAD_min = 0 in every block
    and the deviation is the plain sum of the SAD volume."""
    rng = np.random.default_rng(17)
    W, H, N, M, p = 64, 48, 16, 16, 5
    ref = synth.texture(rng, W, H)
    cur = synth.shifted_copy(ref, -gx, -gy)
    vol = brute_sad_volume(cur, ref, N, M, p)
    assert np.all(vol[gy + p, gx + p] == 0)
    mn, dev = orc.sad_deviation(cur, ref, N, M, p)
    assert np.all(mn == 0)
    assert np.array_equal(dev, vol.sum(axis=(0, 1)))


def test_sad_deviation_blocks_agree_with_the_frame_call(orc):
    """The sampled-block entry (used at frame sizes the whole-frame oracle is
    too slow for) returns the frame call's values at the listed blocks."""
    rng = np.random.default_rng(23)
    W, H, N, M, p = 64, 48, 8, 16, 6
    ref = synth.texture(rng, W, H)
    cur = np.clip(ref.astype(int) + rng.integers(-20, 21, ref.shape), 0, 255).astype(np.uint8)
    mn, dev = orc.sad_deviation(cur, ref, N, M, p)
    blocks = np.array([0, 5, 7, 8, 23, 17], np.int32)
    bmn, bdev = orc.sad_deviation_blocks(cur, ref, N, M, p, blocks)
    assert np.array_equal(bmn, mn.ravel()[blocks]) and np.array_equal(bdev, dev.ravel()[blocks])
    with pytest.raises(Exception):
        orc.sad_deviation_blocks(cur, ref, N, M, p, np.array([24], np.int32))


def test_acbm_full_search_set_shrinks_as_qp_rises(orc):
    """Cond. 1's threshold alpha + beta*Qp^2 grows with Qp and nothing else in
    a block's decision depends on Qp once lambda is held fixed: the blocks
    searched fully at a higher Qp are a subset of those at a lower Qp, and
    the load never grows."""
    frames = synth.load_sequence("textured-fast", 10, seed=500, n_frames=3)
    prev, _, _, _, _ = orc.acbm(frames[1], frames[0], 16, 16, 15, 6595, orc.params(qp=28), None)
    masks, loads = [], []
    for qp in (10, 16, 22, 28, 34, 40):
        _, _, mask, _, load = orc.acbm(frames[2], frames[1], 16, 16, 15, 6595, orc.params(qp=qp), prev)
        masks.append(mask)
        loads.append(load)
    for lo, hi, llo, lhi in zip(masks, masks[1:], loads, loads[1:]):
        assert np.all(hi <= lo) and np.all(lhi <= llo)
    assert masks[0].sum() > masks[-1].sum()


# ---------------------------------------------------------------------------
# FSBM with R coded against the median predictor (Sec. 2.1 R, Sec. 2.2
# differential coding; H.263-style median of left, upper, upper-right)
# ---------------------------------------------------------------------------
def brute_predictor(field, bx, by):
    """H.263 rules restated: left edge -> MV1 = 0; top row -> the predictor is
    MV1; right edge -> MV3 = 0; else the component-wise middle value."""
    BW = field.shape[1]
    mv1 = tuple(field[by, bx - 1]) if bx > 0 else (0, 0)
    if by == 0:
        return mv1
    mv2 = tuple(field[by - 1, bx])
    mv3 = tuple(field[by - 1, bx + 1]) if bx + 1 < BW else (0, 0)
    return tuple(sorted([mv1[c], mv2[c], mv3[c]])[1] for c in range(2))


def brute_fsbm_pred(cur, ref, N, M, p, lam):
    H, W = cur.shape
    BH, BW = H // M, W // N
    vol = brute_sad_volume(cur, ref, N, M, p)
    mvs = np.arange(-p, p + 1)
    bits = {d: len(eg_encode_signed(int(d))) for d in range(-2 * p, 2 * p + 1)}
    MY, MX = np.meshgrid(mvs, mvs, indexing="ij")
    L1 = (np.abs(MY) + np.abs(MX)).ravel()
    field = np.zeros((BH, BW, 2), np.int64)
    Jb = np.zeros((BH, BW), np.int64)
    Sb = np.zeros((BH, BW), np.int64)
    for by in range(BH):
        for bx in range(BW):
            px, py = brute_predictor(field, bx, by)
            R = np.array([[bits[int(x) - px] + bits[int(y) - py] for x in mvs] for y in mvs])
            j = (256 * vol[:, :, by, bx] + lam * R).ravel()
            k = np.lexsort((MX.ravel(), MY.ravel(), L1, j))[0]
            field[by, bx] = (MX.ravel()[k], MY.ravel()[k])
            Jb[by, bx] = j[k]
            Sb[by, bx] = vol[:, :, by, bx].ravel()[k]
    return field, Jb, Sb


def test_median_predictor_edge_rules(orc):
    """Hand-worked fields: interior median per component, the left-edge zero,
    the right-edge zero and the top-row copy of the left vector."""
    f = np.zeros((3, 3, 2), np.int16)
    f[0] = [(5, -1), (-2, 4), (7, 7)]
    f[1] = [(1, 1), (0, 0), (0, 0)]
    assert orc.median_predictor(f, 0, 0) == (0, 0)          # top-left: nothing coded yet
    assert orc.median_predictor(f, 1, 0) == (5, -1)         # top row: left vector
    assert orc.median_predictor(f, 2, 0) == (-2, 4)
    # (1,1): left (1,1), up (-2,4), up-right (7,7) -> (1, 4)
    assert orc.median_predictor(f, 1, 1) == (1, 4)
    # (0,1): left edge -> (0,0), up (5,-1), up-right (-2,4) -> (0, 0)
    assert orc.median_predictor(f, 0, 1) == (0, 0)
    # (2,1): left (0,0), up (7,7), right edge -> (0,0) -> (0, 0)
    assert orc.median_predictor(f, 2, 1) == (0, 0)
    f[1, 1] = (3, -6)
    # (2,1) again: left (3,-6), up (7,7), up-right 0 -> (3, 0)
    assert orc.median_predictor(f, 2, 1) == (3, 0)
    # (0,2): left 0, up (1,1), up-right (3,-6) -> (1, 0)
    assert orc.median_predictor(f, 0, 2) == (1, 0)


def blockwise_motion(W, H, N, M, p, seed):
    """cur: every block copied from the reference at its own random offset in
    [-p, p]^2 (edge clamp), 30 % of blocks flat instead, plus U{-12..12}
    noise: a field with many distinct vectors for the predictor to mix."""
    rng = np.random.default_rng(seed)
    ref = synth.texture(rng, W, H).astype(int)
    cur = np.zeros((H, W), int)
    for by in range(H // M):
        for bx in range(W // N):
            dx, dy = rng.integers(-p, p + 1, 2)
            ys = np.clip(np.arange(by * M, by * M + M) + dy, 0, H - 1)
            xs = np.clip(np.arange(bx * N, bx * N + N) + dx, 0, W - 1)
            cur[by * M:by * M + M, bx * N:bx * N + N] = ref[np.ix_(ys, xs)]
            if rng.random() < 0.3:
                cur[by * M:by * M + M, bx * N:bx * N + N] = rng.integers(100, 110)
    cur = np.clip(cur + rng.integers(-12, 13, cur.shape), 0, 255).astype(np.uint8)
    return cur, ref.astype(np.uint8)


@pytest.mark.parametrize("W,H,N,M,p", [(64, 48, 16, 16, 4), (40, 32, 8, 8, 3), (24, 32, 4, 8, 2)])
def test_fsbm_pred_matches_brute_force(orc, W, H, N, M, p):
    """Block-wise random motion (many distinct neighbour vectors), lambda from
    0 to values where the rate decides most blocks."""
    cur, ref = blockwise_motion(W, H, N, M, p, W + H)
    for lam in (0, 3000, 6595, 20000, 60000, 1 << 20):
        mv, J, sad = orc.fsbm_pred(cur, ref, N, M, p, lam)
        bmv, bJ, bs = brute_fsbm_pred(cur, ref, N, M, p, lam)
        assert np.array_equal(mv, bmv) and np.array_equal(J, bJ) and np.array_equal(sad, bs), lam


def test_fsbm_pred_reduces_to_fsbm_without_rate(orc):
    seq = synth.config_sequence("qcif", seed=3, n_frames=2)
    mv, J, sad = orc.fsbm_pred(seq[1], seq[0], 16, 16, 7, 0)
    fmv, fJ, fs = orc.fsbm(seq[1], seq[0], 16, 16, 7, 0)
    assert np.array_equal(mv, fmv) and np.array_equal(J, fJ) and np.array_equal(sad, fs)


def test_fsbm_pred_follows_a_global_shift(orc):
    """Noise-free global shift g: SAD 0 at g in every block; once the first
    block has g every predictor is g, so R is 2 bits there and the whole field
    is g, J = 2*lambda after the first block."""
    rng = np.random.default_rng(8)
    ref = synth.texture(rng, 64, 64)
    gx, gy = 3, -2
    cur = synth.shifted_copy(ref, -gx, -gy)
    lam = 6595
    mv, J, sad = orc.fsbm_pred(cur, ref, 16, 16, 5, lam)
    assert np.all(mv[..., 0] == gx) and np.all(mv[..., 1] == gy) and np.all(sad == 0)
    assert np.all(J.ravel()[1:] == 2 * lam)


def test_fsbm_pred_blocks_agree_with_the_frame_call(orc):
    """Given the frame call's own field, every block's one-block step
    reproduces it (the sampled check used at large frame sizes)."""
    cur, ref = blockwise_motion(64, 48, 8, 8, 3, 77)
    mv, J, sad = orc.fsbm_pred(cur, ref, 8, 8, 3, 6595)
    blocks = np.arange(mv.shape[0] * mv.shape[1], dtype=np.int32)
    bmv, bJ, bs = orc.fsbm_pred_blocks(cur, ref, 8, 8, 3, 6595, mv, blocks)
    assert np.array_equal(bmv, mv.reshape(-1, 2)) and np.array_equal(bJ, J.ravel())
    assert np.array_equal(bs, sad.ravel())


# ----------------------------------------------------------------- block-list entries
@pytest.mark.parametrize("W,H,N,M,p", [(48, 32, 16, 16, 3), (40, 24, 8, 4, 2), (24, 48, 4, 16, 3)])
def test_fsbm_blocks_match_brute_force(orc, W, H, N, M, p):
    """The block-list full search (the oracle of the large-frame sampled
    checks) against the numpy brute force of Sec. 2.3, on grids with BW != BH
    so that a transposed or mis-scaled block index shows: every block once in
    a shuffled order, plus repeats; outputs follow the list's order."""
    rng = np.random.default_rng(W * H + N * M + p)
    ref = synth.texture(rng, W, H)
    cur = np.clip(np.roll(ref, (1, -2), (0, 1)).astype(int) + rng.integers(-9, 10, ref.shape),
                  0, 255).astype(np.uint8)
    BW, BH = W // N, H // M
    assert BW != BH
    lam = 6595
    wmv, wJ, wS = brute_fsbm(cur, ref, N, M, p, lam)
    blocks = np.concatenate([rng.permutation(BW * BH), rng.integers(0, BW * BH, 5)]).astype(np.int32)
    mv, J, sad = orc.fsbm_blocks(cur, ref, N, M, p, lam, blocks, nthreads=2)
    assert np.array_equal(mv, wmv.reshape(-1, 2)[blocks])
    assert np.array_equal(J, wJ.ravel()[blocks])
    assert np.array_equal(sad, wS.ravel()[blocks])
    fmv, fJ, fS = orc.fsbm(cur, ref, N, M, p, lam)
    assert np.array_equal(mv, fmv.reshape(-1, 2)[blocks]) and np.array_equal(J, fJ.ravel()[blocks])
    with pytest.raises(Exception):
        orc.fsbm_blocks(cur, ref, N, M, p, lam, np.array([BW * BH], np.int32))


@pytest.mark.parametrize("N,M,p", [(16, 16, 4), (8, 16, 3), (16, 8, 5)])
def test_acbm_blocks_agree_with_the_frame_call(orc, N, M, p):
    """Given the frame call's own final field as the current-frame field (and
    the same previous field), the block-list ACBM reproduces every block of
    the frame call (Sec. 3.2: each block's result depends only on its
    predictors' final vectors): vector, J, mask, SAD and load, with the blocks
    listed in a shuffled order on a grid with BW != BH."""
    seq = _acbm_inputs(5 * N + M + p, 112, 64)
    lam = orc.lambda_q8(28)
    prm = orc.params(alpha=300, beta=1)          # a mix of passing and full-searched blocks
    prev = orc.acbm(seq[1], seq[0], N, M, p, lam, prm)[0]
    mv, J, mask, sad, load = orc.acbm(seq[2], seq[1], N, M, p, lam, prm, prev)
    BH, BW = J.shape
    assert BW != BH and mask.any() and not mask.all()
    rng = np.random.default_rng(N * M * p)
    blocks = rng.permutation(BW * BH).astype(np.int32)
    bmv, bJ, bmask, bsad, bload = orc.acbm_blocks(seq[2], seq[1], N, M, p, lam, prm, mv, blocks,
                                                  prev_mv=prev)
    assert np.array_equal(bmv, mv.reshape(-1, 2)[blocks])
    assert np.array_equal(bJ, J.ravel()[blocks])
    assert np.array_equal(bmask, mask.ravel()[blocks])
    assert np.array_equal(bsad, sad.ravel()[blocks])
    assert np.array_equal(bload, load.ravel()[blocks])

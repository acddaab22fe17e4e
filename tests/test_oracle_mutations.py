"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of oracle/me_oracle.c (a dropped
term, a wrong sign or index, a transposed operand, a non-strict comparison,
a wrong neighbourhood ...), compiles it on the CPU and runs the pins of
tests/test_oracle_pins.py against it: at least one pin must fail.  The real
oracle passes all of them (test_oracle_pins.py itself)."""
import os

import pytest

import oracle
import test_oracle_pins as pins

MUTANTS = {
    "mvx/mvy transposed in SAD": (
        "int rx = clampi(x0 + i + mvx, 0, W - 1);", "int rx = clampi(x0 + i + mvy, 0, W - 1);"),
    "wrong sign of mvx": (
        "int rx = clampi(x0 + i + mvx, 0, W - 1);", "int rx = clampi(x0 + i - mvx, 0, W - 1);"),
    "rate term dropped from J": (
        "return 256u * sad + lambda_q8 * (uint32_t)rate_bits(mvx, mvy);", "return 256u * sad;"),
    "R counts mvx twice": (
        "return oracle_mv_bits(mvx) + oracle_mv_bits(mvy); }",
        "return oracle_mv_bits(mvx) + oracle_mv_bits(mvx); }"),
    "Exp-Golomb length off by one": ("    return 2 * lg + 1;", "    return 2 * lg + 2;"),
    "lambda rounding dropped": ("(23552LL * qp + 50) / 100", "(23552LL * qp) / 100"),
    "|mv|_1 tie level dropped": ("    if (l1 != l2) return l1 < l2;\n", ""),
    "raster tie order transposed": (
        "    if (mvy1 != mvy2) return mvy1 < mvy2;\n    return mvx1 < mvx2;",
        "    if (mvx1 != mvx2) return mvx1 < mvx2;\n    return mvy1 < mvy2;"),
    "zero padding instead of edge clamp": (
        "            int b = ref[(size_t)ry * W + rx];",
        "            int b = (x0 + i + mvx < 0 || x0 + i + mvx >= W || y0 + j + mvy < 0 ||"
        " y0 + j + mvy >= H) ? 0 : ref[(size_t)ry * W + rx];"),
    "Intra_SAD not scaled by NM": (
        "int64_t d = (int64_t)NM * cur[(size_t)(by * M + j) * W + bx * N + i] - S;",
        "int64_t d = (int64_t)cur[(size_t)(by * M + j) * W + bx * N + i] - S / NM;"),
    "cond. 1 not strict": ("    int cond1 = lhs1 < rhs1;", "    int cond1 = lhs1 <= rhs1;"),
    "cond. 2 not strict": ("    int cond2 = lhs2 < rhs2;", "    int cond2 = lhs2 <= rhs2;"),
    "cond. 2 missing the NM scale": (
        "    int64_t lhs2 = (int64_t)prm->gamma_den * NM * sad_pbm;",
        "    int64_t lhs2 = (int64_t)prm->gamma_den * sad_pbm;"),
    "beta * Qp instead of beta * Qp^2": (
        "(int64_t)prm->beta * qp * qp", "(int64_t)prm->beta * qp"),
    "right neighbour instead of up-right": (
        "    static const int sp_dy[4] = {0, -1, -1, -1};",
        "    static const int sp_dy[4] = {0, -1, -1, 0};"),
    "up-left dropped from the spatial set": (
        "    static const int sp_dx[4] = {-1, -1, 0, 1};",
        "    static const int sp_dx[4] = {-1, 0, 0, 1};"),
    "temporal set reduced to the co-located block": (
        "    for (int dy = -1; dy <= 1; dy++) {\n        for (int dx = -1; dx <= 1; dx++) {\n"
        "            int nx = bx + dx, ny = by + dy;",
        "    for (int dy = 0; dy <= 0; dy++) {\n        for (int dx = 0; dx <= 0; dx++) {\n"
        "            int nx = bx + dx, ny = by + dy;"),
    "zero predictor dropped": (
        "    pbm_try(&s, cur, ref, W, H, N, M, x0, y0, lambda_q8, 0, 0);\n", ""),
    "refinement never runs": ("    if (prm->refine) {", "    if (0) {"),
    "repeated positions counted twice": ("    if (s->seen[idx]) return;\n", ""),
    "fallback keeps the PBM vector": (
        "        full_search_block(cur, ref, W, H, N, M, p, lambda_q8, bx, by, mvx_o, mvy_o, J_o, sad_o);",
        "        *mvx_o = s.bmx; *mvy_o = s.bmy; *J_o = s.bJ; *sad_o = s.bS;"),
    "fallback load not (2p+1)^2": (
        "        *load_o = (uint32_t)((2 * p + 1) * (2 * p + 1));", "        *load_o = (uint32_t)s.count;"),
    "half-pel average not rounded": (
        "    if (fx && !fy) return (A + B + 1) >> 1;", "    if (fx && !fy) return (A + B) >> 1;"),
    "half-pel diagonal rounding off": (
        "    return (A + B + C + D + 2) >> 2;", "    return (A + B + C + D + 1) >> 2;"),
    "half-pel vertical uses the wrong neighbour": (
        "    if (!fx && fy) return (A + C + 1) >> 1;", "    if (!fx && fy) return (A + B + 1) >> 1;"),
    "half-pel floor division truncates negatives": (
        "    int ax = hx >= 0 ? hx / 2 : -((-hx + 1) / 2);", "    int ax = hx / 2;"),
    "half-pel rate in integer units": (
        "                    uint32_t J = 256u * s + lambda_q8 * (uint32_t)rate_bits(hx, hy);",
        "                    uint32_t J = 256u * s + lambda_q8 * (uint32_t)rate_bits(hx / 2, hy / 2);"),
    "half-pel clip at p instead of 2p": (
        "                    int hx = clampi(cx + dx, -2 * p, 2 * p), hy = clampi(cy + dy, -2 * p, 2 * p);",
        "                    int hx = clampi(cx + dx, -p, p), hy = clampi(cy + dy, -p, p);"),
    "half-pel centre not doubled": (
        "            int cx = 2 * clampi(mv_int[2 * b], -p, p), cy = 2 * clampi(mv_int[2 * b + 1], -p, p);",
        "            int cx = clampi(mv_int[2 * b], -p, p), cy = clampi(mv_int[2 * b + 1], -p, p);"),
    "SAD_deviation window misses the last column": (
        "        for (int u = -p; u <= p; u++) {\n"
        "            uint32_t s = block_sad(cur, ref, W, H, N, M, bx * N, by * M, u, v);",
        "        for (int u = -p; u < p; u++) {\n"
        "            uint32_t s = block_sad(cur, ref, W, H, N, M, bx * N, by * M, u, v);"),
    "SAD_deviation minimum starts at zero": (
        "            if ((u == -p && v == -p) || s < mn) mn = s;",
        "            if (s < mn) mn = s;"),
    "SAD_deviation block origin transposed": (
        "block_sad(cur, ref, W, H, N, M, bx * N, by * M, u, v);",
        "block_sad(cur, ref, W, H, N, M, bx * M, by * N, u, v);"),
    "median predictor takes the largest value": (
        "    return c < lo ? lo : (c > hi ? hi : c);", "    return c > hi ? c : hi;"),
    "top row predicts from the upper neighbours": (
        "    if (by == 0) {\n        *pmx = m1x;", "    if (by < 0) {\n        *pmx = m1x;"),
    "right edge keeps a stale upper-right vector": (
        "    if (bx + 1 < BW) {\n        m3x", "    if (bx < BW) {\n        m3x"),
    "block-list search takes the block index transposed": (
        "lambda_q8, blocks[k] % BW, blocks[k] / BW,", "lambda_q8, blocks[k] / BH, blocks[k] % BH,"),
    "block-list search scales the index by the grid height": (
        "lambda_q8, blocks[k] % BW, blocks[k] / BW,", "lambda_q8, blocks[k] % BH, blocks[k] / BH,"),
    "block-list search writes outputs by block index": (
        "        J_out[k] = J;\n        if (sad_out) sad_out[k] = s;\n    }\n    return OR_OK;\n}\n\ntypedef",
        "        J_out[blocks[k]] = J;\n        if (sad_out) sad_out[k] = s;\n    }\n    return OR_OK;\n}\n\ntypedef"),
    "block-list ACBM takes the block index transposed": (
        "prm, b % BW, b / BW,", "prm, b / BH, b % BH,"),
    "block-list ACBM reads Intra_SAD by list position": (
        "prm, b % BW, b / BW,\n                   intra[b], seen,",
        "prm, b % BW, b / BW,\n                   intra[k], seen,"),
    "predicted rate coded against zero": (
        "(uint32_t)(oracle_mv_bits(mvx - pmx) +", "(uint32_t)(oracle_mv_bits(mvx) +"),
}


def _pin_suite(v):
    yield lambda: pins.test_lambda_is_092_qp_in_q8(v)
    yield lambda: pins.test_mv_bits_match_exp_golomb_encoder(v)
    yield lambda: pins.test_intra_sad_exact_rational_mean(v, 16, 16)
    yield lambda: pins.test_intra_sad_closed_forms(v)
    for args in [(48, 32, 16, 16, 4), (32, 32, 8, 8, 2), (24, 16, 4, 8, 4)]:
        yield lambda args=args: pins.test_fsbm_matches_brute_force(v, *args)
    yield lambda: pins.test_fsbm_recovers_exact_shift(v, 3, -2)
    yield lambda: pins.test_fsbm_tie_breaks(v)
    yield lambda: pins.test_acbm_cond1_strict_and_scaled(v)
    yield lambda: pins.test_acbm_cond2_strict_and_scaled(v)
    yield lambda: pins.test_acbm_forced_fs_equals_fsbm(v, 16, 16, 4)
    yield lambda: pins.test_paper_constants(v)
    yield lambda: pins.test_pbm_zero_predictor_and_ring(v)
    yield lambda: pins.test_pbm_load_counts_distinct_positions(v)
    for nb, helps in [((1, 1), True), ((1, 0), True), ((2, 0), True), ((3, 0), True),
                      ((0, 1), False), ((4, 0), False)]:
        yield lambda nb=nb, helps=helps: pins.test_pbm_spatial_predictors(v, nb, helps)
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            yield lambda dx=dx, dy=dy: pins.test_pbm_temporal_predictors(v, (dx, dy), True)
    yield lambda: pins.test_acbm_invariants_on_a_sequence(v)
    for args in [(48, 32, 16, 16, 4), (24, 16, 4, 8, 2)]:
        yield lambda args=args: pins.test_halfpel_matches_brute_force(v, *args)
    for hx0, hy0 in [(3, -1), (-1, 2), (1, 1), (-3, -3)]:
        yield lambda hx0=hx0, hy0=hy0: pins.test_halfpel_recovers_exact_half_pel_shift(v, hx0, hy0)
    yield lambda: pins.test_halfpel_flat_frame_keeps_the_cheapest_position(v)
    for args in [(48, 32, 16, 16, 4), (24, 16, 4, 8, 2), (32, 48, 16, 8, 5)]:
        yield lambda args=args: pins.test_sad_deviation_matches_sad_volume(v, *args)
    yield lambda: pins.test_acbm_full_search_set_shrinks_as_qp_rises(v)
    yield lambda: pins.test_median_predictor_edge_rules(v)
    for args in [(64, 48, 16, 16, 4), (40, 32, 8, 8, 3)]:
        yield lambda args=args: pins.test_fsbm_pred_matches_brute_force(v, *args)
    yield lambda: pins.test_fsbm_pred_reduces_to_fsbm_without_rate(v)
    yield lambda: pins.test_fsbm_pred_follows_a_global_shift(v)
    yield lambda: pins.test_sad_deviation_closed_forms(v)
    yield lambda: pins.test_sad_deviation_of_a_known_global_shift(v, 3, -2)
    for args in [(48, 32, 16, 16, 3), (24, 48, 4, 16, 3)]:
        yield lambda args=args: pins.test_fsbm_blocks_match_brute_force(v, *args)
    yield lambda: pins.test_acbm_blocks_agree_with_the_frame_call(v, 8, 16, 3)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation target not unique: {old!r}"
    so = oracle.compile_variant(src.replace(old, new), os.path.join(str(tmp_path), "mut.so"))
    v = oracle.Variant(so)
    for check in _pin_suite(v):
        try:
            check()
        except Exception:
            return      # caught
    pytest.fail(f"no pin caught the mutant: {name}")


def test_unmutated_copy_passes_all_pins(tmp_path):
    so = oracle.compile_variant(oracle.source_text(), os.path.join(str(tmp_path), "same.so"))
    v = oracle.Variant(so)
    for check in _pin_suite(v):
        check()

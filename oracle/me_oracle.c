/*
 * me_oracle.c -- plain, slow CPU oracle for integer-pel block-matching motion
 * estimation: full search (FSBM) and adaptive cost block matching (ACBM).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA library is checked against.  It shares no code, header, table or
 * constant with the library under paper_0710_4819_gb300/; only tests/, the
 * smoke check in __graft_entry__.py and the cpu_baseline / reference legs of
 * bench.py may load it.  Nothing on the product path may call it.
 *
 * Everything is integer arithmetic and written for a reader checking it
 * against the paper (Lopez, Callico, Lopez, Sarmiento, "A High Quality/Low
 * Computational Cost Technique for Block Matching Motion Estimation"):
 *
 *   Sec. 2.1, eq. J      J(mv) = D(mv) + lambda * R(mv)
 *   Sec. 2.1, eq. SAD    D = SAD(mvx,mvy) = sum_{i<N} sum_{j<M}
 *                              |p_t(i,j) - p_{t-1}(i+mvx, j+mvy)|
 *                        i runs over N and pairs with mvx, so N is the block
 *                        width and mvx the horizontal component.
 *   Sec. 2.2             PBM: predictors from the spatio-temporal
 *                        neighbourhood (Fig. 2), keep the best, refine.
 *   Sec. 2.3             FSBM: all (2p+1)^2 integer positions.
 *   Sec. 3.1, eq. Intra_SAD   sum |p_t(i,j) - mu|, mu = block mean.
 *   Sec. 3.1, eq. SAD_deviation  sum over the evaluated positions of
 *                        |SAD(u,v) - SAD_min|, SAD_min the least SAD among
 *                        them (here: the (2p+1)^2 positions of the full search).
 *   Sec. 3.2             ACBM: Intra_SAD, then PBM, then
 *                        cond. 1  Intra_SAD + SAD_PBM < alpha + beta*Qp^2
 *                        cond. 2  SAD_PBM < gamma * Intra_SAD
 *                        and a full search only when neither holds.
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - reference pixels outside the frame take the nearest edge pixel;
 *   - lambda = 0.92*Qp, carried in Q8 fixed point: lambda_q8 = round(235.52*Qp);
 *     the cost is kept as J_q8 = 256*SAD + lambda_q8*R;
 *   - R(mv) = L(mvx) + L(mvy), L = length of the signed Exp-Golomb code of the
 *     component in integer-pel units (motion vector coded against zero);
 *   - ties: lowest J, then smallest |mvx|+|mvy|, then smaller mvy, then
 *     smaller mvx;
 *   - Intra_SAD is carried scaled by NM so the real mean needs no rounding:
 *     IntraSAD_x = sum |NM*p - S| = NM * Intra_SAD, S = sum of the block;
 *   - PBM predictors: final vectors of the left, up-left, up and up-right
 *     blocks of the current frame; the 3x3 blocks around the block in the
 *     previous frame's field; and (0,0).  Blocks outside the grid are skipped,
 *     each component is clipped to [-p,p], repeated positions are evaluated
 *     once.  PBM keeps the lowest J (equal to "lowest SAD" when lambda = 0);
 *   - refinement: one pass over the 8 integer neighbours of the best
 *     predictor (clipped to [-p,p], positions already evaluated skipped);
 *   - SAD_PBM is the SAD of the refined PBM winner;
 *   - the load of a block is the number of distinct positions evaluated:
 *     (2p+1)^2 when the full search ran.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_SHAPE 2
#define OR_ERR_NOMEM 4

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
static int absi(int v) { return v < 0 ? -v : v; }

/* lambda "proportional to Qp" (Sec. 2.1): 0.92*Qp in Q8, rounded half up. */
uint32_t oracle_lambda_q8(int qp) { return (uint32_t)((23552LL * qp + 50) / 100); }

/* Bits of one motion-vector component: signed Exp-Golomb code length.
 * v > 0 maps to code number 2v-1, v <= 0 to -2v; a code number k takes
 * 2*floor(log2(k+1)) + 1 bits. */
int oracle_mv_bits(int v)
{
    unsigned k = v > 0 ? 2u * (unsigned)v - 1u : 2u * (unsigned)(-v);
    unsigned x = k + 1u;
    int lg = 0;
    while (x > 1u) { x >>= 1; lg++; }
    return 2 * lg + 1;
}

/* R(mvx,mvy) of eq. J: bits of both components. */
static int rate_bits(int mvx, int mvy) { return oracle_mv_bits(mvx) + oracle_mv_bits(mvy); }

/* eq. SAD for the block whose top-left pixel is (x0,y0), with the reference
 * pixel (x0+i+mvx, y0+j+mvy) taken at the nearest in-frame position. */
static uint32_t block_sad(const uint8_t *cur, const uint8_t *ref, int W, int H,
                          int N, int M, int x0, int y0, int mvx, int mvy)
{
    uint32_t s = 0;
    for (int j = 0; j < M; j++) {
        for (int i = 0; i < N; i++) {
            int a = cur[(size_t)(y0 + j) * W + (x0 + i)];
            int rx = clampi(x0 + i + mvx, 0, W - 1);
            int ry = clampi(y0 + j + mvy, 0, H - 1);
            int b = ref[(size_t)ry * W + rx];
            s += (uint32_t)absi(a - b);
        }
    }
    return s;
}

/* eq. J with the Q8 lambda: J_q8 = 256*SAD + lambda_q8*R. */
static uint32_t cost_q8(uint32_t sad, uint32_t lambda_q8, int mvx, int mvy)
{
    return 256u * sad + lambda_q8 * (uint32_t)rate_bits(mvx, mvy);
}

/* The tie-broken order on candidates: is (J1, mv1) better than (J2, mv2)? */
static int better(uint32_t J1, int mvx1, int mvy1, uint32_t J2, int mvx2, int mvy2)
{
    if (J1 != J2) return J1 < J2;
    int l1 = absi(mvx1) + absi(mvy1), l2 = absi(mvx2) + absi(mvy2);
    if (l1 != l2) return l1 < l2;
    if (mvy1 != mvy2) return mvy1 < mvy2;
    return mvx1 < mvx2;
}

static int check_shape(int W, int H, int N, int M, int p, uint32_t lambda_q8)
{
    if (!(N == 4 || N == 8 || N == 16) || !(M == 4 || M == 8 || M == 16)) return OR_ERR_ARG;
    if (p < 1 || p > 64) return OR_ERR_ARG;
    if (lambda_q8 > (1u << 20)) return OR_ERR_ARG;
    if (W < N || H < M || W > 16384 || H > 16384) return OR_ERR_SHAPE;
    if (W % N != 0 || H % M != 0) return OR_ERR_SHAPE;
    return OR_OK;
}

/* Eq. Intra_SAD (Sec. 3.1) for every block, scaled by NM:
 * out[b] = sum |NM*p - S| = NM * sum |p - S/NM|. */
int oracle_intra_sad(const uint8_t *cur, int W, int H, int N, int M, uint32_t *out)
{
    if (!cur || !out) return OR_ERR_ARG;
    int st = check_shape(W, H, N, M, 1, 0);
    if (st) return st;
    int BW = W / N, BH = H / M, NM = N * M;
    for (int by = 0; by < BH; by++) {
        for (int bx = 0; bx < BW; bx++) {
            int64_t S = 0;
            for (int j = 0; j < M; j++)
                for (int i = 0; i < N; i++) S += cur[(size_t)(by * M + j) * W + bx * N + i];
            int64_t acc = 0;
            for (int j = 0; j < M; j++)
                for (int i = 0; i < N; i++) {
                    int64_t d = (int64_t)NM * cur[(size_t)(by * M + j) * W + bx * N + i] - S;
                    acc += d < 0 ? -d : d;
                }
            out[by * BW + bx] = (uint32_t)acc;
        }
    }
    return OR_OK;
}

/* Full search for one block (Sec. 2.3): every mv in [-p,p]^2, keep the best
 * under the tie-broken order. */
static void full_search_block(const uint8_t *cur, const uint8_t *ref, int W, int H, int N, int M,
                              int p, uint32_t lambda_q8, int bx, int by,
                              int *mvx_o, int *mvy_o, uint32_t *J_o, uint32_t *sad_o)
{
    int x0 = bx * N, y0 = by * M;
    int bmx = 0, bmy = 0;
    uint32_t bJ = 0, bS = 0;
    int have = 0;
    for (int mvy = -p; mvy <= p; mvy++) {
        for (int mvx = -p; mvx <= p; mvx++) {
            uint32_t s = block_sad(cur, ref, W, H, N, M, x0, y0, mvx, mvy);
            uint32_t J = cost_q8(s, lambda_q8, mvx, mvy);
            if (!have || better(J, mvx, mvy, bJ, bmx, bmy)) {
                have = 1; bJ = J; bS = s; bmx = mvx; bmy = mvy;
            }
        }
    }
    *mvx_o = bmx; *mvy_o = bmy; *J_o = bJ; *sad_o = bS;
}

/* FSBM over a whole frame.  mv_out is [BH][BW][2] as (mvx, mvy); sad_out may
 * be NULL.  nthreads > 1 splits the block loop over OpenMP threads; every
 * block is independent, so the result does not depend on it. */
int oracle_fsbm(const uint8_t *cur, const uint8_t *ref, int W, int H, int N, int M, int p,
                uint32_t lambda_q8, int16_t *mv_out, uint32_t *J_out, uint32_t *sad_out,
                int nthreads)
{
    if (!cur || !ref || !mv_out || !J_out) return OR_ERR_ARG;
    int st = check_shape(W, H, N, M, p, lambda_q8);
    if (st) return st;
    int BW = W / N, BH = H / M;
    int nb = BW * BH;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int b = 0; b < nb; b++) {
        int mx, my;
        uint32_t J, s;
        full_search_block(cur, ref, W, H, N, M, p, lambda_q8, b % BW, b / BW, &mx, &my, &J, &s);
        mv_out[2 * b] = (int16_t)mx;
        mv_out[2 * b + 1] = (int16_t)my;
        J_out[b] = J;
        if (sad_out) sad_out[b] = s;
    }
    return OR_OK;
}

/* FSBM for a list of blocks only (sampled checks of large frames).
 * blocks[k] is a block index by*BW+bx; outputs are indexed by k. */
int oracle_fsbm_blocks(const uint8_t *cur, const uint8_t *ref, int W, int H, int N, int M,
                       int p, uint32_t lambda_q8, const int32_t *blocks, int nblocks,
                       int16_t *mv_out, uint32_t *J_out, uint32_t *sad_out, int nthreads)
{
    if (!cur || !ref || !blocks || !mv_out || !J_out || nblocks < 0) return OR_ERR_ARG;
    int st = check_shape(W, H, N, M, p, lambda_q8);
    if (st) return st;
    int BW = W / N, BH = H / M;
    for (int k = 0; k < nblocks; k++)
        if (blocks[k] < 0 || blocks[k] >= BW * BH) return OR_ERR_ARG;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int k = 0; k < nblocks; k++) {
        int mx, my;
        uint32_t J, s;
        full_search_block(cur, ref, W, H, N, M, p, lambda_q8, blocks[k] % BW, blocks[k] / BW,
                          &mx, &my, &J, &s);
        mv_out[2 * k] = (int16_t)mx;
        mv_out[2 * k + 1] = (int16_t)my;
        J_out[k] = J;
        if (sad_out) sad_out[k] = s;
    }
    return OR_OK;
}

typedef struct {
    int32_t alpha, beta, gamma_num, gamma_den, qp, refine;
} oracle_acbm_params;

static int check_params(const oracle_acbm_params *prm)
{
    if (!prm) return OR_ERR_ARG;
    if (prm->gamma_den < 1 || prm->gamma_num < 0) return OR_ERR_ARG;
    if (prm->qp < 0 || prm->qp > 1023) return OR_ERR_ARG;
    if (prm->refine != 0 && prm->refine != 1) return OR_ERR_ARG;
    return OR_OK;
}

/* Book-keeping of one block's PBM search: which window positions have been
 * evaluated (for the load count) and the best one so far. */
typedef struct {
    int p;
    unsigned char *seen; /* (2p+1)^2 flags, index (mvy+p)*(2p+1) + (mvx+p) */
    int count;
    int have;
    int bmx, bmy;
    uint32_t bJ, bS;
} pbm_state;

static void pbm_try(pbm_state *s, const uint8_t *cur, const uint8_t *ref, int W, int H, int N,
                    int M, int x0, int y0, uint32_t lambda_q8, int mvx, int mvy)
{
    mvx = clampi(mvx, -s->p, s->p);
    mvy = clampi(mvy, -s->p, s->p);
    int idx = (mvy + s->p) * (2 * s->p + 1) + (mvx + s->p);
    if (s->seen[idx]) return;
    s->seen[idx] = 1;
    s->count++;
    uint32_t sad = block_sad(cur, ref, W, H, N, M, x0, y0, mvx, mvy);
    uint32_t J = cost_q8(sad, lambda_q8, mvx, mvy);
    if (!s->have || better(J, mvx, mvy, s->bJ, s->bmx, s->bmy)) {
        s->have = 1; s->bJ = J; s->bS = sad; s->bmx = mvx; s->bmy = mvy;
    }
}

/* One ACBM block (Sec. 3.2) given the vectors it may use as predictors.
 * cur_field holds the final vectors of the blocks already done in this frame
 * (only the left, up-left, up and up-right entries are read); prev_field is
 * the previous frame's field (NULL = all zero).  intra_x is the scaled
 * Intra_SAD of the block. */
static void acbm_block(const uint8_t *cur, const uint8_t *ref, int W, int H, int N, int M, int p,
                       uint32_t lambda_q8, const int16_t *cur_field, const int16_t *prev_field,
                       const oracle_acbm_params *prm, int bx, int by, uint32_t intra_x,
                       unsigned char *seen, int *mvx_o, int *mvy_o, uint32_t *J_o,
                       uint32_t *sad_o, uint8_t *mask_o, uint32_t *load_o)
{
    int BW = W / N, BH = H / M, NM = N * M;
    int x0 = bx * N, y0 = by * M;
    pbm_state s;
    s.p = p; s.seen = seen; s.count = 0; s.have = 0;
    s.bmx = s.bmy = 0; s.bJ = s.bS = 0;
    memset(seen, 0, (size_t)(2 * p + 1) * (2 * p + 1));

    /* PBM step 1 + 2 (Sec. 2.2): predictors that are already computed. The
     * spatial ones are the current-frame blocks before this one in raster
     * order that touch it: left, up-left, up, up-right.  The blocks right of
     * and below it (mv5_t..mv8_t in Fig. 2) are not computed yet. */
    static const int sp_dx[4] = {-1, -1, 0, 1};
    static const int sp_dy[4] = {0, -1, -1, -1};
    for (int k = 0; k < 4; k++) {
        int nx = bx + sp_dx[k], ny = by + sp_dy[k];
        if (nx < 0 || nx >= BW || ny < 0 || ny >= BH) continue;
        const int16_t *v = cur_field + 2 * (ny * BW + nx);
        pbm_try(&s, cur, ref, W, H, N, M, x0, y0, lambda_q8, v[0], v[1]);
    }
    /* Temporal predictors: the 3x3 blocks around this one, previous frame. */
    for (int dy = -1; dy <= 1; dy++) {
        for (int dx = -1; dx <= 1; dx++) {
            int nx = bx + dx, ny = by + dy;
            if (nx < 0 || nx >= BW || ny < 0 || ny >= BH) continue;
            int mvx = 0, mvy = 0;
            if (prev_field) {
                mvx = prev_field[2 * (ny * BW + nx)];
                mvy = prev_field[2 * (ny * BW + nx) + 1];
            }
            pbm_try(&s, cur, ref, W, H, N, M, x0, y0, lambda_q8, mvx, mvy);
        }
    }
    /* The zero vector. */
    pbm_try(&s, cur, ref, W, H, N, M, x0, y0, lambda_q8, 0, 0);

    /* PBM step 3: refinement around the best predictor, on the integer grid. */
    if (prm->refine) {
        int cx = s.bmx, cy = s.bmy;
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++)
                if (dx != 0 || dy != 0)
                    pbm_try(&s, cur, ref, W, H, N, M, x0, y0, lambda_q8, cx + dx, cy + dy);
    }

    /* Sec. 3.2: the two stopping conditions, in exact integers.
     * cond. 1: Intra_SAD + SAD_PBM < alpha + beta*Qp^2, times NM.
     * cond. 2: SAD_PBM < (gamma_num/gamma_den) * Intra_SAD, times NM*gamma_den. */
    int64_t sad_pbm = s.bS;
    int64_t qp = prm->qp;
    int64_t lhs1 = (int64_t)intra_x + (int64_t)NM * sad_pbm;
    int64_t rhs1 = (int64_t)NM * ((int64_t)prm->alpha + (int64_t)prm->beta * qp * qp);
    int cond1 = lhs1 < rhs1;
    int64_t lhs2 = (int64_t)prm->gamma_den * NM * sad_pbm;
    int64_t rhs2 = (int64_t)prm->gamma_num * (int64_t)intra_x;
    int cond2 = lhs2 < rhs2;

    if (cond1 || cond2) {
        *mvx_o = s.bmx; *mvy_o = s.bmy; *J_o = s.bJ; *sad_o = s.bS;
        *mask_o = 0;
        *load_o = (uint32_t)s.count;
    } else {
        /* A critical block: the full search decides (Sec. 3.2). */
        full_search_block(cur, ref, W, H, N, M, p, lambda_q8, bx, by, mvx_o, mvy_o, J_o, sad_o);
        *mask_o = 1;
        *load_o = (uint32_t)((2 * p + 1) * (2 * p + 1));
    }
}

/* ACBM over a whole frame, blocks in raster order (every predictor a block
 * uses is final by then).  prev_mv may be NULL (first frame pair: zeros).
 * sad_out and load_out may be NULL. */
int oracle_acbm(const uint8_t *cur, const uint8_t *ref, int W, int H, int N, int M, int p,
                uint32_t lambda_q8, const int16_t *prev_mv, const oracle_acbm_params *prm,
                int16_t *mv_out, uint32_t *J_out, uint8_t *mask_out, uint32_t *sad_out,
                uint32_t *load_out)
{
    if (!cur || !ref || !mv_out || !J_out || !mask_out) return OR_ERR_ARG;
    int st = check_shape(W, H, N, M, p, lambda_q8);
    if (st) return st;
    st = check_params(prm);
    if (st) return st;
    int BW = W / N, BH = H / M, nb = BW * BH;
    uint32_t *intra = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)nb);
    unsigned char *seen = (unsigned char *)malloc((size_t)(2 * p + 1) * (2 * p + 1));
    if (!intra || !seen) { free(intra); free(seen); return OR_ERR_NOMEM; }
    oracle_intra_sad(cur, W, H, N, M, intra);
    for (int by = 0; by < BH; by++) {
        for (int bx = 0; bx < BW; bx++) {
            int b = by * BW + bx, mx, my;
            uint32_t J, s, load;
            uint8_t mask;
            acbm_block(cur, ref, W, H, N, M, p, lambda_q8, mv_out, prev_mv, prm, bx, by,
                       intra[b], seen, &mx, &my, &J, &s, &mask, &load);
            mv_out[2 * b] = (int16_t)mx;
            mv_out[2 * b + 1] = (int16_t)my;
            J_out[b] = J;
            mask_out[b] = mask;
            if (sad_out) sad_out[b] = s;
            if (load_out) load_out[b] = load;
        }
    }
    free(intra);
    free(seen);
    return OR_OK;
}

/* ACBM for a list of blocks, each evaluated against a given current-frame
 * field (for instance the one another implementation produced): this checks
 * single blocks of frames too large for a whole-frame run.  cur_field is the
 * full [BH][BW][2] field whose left/up-left/up/up-right entries serve as the
 * spatial predictors. */
int oracle_acbm_blocks(const uint8_t *cur, const uint8_t *ref, int W, int H, int N, int M, int p,
                       uint32_t lambda_q8, const int16_t *prev_mv, const int16_t *cur_field,
                       const oracle_acbm_params *prm, const int32_t *blocks, int nblocks,
                       int16_t *mv_out, uint32_t *J_out, uint8_t *mask_out, uint32_t *sad_out,
                       uint32_t *load_out)
{
    if (!cur || !ref || !cur_field || !blocks || !mv_out || !J_out || !mask_out || nblocks < 0)
        return OR_ERR_ARG;
    int st = check_shape(W, H, N, M, p, lambda_q8);
    if (st) return st;
    st = check_params(prm);
    if (st) return st;
    int BW = W / N, BH = H / M, nb = BW * BH;
    for (int k = 0; k < nblocks; k++)
        if (blocks[k] < 0 || blocks[k] >= nb) return OR_ERR_ARG;
    uint32_t *intra = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)nb);
    unsigned char *seen = (unsigned char *)malloc((size_t)(2 * p + 1) * (2 * p + 1));
    if (!intra || !seen) { free(intra); free(seen); return OR_ERR_NOMEM; }
    oracle_intra_sad(cur, W, H, N, M, intra);
    for (int k = 0; k < nblocks; k++) {
        int b = blocks[k], mx, my;
        uint32_t J, s, load;
        uint8_t mask;
        acbm_block(cur, ref, W, H, N, M, p, lambda_q8, cur_field, prev_mv, prm, b % BW, b / BW,
                   intra[b], seen, &mx, &my, &J, &s, &mask, &load);
        mv_out[2 * k] = (int16_t)mx;
        mv_out[2 * k + 1] = (int16_t)my;
        J_out[k] = J;
        mask_out[k] = mask;
        if (sad_out) sad_out[k] = s;
        if (load_out) load_out[k] = load;
    }
    free(intra);
    free(seen);
    return OR_OK;
}

/* ------------------------------------------------------------------------
 * Half-pel refinement (Sec. 2.2: the best predictor "is normally refined to
 * half-pel accuracy"; Sec. 2.3: the full search count 969 = 961 integer +
 * 8 half-pel positions).  For every block, starting from its integer vector
 * (mvx, mvy), the 9 positions (2*mvx + dx, 2*mvy + dy), dx, dy in {-1,0,1},
 * in half-pel units, each component clipped to [-2p, 2p]; repeated positions
 * are evaluated once (the integer vector itself is first clipped to
 * [-p, p]).  Readings (the paper gives none of these details):
 *   - the reference at a half-pel position is the bilinear average of the
 *     integer pixels around it, rounded half up, as in H.263 (the encoder the
 *     paper's experiments use): a half step in x averages A and B with
 *     (A + B + 1) >> 1, in y A and C likewise, in both (A+B+C+D+2) >> 2;
 *     integer pixels outside the frame take the nearest edge pixel;
 *   - the cost is J_q8 = 256*SAD + lambda_q8*(L(hx) + L(hy)) with L the
 *     signed Exp-Golomb length of the component in half-pel units;
 *   - ties as for integer positions on the half-pel grid: lowest J, then
 *     smallest |hx|+|hy|, then smaller hy, then smaller hx.
 * Output: the best position in half-pel units, its J_q8 and its SAD.
 * ------------------------------------------------------------------------ */

/* Reference value at half-pel position (X*2 + hx, Y*2 + hy) / 2 of the pixel
 * (X, Y) of the block, i.e. at (X + hx/2, Y + hy/2). */
static int halfpel_ref(const uint8_t *ref, int W, int H, int X, int Y, int hx, int hy)
{
    /* floor division by 2 and the half-step flags */
    int ax = hx >= 0 ? hx / 2 : -((-hx + 1) / 2);
    int ay = hy >= 0 ? hy / 2 : -((-hy + 1) / 2);
    int fx = hx - 2 * ax, fy = hy - 2 * ay;
    int x0 = clampi(X + ax, 0, W - 1), x1 = clampi(X + ax + 1, 0, W - 1);
    int y0 = clampi(Y + ay, 0, H - 1), y1 = clampi(Y + ay + 1, 0, H - 1);
    int A = ref[(size_t)y0 * W + x0];
    if (!fx && !fy) return A;
    int B = ref[(size_t)y0 * W + x1];
    int C = ref[(size_t)y1 * W + x0];
    if (fx && !fy) return (A + B + 1) >> 1;
    if (!fx && fy) return (A + C + 1) >> 1;
    int D = ref[(size_t)y1 * W + x1];
    return (A + B + C + D + 2) >> 2;
}

static uint32_t halfpel_sad(const uint8_t *cur, const uint8_t *ref, int W, int H, int N, int M,
                            int x0, int y0, int hx, int hy)
{
    uint32_t s = 0;
    for (int j = 0; j < M; j++)
        for (int i = 0; i < N; i++) {
            int a = cur[(size_t)(y0 + j) * W + (x0 + i)];
            s += (uint32_t)absi(a - halfpel_ref(ref, W, H, x0 + i, y0 + j, hx, hy));
        }
    return s;
}

int oracle_halfpel(const uint8_t *cur, const uint8_t *ref, int W, int H, int N, int M, int p,
                   uint32_t lambda_q8, const int16_t *mv_int, int16_t *mv_half_out,
                   uint32_t *J_out, uint32_t *sad_out)
{
    if (!cur || !ref || !mv_int || !mv_half_out || !J_out) return OR_ERR_ARG;
    int st = check_shape(W, H, N, M, p, lambda_q8);
    if (st) return st;
    int BW = W / N, BH = H / M;
    for (int by = 0; by < BH; by++)
        for (int bx = 0; bx < BW; bx++) {
            int b = by * BW + bx;
            /* the integer vector is first taken inside the window */
            int cx = 2 * clampi(mv_int[2 * b], -p, p), cy = 2 * clampi(mv_int[2 * b + 1], -p, p);
            int seen[9][2], nseen = 0;
            int bestx = 0, besty = 0, have = 0;
            uint32_t bestJ = 0, bestS = 0;
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    int hx = clampi(cx + dx, -2 * p, 2 * p), hy = clampi(cy + dy, -2 * p, 2 * p);
                    int dup = 0;
                    for (int k = 0; k < nseen; k++)
                        if (seen[k][0] == hx && seen[k][1] == hy) dup = 1;
                    if (dup) continue;
                    seen[nseen][0] = hx;
                    seen[nseen][1] = hy;
                    nseen++;
                    uint32_t s = halfpel_sad(cur, ref, W, H, N, M, bx * N, by * M, hx, hy);
                    uint32_t J = 256u * s + lambda_q8 * (uint32_t)rate_bits(hx, hy);
                    if (!have || better(J, hx, hy, bestJ, bestx, besty)) {
                        bestJ = J; bestS = s; bestx = hx; besty = hy; have = 1;
                    }
                }
            mv_half_out[2 * b] = (int16_t)bestx;
            mv_half_out[2 * b + 1] = (int16_t)besty;
            J_out[b] = bestJ;
            if (sad_out) sad_out[b] = bestS;
        }
    return OR_OK;
}

/* ------------------------------------------------------------------------
 * SAD_deviation (Sec. 3.1): for every block, over all (2p+1)^2 positions of
 * the full search, SAD_deviation = sum_{u,v} |SAD(u,v) - SAD_min| with
 * SAD_min the smallest SAD of the window (a SAD minimum, not the J one).
 * Written out term by term.  Outputs per block: SAD_min and SAD_deviation.
 * ------------------------------------------------------------------------ */
static void sad_deviation_block(const uint8_t *cur, const uint8_t *ref, int W, int H, int N,
                                int M, int p, int bx, int by, uint32_t *vol,
                                uint32_t *sad_min, uint32_t *sad_dev)
{
    int n = 2 * p + 1;
    uint32_t mn = 0;
    for (int v = -p; v <= p; v++)
        for (int u = -p; u <= p; u++) {
            uint32_t s = block_sad(cur, ref, W, H, N, M, bx * N, by * M, u, v);
            vol[(v + p) * n + (u + p)] = s;
            if ((u == -p && v == -p) || s < mn) mn = s;
        }
    uint64_t dev = 0;
    for (int k = 0; k < n * n; k++)
        dev += (uint64_t)(vol[k] > mn ? vol[k] - mn : mn - vol[k]);
    *sad_min = mn;
    *sad_dev = (uint32_t)dev;
}

int oracle_sad_deviation(const uint8_t *cur, const uint8_t *ref, int W, int H, int N, int M,
                         int p, uint32_t *sad_min_out, uint32_t *sad_dev_out)
{
    if (!cur || !ref || !sad_min_out || !sad_dev_out) return OR_ERR_ARG;
    int st = check_shape(W, H, N, M, p, 0);
    if (st) return st;
    int BW = W / N, BH = H / M, n = 2 * p + 1;
    uint32_t *vol = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n * n);
    if (!vol) return OR_ERR_NOMEM;
    for (int by = 0; by < BH; by++)
        for (int bx = 0; bx < BW; bx++)
            sad_deviation_block(cur, ref, W, H, N, M, p, bx, by, vol, &sad_min_out[by * BW + bx],
                                &sad_dev_out[by * BW + bx]);
    free(vol);
    return OR_OK;
}

/* The same for a list of block indices (raster order), outputs per listed block. */
int oracle_sad_deviation_blocks(const uint8_t *cur, const uint8_t *ref, int W, int H, int N,
                                int M, int p, const int *blocks, int nblocks,
                                uint32_t *sad_min_out, uint32_t *sad_dev_out)
{
    if (!cur || !ref || !blocks || !sad_min_out || !sad_dev_out || nblocks < 0) return OR_ERR_ARG;
    int st = check_shape(W, H, N, M, p, 0);
    if (st) return st;
    int BW = W / N, BH = H / M, n = 2 * p + 1;
    for (int k = 0; k < nblocks; k++)
        if (blocks[k] < 0 || blocks[k] >= BW * BH) return OR_ERR_ARG;
    uint32_t *vol = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n * n);
    if (!vol) return OR_ERR_NOMEM;
    for (int k = 0; k < nblocks; k++)
        sad_deviation_block(cur, ref, W, H, N, M, p, blocks[k] % BW, blocks[k] / BW, vol,
                            &sad_min_out[k], &sad_dev_out[k]);
    free(vol);
    return OR_OK;
}

/* ------------------------------------------------------------------------
 * FSBM with a differentially coded vector (Sec. 2.1: R is the bits needed to
 * transmit the vector; Sec. 2.2: vectors are coded differentially in the
 * standards).  The predictor is the H.263-style median: component-wise median
 * of the final vectors of the left (MV1), upper (MV2) and upper-right (MV3)
 * blocks, where a block on the left edge takes MV1 = (0,0), a block on the
 * right edge takes MV3 = (0,0), and a block in the top row takes
 * MV2 = MV3 = MV1.  R(mv) = L(mvx - pmx) + L(mvy - pmy), L the signed
 * Exp-Golomb length; ties as for FSBM.  Blocks in raster order: every
 * predictor is final when it is read.
 * ------------------------------------------------------------------------ */
static int median3(int a, int b, int c)
{
    int lo = a < b ? a : b, hi = a < b ? b : a;
    return c < lo ? lo : (c > hi ? hi : c);
}

void oracle_median_predictor(const int16_t *mv, int BW, int bx, int by, int *pmx, int *pmy)
{
    int m1x = 0, m1y = 0, m2x, m2y, m3x = 0, m3y = 0;
    if (bx > 0) { m1x = mv[2 * (by * BW + bx - 1)]; m1y = mv[2 * (by * BW + bx - 1) + 1]; }
    if (by == 0) {
        *pmx = m1x;
        *pmy = m1y;
        return;
    }
    m2x = mv[2 * ((by - 1) * BW + bx)];
    m2y = mv[2 * ((by - 1) * BW + bx) + 1];
    if (bx + 1 < BW) {
        m3x = mv[2 * ((by - 1) * BW + bx + 1)];
        m3y = mv[2 * ((by - 1) * BW + bx + 1) + 1];
    }
    *pmx = median3(m1x, m2x, m3x);
    *pmy = median3(m1y, m2y, m3y);
}

/* Full search of one block with the rate coded against (pmx, pmy). */
static void pred_search_block(const uint8_t *cur, const uint8_t *ref, int W, int H, int N, int M,
                              int p, uint32_t lambda_q8, int bx, int by, int pmx, int pmy,
                              int *mvx_o, int *mvy_o, uint32_t *J_o, uint32_t *sad_o)
{
    int bmx = 0, bmy = 0, have = 0;
    uint32_t bJ = 0, bS = 0;
    for (int mvy = -p; mvy <= p; mvy++)
        for (int mvx = -p; mvx <= p; mvx++) {
            uint32_t s = block_sad(cur, ref, W, H, N, M, bx * N, by * M, mvx, mvy);
            uint32_t J = 256u * s + lambda_q8 * (uint32_t)(oracle_mv_bits(mvx - pmx) +
                                                           oracle_mv_bits(mvy - pmy));
            if (!have || better(J, mvx, mvy, bJ, bmx, bmy)) {
                have = 1; bJ = J; bS = s; bmx = mvx; bmy = mvy;
            }
        }
    *mvx_o = bmx; *mvy_o = bmy; *J_o = bJ; *sad_o = bS;
}

int oracle_fsbm_pred(const uint8_t *cur, const uint8_t *ref, int W, int H, int N, int M, int p,
                     uint32_t lambda_q8, int16_t *mv_out, uint32_t *J_out, uint32_t *sad_out)
{
    if (!cur || !ref || !mv_out || !J_out) return OR_ERR_ARG;
    int st = check_shape(W, H, N, M, p, lambda_q8);
    if (st) return st;
    int BW = W / N, BH = H / M;
    for (int by = 0; by < BH; by++)
        for (int bx = 0; bx < BW; bx++) {
            int pmx, pmy, mx, my;
            uint32_t J, s;
            oracle_median_predictor(mv_out, BW, bx, by, &pmx, &pmy);
            pred_search_block(cur, ref, W, H, N, M, p, lambda_q8, bx, by, pmx, pmy, &mx, &my, &J, &s);
            int b = by * BW + bx;
            mv_out[2 * b] = (int16_t)mx;
            mv_out[2 * b + 1] = (int16_t)my;
            J_out[b] = J;
            if (sad_out) sad_out[b] = s;
        }
    return OR_OK;
}

/* The listed blocks only, each with its predictor taken from `field` (a
 * whole [BH][BW][2] field, e.g. a result under test): checks every listed
 * block's own step at frame sizes the sequential frame call is too slow for. */
int oracle_fsbm_pred_blocks(const uint8_t *cur, const uint8_t *ref, int W, int H, int N, int M,
                            int p, uint32_t lambda_q8, const int16_t *field, const int32_t *blocks,
                            int nblocks, int16_t *mv_out, uint32_t *J_out, uint32_t *sad_out)
{
    if (!cur || !ref || !field || !blocks || !mv_out || !J_out || !sad_out || nblocks < 0)
        return OR_ERR_ARG;
    int st = check_shape(W, H, N, M, p, lambda_q8);
    if (st) return st;
    int BW = W / N, BH = H / M;
    for (int k = 0; k < nblocks; k++)
        if (blocks[k] < 0 || blocks[k] >= BW * BH) return OR_ERR_ARG;
    for (int k = 0; k < nblocks; k++) {
        int bx = blocks[k] % BW, by = blocks[k] / BW, pmx, pmy, mx, my;
        oracle_median_predictor(field, BW, bx, by, &pmx, &pmy);
        pred_search_block(cur, ref, W, H, N, M, p, lambda_q8, bx, by, pmx, pmy, &mx, &my,
                          &J_out[k], &sad_out[k]);
        mv_out[2 * k] = (int16_t)mx;
        mv_out[2 * k + 1] = (int16_t)my;
    }
    return OR_OK;
}

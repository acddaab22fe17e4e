/*
 * me.h -- C ABI of the GB300 (sm_103a) block-matching motion-estimation
 * library: integer-pel full search (FSBM) and adaptive cost block matching
 * (ACBM) after Lopez, Callico, Lopez and Sarmiento, "A High Quality/Low
 * Computational Cost Technique for Block Matching Motion Estimation".
 *
 * Conventions shared by every call
 * --------------------------------
 * Frames: 8-bit luma, row-major, W columns by H rows, pitch W bytes.
 * Blocks: N x M pixels with N the width and M the height (the SAD of Sec. 2.1
 *   sums i < N with i paired with mvx).  N, M in {4, 8, 16}; W % N == 0 and
 *   H % M == 0 (the caller pads, e.g. 1080 -> 1088 rows).  BW = W/N blocks
 *   per row, BH = H/M block rows; per-block outputs are [BH][BW] row-major.
 * Search range: mv in [-p, p]^2, 1 <= p <= 64.  A reference pixel outside
 *   the frame takes the value of the nearest edge pixel.
 * Motion vectors: int16 pairs (mvx, mvy), [BH][BW][2].  The candidate block
 *   of mv is ref(x0+i+mvx, y0+j+mvy): content that moved right by d is
 *   matched at mvx = -d.
 * Cost (Sec. 2.1, eq. J): J = SAD + lambda*R, carried in Q8 fixed point as
 *   J_q8 = 256*SAD + lambda_q8*R, R(mv) = L(mvx) + L(mvy), L = length of the
 *   signed Exp-Golomb code of a component (1, 3, 3, 5, 5, 5, 5, 7, ...).
 *   lambda_q8 <= 2^20.  Ties: lowest J_q8, then smallest |mvx|+|mvy|, then
 *   smaller mvy, then smaller mvx -- one exact answer per block.
 * Pointers: every array argument of the frame calls is a DEVICE pointer of the
 *   current device, owned by the caller; "nullable" outputs may be NULL.
 *   Frame pointers (cur, ref) must be 4-byte aligned.  Work is enqueued on
 *   `stream` (a cudaStream_t; NULL = legacy default stream) and the call
 *   returns without waiting unless stated.  Scratch memory, where a call needs
 *   it, comes from a library-owned stream-ordered pool of the current device
 *   (allocated and released on `stream`, cached between calls).
 * Errors: every call returns an me_status; on ME_ERR_ARG / ME_ERR_SHAPE
 *   nothing was enqueued.  ME_ERR_CUDA reports a failed CUDA call (the text
 *   of the last one is available from me_last_error()).
 * Threads: the frame calls may be used from several host threads at once;
 *   a batch or server object belongs to one host thread at a time.
 */
#ifndef ME_H_
#define ME_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *me_stream_t; /* identical to cudaStream_t */

typedef enum {
    ME_OK = 0,
    ME_ERR_ARG = 1,      /* NULL pointer, N/M/p/lambda/params out of range */
    ME_ERR_SHAPE = 2,    /* W % N or H % M nonzero, or W/H out of range     */
    ME_ERR_CUDA = 3,     /* a CUDA call failed                               */
    ME_ERR_NOMEM = 4,    /* device or host allocation failed / over budget   */
    ME_ERR_TIMEOUT = 5,  /* a bounded device wait gave up                    */
    ME_ERR_BUSY = 6,     /* request not finished yet / queue full            */
    ME_ERR_NOTFOUND = 7  /* unknown stream or request id                     */
} me_status;

/* Text for a status code (static storage). */
const char *me_status_string(int status);
/* Text of the last CUDA error seen by this host thread ("" if none); a server
 * call that reports its worker thread's error passes that text on. */
const char *me_last_error(void);

/* ----------------------------------------------------------------- cost */

/* lambda of eq. J, "proportional to Qp" (Sec. 2.1); read as 0.92*Qp and
 * returned in Q8: (23552*qp + 50) / 100.  qp in [0, 1023], else 0. */
uint32_t me_lambda_q8(int32_t qp);

/* L(v): bits of the signed Exp-Golomb code of one MV component (the R term of
 * eq. J is L(mvx) + L(mvy)).  Any int16 v. */
int32_t me_mv_bits(int32_t v);

/* ACBM parameters (Sec. 3.2).  cond. 1: Intra_SAD + SAD_PBM < alpha + beta*qp^2;
 * cond. 2: SAD_PBM < (gamma_num/gamma_den)*Intra_SAD; both tested in exact
 * integers.  refine = 1 adds the +-1 integer ring around the best predictor
 * (Sec. 2.2, third PBM step), 0 skips it.  Valid: gamma_den >= 1,
 * gamma_num >= 0, qp in [0, 1023], refine in {0, 1}. */
typedef struct {
    int32_t alpha, beta, gamma_num, gamma_den;
    int32_t qp;
    int32_t refine;
} me_acbm_params;

/* The paper's choice alpha = 1000, beta = 8, gamma = 1/4 (Sec. 4), refine 1. */
me_acbm_params me_acbm_default_params(int32_t qp);

/* ----------------------------------------------------------------- frame calls */

/* Edge-clamped copy of a reference frame with a margin of P = 16*ceil(p/16)
 * pixels on every side, laid out with a 16-byte aligned pitch
 * (the first step of every search; exposed for tests).  out[(y+P)*pitch + x+P]
 * = ref[clamp(y)*W + clamp(x)] for y in [-P, H+P), x in [-P, pitch-P).
 * me_padded_geometry gives pitch, rows = H + 2P, and P.  out must hold
 * pitch*rows bytes. */
int me_padded_geometry(int W, int H, int p, int *pitch, int *rows, int *P);
int me_pad_ref(const uint8_t *ref, int W, int H, int p, uint8_t *out, me_stream_t stream);

/* Scaled Intra_SAD of every block (Sec. 3.1, eq. Intra_SAD):
 * out[b] = sum |N*M*pix - S| = N*M*Intra_SAD with S the block sum, so the
 * block mean needs no rounding.  out is [BH][BW] uint32. */
int me_intra_sad(const uint8_t *cur, int W, int H, int N, int M, uint32_t *out,
                 me_stream_t stream);

/* FSBM (Sec. 2.3): for each block the minimum of J over all (2p+1)^2 integer
 * positions.  mv_out [BH][BW][2], J_out [BH][BW] (J_q8), sad_out [BH][BW]
 * (nullable).  One kernel launch; no scratch memory. */
int me_fsbm(const uint8_t *cur, const uint8_t *ref, int W, int H, int N, int M, int p,
            uint32_t lambda_q8, int16_t *mv_out, uint32_t *J_out, uint32_t *sad_out,
            me_stream_t stream);

/* ACBM (Sec. 3.2) for one frame pair.  Per block: Intra_SAD, then PBM over the
 * predictors (final vectors of the left, up-left, up and up-right blocks of
 * this frame; the 3x3 blocks around it in prev_mv_field; (0,0)), each clipped
 * to [-p,p] and evaluated once, best by J, then the +-1 ring; then cond. 1 /
 * cond. 2; a block meeting neither gets the full search.
 * prev_mv_field [BH][BW][2] is the previous frame's output (NULL = zeros).
 * Outputs: mv_out, J_out, fullsearch_mask_out (1 = full search ran),
 * sad_out (nullable), load_out (nullable; distinct positions evaluated,
 * (2p+1)^2 for a full-searched block).  Every predictor is final when
 * read.  Two forms, the same outputs; the first call with a shape times both
 * (see me_tune_log) and later calls use the faster:
 *  - the wave graph: the blocks as anti-diagonal waves x + 2y = w; the
 *    frame's launches (a prologue, the early full searches of the blocks
 *    that fail with their temporal predictors, then one kernel per wave) are
 *    captured once per (device, W, H, N, M, p) into a CUDA graph with its
 *    own scratch (the padded reference plus 16 bytes per block, about
 *    pitch*rows + 16*BW*BH bytes) and replayed;
 *  - the persistent kernel of me_acbm_sequence over this one pair (K = 1),
 *    with its own plan; a bounded wait that ran out is reported by
 *    me_acbm_sequence_status(W, H, N, M, p, 1).
 * Both are allocated at the first call with that shape and kept until the
 * process exits; calls with the same shape run one after another on the
 * GPU, whatever their streams.  The first call with a new shape allocates,
 * tunes and captures, so make it outside any stream capture of your own;
 * calls made while their stream is being captured use the wave graph. */
int me_acbm(const uint8_t *cur, const uint8_t *ref, int W, int H, int N, int M, int p,
            uint32_t lambda_q8, const int16_t *prev_mv_field, const me_acbm_params *prm,
            int16_t *mv_out, uint32_t *J_out, uint8_t *fullsearch_mask_out, uint32_t *sad_out,
            uint32_t *load_out, me_stream_t stream);

/* ----------------------------------------------------------------- sequences */

/* FSBM over K consecutive frame pairs in one launch (1 <= K <= 64).
 * frames is a HOST array of K+1 device frame pointers: pair k has reference
 * frames[k] and current frame frames[k+1].  Outputs are [K][BH][BW] (x2 for
 * mv), pair k at offset k*BW*BH.  No scratch memory.  For 16x16 blocks (and
 * p <= 34) the launch is one persistent CTA per SM in which staging warps
 * fill two shared-memory buffers while searching warps work on the other
 * (me_fsbm uses the same kernel for one pair). */
int me_fsbm_sequence(const uint8_t *const *frames, int K, int W, int H, int N, int M, int p,
                     uint32_t lambda_q8, int16_t *mv_out, uint32_t *J_out, uint32_t *sad_out,
                     me_stream_t stream);

/* Waits for `stream`; ME_ERR_TIMEOUT if a bounded wait inside a
 * me_fsbm_sequence run since the last call gave up (the persistent form used
 * for 16x16 blocks, whose staging and searching warps hand buffers to each
 * other; its outputs are then incomplete), else ME_OK.  Clears the record. */
int me_fsbm_sequence_status(me_stream_t stream);

/* ACBM over K consecutive frame pairs in one persistent launch: pair k's
 * previous field is pair k-1's output (prev_mv_field for pair 0, NULL =
 * zeros), exactly as K chained me_acbm calls, with identical outputs.  The
 * method's causal order (Sec. 2.2) lets the pairs overlap: a block of pair k
 * needs only its spatial neighbours of pair k and its 3x3 neighbourhood of
 * pair k-1, so blocks are claimed in order of (wave + 4k) and each waits
 * (bounded) for those predecessors; many pairs are in flight at once.
 * Scratch: one cached plan per (device, W, H, N, M, p, K) with K padded
 * references, Intra_SAD and ready flags (allocated at the first call, kept
 * until exit); runs with the same plan are ordered on the GPU.
 * me_acbm_sequence_status waits for the stream and reports ME_ERR_TIMEOUT if
 * a bounded wait of the last run gave up. */
int me_acbm_sequence(const uint8_t *const *frames, int K, int W, int H, int N, int M, int p,
                     uint32_t lambda_q8, const int16_t *prev_mv_field, const me_acbm_params *prm,
                     int16_t *mv_out, uint32_t *J_out, uint8_t *fullsearch_mask_out,
                     uint32_t *sad_out, uint32_t *load_out, me_stream_t stream);
int me_acbm_sequence_status(int W, int H, int N, int M, int p, int K, me_stream_t stream);

/* ------------------------------------------------------------ half-pel */

/* Half-pel refinement of an integer vector field (Sec. 2.2: the best vector
 * is normally refined to half-pel accuracy; Sec. 2.3: the 8 half-pel
 * positions around it).  For every block, with (mvx, mvy) = mv_int clipped to
 * [-p, p]: the positions (2*mvx + dx, 2*mvy + dy), dx, dy in {-1,0,1}, in
 * half-pel units, each component clipped to [-2p, 2p], repeated ones once.
 * The reference at a half-pel position is the bilinear average of the
 * integer pixels around it, H.263 rounding ((A+B+1)>>1 along one axis,
 * (A+B+C+D+2)>>2 along both), pixels outside the frame at the nearest edge.
 * Cost J_q8 = 256*SAD + lambda_q8*(L(hx)+L(hy)), L = me_mv_bits in half-pel
 * units; ties: lowest J, then |hx|+|hy|, then hy, then hx.
 * mv_int: device [BH][BW][2] int16 (e.g. the output of me_fsbm or me_acbm);
 * mv_half_out: device [BH][BW][2] int16 in half-pel units; J_out, sad_out
 * (nullable): device [BH][BW].  Same argument checks as me_fsbm; no scratch
 * memory; asynchronous on `stream`. */
int me_halfpel(const uint8_t *cur, const uint8_t *ref, int W, int H, int N, int M, int p,
               uint32_t lambda_q8, const int16_t *mv_int, int16_t *mv_half_out, uint32_t *J_out,
               uint32_t *sad_out, me_stream_t stream);

/* me_halfpel for K consecutive frame pairs in one launch: frames is a host
 * array of K+1 device frame pointers (pair k: reference frames[k], current
 * frames[k+1]); mv_int and the outputs are [K][BH][BW] (x2 for vectors). */
int me_halfpel_sequence(const uint8_t *const *frames, int K, int W, int H, int N, int M, int p,
                        uint32_t lambda_q8, const int16_t *mv_int, int16_t *mv_half_out,
                        uint32_t *J_out, uint32_t *sad_out, me_stream_t stream);

/* ------------------------------------- FSBM with a predicted vector rate */

/* FSBM where the vector is coded against a predictor (Sec. 2.1: R is the
 * bits that transmit the vector; Sec. 2.2: the standards code vectors
 * differentially).  pm = the H.263-style median predictor: component-wise
 * median of the final vectors of the left (MV1), upper (MV2) and upper-right
 * (MV3) blocks; MV1 = (0,0) on the left edge, MV3 = (0,0) on the right edge,
 * and in the top row the predictor is MV1.  R = L(mvx - pmx) + L(mvy - pmy)
 * with L = me_mv_bits; J_q8 = 256*SAD + lambda_q8*R; ties as me_fsbm.
 * Blocks depend on their neighbours' results, so the search is a wavefront:
 * one launch computes every candidate's SAD (uint16 volume), a second,
 * persistent one takes the blocks in anti-diagonal order with bounded waits.
 * Outputs as me_fsbm (mv_out, J_out required; sad_out nullable).  Scratch:
 * one cached plan per (device, W, H, N, M, p, K) holding the SAD volume
 * (2*ceil8((2p+1)^2) bytes per block and pair) and per-block flags,
 * allocated at the first call and kept until exit; runs with one plan are
 * ordered on the GPU. */
int me_fsbm_pred(const uint8_t *cur, const uint8_t *ref, int W, int H, int N, int M, int p,
                 uint32_t lambda_q8, int16_t *mv_out, uint32_t *J_out, uint32_t *sad_out,
                 me_stream_t stream);

/* me_fsbm_pred for K independent consecutive pairs (pair k: reference
 * frames[k], current frames[k+1]; frames a host array of K+1 device
 * pointers, 1 <= K <= 64) in the same two launches; outputs [K][BH][BW]. */
int me_fsbm_pred_sequence(const uint8_t *const *frames, int K, int W, int H, int N, int M, int p,
                          uint32_t lambda_q8, int16_t *mv_out, uint32_t *J_out, uint32_t *sad_out,
                          me_stream_t stream);

/* Waits for `stream` and reports ME_ERR_TIMEOUT if a bounded wait of the last
 * me_fsbm_pred / me_fsbm_pred_sequence run with this shape gave up (its
 * outputs are then incomplete), else ME_OK.  K = 1 for me_fsbm_pred. */
int me_fsbm_pred_status(int W, int H, int N, int M, int p, int K, me_stream_t stream);

/* ------------------------------------------------- SAD statistics (Sec. 3.1) */

/* FSBM (as me_fsbm) plus, for every block, the two statistics of the full
 * search's SAD surface that Sec. 3.1 introduces: SAD_min, the least SAD over
 * the (2p+1)^2 positions (a SAD minimum, independent of lambda), and
 * SAD_deviation = sum over those positions of |SAD(u,v) - SAD_min|.
 * mv_out [BH][BW][2] and J_out [BH][BW] (both nullable) are the FSBM result
 * for lambda_q8; sad_min_out, sad_dev_out: device [BH][BW] uint32 (required;
 * SAD_deviation < 2^31 for every allowed shape).  Same argument checks as
 * me_fsbm; one launch; no scratch memory; asynchronous on `stream`. */
int me_sad_deviation(const uint8_t *cur, const uint8_t *ref, int W, int H, int N, int M, int p,
                     uint32_t lambda_q8, int16_t *mv_out, uint32_t *J_out,
                     uint32_t *sad_min_out, uint32_t *sad_dev_out, me_stream_t stream);

/* The known-motion experiment of Sec. 3.1 (Fig. 3) in one launch: frames is a
 * host array of K+1 device frame pointers (1 <= K <= 64); frames[0] is the
 * original frame and frames[k], k >= 1, the original displaced by the known
 * global vector true_mv[k-1] (device [K][2] int16, (gx, gy), given as the
 * motion vector a block matcher should find).  For every moved frame k and
 * block b, index (k-1)*BH*BW + b: the FSBM vector of frames[k] against
 * frames[0] (mv_out, [K][BH][BW][2]), the scaled Intra_SAD of the block of
 * frames[k] (intra_out, N*M*Intra_SAD as me_intra_sad), SAD_min and
 * SAD_deviation (as me_sad_deviation), and the vector error
 * err_out = min(|mvx - gx| + |mvy - gy|, 255) (uint8; 0 = true vector).
 * mv_out, intra_out and err_out are nullable; sad_min_out and sad_dev_out are
 * required.  Same argument checks as me_fsbm; asynchronous on `stream`. */
int me_motion_study(const uint8_t *const *frames, int K, int W, int H, int N, int M, int p,
                    uint32_t lambda_q8, const int16_t *true_mv, int16_t *mv_out,
                    uint32_t *intra_out, uint32_t *sad_min_out, uint32_t *sad_dev_out,
                    uint8_t *err_out, me_stream_t stream);

/* ----------------------------------------------------------------- batches */

/* Many independent streams of uneven size in one launch per step (an
 * extension of the per-frame calls; the paper has one sequence at a time).
 * A batch fixes the list of stream shapes (one block shape N x M for all
 * streams; W, H and p may differ); each run takes one frame pair per stream
 * through FSBM or ACBM in a single persistent kernel (with the padding and
 * Intra_SAD prologue for ACBM), captured once into a CUDA graph and replayed.
 * Outputs are identical to running each stream alone with me_fsbm / me_acbm.
 * Device memory (padded references, Intra_SAD, flags) is allocated once at
 * the first run and released by me_batch_destroy. */
typedef struct me_batch me_batch;

typedef enum { ME_MODE_FSBM = 0, ME_MODE_ACBM = 1 } me_mode;

typedef struct {
    const uint8_t *cur, *ref;    /* device frames of this stream                 */
    const int16_t *prev_mv;      /* ACBM: previous field, NULL = zeros           */
    int16_t *mv_out;             /* [BH][BW][2]                                  */
    uint32_t *J_out;             /* [BH][BW]                                     */
    uint8_t *mask_out;           /* ACBM: [BH][BW] (required), FSBM: ignored     */
    uint32_t *sad_out;           /* nullable                                     */
    uint32_t *load_out;          /* nullable                                     */
    uint32_t lambda_q8;
    me_acbm_params prm;          /* ACBM only                                    */
} me_batch_item;

int me_batch_create(me_batch **out);
/* Adds a stream shape; returns its index in *index.  Not allowed after the
 * first me_batch_run. */
int me_batch_add_stream(me_batch *b, int W, int H, int N, int M, int p, int *index);
/* One step: items[k] belongs to stream k (all streams, in order).  Enqueued on
 * stream; me_batch_sync then reports ME_ERR_TIMEOUT if a bounded device wait
 * gave up, in which case the outputs are unspecified.  Successive runs of one
 * batch share its device tables: issue them on one stream (or order them). */
int me_batch_run(me_batch *b, int mode, const me_batch_item *items, int n_items,
                 me_stream_t stream);
/* Blocks until the last run on the given stream finished; reports its status
 * (ME_ERR_TIMEOUT if a bounded wait inside the step gave up). */
int me_batch_sync(me_batch *b, me_stream_t stream);
/* Test hook for failure detection, before the first run: every device wait
 * of the ACBM step gives up after timeout_ns nanoseconds (default 1 s), and
 * block skip_block of stream skip_stream (-1: none) never publishes its
 * vector, so the blocks that depend on it time out and the step reports
 * ME_ERR_TIMEOUT instead of hanging. */
int me_batch_set_fault(me_batch *b, long long timeout_ns, int skip_stream, int skip_block);
void me_batch_destroy(me_batch *b);

/* ----------------------------------------------------------------- serving */

/* A request server with continuous batching (an extension for serving many
 * live streams; the paper has one sequence at a time).  Each stream submits
 * its frames in order from host memory; the server keeps the stream's last
 * frame (the reference) and last motion field resident in device memory, so a
 * request is one new frame and its result is the motion field of the pair
 * (previous frame, this frame).  A worker thread keeps up to max_inflight
 * steps on the GPU; each step takes the oldest pending request of every
 * stream not already on the GPU and runs them in one persistent launch, so
 * requests that arrive while steps are running join the next step as soon as
 * a slot frees.  Results are identical to me_acbm / me_fsbm on the same frames.
 * Streams are admitted against device_budget_bytes (their resident state:
 * two frames, two fields, the outputs and the padded reference). */
typedef struct me_server me_server;

typedef struct {
    long long device_budget_bytes; /* admission budget for resident stream state */
    int max_inflight;              /* steps on the GPU at once, 1..8              */
    int mode;                      /* ME_MODE_ACBM or ME_MODE_FSBM                */
    int N, M;                      /* block size of every stream                  */
} me_server_config;

typedef struct {
    int has_result;      /* 0 for a stream's first frame (it only becomes the reference) */
    int status;          /* ME_OK, or ME_ERR_TIMEOUT if a bounded device wait gave up   */
    double latency_ms;   /* submit -> results in host memory                            */
    /* host buffers the caller provides (each nullable), [BH][BW](x2 for mv) */
    int16_t *mv;
    uint32_t *J;
    uint8_t *mask;       /* ACBM only */
    uint32_t *sad;
    uint32_t *load;      /* ACBM only */
} me_server_result;

int me_server_create(const me_server_config *cfg, me_server **out);
/* Opens a stream of W x H frames with search range p; prm NULL = the paper's
 * parameters for qp.  ME_ERR_NOMEM: the stream does not fit the budget now
 * (retry after another stream closed). */
int me_server_open_stream(me_server *s, int W, int H, int p, const me_acbm_params *prm,
                          int32_t qp, int *stream_id);
/* Queues one frame (W*H bytes of host memory, copied before returning). */
int me_server_submit(me_server *s, int stream_id, const uint8_t *frame, long long *request_id);
/* ME_ERR_BUSY while pending; on completion copies the results into res's
 * buffers, returns the request's status and forgets the request. */
int me_server_poll(me_server *s, long long request_id, me_server_result *res);
/* As poll, waiting up to timeout_ms (ME_ERR_BUSY if still pending). */
int me_server_wait(me_server *s, long long request_id, int timeout_ms, me_server_result *res);
/* Closes a stream; its memory returns to the budget once its work is done. */
int me_server_close_stream(me_server *s, int stream_id);
/* Budget in use, open streams and pending requests; returns the server's
 * status (ME_OK unless a CUDA error stopped it). */
int me_server_stats(me_server *s, long long *used_bytes, int *open_streams, int *pending);
/* Text describing the last step whose bounded device wait gave up (its
 * control block: claimed blocks, queue head and tail), "" if none. */
const char *me_server_diagnostics(me_server *s);
void me_server_destroy(me_server *s);

/* The same ACBM as me_acbm, for callers that cannot allocate device memory:
 * a host application or engine that owns every device allocation under a
 * fixed budget, a plugin loaded into another process's CUDA context, or code
 * that must not allocate after start-up.  The paper has no counterpart; this
 * is a deployment variant.  It allocates nothing: its scratch memory is one
 * fixed device array of 4 MiB inside the library, which every GPU that loads
 * the library holds until the process exits.  A call needs the padded
 * reference, (16*ceil(W/16) + 2P + 16) x (H + 2P) bytes with
 * P = 16*ceil(p/16), plus 16 bytes per block: frames up to 1920x1088 fit at
 * any p for every block shape of 4x8 / 8x4 pixels or larger; 4x4 blocks fit
 * frames up to 1280x720 (not 1920x1088).  Arguments, outputs and errors are
 * those of me_acbm; a frame whose scratch would exceed the array returns
 * ME_ERR_NOMEM before anything is enqueued.
 * The first call on each device looks up the array's device address (with
 * that device current); make that first call before any stream capture.
 * Every call on a device shares the one array, and a call leaves its contents
 * behind (the parts that must start at zero are cleared by each call on its
 * stream).  Calls whose GPU work overlaps -- on different streams, or from
 * several host threads -- race on the array and give wrong results: issue
 * them on one stream, or order them with events. */
int me_acbm_noalloc(const uint8_t *cur, const uint8_t *ref, int W, int H, int N, int M, int p,
                    uint32_t lambda_q8, const int16_t *prev_mv_field, const me_acbm_params *prm,
                    int16_t *mv_out, uint32_t *J_out, uint8_t *fullsearch_mask_out,
                    uint32_t *sad_out, uint32_t *load_out, me_stream_t stream);

/* ----------------------------------------------------------------- peak probe */

/* Measures the integer-pipe rate of a packed-SAD instruction form on the
 * current device with no memory traffic (the roofline denominator of the SAD
 * kernels).  variant 0: vabsdiff4 with accumulate (the form the kernels
 * use); 1: per-byte absolute difference + dp4a byte sum; 2: __vsadu4 + add;
 * 3: per-byte max - min + dp4a; 4: vabsdiff2 with accumulate (16-bit lanes).
 * Writes absolute differences per second, and operations per SM clock per
 * SM (from the SM cycle counter).  Synchronous. */
int me_sad_peak(int variant, double *absdiff_per_s, double *lane_ops_per_clk_per_sm,
                me_stream_t stream);

/* ----------------------------------------------------------------- autotuner */

/* The library tunes its launch forms by measurement (not a paper item; the
 * paper has no implementation): on the first call of a shape, me_fsbm,
 * me_fsbm_sequence and me_acbm_sequence time every candidate launch form
 * (run length of the full searches, per-group or pipelined full-search
 * kernel, the CTA roles of the ACBM sequence kernel) with CUDA events on the
 * caller's stream, synchronising it, and keep the fastest for the rest of the
 * process.  Every candidate computes the same outputs.  A first call made
 * while the stream is being captured into a CUDA graph, or with the
 * environment variable ME_TUNE=0, takes the cost model's choice without
 * timing; ME_TUNE_FORCE=<i> runs candidate i of every tuned call (tests).
 *
 * me_tune_log writes one text line per tuned shape -- the shape, the model's
 * and the chosen candidate and every candidate's best time in ms (-1: not
 * timed) -- NUL-terminated into buf (at most len bytes, truncated), and
 * returns the bytes the whole text needs including the NUL. */
int me_tune_log(char *buf, int len);

#ifdef __cplusplus
}
#endif
#endif /* ME_H_ */

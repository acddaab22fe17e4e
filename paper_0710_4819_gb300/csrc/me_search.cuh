// me_search.cuh -- kernels of the frame path shared by the per-frame calls and
// the batched/persistent paths: reference padding, Intra_SAD, the PBM stage of
// ACBM for one block (one warp), and the full-search plan (tile choice).
#pragma once
#include <cstdio>
#include <functional>
#include <vector>

#include "../../include/me.h"
#include "me_device.cuh"

// Compile-time self-checks (ME_DEBUG_CHECKS): an index outside its buffer is
// printed (first few only) and the access is skipped.  Off by default.
#ifdef ME_DEBUG_CHECKS
static __device__ int g_me_check_count = 0;
#define ME_CHECK(cond, ...)                                              \
  ((cond) ? true                                                         \
          : ((atomicAdd(&g_me_check_count, 1) < 16 ? printf(__VA_ARGS__) : 0), false))
#else
#define ME_CHECK(cond, ...) true
#endif

namespace me {

// Per-call arguments of ACBM (device pointers and parameters).
struct AcbmArgs {
  const uint8_t* cur;
  const uint8_t* ref;
  const int16_t* prev;     // may be null (= zero field)
  int16_t* mv;
  uint32_t* J;
  uint8_t* mask;
  uint32_t* sad;           // may be null
  uint32_t* load;          // may be null
  uint32_t lam;
  int32_t alpha, beta, gnum, gden, qp, refine;
};

// Padded-reference geometry: margin P = 16*ceil(p/16) on every side, pitch a
// multiple of 16 with 16 extra bytes on the right so that a row segment read
// as whole words (one word past its end) stays inside the row.
struct PadGeom {
  int P, pitch, rows;
};
__host__ __device__ inline PadGeom pad_geom(int W, int H, int p) {
  PadGeom g;
  g.P = (p + 15) / 16 * 16;
  g.pitch = (W + 15) / 16 * 16 + 2 * g.P + 16;
  g.rows = H + 2 * g.P;
  return g;
}

// ---------------------------------------------------------------------------
// a1: edge-clamped padded reference, one thread per 16 output bytes.
// ---------------------------------------------------------------------------
__global__ void k_pad_ref(const uint8_t* __restrict__ ref, int W, int H, PadGeom g,
                          uint8_t* __restrict__ out);

// ---------------------------------------------------------------------------
// a2: scaled Intra_SAD per block (eq. Intra_SAD, Sec. 3.1): one warp per block.
// ---------------------------------------------------------------------------
template <int N, int M>
__device__ __forceinline__ uint32_t warp_intra_sad(const uint8_t* __restrict__ cur, int W, int x0,
                                                   int y0) {
  constexpr int NM = N * M;
  const int lane = threadIdx.x & 31;
  int v[(NM + 31) / 32];
  int s = 0;
#pragma unroll
  for (int k = 0; k < (NM + 31) / 32; k++) {
    int i = lane + 32 * k;
    v[k] = i < NM ? (int)cur[(size_t)(y0 + i / N) * W + x0 + (i % N)] : 0;
    s += v[k];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  int d = 0;
#pragma unroll
  for (int k = 0; k < (NM + 31) / 32; k++) {
    int i = lane + 32 * k;
    if (i < NM) d += abs(NM * v[k] - s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  return (uint32_t)d;
}

// ---------------------------------------------------------------------------
// The search window of one block, staged in shared memory by one warp so that
// the PBM candidates are evaluated without further global-memory round trips.
// The window covers padded-reference columns [A, A + 16*chunks) with A the
// 16-byte boundary at or left of the block's column x0 + P - p, and rows
// y0 + P - p .. y0 + P + p + M - 1.
// ---------------------------------------------------------------------------
struct PbmWin {
  int s0;      // byte offset of column x0 - p inside the staged row
  int chunks;  // 16-byte chunks per staged row
  int wp;      // staged row pitch in words (4 * chunks)
  int rows;    // M + 2p
};

__host__ __device__ inline PbmWin pbm_win(int N, int M, int p, int x0, int P) {
  PbmWin w;
  const int X = x0 + P - p;
  w.s0 = X & 15;
  w.chunks = (w.s0 + N + 2 * p + 4 + 15) / 16;  // + one spare word for the funnel shift
  w.wp = 4 * w.chunks;
  w.rows = M + 2 * p;
  return w;
}

// Upper bound of the staged words for any block (for shared-memory sizing).
__host__ __device__ inline int pbm_win_words(int N, int M, int p) {
  return 4 * ((15 + N + 2 * p + 4 + 15) / 16) * (M + 2 * p);
}

// Part of one candidate's SAD computed by a single lane from the staged
// window: rows j0 .. j0+nrows-1 of the block, each read as N/4+1 words and
// shifted into place.  Not inlined and rolled, so the PBM code stays small and
// in the instruction cache between blocks, when other code has run on the SM.
template <int N, int M>
__device__ __noinline__ uint32_t lane_sad_rows(const uint32_t* curs, const uint32_t* win, PbmWin wg,
                                               int p, int mvx, int mvy, int j0, int nrows) {
  constexpr int NW = N / 4;
  const int o = wg.s0 + p + mvx;
  if (!ME_CHECK(p + mvy + j0 >= 0 && p + mvy + j0 + nrows <= wg.rows && o >= 0 &&
                    (o >> 2) + NW < wg.wp,
                "ME_CHECK lane_sad_rows p %d mv %d,%d j0 %d rows %d wp %d s0 %d\n", p, mvx, mvy,
                j0, wg.rows, wg.wp, wg.s0))
    return 0;
  const uint32_t* rp = win + (p + mvy + j0) * wg.wp + (o >> 2);
  const uint32_t* cp = curs + j0 * NW;
  const unsigned sh = 8u * (unsigned)(o & 3);
  uint32_t acc = 0;
#pragma unroll 4
  for (int j = 0; j < nrows; j++) {
    uint32_t wv[NW + 1];
#pragma unroll
    for (int w = 0; w <= NW; w++) wv[w] = rp[j * wg.wp + w];
#pragma unroll
    for (int w = 0; w < NW; w++) acc = sad4(cp[j * NW + w], __funnelshift_r(wv[w], wv[w + 1], sh), acc);
  }
  return acc;
}

// Result of the PBM stage for one block (valid in every lane of the warp).
struct PbmResult {
  unsigned long long key;  // best PBM candidate
  int load;                // distinct positions evaluated
  bool pass;               // cond. 1 or cond. 2 holds
};

// The published state of a block in the persistent kernels: the run's epoch
// in the high word and the block's final vector in the low word (mvx in bits
// 0-15, mvy in bits 16-31), so a block waiting for a predecessor receives the
// predictor with the flag, in the same load.
__host__ __device__ __forceinline__ unsigned long long pub_word(int epoch, int mvx, int mvy) {
  return ((unsigned long long)(uint32_t)epoch << 32) |
         ((unsigned long long)(uint16_t)(int16_t)mvy << 16) | (unsigned long long)(uint16_t)(int16_t)mvx;
}
__host__ __device__ __forceinline__ int pub_epoch(unsigned long long w) { return (int)(w >> 32); }
__host__ __device__ __forceinline__ int pub_mvx(unsigned long long w) { return (int)(int16_t)(uint16_t)(w & 0xffffu); }
__host__ __device__ __forceinline__ int pub_mvy(unsigned long long w) {
  return (int)(int16_t)(uint16_t)((w >> 16) & 0xffffu);
}

// ---------------------------------------------------------------------------
// Role of a CTA of the two-role persistent kernels (0: PBM warps, 1: full
// searches), called by one thread.  The first two CTAs of a launch take one
// role each, so both roles are resident from the start whatever else holds
// the GPU; after that the first CTA on an SM runs PBM and the second the full
// searches, so every SM hosts one of each.  (Arrival order alone does not
// pair the CTAs of an SM: the block scheduler may give both CTAs of an SM the
// same parity, leaving half the SMs with two PBM CTAs and half with two
// search CTAs.)
// ---------------------------------------------------------------------------
constexpr int kRoleSlots = 1024;   // > any %smid

// search_every > 0: the CTAs of every search_every-th SM (by %smid) all take
// the search role (more search CTAs than PBM CTAs).  With cps CTAs per SM,
// the first pbm_per_sm CTAs to arrive on an SM run PBM and the rest search.
__device__ __forceinline__ int cta_role(int* started, int* sm_arr, int search_every = 0,
                                        int cps = 2, int pbm_per_sm = 1) {
  const int arr = atomicAdd(started, 1);
  unsigned smid;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
  const int sa = atomicAdd(sm_arr + (smid & (kRoleSlots - 1)), 1);
  if (arr < 2) return arr;
  if (search_every > 0 && smid % (unsigned)search_every == 0) return 1;
  return sa % cps < pbm_per_sm ? 0 : 1;
}

// ---------------------------------------------------------------------------
// Warp-wide bounded wait of the persistent kernels: every lane with a
// non-null flag f waits until its word carries epoch `want` (pub_word) and
// gets the word back.  One load per lane first; then every pending lane
// re-reads its own flag after each short sleep (32, then 64 ns), all at
// once: the dependency chain is bound by how soon a published flag is seen,
// and polling one pending flag at a time added a round trip per flag.  The
// decision to give up is lane 0's, for the whole warp: after `lim` SM
// cycles (recording ME_ERR_TIMEOUT and `item` in *err / *err_item) or as
// soon as *err is set by another wait.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long warp_wait_flags(const unsigned long long* f, int want,
                                                              int* err, int* err_item,
                                                              long long lim, int item) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const volatile int* verr = err;
  unsigned long long w = 0;
  bool need = false;
  if (f) {
    w = *reinterpret_cast<const volatile unsigned long long*>(f);
    need = pub_epoch(w) != want;
  }
  unsigned pend = __ballot_sync(FULL, need);
  if (!pend) return w;
  const long long t0 = clock64();
  unsigned ns = 32;
  while (pend) {
    __nanosleep(ns);
    if (ns < 64) ns *= 2;
    if (need) {
      w = *reinterpret_cast<const volatile unsigned long long*>(f);
      need = pub_epoch(w) != want;
    }
    int stop = 0;
    if (lane == 0) {
      if (*verr != 0) {
        stop = 1;
      } else if (clock64() - t0 > lim) {
        atomicExch(err, (int)ME_ERR_TIMEOUT);
        atomicExch(err_item, item);
        stop = 1;
      }
    }
    pend = __ballot_sync(FULL, need);
    if (__shfl_sync(FULL, stop, 0)) break;
  }
  return w;
}

// Spin-wait bounds are counted in SM clock cycles (the SM-local cycle counter
// is cheap to read, unlike the global timer); the host converts a timeout to
// cycles at the device's peak SM clock (wait_cycles in me_host.h), so a wait
// lasts at least the timeout at any clock.

// ---------------------------------------------------------------------------
// PBM of one block by one warp, in two parts so that the memory traffic that
// does not depend on other blocks can be in flight while the warp waits for
// its predecessors:
//
//   pbm_stage: queue the current block (4-byte copies) and the whole search
//              window (16-byte copies) as asynchronous global-to-shared copies;
//   pbm_eval : with the lane's predictor in hand (lanes 0-3 the spatial ones:
//              left, up-left, up, up-right; lanes 4-12 the 3x3 temporal ones;
//              lane 13 the zero vector), wait for the copies, evaluate every
//              distinct clipped predictor (Sec. 2.2 steps 1-2), the +-1 ring
//              around the best (step 3, skipping positions already evaluated)
//              and the two conditions of Sec. 3.2 (a5 + a6 + a9).
//
// curs: this warp's M*N/4 words for the current block; win: its window area
// (pbm_win_words words).  Both in shared memory.
// ---------------------------------------------------------------------------
template <int N, int M>
__device__ __forceinline__ PbmWin pbm_stage(const uint8_t* __restrict__ cur,
                                            const uint8_t* __restrict__ refpad, const PadGeom& pg,
                                            int W, int p, int x0, int y0, uint32_t* curs,
                                            uint32_t* win) {
  constexpr int NW = N / 4;
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < M * NW; i += 32) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(curs + i);
    const void* g = cur + (size_t)(y0 + i / NW) * W + x0 + 4 * (i % NW);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(g) : "memory");
  }
  const PbmWin wg = pbm_win(N, M, p, x0, pg.P);
  const int rpp = 32 / wg.chunks;          // rows per pass (chunks <= 11 for p <= 64)
  const int rl = lane / wg.chunks, cl = lane - (lane / wg.chunks) * wg.chunks;
  const uint8_t* src = refpad + (size_t)(y0 + pg.P - p) * pg.pitch + ((x0 + pg.P - p) & ~15);
  if (rl < rpp) {
    for (int r = rl; r < wg.rows; r += rpp) {
      const unsigned dst = (unsigned)__cvta_generic_to_shared(win + r * wg.wp + 4 * cl);
      const void* g = src + (size_t)r * pg.pitch + 16 * cl;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(g) : "memory");
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  return wg;
}

// Lane 0 of pbm_eval writes globaltimer stamps to tr[0..2] when tr is not
// null (copies waited for, predictors evaluated, ring evaluated).
__device__ __forceinline__ void pbm_stamp(unsigned long long* tr, int i) {
  if (tr && (threadIdx.x & 31) == 0) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    tr[i] = t;
  }
}

// The best candidate of a set: its key, vector and SAD (valid in every
// lane; key kNoKey when the set was empty).
struct PbmBest {
  unsigned long long key;
  int mvx, mvy;
  uint32_t sad;
};

__device__ __forceinline__ PbmBest pbm_better(const PbmBest& a, const PbmBest& b) {
  return b.key < a.key ? b : a;
}

// Candidates held by lanes (position ex, ey; act: to evaluate), each
// candidate's rows split over `parts` lanes (2, 4 or 8, at most M): lane
// c*parts + q sums rows q*M/parts .. (q+1)*M/parts-1 of the candidate held
// by lane c.  The minimum key is taken with two 32-bit warp reductions and
// the winner's vector and SAD are read from its lane (no key decoding).  Not
// inlined: the three calls share one copy, so the PBM code stays small and in
// the instruction cache when other code has run on the SM.
template <int N, int M>
__device__ __noinline__ PbmBest pbm_eval_set(int ex, int ey, bool act, int parts,
                                                const PbmWin& wg, int p, uint32_t lam,
                                                const uint32_t* curs, const uint32_t* win) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int c = lane / parts, q = lane - c * parts;
  const int ccx = __shfl_sync(FULL, ex, c), ccy = __shfl_sync(FULL, ey, c);
  const bool cact = __shfl_sync(FULL, act ? 1 : 0, c) != 0;
  uint32_t s = cact ? lane_sad_rows<N, M>(curs, win, wg, p, ccx, ccy, q * (M / parts), M / parts) : 0u;
  for (int o = 1; o < parts; o <<= 1) s += __shfl_xor_sync(FULL, s, o);
  const unsigned long long key =
      cact && q == 0 ? make_key(256u * s + lam * (uint32_t)(mv_bits(ccx) + mv_bits(ccy)), ccx, ccy, p)
                     : kNoKey;
  PbmBest r;
  r.key = warp_min64_redux(key);
  const unsigned w = __ballot_sync(FULL, key == r.key && key != kNoKey);
  const int src = w ? __ffs(w) - 1 : 0;
  r.mvx = __shfl_sync(FULL, ccx, src);
  r.mvy = __shfl_sync(FULL, ccy, src);
  r.sad = __shfl_sync(FULL, s, src);
  return r;
}

// PBM in two parts, so that the predictors known early can be evaluated
// while the warp still waits for its spatial neighbours:
//   pbm_part_a: the distinct clipped positions among the temporal predictors
//               and the zero vector (lanes 4-13), best by J;
//   pbm_part_b: the spatial predictors (lanes 0-3) not already evaluated,
//               the +-1 ring around the best of all predictors (skipping
//               positions already evaluated) and the two conditions.
// Together they evaluate exactly the distinct positions of Sec. 2.2 steps
// 1-3 (which lane evaluates a repeated position does not matter: its key is
// the same).  Every lane passes its own predictor (cx, cy, valid).
struct PbmPart {
  PbmBest best;
  int load;
};

__device__ __forceinline__ int pbm_code(int cx, int cy, bool valid, int p) {
  const int lane = threadIdx.x & 31;
  return valid ? ((clampi(cy, -p, p) + p) << 8) + (clampi(cx, -p, p) + p) : -1 - lane;
}

template <int N, int M>
__device__ PbmPart pbm_part_a(int cx, int cy, bool valid, const PbmWin& wg, int p, uint32_t lam,
                              const uint32_t* curs, const uint32_t* win,
                              unsigned long long* tr = nullptr) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncwarp();
  pbm_stamp(tr, 0);
  const bool mine = valid && lane >= 4 && lane < 14;
  const int code = pbm_code(cx, cy, mine, p);
  // repeated among lanes 4-13: an earlier lane of them holds the same code
  const unsigned same = __match_any_sync(FULL, code);
  const bool dup = (same & ((1u << lane) - 1u) & 0x3FF0u) != 0;
  const bool act = mine && !dup;
  PbmPart r;
  r.best = pbm_eval_set<N, M>(clampi(cx, -p, p), clampi(cy, -p, p), act, 2, wg, p, lam, curs, win);
  r.load = __popc(__ballot_sync(FULL, act));
  return r;
}

// The +-1 ring around part a's best, evaluated early (while the warp waits
// for its spatial neighbours): ring positions equal to a temporal or zero
// predictor, or to an earlier ring lane's, are skipped, as in part b.  Part b
// uses it when no spatial predictor beats part a's best, so that the ring is
// the same one (positions equal to a spatial predictor then only drop out of
// the load count: their keys are already in the running best).
struct PbmRing {
  PbmBest best;   // best of the ring's evaluated positions (kNoKey: none)
  int rcode;      // this lane's ring position (lanes 0-7)
  bool act;       // this lane's position was evaluated
  bool valid;     // the early ring exists
};

__device__ __forceinline__ PbmRing pbm_no_ring() {
  PbmRing r;
  r.best.key = kNoKey;
  r.best.mvx = r.best.mvy = 0;
  r.best.sad = 0u;
  r.rcode = -1;
  r.act = false;
  r.valid = false;
  return r;
}

template <int N, int M>
__device__ PbmRing pbm_ring_early(int cx, int cy, bool valid, const PbmPart& pa, const PbmWin& wg,
                                  int p, uint32_t lam, const uint32_t* curs, const uint32_t* win) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  // the temporal and zero predictors' codes (lanes 4-13)
  const bool is_tz = valid && lane >= 4 && lane < 14;
  const int ecode = is_tz ? pbm_code(cx, cy, true, p) : -1;
  int rcode = -100 - lane;
  int ex = 0, ey = 0;
  if (lane < 8) {
    const int o = lane < 4 ? lane : lane + 1;  // skip the centre of the 3x3
    ex = clampi(pa.best.mvx + o % 3 - 1, -p, p);
    ey = clampi(pa.best.mvy + o / 3 - 1, -p, p);
    rcode = ((ey + p) << 8) + (ex + p);
  }
  bool rdup = false;
#pragma unroll
  for (int l = 4; l < 14; l++) rdup |= (__shfl_sync(FULL, ecode, l) == rcode);
  const unsigned rsame = __match_any_sync(FULL, rcode);
  rdup |= (rsame & ((1u << lane) - 1u)) != 0;
  PbmRing r;
  r.act = lane < 8 && !rdup;
  r.rcode = rcode;
  r.best = pbm_eval_set<N, M>(ex, ey, r.act, 4, wg, p, lam, curs, win);
  r.valid = true;
  return r;
}

template <int N, int M>
__device__ PbmResult pbm_part_b(int cx, int cy, bool valid, const PbmPart& pa, const PbmWin& wg,
                                int p, uint32_t lam, uint32_t intra_x, int32_t alpha,
                                int32_t beta, int32_t gnum, int32_t gden, int32_t qp,
                                int32_t refine, const uint32_t* curs, const uint32_t* win,
                                unsigned long long* tr = nullptr,
                                const PbmRing& early = pbm_no_ring()) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  // every predictor's code (lanes 0-13); a spatial one repeating a temporal
  // one, or an earlier spatial one, is not evaluated again
  const bool is_pred = valid && lane < 14;
  const int code = pbm_code(cx, cy, is_pred, p);
  const unsigned same = __match_any_sync(FULL, code);
  const bool dup = (same & (0x3FF0u | ((1u << lane) - 1u))) != 0;
  const bool actb = is_pred && lane < 4 && !dup;
  PbmBest best = pbm_better(pa.best, pbm_eval_set<N, M>(clampi(cx, -p, p), clampi(cy, -p, p), actb,
                                                        M >= 8 ? 8 : 4, wg, p, lam, curs, win));
  int load = pa.load + __popc(__ballot_sync(FULL, actb));
  pbm_stamp(tr, 1);
  if (refine && early.valid && best.key == pa.best.key) {
    // no spatial predictor beat part a's best: the early ring is this ring;
    // its positions equal to a spatial predictor leave the load count
    const int scode = is_pred && lane < 4 ? code : -1;
    bool sdup = false;
#pragma unroll
    for (int l = 0; l < 4; l++) sdup |= (__shfl_sync(FULL, scode, l) == early.rcode);
    best = pbm_better(best, early.best);
    load += __popc(__ballot_sync(FULL, early.act && !sdup));
    pbm_stamp(tr, 2);
  } else if (refine) {
    // every predictor's position has been evaluated (by its lane or by the
    // lane it repeats), so a ring position equal to any predictor's is skipped
    const int ecode = is_pred ? code : -1;
    int rcode = -100 - lane;
    int ex = 0, ey = 0;
    if (lane < 8) {
      const int o = lane < 4 ? lane : lane + 1;  // skip the centre of the 3x3
      ex = clampi(best.mvx + o % 3 - 1, -p, p);
      ey = clampi(best.mvy + o / 3 - 1, -p, p);
      rcode = ((ey + p) << 8) + (ex + p);
    }
    bool rdup = false;
#pragma unroll
    for (int l = 0; l < 14; l++) rdup |= (__shfl_sync(FULL, ecode, l) == rcode);
    // repeated among the ring's own lanes: an earlier ring lane holds it
    const unsigned rsame = __match_any_sync(FULL, rcode);
    rdup |= (rsame & ((1u << lane) - 1u)) != 0;
    const bool act = lane < 8 && !rdup;
    best = pbm_better(best, pbm_eval_set<N, M>(ex, ey, act, 4, wg, p, lam, curs, win));
    load += __popc(__ballot_sync(FULL, act));
    pbm_stamp(tr, 2);
  }
  // Sec. 3.2 conditions in exact integers (intra_x = NM * Intra_SAD)
  const long long NM = N * M, sad = best.sad, q = qp;
  const bool c1 = (long long)intra_x + NM * sad < NM * ((long long)alpha + (long long)beta * q * q);
  const bool c2 = (long long)gden * NM * sad < (long long)gnum * (long long)intra_x;
  PbmResult res;
  res.key = best.key;
  res.load = load;
  res.pass = c1 || c2;
  return res;
}

// Whether a block whose PBM winner had this key would fail both conditions
// (used on part a's best to start a likely full search early).
template <int N, int M>
__device__ __forceinline__ bool pbm_would_fail(const PbmBest& b, int p, uint32_t lam,
                                               uint32_t intra_x, int32_t alpha, int32_t beta,
                                               int32_t gnum, int32_t gden, int32_t qp) {
  const long long NM = N * M, sad = b.sad, q = qp;
  const bool c1 = (long long)intra_x + NM * sad < NM * ((long long)alpha + (long long)beta * q * q);
  const bool c2 = (long long)gden * NM * sad < (long long)gnum * (long long)intra_x;
  return !(c1 || c2);
}

// The whole PBM stage of one block with every predictor in hand.
template <int N, int M>
__device__ PbmResult pbm_eval(int cx, int cy, bool valid, const PbmWin& wg, int p, uint32_t lam,
                              uint32_t intra_x, int32_t alpha, int32_t beta, int32_t gnum,
                              int32_t gden, int32_t qp, int32_t refine, const uint32_t* curs,
                              const uint32_t* win, unsigned long long* tr = nullptr) {
  const PbmPart pa = pbm_part_a<N, M>(cx, cy, valid, wg, p, lam, curs, win, tr);
  return pbm_part_b<N, M>(cx, cy, valid, pa, wg, p, lam, intra_x, alpha, beta, gnum, gden, qp,
                          refine, curs, win, tr);
}

// PBM of block (bx, by) with its predictors read from the current-frame field
// `field` (final vectors of earlier waves) and the previous field `prev`
// (nullable: zero vectors): the per-frame path, where a kernel boundary orders
// every predictor before its reader.
template <int N, int M>
__device__ PbmResult warp_pbm(const uint8_t* __restrict__ cur, const uint8_t* __restrict__ refpad,
                              const PadGeom& pg, int W, int H, int p, uint32_t lam,
                              const int16_t* field, const int16_t* prev,
                              int bx, int by, uint32_t intra_x, int32_t alpha, int32_t beta,
                              int32_t gnum, int32_t gden, int32_t qp, int32_t refine,
                              uint32_t* curs, uint32_t* win) {
  const int lane = threadIdx.x & 31;
  const int BW = W / N, BH = H / M;
  const PbmWin wg = pbm_stage<N, M>(cur, refpad, pg, W, p, bx * N, by * M, curs, win);
  int cx = 0, cy = 0;
  bool valid = false;
  if (lane < 4) {
    const int dx = (lane < 2) ? -1 : (lane == 2 ? 0 : 1);
    const int dy = (lane == 0) ? 0 : -1;
    const int nx = bx + dx, ny = by + dy;
    if (nx >= 0 && nx < BW && ny >= 0) {
      cx = field[2 * (ny * BW + nx)];
      cy = field[2 * (ny * BW + nx) + 1];
      valid = true;
    }
  } else if (lane < 13) {
    const int t = lane - 4, nx = bx + t % 3 - 1, ny = by + t / 3 - 1;
    if (nx >= 0 && nx < BW && ny >= 0 && ny < BH) {
      if (prev) {
        cx = prev[2 * (ny * BW + nx)];
        cy = prev[2 * (ny * BW + nx) + 1];
      }
      valid = true;
    }
  } else if (lane == 13) {
    valid = true;
  }
  return pbm_eval<N, M>(cx, cy, valid, wg, p, lam, intra_x, alpha, beta, gnum, gden, qp, refine,
                        curs, win);
}

// ---------------------------------------------------------------------------
// Full-search tile plan: run length T, blocks per CTA and threads per CTA.
// ---------------------------------------------------------------------------
struct FsPlan {
  int T, G, threads;   // run length, threads per block, threads per CTA
  size_t smem;
  int S;               // CTAs sharing one block (column slices); 1 = whole block
};

// Chooses among the instantiated run lengths with a small cost model
// (SAD, load and epilogue instructions per useful candidate, lanes idle in the
// last round, shared-memory staging).  bpc_max = 1 forces one block per CTA.
FsPlan fs_plan(int N, int M, int p, int bpc_max);
std::vector<FsPlan> fs_plans_ranked(int N, int M, int p, int bpc_max, int k);
FsPlan fs_plan_latency(int N, int M, int p);
FsPlan fs_plan_fixed(int N, int M, int T, int p, int thr, int bpc_max, size_t smem_limit);

// The pipelined persistent full search (16x16 blocks, windows of 8 blocks
// within the compile-time pitch): K frame pairs frames[k] -> frames[k+1]
// (host array of device pointers) in one launch; outputs [K][BH][BW].
bool fsbm_pipe_applies(int N, int M, int p);
int launch_fsbm_pipe(const uint8_t* const* frames, int K, int W, int H, int p, uint32_t lam,
                     int16_t* mv_out, uint32_t* J_out, uint32_t* sad_out, cudaStream_t s);

// Outputs of the pipelined search in its three modes: kPipeKeys (mv, J, sad;
// each nullable), kPipeStats (also smin, sdev: SAD_min and SAD_deviation,
// required), kPipeVolume (every candidate's SAD: vol + block * vstride +
// (mvy+p)*(2p+1) + (mvx+p), uint16).  ref_fixed: every pair k compares
// frames[k+1] with frames[0] instead of frames[k].
enum { kPipeKeys = 0, kPipeStats = 1, kPipeVolume = 2 };
struct PipeOut {
  int16_t* mv;
  uint32_t* J;
  uint32_t* sad;
  uint32_t* smin;
  uint32_t* sdev;
  uint16_t* vol;
  int vstride;
  int ref_fixed;
};
int launch_fsbm_pipe_mode(int mode, const uint8_t* const* frames, int K, int W, int H, int p,
                          uint32_t lam, const PipeOut& out, cudaStream_t s, int T = 0);

// The full search of K pairs (frames[k] -> frames[k+1], outputs [K][BH][BW])
// in the launch form the autotuner picked for the shape (timed on the first
// call; every form gives the same outputs).
int fsbm_tuned(const uint8_t* const* frames, int K, int W, int H, int N, int M, int p,
               uint32_t lam, int16_t* mv_out, uint32_t* J_out, uint32_t* sad_out, cudaStream_t s);

// ACBM of one pair in the form the autotuner picked for the shape: candidate
// 0 is `waves` (the per-frame wave graph), the others the persistent
// two-role kernel over this one pair (the launch forms of the sequence plan
// with K = 1).  Every form gives the same outputs.  While s is being
// captured, `waves` runs.
int acbm_pair_tuned(const AcbmArgs& a, int W, int H, int N, int M, int p, cudaStream_t s,
                    const std::function<int()>& waves);

// Calls FN<N, M, T>(...) for the run lengths instantiated per block shape
// (pl.T chooses among them for 16x16); expects N, M and pl in scope.
#define ME_DISPATCH_FS(FN, ...)                                                      \
  do {                                                                               \
    if (N == 16 && M == 16) {                                                        \
      switch (pl.T) {                                                                \
        case 8: return FN<16, 16, 8>(__VA_ARGS__);                                   \
        case 11: return FN<16, 16, 11>(__VA_ARGS__);                                 \
        case 13: return FN<16, 16, 13>(__VA_ARGS__);                                 \
        case 16: return FN<16, 16, 16>(__VA_ARGS__);                                 \
      }                                                                              \
    }                                                                                \
    if (N == 16 && M == 8) return FN<16, 8, 8>(__VA_ARGS__);                         \
    if (N == 16 && M == 4) return FN<16, 4, 8>(__VA_ARGS__);                         \
    if (N == 8 && M == 16) return FN<8, 16, 8>(__VA_ARGS__);                         \
    if (N == 8 && M == 8) return FN<8, 8, 8>(__VA_ARGS__);                           \
    if (N == 8 && M == 4) return FN<8, 4, 8>(__VA_ARGS__);                           \
    if (N == 4 && M == 16) return FN<4, 16, 8>(__VA_ARGS__);                         \
    if (N == 4 && M == 8) return FN<4, 8, 8>(__VA_ARGS__);                           \
    if (N == 4 && M == 4) return FN<4, 4, 8>(__VA_ARGS__);                           \
    return ME_ERR_ARG;                                                               \
  } while (0)

// Scratch layout of one ACBM frame (the call's arguments, padded reference,
// scaled Intra_SAD per block, and per block the key and state word of its
// early full search), in bytes from the start of one 256-byte aligned region.
struct AcbmScratch {
  size_t off_args, off_pad, off_intra, off_keys, off_done, total;
};
AcbmScratch acbm_scratch_layout(int W, int H, int N, int M, int p);

// Enqueues the whole ACBM frame on s, using `scratch` (acbm_scratch_layout
// bytes; every part that must start at zero is cleared on the stream first).
int enqueue_acbm(const AcbmArgs& a, int W, int H, int N, int M, int p, uint8_t* scratch,
                 cudaStream_t s);

}  // namespace me

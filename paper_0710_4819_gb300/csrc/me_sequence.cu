// me_sequence.cu -- FSBM and ACBM over K consecutive frame pairs of one
// sequence in one launch each.
//
// FSBM (Sec. 2.3): no dependencies between blocks or pairs.  Launch forms,
// chosen per shape by the autotuner: the per-group kernel with one grid row
// per pair (k_fsbm_seq); the pipelined persistent search for 16x16 blocks at
// p <= 34 (k_fsbm_pipe: producer warps stage block groups' shifted windows
// while consumer warps search, mbarrier hand-over); the table-driven
// pipelined search for every shape and p <= 64 (k_fsbm_pipe_tab: groups of
// adjacent blocks searched in bands of candidate rows, from a sequence or
// from the batch's group table).
//
// ACBM (Sec. 3.2): the causal order of the method (Sec. 2.2: spatial
// predictors must be final in the current frame; temporal predictors come
// from the previous frame's field) allows pairs to overlap: block (x, y) of
// pair k needs the final vectors of its left, up-left, up and up-right
// neighbours in pair k (anti-diagonal waves w-1 .. w-3, with w = x + 2y) and
// of its 3x3 neighbourhood in pair k-1 (waves up to w+3).  Claiming all
// blocks of all pairs in the order w + L*k (L >= 4) therefore puts every
// dependency first, and one persistent launch (k_acbm_seq: PBM CTAs and
// full-search CTAs) walks the whole sequence with L waves between
// consecutive pairs instead of a full frame: the GPU sees many pairs in
// flight at once.  Each block waits (bounded in time) for its 4 + 9
// predecessors' flags.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "me_device.cuh"
#include "me_host.h"
#include "me_search.cuh"
#include "me_batch_types.h"

namespace me {

constexpr int kSeqMax = 64;     // frame pairs per call
constexpr int kSeqThreads = 256;
constexpr int kSeqLag = 4;      // waves between consecutive pairs in the claim order (least)
// Claim orders the plan holds: lags of 4 (the least that keeps every
// predecessor claimed before its block), 5 and 6 waves between pairs; a
// longer lag claims a pair's blocks later, when their temporal predecessors
// are more likely finished, so PBM warps wait less while holding a block.
constexpr int kSeqLags[] = {4, 5, 6};
constexpr int kSeqNLags = 3;
// The model's role split of k_acbm_seq: every kSeqSearchEvery-th SM (by
// %smid) hosts two search CTAs instead of one PBM and one search CTA.
// Measured at 1080p p=32 (59 pairs): one of each on every SM 0.1196 ms of
// ACBM per pair; two search CTAs on every 8th / 4th / 3rd / 2nd SM 0.1159 /
// 0.1119 / 0.1097 / 0.1113 ms; without occlusions (1.5 % of blocks searched)
// 0.0841 / - / 0.0834 / 0.0844 / 0.0911 ms.  The autotuner also times the
// 2nd and 4th SM splits.
constexpr int kSeqSearchEvery = 3;
constexpr int kSeqSP = 193;     // compile-time shifted-word pitch of the main FSBM build (odd:
                                // rows of different runs start on different banks)

struct SeqFrames {
  const uint8_t* f[kSeqMax + 1];  // f[k] = reference of pair k, f[k+1] = its current frame
};

struct SeqArgs {
  const int16_t* prev0;  // field before pair 0 (nullable)
  int16_t* mv;           // [K][BH][BW][2]
  uint32_t* J;           // [K][BH][BW]
  uint8_t* mask;
  uint32_t* sad;         // nullable
  uint32_t* load;        // nullable
  uint32_t lam;
  int32_t alpha, beta, gnum, gden, qp, refine;
};

// Control block of a run.  Counters that many warps update or poll each sit
// on their own 128-byte line: an atomic on a line that 1000+ warps keep
// reading waits behind those reads for microseconds.
struct SeqCtrl {
  int epoch, error, err_item;   // read-mostly (error is written only on failure)
  long long timeout_cycles;     // bound of every spin-wait (SM clock cycles)
  alignas(128) int next;        // PBM claims
  alignas(128) int fs_head;     // search-CTA claims
  alignas(128) int fs_tail;     // queue appends
  alignas(128) int pbm_done;    // blocks through PBM
  alignas(128) int started;     // CTA arrivals (roles)
  int sm_arr[kRoleSlots];       // CTA arrivals per SM (roles)
};

// ------------------------------------------------------------------ FSBM

template <int N, int M, int T, int SP = 0>
__global__ void __launch_bounds__(kMaxThreads) k_fsbm_seq(SeqFrames fr, int W, int H, int p, int G,
                                                          uint32_t lam, int16_t* __restrict__ mv_out,
                                                          uint32_t* __restrict__ J_out,
                                                          uint32_t* __restrict__ sad_out) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ unsigned long long keys[16];
  const int k = blockIdx.y;
  const int BW = W / N, nbf = BW * (H / M);
  const int bpc = blockDim.x / G;
  const int gpr = (BW + bpc - 1) / bpc;
  const int by = blockIdx.x / gpr, bx0 = (blockIdx.x % gpr) * bpc;
  const int nb = min(bpc, BW - bx0);
  const FsGeom g = fs_geom<N, M, T>(p, nb, G, 0, 0, SP);
  fs_group<N, M, T, SP>(fr.f[k + 1], fr.f[k], W, H, bx0 * N, by * M, g, lam, smem, keys);
  if ((int)threadIdx.x < nb) {
    const Decoded d = decode_key(keys[threadIdx.x], p, lam);
    const size_t b = (size_t)k * nbf + by * BW + bx0 + threadIdx.x;
    mv_out[2 * b] = (int16_t)d.mvx;
    mv_out[2 * b + 1] = (int16_t)d.mvy;
    J_out[b] = d.J;
    if (sad_out) sad_out[b] = d.sad;
  }
}

// ------------------------------------------------------------------ FSBM, pipelined
//
// The same full search as k_fsbm_seq as one persistent CTA per SM that
// overlaps staging with searching.  Four producer warps stage the windows of
// the CTA's groups (kPipeBpc adjacent blocks of one block row of one pair;
// groups blockIdx.x, blockIdx.x + gridDim.x, ...) into two shared-memory
// buffers in turn; twelve consumer warps (three per scheduler) run the
// searches.  A group's runs (block-major, then segment, then column) are
// dealt in rounds of 32, one per lane, each consumer warp taking a fixed
// contiguous range of rounds, and a warp moves on to the next group as soon
// as its own rounds are done -- the uneven shares of a group (2600 runs over
// 12 warps at p = 32) no longer leave lanes or warps idle until the slowest
// finishes, and staging is off the search's path.  When every consumer
// thread has arrived on a buffer's empty barrier, the producers write that
// group's results (per-block minima kept in shared memory) and restage the
// buffer.  Every wait is bounded (SM cycle count); a wait that gives up
// records ME_ERR_TIMEOUT for me_fsbm_sequence_status.  The producer count is
// a build-time setting (ME_PIPE_PRODUCERS) for sweeps.
constexpr int kPipeThreads = 512;
#ifndef ME_PIPE_PRODUCERS
#define ME_PIPE_PRODUCERS 4
#endif
constexpr int kPipeProducers = ME_PIPE_PRODUCERS;               // warps
constexpr int kPipeConsumers = kPipeThreads / 32 - kPipeProducers;
constexpr int kPipeBpc = 8;

__device__ int g_fsbm_pipe_error = 0;

template <int N, int M, int T>
__host__ __device__ inline size_t pipe_smem_bytes(int p) {
  const FsGeom g = fs_geom<N, M, T>(p, kPipeBpc, 32, 0, 0, kSeqSP);
  const size_t words = 3 * (size_t)g.rows + (size_t)g.rows * g.wbw +
                       2 * ((size_t)kPipeBpc * M * (N / 4) + (size_t)g.rows * kSeqSP);
  return 4 * words;
}

// Shared-memory barrier objects (mbarrier) hand the two buffers between the
// roles: full[b] completes a phase when the producers have staged a group
// into buffer b, empty[b] when every consumer thread is through it.  A
// waiting thread sleeps in the barrier's try_wait (suspend-time hint), so
// waiting costs no issue slots; the wait is bounded by the SM cycle count and
// gives up early when another wait has (err).
__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(a) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, volatile int* err,
                                          long long lim) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  const long long t0 = clock64();
  for (;;) {
    unsigned done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(a), "r"(parity), "r"(20000u)
        : "memory");
    if (done) return true;
    if (*err) return false;
    if (clock64() - t0 > lim) {
      *err = 1;
      atomicExch(&g_fsbm_pipe_error, (int)ME_ERR_TIMEOUT);
      return false;
    }
  }
}

// MODE: kPipeKeys (the search: best key per block), kPipeStats (also the sum
// and the minimum of the SAD over the window per block: SAD_min and
// SAD_deviation, Sec. 3.1), kPipeVolume (every candidate's SAD to a volume).
template <int N, int M, int T, int MODE>
__global__ void __launch_bounds__(kPipeThreads, 1) k_fsbm_pipe(SeqFrames fr, int W, int H, int p,
                                                              uint32_t lam, int groups, long long lim,
                                                              PipeOut out) {
  constexpr int NW = N / 4, B = kPipeBpc, SP = kSeqSP;
  constexpr int PT = 32 * kPipeProducers, CT = 32 * kPipeConsumers;
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ unsigned long long red[2][B];
  __shared__ uint32_t ssum_s[2][B], smin_s[2][B];
  __shared__ __align__(8) uint64_t full_bar[2], empty_bar[2];
  __shared__ int err_s, go_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned FULL = 0xffffffffu;
  const FsGeom g = fs_geom<N, M, T>(p, B, 32, 0, 0, SP);
  const int n = g.n, nc = g.nc;
  const int BW = W / N, BH = H / M, nbf = BW * BH;
  const int gpr = (BW + B - 1) / B;
  uint32_t* tabJ = smem;
  uint32_t* tabK = tabJ + g.rows;
  uint32_t* tabQ = tabK + g.rows;
  uint32_t* raw = tabQ + g.rows;                        // [rows][wbw], producers only
  // buffer b: current blocks [B][M][NW], then shifted words [rows][SP]
  const int bstride = B * M * NW + g.rows * SP;
  uint32_t* const buf0 = raw + g.rows * g.wbw;
  const int fast = key_mode(N, M, p, lam);
  const int rb = rank_bits(p);
  for (int r = tid; r < g.rows; r += kPipeThreads) {
    const int mvy = r - p;
    const int a = mvy < 0 ? -mvy : mvy;
    tabJ[r] = lam * (uint32_t)mv_bits(mvy);
    tabK[r] = ((uint32_t)a << 17) + (uint32_t)r * (uint32_t)n;
    tabQ[r] = tabq_value(fast, tabJ[r], mvy, p);
  }
  if (tid < 2 * B) {
    red[tid / B][tid % B] = kNoKey;
    ssum_s[tid / B][tid % B] = 0u;
    smin_s[tid / B][tid % B] = 0xffffffffu;
  }
  if (tid == 0) {
    err_s = 0;
    mbar_init(&full_bar[0], PT);
    mbar_init(&full_bar[1], PT);
    mbar_init(&empty_bar[0], CT);
    mbar_init(&empty_bar[1], CT);
  }
  __syncthreads();
  const int mine = groups > (int)blockIdx.x ? (groups - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (warp < kPipeProducers) {
    // ---------------- producers: stage group i into buffer i & 1; once its
    // consumers are through group i - 2 in that buffer, write that group's
    // results first
    const int pt = tid;
    // results of group j (its consumers done): the per-block minima -> outputs
    auto finish = [&](int j) {
      const int b = j & 1;
      if (pt == 0) go_s = mbar_wait(&empty_bar[b], (unsigned)((j >> 1) & 1), &err_s, lim) ? 1 : 0;
      asm volatile("bar.sync 1, %0;" ::"r"(PT) : "memory");
      const bool go = go_s != 0;
      asm volatile("bar.sync 1, %0;" ::"r"(PT) : "memory");
      if (!go) return false;
      const int gj = (int)blockIdx.x + j * (int)gridDim.x;
      const int k = gj / (BH * gpr), rem = gj - k * (BH * gpr);
      const int by = rem / gpr, bx0 = (rem - by * gpr) * B;
      if (MODE != kPipeVolume && pt < B) {
        if (bx0 + pt < BW) {
          const Decoded d = decode_key(red[b][pt], p, lam);
          const size_t o = (size_t)k * nbf + (size_t)by * BW + bx0 + pt;
          if (out.mv) {
            out.mv[2 * o] = (int16_t)d.mvx;
            out.mv[2 * o + 1] = (int16_t)d.mvy;
          }
          if (out.J) out.J[o] = d.J;
          if (out.sad) out.sad[o] = d.sad;
          if (MODE == kPipeStats) {
            // every term of sum |SAD - SAD_min| is non-negative
            out.smin[o] = smin_s[b][pt];
            out.sdev[o] = ssum_s[b][pt] - (uint32_t)(n * n) * smin_s[b][pt];
          }
        }
        red[b][pt] = kNoKey;
        ssum_s[b][pt] = 0u;
        smin_s[b][pt] = 0xffffffffu;
      }
      return true;
    };
    bool ok = true;
    for (int i = 0; i < mine && ok; i++) {
      const int b = i & 1;
      if (i >= 2 && !finish(i - 2)) { ok = false; break; }
      const int gi = (int)blockIdx.x + i * (int)gridDim.x;
      const int k = gi / (BH * gpr), rem = gi - k * (BH * gpr);
      const int by = rem / gpr, bx0 = (rem - by * gpr) * B;
      const int x0 = bx0 * N, y0 = by * M;
      const uint8_t* __restrict__ cur = fr.f[k + 1];
      const uint8_t* __restrict__ ref = fr.f[out.ref_fixed ? 0 : k];
      uint32_t* cw = buf0 + b * bstride;
      for (int e = pt; e < B * M * NW; e += PT) {
        const int blk = e / (M * NW), rm = e % (M * NW), j = rm / NW, w = rm % NW;
        cw[e] = bx0 + blk < BW
                    ? *reinterpret_cast<const uint32_t*>(cur + (size_t)(y0 + j) * W + x0 + blk * N + 4 * w)
                    : 0u;
      }
      // raw window rows from the aligned word at or left of column x0 - p:
      // producer warp pw takes rows pw, pw + kPipeProducers, ...; its lanes
      // the words of a row (wbw <= 64).  Windows inside the frame are copied
      // asynchronously; the others are clamped byte by byte.
      const int pw = warp;
      const int wx0 = x0 - p;
      const int A0 = (wx0 >> 2) << 2;
      const int s0 = wx0 - A0;
      const bool inside = A0 >= 0 && A0 + 4 * g.wbw <= W;
      for (int r = pw; r < g.rows; r += kPipeProducers) {
        const uint8_t* rowp = ref + (size_t)clampi(y0 - p + r, 0, H - 1) * W + A0;
        uint32_t* dst = raw + r * g.wbw;
        for (int q = lane; q < g.wbw; q += 32) {
          if (inside) {
            const unsigned d = (unsigned)__cvta_generic_to_shared(dst + q);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(rowp + 4 * q)
                         : "memory");
          } else {
            uint32_t v = 0;
#pragma unroll
            for (int bb = 0; bb < 4; bb++)
              v |= (uint32_t)ref[(size_t)clampi(y0 - p + r, 0, H - 1) * W +
                                 clampi(A0 + 4 * q + bb, 0, W - 1)] << (8 * bb);
            dst[q] = v;
          }
        }
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
      asm volatile("bar.sync 1, %0;" ::"r"(PT) : "memory");
      // shifted words: sh[r][o] = raw bytes s0+o .. s0+o+3, four consecutive
      // o per lane from the three raw words that hold them
      uint32_t* sh = cw + B * M * NW;
      const int quads = (g.pos + 3) >> 2;
      for (int r = pw; r < g.rows; r += kPipeProducers) {
        for (int qd = lane; qd < quads; qd += 32) {
          const int o = 4 * qd;
          // (the third word may lie past the row, and is then not used)
          const uint32_t* row = raw + r * g.wbw + ((s0 + o) >> 2);
          const uint32_t w0 = row[0], w1 = row[1], w2 = row[2];
          const int t0 = (s0 + o) & 3;
          uint32_t* dst = sh + r * SP + o;
#pragma unroll
          for (int d = 0; d < 4; d++) {
            const int t = t0 + d;            // byte offset from w0, 0 .. 6
            if (o + d < g.pos)
              dst[d] = t < 4 ? __funnelshift_r(w0, w1, 8 * t) : __funnelshift_r(w1, w2, 8 * (t - 4));
          }
        }
      }
      // every producer's stores before its arrival (raw is rewritten only
      // after the next group's first producer barrier)
      asm volatile("bar.sync 1, %0;" ::"r"(PT) : "memory");
      mbar_arrive(&full_bar[b]);
    }
    // the last two groups' results
    for (int j = mine - 2; ok && j < mine; j++)
      if (j >= 0 && !finish(j)) ok = false;
    return;
  }

  // ---------------- consumers
  // A group's R warp-tasks (32 consecutive tasks each) are dealt round robin
  // over the consumer warps, continuing from where the previous group's
  // dealing stopped: the warps that took one more warp-task of this group
  // take one fewer of the next, so no warp is the slowest of every group.
  const int cw_id = warp - kPipeProducers;
  const int F = B * g.tasks;
  const int R = (F + 31) >> 5;
  constexpr int KC = kPipeConsumers;
  // one step = 32 * KC tasks = dblk whole blocks + dseg runs + dcol columns
  const int dblk = (32 * KC) / g.tasks, drem = 32 * KC - dblk * g.tasks;
  const int dseg = drem / nc, dcol = drem - (drem / nc) * nc;
  uint32_t c[M][NW];
  for (int i = 0; i < mine; i++) {
    const int b = i & 1;
    int ok = 1;
    if (lane == 0) ok = mbar_wait(&full_bar[b], (unsigned)((i >> 1) & 1), &err_s, lim) ? 1 : 0;
    ok = __shfl_sync(FULL, ok, 0);
    if (!ok) break;
    __syncwarp();
    // every lane acquires the producers' stores itself (the phase is complete)
    mbar_wait(&full_bar[b], (unsigned)((i >> 1) & 1), &err_s, lim);
    const int gi = (int)blockIdx.x + i * (int)gridDim.x;
    const int gk = gi / (BH * gpr), rem = gi - gk * (BH * gpr);
    const int bx0 = (rem % gpr) * B;
    const int nb = min(B, BW - bx0);
    // MODE kPipeVolume: the group's first block in the volume
    uint16_t* vg = MODE == kPipeVolume
                       ? out.vol + ((size_t)gk * nbf + (size_t)(rem / gpr) * BW + bx0) * out.vstride
                       : nullptr;
    const uint32_t* cwb = buf0 + b * bstride;
    const uint32_t* sh = cwb + B * M * NW;
    const int qs = (cw_id - (int)(((long long)i * R) % KC) + KC) % KC;
    int f = 32 * qs + lane;
    int blk = f / g.tasks;
    const int t0 = f - blk * g.tasks;
    int seg = t0 / nc, col = t0 - (t0 / nc) * nc;
    for (int q = qs; q < R; q += KC, f += 32 * KC) {
      if (f < F && blk < nb) {
#pragma unroll
        for (int j = 0; j < M; j++)
#pragma unroll
          for (int w = 0; w < NW; w++) c[j][w] = cwb[(blk * M + j) * NW + w];
        const int row0 = seg * T;
        uint32_t acc[T];
        fs_run_sads<N, M, T>(c, sh + row0 * SP + blk * N + col, SP, acc);
        if (MODE == kPipeVolume) {
          uint16_t* vb = vg + (size_t)blk * out.vstride + col;
#pragma unroll
          for (int kk = 0; kk < T; kk++)
            if (row0 + kk < n) vb[(row0 + kk) * n] = (uint16_t)acc[kk];
        } else {
          atomicMin(&red[b][blk], fs_run_key<T>(acc, row0, col, p, n, lam, rb, fast, tabJ, tabK, tabQ));
        }
        if (MODE == kPipeStats) {
          uint32_t sum = 0u, mn = 0xffffffffu;
#pragma unroll
          for (int kk = 0; kk < T; kk++)
            if (row0 + kk < n) {
              sum += acc[kk];
              mn = min(mn, acc[kk]);
            }
          atomicAdd(&ssum_s[b][blk], sum);
          atomicMin(&smin_s[b][blk], mn);
        }
      }
      col += dcol;
      if (col >= nc) { col -= nc; seg++; }
      seg += dseg;
      if (seg >= g.nseg) { seg -= g.nseg; blk++; }
      blk += dblk;
    }
    mbar_arrive(&empty_bar[b]);
  }
}

// ------------------------------------------------------------------ pipelined search, any p
//
// The pipelined full search for every block shape at every search range
// p <= 64, driven by a table of block groups: the same producer/consumer
// pipeline as k_fsbm_pipe (4 producer warps stage a work item into one of
// two shared buffers while 12 consumer warps search the other), with a fixed
// shifted-word pitch of kTabSP words.  A group is tab_bpc(p) adjacent blocks
// of one block row (16x16: 8 at p = 64, 12 at p = 32, 14 at p = 16; narrower
// blocks more).  Its candidate rows (mvy) are split into bands of at most
// TabCfg::HB rows (65 for 16x16: five runs of 13; 72 for the other shapes:
// nine runs of 8), one work item per band: a window band of HB + M - 1 rows
// is staged at a time, so that the shifted words of many blocks fit the
// buffers at any p and the producers' staging is spread over more SAD work.
// The bands of a group meet in the per-block minimum (red), which the
// producers decode after the group's last band.  Groups come from one of
// two sources:
//   - a sequence of K pairs (frames[k] -> frames[k+1]) of one shape, groups
//     dealt to CTAs round robin;
//   - a batch of streams of any sizes and ranges (the batch API's stream and
//     group tables), groups claimed from a counter, largest work first.
// The tables of costs per row depend on p and lambda, so the producers stage
// them with each work item.
constexpr int kTabSP = 253;

template <int N, int M>
struct TabCfg {
  static constexpr int T = (N == 16 && M == 16) ? 13 : 8;              // run length
  static constexpr int HB = ((65 + T - 1) / T) * T;                    // candidate rows per band
  static constexpr int RB = HB + M - 1;                                // staged rows per band
  static constexpr int RT = 2 * HB;                                    // cost-table rows (p <= 64)
  static constexpr int B = 256 / N;                                    // blocks per group, at most
  static constexpr int WBW = (kTabSP + 6) / 4 + 1;                     // raw words per row
  static constexpr int BST = B * M * (N / 4) + 3 * RT + RB * kTabSP;   // words per buffer
};

template <int N>
__host__ __device__ inline int tab_bpc(int p) {
  const int b = (kTabSP - (2 * p + 1) - (N - 4)) / N + 1;
  return b < 256 / N ? b : 256 / N;
}

// Bands of a group at range p (one while 2p+1 <= HB, else two).
template <int N, int M>
__host__ __device__ inline int tab_nbands(int p) {
  return 2 * p + 1 <= TabCfg<N, M>::HB ? 1 : 2;
}

struct TabArgs {
  // sequence source (shp == nullptr)
  SeqFrames fr;
  int W, H, p, K;
  uint32_t lam;
  int16_t* mv;
  uint32_t* J;
  uint32_t* sad;
  // batch source
  const BShape* shp;
  const BStream* st;
  const BFsEntry* ent;
  int ngroups;
  int* ctr;         // group claims (batch); null: round robin
  int* err;         // the caller's error word; null: g_fsbm_pipe_error
  long long lim;    // bound of every wait, SM cycles
};

struct TabGroup {
  const uint8_t* cur;
  const uint8_t* ref;
  int16_t* mv;
  uint32_t* J;
  uint32_t* sad;
  int W, H, p, x0, y0, nb;
  long long obase;  // output index of the group's first block
  uint32_t lam;
};

template <int N, int M>
__device__ __forceinline__ TabGroup tab_group(const TabArgs& A, int gi) {
  TabGroup G;
  if (A.shp == nullptr) {
    const int BW = A.W / N, BH = A.H / M, bpc = tab_bpc<N>(A.p);
    const int gpr = (BW + bpc - 1) / bpc;
    const int k = gi / (BH * gpr), rem = gi - k * (BH * gpr);
    const int by = rem / gpr, bx0 = (rem - by * gpr) * bpc;
    G.cur = A.fr.f[k + 1];
    G.ref = A.fr.f[k];
    G.mv = A.mv;
    G.J = A.J;
    G.sad = A.sad;
    G.W = A.W;
    G.H = A.H;
    G.p = A.p;
    G.lam = A.lam;
    G.x0 = bx0 * N;
    G.y0 = by * M;
    G.nb = min(bpc, BW - bx0);
    G.obase = (long long)k * BW * BH + (long long)by * BW + bx0;
  } else {
    const BFsEntry e = A.ent[gi];
    const BShape& s = A.shp[e.stream];
    const BStream& a = A.st[e.stream];
    G.cur = a.cur;
    G.ref = a.ref;
    G.mv = a.mv;
    G.J = a.J;
    G.sad = a.sad;
    G.W = s.W;
    G.H = s.H;
    G.p = s.p;
    G.lam = a.lam;
    G.x0 = e.bx0 * N;
    G.y0 = e.by * M;
    G.nb = e.nb;
    G.obase = (long long)e.by * (s.W / N) + e.bx0;
  }
  return G;
}

template <int N, int M>
__host__ __device__ inline size_t tab_smem_bytes() {
  using C = TabCfg<N, M>;
  return 4 * ((size_t)C::RB * C::WBW + 2 * (size_t)C::BST);
}

template <int N, int M>
__global__ void __launch_bounds__(kPipeThreads, 1) k_fsbm_pipe_tab(TabArgs A) {
  using C = TabCfg<N, M>;
  constexpr int NW = N / 4, T = C::T, SP = kTabSP, RB = C::RB, RT = C::RT, HB = C::HB, B = C::B;
  constexpr int WBW = C::WBW;
  constexpr int PT = 32 * kPipeProducers, CT = 32 * kPipeConsumers;
  constexpr int BST = C::BST;   // words per buffer
  extern __shared__ __align__(16) uint32_t smem[];
  // per group slot (two groups can be in flight): the group and its blocks'
  // running minima over the bands searched so far
  __shared__ unsigned long long red[2][B];
  __shared__ TabGroup grp[2];
  // per buffer: the work item's group (-1: end mark), group slot, first
  // candidate row of its band, candidate rows, last band of its group
  __shared__ int gid_s[2], slot_s[2], r0_s[2], nrow_s[2], last_s[2];
  __shared__ __align__(8) uint64_t full_bar[2], empty_bar[2];
  __shared__ int err_s, go_s, claim_s, band_s, newg_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned FULL = 0xffffffffu;
  uint32_t* raw = smem;                       // [RB][WBW], producers only
  uint32_t* const buf0 = raw + RB * WBW;      // buffer b: cur [B][M][NW], tabJ/K/Q [RT], sh [RB][SP]
  int* const errw = A.err ? A.err : &g_fsbm_pipe_error;
  for (int i = tid; i < 2 * B; i += blockDim.x) red[i / B][i % B] = kNoKey;
  if (tid == 0) {
    err_s = 0;
    mbar_init(&full_bar[0], PT);
    mbar_init(&full_bar[1], PT);
    mbar_init(&empty_bar[0], CT);
    mbar_init(&empty_bar[1], CT);
  }
  __syncthreads();

  if (warp < kPipeProducers) {
    const int pt = tid;
    // the decisions of producer thread 0: current group, its band, its bands
    int cur_g = -1, cur_band = 0, cur_nb = 0, gj = 0, gcount = 0;
    auto finish = [&](int j) {
      const int b = j & 1;
      if (pt == 0) {
        const bool w = mbar_wait(&empty_bar[b], (unsigned)((j >> 1) & 1), &err_s, A.lim);
        if (!w) atomicExch(errw, (int)ME_ERR_TIMEOUT);
        go_s = w ? 1 : 0;
      }
      asm volatile("bar.sync 1, %0;" ::"r"(PT) : "memory");
      const bool go = go_s != 0;
      asm volatile("bar.sync 1, %0;" ::"r"(PT) : "memory");
      if (!go) return false;
      if (last_s[b]) {
        const int sl = slot_s[b];
        const TabGroup& G = grp[sl];
        for (int e = pt; e < B; e += PT) {
          if (e < G.nb) {
            const Decoded d = decode_key(red[sl][e], G.p, G.lam);
            const long long o = G.obase + e;
            if (G.mv) {
              G.mv[2 * o] = (int16_t)d.mvx;
              G.mv[2 * o + 1] = (int16_t)d.mvy;
            }
            if (G.J) G.J[o] = d.J;
            if (G.sad) G.sad[o] = d.sad;
          }
          red[sl][e] = kNoKey;
        }
      }
      // the buffer's item fields and grp[] are rewritten after this
      asm volatile("bar.sync 1, %0;" ::"r"(PT) : "memory");
      return true;
    };
    bool ok = true;
    int i = 0;
    for (;; i++) {
      const int b = i & 1;
      if (pt == 0) {
        // the next band of the current group, or the first band of the next
        if (cur_g >= 0 && cur_band + 1 < cur_nb) {
          cur_band++;
          newg_s = 0;
        } else {
          cur_g = A.ctr ? atomicAdd(A.ctr, 1) : (int)blockIdx.x + gj * (int)gridDim.x;
          gj++;
          cur_band = 0;
          cur_nb = cur_g < A.ngroups ? tab_nbands<N, M>(tab_group<N, M>(A, cur_g).p) : 1;
          newg_s = 1;
        }
        claim_s = cur_g;
        band_s = cur_band;
      }
      asm volatile("bar.sync 1, %0;" ::"r"(PT) : "memory");
      const int gi = claim_s, band = band_s, newg = newg_s;
      if (i >= 2 && !finish(i - 2)) { ok = false; break; }   // (its barriers order the reads above)
      if (gi >= A.ngroups) break;
      const TabGroup G = tab_group<N, M>(A, gi);
      const int p = G.p, n = 2 * p + 1, nbands = tab_nbands<N, M>(p);
      const int R0 = band * HB, nrow = min(n - R0, HB), nseg = (nrow + T - 1) / T;
      const int rows = nseg * T + M - 1;
      if (pt == 0) {
        if (newg) {
          grp[gcount & 1] = G;
          gcount++;
        }
        gid_s[b] = gi;
        slot_s[b] = (gcount - 1) & 1;
        r0_s[b] = R0;
        nrow_s[b] = nrow;
        last_s[b] = band == nbands - 1 ? 1 : 0;
      }
      const int pos = (G.nb - 1) * N + n + N - 4;
      uint32_t* cw = buf0 + b * BST;
      uint32_t* tabJ = cw + B * M * NW;
      uint32_t* tabK = tabJ + RT;
      uint32_t* tabQ = tabK + RT;
      uint32_t* sh = tabQ + RT;
      for (int e = pt; e < G.nb * M * NW; e += PT) {
        const int blk = e / (M * NW), rm = e % (M * NW), j = rm / NW, w = rm % NW;
        cw[e] = *reinterpret_cast<const uint32_t*>(G.cur + (size_t)(G.y0 + j) * G.W + G.x0 + blk * N +
                                                  4 * w);
      }
      // costs of every candidate row of the group (indexed by the row in the
      // whole window, r = mvy + p)
      const int kmode = key_mode(N, M, p, G.lam);
      for (int r = pt; r < nbands * HB; r += PT) {
        const int mvy = r - p;
        const int am = mvy < 0 ? -mvy : mvy;
        tabJ[r] = G.lam * (uint32_t)mv_bits(mvy);
        tabK[r] = ((uint32_t)am << 17) + (uint32_t)r * (uint32_t)n;
        tabQ[r] = tabq_value(kmode, tabJ[r], mvy, p);
      }
      // raw window rows of the band, from the aligned word at or left of
      // column x0 - p
      const int wbw = (pos + 6) / 4 + 1;
      const int wx0 = G.x0 - p;
      const int A0 = (wx0 >> 2) << 2;
      const int s0 = wx0 - A0;
      const bool inside = A0 >= 0 && A0 + 4 * wbw <= G.W;
      for (int r = warp; r < rows; r += kPipeProducers) {
        const size_t yrow = (size_t)clampi(G.y0 - p + R0 + r, 0, G.H - 1) * G.W;
        uint32_t* dst = raw + r * WBW;
        for (int q = lane; q < wbw; q += 32) {
          if (inside) {
            const unsigned d = (unsigned)__cvta_generic_to_shared(dst + q);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(G.ref + yrow + A0 + 4 * q)
                         : "memory");
          } else {
            uint32_t v = 0;
#pragma unroll
            for (int bb = 0; bb < 4; bb++)
              v |= (uint32_t)G.ref[yrow + clampi(A0 + 4 * q + bb, 0, G.W - 1)] << (8 * bb);
            dst[q] = v;
          }
        }
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
      asm volatile("bar.sync 1, %0;" ::"r"(PT) : "memory");
      // shifted words: sh[r][o] = raw bytes s0+o .. s0+o+3, four per lane
      const int quads = (pos + 3) >> 2;
      for (int r = warp; r < rows; r += kPipeProducers) {
        for (int qd = lane; qd < quads; qd += 32) {
          const int o = 4 * qd;
          const uint32_t* row = raw + r * WBW + ((s0 + o) >> 2);
          const uint32_t w0 = row[0], w1 = row[1], w2 = row[2];
          const int t0 = (s0 + o) & 3;
          uint32_t* dst = sh + r * SP + o;
#pragma unroll
          for (int d = 0; d < 4; d++) {
            const int t = t0 + d;
            if (o + d < pos)
              dst[d] = t < 4 ? __funnelshift_r(w0, w1, 8 * t) : __funnelshift_r(w1, w2, 8 * (t - 4));
          }
        }
      }
      asm volatile("bar.sync 1, %0;" ::"r"(PT) : "memory");
      mbar_arrive(&full_bar[b]);
    }
    if (ok) {
      // buffer i & 1 is free (item i - 2 finished): it carries the end mark
      const int b = i & 1;
      if (pt == 0) gid_s[b] = -1;
      asm volatile("bar.sync 1, %0;" ::"r"(PT) : "memory");
      mbar_arrive(&full_bar[b]);
      if (i >= 1) finish(i - 1);
    }
    return;
  }

  // ---------------- consumers
  // warp-tasks dealt round robin over the consumer warps, continuing across
  // work items (roff: where the previous item's dealing stopped)
  const int cw_id = warp - kPipeProducers;
  constexpr int KC = kPipeConsumers;
  int roff = 0;
  uint32_t c[M][NW];
  for (int i = 0;; i++) {
    const int b = i & 1;
    int okw = 1;
    if (lane == 0) okw = mbar_wait(&full_bar[b], (unsigned)((i >> 1) & 1), &err_s, A.lim) ? 1 : 0;
    okw = __shfl_sync(FULL, okw, 0);
    if (!okw) {
      if (lane == 0) atomicExch(errw, (int)ME_ERR_TIMEOUT);
      break;
    }
    __syncwarp();
    mbar_wait(&full_bar[b], (unsigned)((i >> 1) & 1), &err_s, A.lim);
    if (gid_s[b] < 0) break;
    const int sl = slot_s[b], R0 = r0_s[b], nrow = nrow_s[b];
    const TabGroup& G = grp[sl];
    const int p = G.p, n = 2 * p + 1, nc = n, nseg = (nrow + T - 1) / T;
    const int tasks = nc * nseg, F = G.nb * tasks, Rr = (F + 31) >> 5;
    const int qs = (cw_id - roff + KC) % KC;
    roff = (roff + Rr) % KC;
    // one step = 32 * KC tasks = dblk whole blocks + dseg runs + dcol columns
    const int dblk = (32 * KC) / tasks, drem = 32 * KC - dblk * tasks;
    const int dseg = drem / nc, dcol = drem - (drem / nc) * nc;
    const uint32_t lam = G.lam;
    const int fast = key_mode(N, M, p, lam);
    const int rb = rank_bits(p);
    const uint32_t* cwb = buf0 + b * BST;
    const uint32_t* tabJ = cwb + B * M * NW;
    const uint32_t* tabK = tabJ + RT;
    const uint32_t* tabQ = tabK + RT;
    const uint32_t* sh = tabQ + RT;
    int f = 32 * qs + lane;
    int blk = f / tasks;
    const int t0 = f - blk * tasks;
    int seg = t0 / nc, col = t0 - (t0 / nc) * nc;
    for (int q = qs; q < Rr; q += KC, f += 32 * KC) {
      if (f < F) {
#pragma unroll
        for (int j = 0; j < M; j++)
#pragma unroll
          for (int w = 0; w < NW; w++) c[j][w] = cwb[(blk * M + j) * NW + w];
        const int row0 = seg * T;
        uint32_t acc[T];
        fs_run_sads<N, M, T>(c, sh + row0 * SP + blk * N + col, SP, acc);
        atomicMin(&red[sl][blk],
                  fs_run_key<T>(acc, R0 + row0, col, p, n, lam, rb, fast, tabJ, tabK, tabQ));
      }
      col += dcol;
      if (col >= nc) { col -= nc; seg++; }
      seg += dseg;
      if (seg >= nseg) { seg -= nseg; blk++; }
      blk += dblk;
    }
    mbar_arrive(&empty_bar[b]);
  }
}

// ------------------------------------------------------------------ ACBM


// Speculative full searches of the ACBM sequence: the queue word of such a
// search carries kSeqSpecBit beside the block; the block's state word (bdone,
// cleared by the prologue) collects kSeqSearched (the search's key is in
// bkey) and kSeqFailed (PBM failed): whichever comes second publishes.
constexpr int kSeqSpecBit = 1 << 30;
constexpr int kSeqSearched = 1, kSeqFailed = 2;

// Publishes block o (pair k, block b of the pair) with the full-search key:
// the flag word first (it carries the vector), then the outputs.
__device__ __forceinline__ void seq_publish_fs(const SeqArgs& a, unsigned long long* flags, int epoch,
                                               int o, int k, int b, int nbf, int p, int n,
                                               unsigned long long key) {
  const Decoded d = decode_key(key, p, a.lam);
  atomicExch(flags + o, pub_word(epoch, d.mvx, d.mvy));
  int16_t* field = a.mv + (size_t)k * nbf * 2;
  field[2 * b] = (int16_t)d.mvx;
  field[2 * b + 1] = (int16_t)d.mvy;
  a.J[o] = d.J;
  a.mask[o] = 1;
  if (a.sad) a.sad[o] = d.sad;
  if (a.load) a.load[o] = (uint32_t)(n * n);
}

__global__ void k_seq_begin(SeqCtrl* c) {
  for (int i = threadIdx.x; i < kRoleSlots; i += blockDim.x) c->sm_arr[i] = 0;
  if (threadIdx.x != 0) return;
  c->epoch += 1;
  c->next = 0;
  c->error = 0;
  c->err_item = -1;
  c->fs_head = 0;
  c->fs_tail = 0;
  c->pbm_done = 0;
  c->started = 0;
}

// Padded references and scaled Intra_SAD of all K pairs.
template <int N, int M>
__global__ void __launch_bounds__(256) k_seq_prologue(SeqFrames fr, int K, PadGeom pg, int W, int H,
                                                      uint8_t* __restrict__ refpad,
                                                      uint32_t* __restrict__ intra,
                                                      unsigned long long* __restrict__ bkey,
                                                      int* __restrict__ bdone) {
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthr = (long long)gridDim.x * blockDim.x;
  const int chunks = pg.pitch / 16;
  const long long per = (long long)pg.rows * chunks;
  for (long long i = gtid; i < per * K; i += nthr) {
    const int k = (int)(i / per);
    const long long j = i - (long long)k * per;
    const int y = (int)(j / chunks), cx = (int)(j % chunks) * 16;
    const uint8_t* src = fr.f[k] + (size_t)clampi(y - pg.P, 0, H - 1) * W;
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      uint32_t v = 0;
#pragma unroll
      for (int b = 0; b < 4; b++) v |= (uint32_t)src[clampi(cx + 4 * q + b - pg.P, 0, W - 1)] << (8 * b);
      w[q] = v;
    }
    *reinterpret_cast<uint4*>(refpad + (size_t)k * pg.pitch * pg.rows + (size_t)y * pg.pitch + cx) =
        make_uint4(w[0], w[1], w[2], w[3]);
  }
  const int BW = W / N, nbf = BW * (H / M);
  const long long warps = nthr / 32;
  for (long long g = gtid / 32; g < (long long)nbf * K; g += warps) {
    const int k = (int)(g / nbf), b = (int)(g - (long long)k * nbf);
    const uint32_t v = warp_intra_sad<N, M>(fr.f[k + 1], W, (b % BW) * N, (b / BW) * M);
    if ((threadIdx.x & 31) == 0) {
      intra[g] = v;
      bkey[g] = kNoKey;   // merge state of a sliced full search
      bdone[g] = 0;
    }
  }
}

// Shared memory (words) of one search group of k_acbm_seq: the block's raw
// window in the PBM layout and its current pixels, the shifted words and the
// per-row cost tables.
template <int N, int M, int T>
__host__ __device__ inline size_t seq_group_words(int p, int ng) {
  const FsGeom g = fs_geom<N, M, T>(p, 1, ng);
  // a multiple of 4 words: each group's window starts 16-byte aligned (its
  // rows arrive by 16-byte asynchronous copies)
  const size_t w = (size_t)pbm_win_words(N, M, p) + M * (N / 4) + (size_t)g.rows * g.pos + 3 * (size_t)g.rows;
  return (w + 3) & ~(size_t)3;
}

// One search group of k_acbm_seq: ng threads (index gt) of the search CTA
// that take queued blocks one at a time and search each in full, with named
// barrier `bar` among themselves (a CTA can hold two groups, so that one
// group stages its window while the other searches).  A group takes the
// next queue slot, waits (bounded) for its entry or for the end of the run,
// stages the block's window from the pair's padded reference by 16-byte
// asynchronous copies, builds the shifted words, runs its share of the
// (2p+1) x ceil((2p+1)/T) runs, and publishes the block (a speculative
// search only if its block has failed PBM, see kSeqSpecBit).  LR: the
// current block is read from shared memory row by row (fs_run_sads_lr), for
// the three-CTAs-per-SM build.
template <int N, int M, int T, bool LR = false>
__device__ void seq_search_group(const SeqFrames& fr, const SeqArgs& a, int W, int H, int p,
                                 const PadGeom& pg, const uint8_t* __restrict__ refpad,
                                 unsigned long long* __restrict__ flags, int total, SeqCtrl* ctrl,
                                 unsigned long long* __restrict__ q,
                                 unsigned long long* __restrict__ bkey, int* __restrict__ bdone,
                                 int epoch, long long timeout, uint32_t* gs, int gt, int ng, int bar,
                                 volatile int* s_item, unsigned long long* s_red) {
  constexpr int NW = N / 4;
  const int lane = threadIdx.x & 31;
  const int BW = W / N, nbf = BW * (H / M);
  const size_t padsz = (size_t)pg.pitch * pg.rows;
  const int n = 2 * p + 1;
  const int wwin = pbm_win_words(N, M, p);
  const FsGeom g = fs_geom<N, M, T>(p, 1, ng);
  uint32_t* raw = gs;                        // window [rows][wp] + current block
  uint32_t* sh = gs + wwin + M * NW;         // [g.rows][g.pos]
  uint32_t* tabJ = sh + g.rows * g.pos;
  uint32_t* tabK = tabJ + g.rows;
  uint32_t* tabQ = tabK + g.rows;
  const int fast = key_mode(N, M, p, a.lam);
  const int rb = rank_bits(p);
  for (int r = gt; r < g.rows; r += ng) {
    const int mvy = r - p;
    const int am = mvy < 0 ? -mvy : mvy;
    tabJ[r] = a.lam * (uint32_t)mv_bits(mvy);
    tabK[r] = ((uint32_t)am << 17) + (uint32_t)r * (uint32_t)n;
    tabQ[r] = tabq_value(fast, tabJ[r], mvy, p);
  }
  if (gt == 0) *s_red = kNoKey;
  for (;;) {
    if (gt == 0) {
      const int slot = atomicAdd(&ctrl->fs_head, 1);
      // the queue holds at most `total` entries: a slot beyond can never be
      // filled, so the group is done without touching it
      const volatile unsigned long long* rd = q + (slot < total ? slot : 0);
      const volatile int* done = &ctrl->pbm_done;
      const volatile int* tail = &ctrl->fs_tail;
      const volatile int* err = &ctrl->error;
      const long long t0 = clock64();
      int got = -1;
      unsigned nsl = 32;
      for (int it = 0;; it++) {
        if (slot >= total) break;
        const unsigned long long e = *rd;
        if (pub_epoch(e) == epoch) { got = (int)(uint32_t)e; break; }
        if ((it & 7) == 7) {
          if (*done == total && *tail <= slot) break;   // no more blocks will come
          if (*err != 0) break;
          if (clock64() - t0 > timeout) {
            atomicExch(&ctrl->error, (int)ME_ERR_TIMEOUT);
            break;
          }
        }
        __nanosleep(nsl);
        if (nsl < 64) nsl *= 2;   // a queued search starts on the chain's clock
      }
      *s_item = got;
    }
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(ng) : "memory");
    const int item = *s_item;
    if (item == -1) break;
    const bool specj = (item & kSeqSpecBit) != 0;
    const int o = item & ~kSeqSpecBit;
    if (o >= total) {
      // not a block of this run: report it instead of touching memory
      if (gt == 0) atomicExch(&ctrl->error, (int)ME_ERR_CUDA);
      asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(ng) : "memory");
      continue;
    }
    const int k = o / nbf, b = o - k * nbf;
    const int x0 = (b % BW) * N, y0 = (b / BW) * M;
    const PbmWin wg = pbm_win(N, M, p, x0, pg.P);
    {
      const uint8_t* cur = fr.f[k + 1];
      for (int i = gt; i < M * NW; i += ng) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(raw + wwin + i);
        const void* src = cur + (size_t)(y0 + i / NW) * W + x0 + 4 * (i % NW);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
      }
      const uint8_t* base = refpad + (size_t)k * padsz + (size_t)(y0 + pg.P - p) * pg.pitch +
                            ((x0 + pg.P - p) & ~15);
      for (int i = gt; i < wg.rows * wg.chunks; i += ng) {
        const int r = i / wg.chunks, c = i - r * wg.chunks;
        const unsigned dst = (unsigned)__cvta_generic_to_shared(raw + r * wg.wp + 4 * c);
        const void* src = base + (size_t)r * pg.pitch + 16 * c;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      asm volatile("cp.async.wait_all;" ::: "memory");
    }
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(ng) : "memory");
    // shifted words: sh[r][o] = window bytes s0+o .. s0+o+3 of row r (rows
    // past the window's last row only feed candidates beyond 2p: any row),
    // a row per warp of the group, four consecutive words per lane
    {
      const int gw = gt >> 5, ngw = ng >> 5, quads = (g.pos + 3) >> 2;
      for (int r = gw; r < g.rows; r += ngw) {
        const uint32_t* row = raw + (r < wg.rows ? r : wg.rows - 1) * wg.wp;
        for (int qd = lane; qd < quads; qd += 32) {
          const int oo = 4 * qd;
          const uint32_t* rw = row + ((wg.s0 + oo) >> 2);
          const uint32_t w0 = rw[0], w1 = rw[1], w2 = rw[2];
          const int t0 = (wg.s0 + oo) & 3;
          uint32_t* dst = sh + r * g.pos + oo;
#pragma unroll
          for (int d = 0; d < 4; d++) {
            const int t = t0 + d;
            if (oo + d < g.pos)
              dst[d] = t < 4 ? __funnelshift_r(w0, w1, 8 * t) : __funnelshift_r(w1, w2, 8 * (t - 4));
          }
        }
      }
    }
    uint32_t c[LR ? 1 : M][LR ? 1 : NW];
    if constexpr (!LR) {
#pragma unroll
      for (int j = 0; j < M; j++)
#pragma unroll
        for (int w = 0; w < NW; w++) c[j][w] = raw[wwin + j * NW + w];
    }
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(ng) : "memory");
    unsigned long long best = kNoKey;
    {
      const int nc = g.nc;
      int seg = gt / nc, col = gt - (gt / nc) * nc;
      const int dseg = ng / nc, dcol = ng - (ng / nc) * nc;
      for (int t = gt; t < g.tasks; t += ng) {
        const int row0 = seg * T;
        uint32_t acc[T];
        if constexpr (LR)
          fs_run_sads_lr<N, M, T>(raw + wwin, sh + row0 * g.pos + col, g.pos, acc);
        else
          fs_run_sads<N, M, T>(c, sh + row0 * g.pos + col, g.pos, acc);
        best = umin64(best, fs_run_key<T>(acc, row0, col, p, n, a.lam, rb, fast, tabJ, tabK, tabQ));
        seg += dseg;
        col += dcol;
        if (col >= nc) { col -= nc; seg++; }
      }
    }
    best = warp_min64(best);
    if (lane == 0 && best != kNoKey) atomicMin(s_red, best);
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(ng) : "memory");
    if (gt == 0) {
      const unsigned long long key = *s_red;
      *s_red = kNoKey;
      bool pub = true;
      if (specj) {
        bkey[o] = key;
        __threadfence();
        pub = (atomicOr(bdone + o, kSeqSearched) & kSeqFailed) != 0;
      }
      if (pub) seq_publish_fs(a, flags, epoch, o, k, b, nbf, p, n, key);
    }
  }
}

// Two roles in one launch (cta_role: one CTA of each per SM).  PBM CTAs: each
// warp claims blocks on its own in the (wave + 4*pair) order (the item table
// maps a claim to its block), queues the block's current pixels and search
// window as asynchronous copies, waits for the block's predecessors (whose
// flag words carry their final vectors), runs PBM and the two conditions, and
// either publishes the block or appends it to the full-search queue; then it
// claims the next block.  Search CTAs take queued blocks in order and search
// each with the whole CTA.  A PBM warp only waits for blocks claimed before
// its own, and a search CTA only for a queue entry that a running PBM warp
// will write (or for the end of the run), so every wait ends; each wait is
// also bounded in time.  MINB = 3: three CTAs per SM (cps = 3, pbm_per_sm of
// them PBM), registers held to a third of the SM's, search groups only, with
// the low-register SAD runs.
template <int N, int M, int T, int MINB = 2>
__global__ void __launch_bounds__(kSeqThreads, MINB) k_acbm_seq(SeqFrames fr, SeqArgs a, int W, int H,
                                                             int p, PadGeom pg,
                                                             const uint8_t* __restrict__ refpad,
                                                             const uint32_t* __restrict__ intra,
                                                             unsigned long long* __restrict__ flags,
                                                             const int* __restrict__ items,
                                                             int total, SeqCtrl* ctrl,
                                                             unsigned long long* __restrict__ q,
                                                             unsigned long long* __restrict__ bkey,
                                                             int* __restrict__ bdone, int S,
                                                             int pbm_warps, int search_every,
                                                             int spec, int sgroups, int cps,
                                                             int pbm_per_sm, int early) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ unsigned long long keys[16];
  __shared__ int s_item, s_role, s_slice;
  const unsigned FULL = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int BW = W / N, BH = H / M, nbf = BW * BH;
  const int epoch = *reinterpret_cast<volatile int*>(&ctrl->epoch);
  const long long timeout = ctrl->timeout_cycles;
  const size_t padsz = (size_t)pg.pitch * pg.rows;
  const int n = 2 * p + 1;
  if (tid == 0) s_role = cta_role(&ctrl->started, ctrl->sm_arr, search_every, cps, pbm_per_sm);
  __syncthreads();

  if (s_role == 0) {
    // ---------------------------------------------------------------- PBM warps
    if (warp >= pbm_warps) return;   // shared memory holds pbm_warps windows
    const int wwords = pbm_win_words(N, M, p) + M * (N / 4);
    uint32_t* win = smem + warp * wwords;
    uint32_t* curs = win + pbm_win_words(N, M, p);
    // lane 0 holds the next claim (item index and its block)
    int nxt = 0, onxt = 0;
    if (lane == 0) {
      nxt = atomicAdd(&ctrl->next, 1);
      if (nxt < total) onxt = items[nxt];
    }
    for (;;) {
      const int i = __shfl_sync(FULL, nxt, 0);
      if (i >= total) break;
      const int o = __shfl_sync(FULL, onxt, 0);
      const int k = o / nbf, b = o - k * nbf;
      const int bx = b % BW, by = b / BW;
      const PbmWin wg = pbm_stage<N, M>(fr.f[k + 1], refpad + (size_t)k * padsz, pg, W, p, bx * N,
                                        by * M, curs, win);
      const uint32_t ix = intra[o];
      // predictors: lanes 0-3 the spatial ones in pair k, lanes 4-12 the 3x3
      // of pair k-1 (or of the caller's field before pair 0), lane 13 zero
      int cx = 0, cy = 0, nidx = -1;
      bool valid = false;
      if (lane < 4) {
        const int dx = (lane < 2) ? -1 : (lane == 2 ? 0 : 1);
        const int dy = (lane == 0) ? 0 : -1;
        const int nx = bx + dx, ny = by + dy;
        if (nx >= 0 && nx < BW && ny >= 0) {
          nidx = k * nbf + ny * BW + nx;
          valid = true;
        }
      } else if (lane < 13) {
        const int t = lane - 4, nx = bx + t % 3 - 1, ny = by + t / 3 - 1;
        if (nx >= 0 && nx < BW && ny >= 0 && ny < BH) {
          valid = true;
          if (k > 0) {
            nidx = (k - 1) * nbf + ny * BW + nx;
          } else if (a.prev0) {
            cx = a.prev0[2 * (ny * BW + nx)];
            cy = a.prev0[2 * (ny * BW + nx) + 1];
          }
        }
      } else if (lane == 13) {
        valid = true;
      }
      // the temporal predecessors first (pair k-1: usually finished already)
      {
        const bool tl = lane >= 4 && nidx >= 0;
        const unsigned long long w = warp_wait_flags(tl ? flags + nidx : nullptr, epoch,
                                                     &ctrl->error, &ctrl->err_item, timeout, i);
        if (tl) {
          cx = pub_mvx(w);
          cy = pub_mvy(w);
        }
      }
      const PbmPart pa = pbm_part_a<N, M>(cx, cy, valid, wg, p, a.lam, curs, win);
      // A block whose temporal and zero predictors already fail both
      // conditions nearly always fails with its spatial ones too: its full
      // search is queued now (speculatively), while the warp waits for the
      // spatial neighbours.  The block's final result does not depend on
      // the guess: a search whose block passes PBM is discarded.
      const bool sp = spec && pbm_would_fail<N, M>(pa.best, p, a.lam, ix, a.alpha, a.beta, a.gnum,
                                                   a.gden, a.qp);
      if (sp && lane == 0) {
        const int slot = atomicAdd(&ctrl->fs_tail, 1);
        atomicExch(q + slot, ((unsigned long long)(uint32_t)epoch << 32) | (uint32_t)o | kSeqSpecBit);
      }
      // the ring around part a's best, evaluated now if a spatial neighbour
      // is still running (part b uses it when no spatial predictor beats
      // part a's best; the result never depends on it)
      PbmRing ring0 = pbm_no_ring();
      if (a.refine && early) {
        bool ready = true;
        if (lane < 4 && nidx >= 0)
          ready = pub_epoch(*reinterpret_cast<const volatile unsigned long long*>(flags + nidx)) == epoch;
        if (!__all_sync(FULL, ready))
          ring0 = pbm_ring_early<N, M>(cx, cy, valid, pa, wg, p, a.lam, curs, win);
      }
      {
        const bool sl = lane < 4 && nidx >= 0;
        const unsigned long long w = warp_wait_flags(sl ? flags + nidx : nullptr, epoch,
                                                     &ctrl->error, &ctrl->err_item, timeout, i);
        if (sl) {
          cx = pub_mvx(w);
          cy = pub_mvy(w);
        }
      }
      const PbmResult r = pbm_part_b<N, M>(cx, cy, valid, pa, wg, p, a.lam, ix, a.alpha, a.beta,
                                           a.gnum, a.gden, a.qp, a.refine, curs, win, nullptr,
                                           ring0);
      if (lane == 0) {
        if (r.pass) {
          // the flag word carries the vector: publish first, outputs after
          const Decoded d = decode_key(r.key, p, a.lam);
          atomicExch(flags + o, pub_word(epoch, d.mvx, d.mvy));
          int16_t* field = a.mv + (size_t)k * nbf * 2;
          field[2 * b] = (int16_t)d.mvx;
          field[2 * b + 1] = (int16_t)d.mvy;
          a.J[o] = d.J;
          a.mask[o] = 0;
          if (a.sad) a.sad[o] = d.sad;
          if (a.load) a.load[o] = (uint32_t)r.load;
        } else if (sp) {
          // the speculative search publishes if it finishes after this
          // decision; if it finished before, its key is here to publish
          const int old = atomicOr(bdone + o, kSeqFailed);
          if (old & kSeqSearched) {
            __threadfence();
            seq_publish_fs(a, flags, epoch, o, k, b, nbf, p, n,
                           *reinterpret_cast<volatile unsigned long long*>(bkey + o));
          }
        } else {
          // S queue entries (one per column slice; slot % S is the slice),
          // each = epoch and block in one word; the tail count is ordered
          // before this warp's pbm_done increment
          const int slot = atomicAdd(&ctrl->fs_tail, S);
          for (int sl = 0; sl < S; sl++)
            atomicExch(q + slot + sl, ((unsigned long long)(uint32_t)epoch << 32) | (uint32_t)o);
        }
        __threadfence();
        atomicAdd(&ctrl->pbm_done, 1);
        // the next claim, once this block is out of the warp's hands (a claim
        // taken earlier would sit behind this block's wait)
        nxt = atomicAdd(&ctrl->next, 1);
        onxt = nxt < total ? items[nxt] : 0;
      }
      __syncwarp();
    }
  } else if (sgroups > 0 || MINB >= 3) {
    // ---------------------------------------------------------------- search groups
    __shared__ int s_gitem[2];
    __shared__ unsigned long long s_gred[2];
    const int ng = kSeqThreads / (sgroups > 0 ? sgroups : 1), gid = tid / ng;
    seq_search_group<N, M, T, (MINB >= 3)>(fr, a, W, H, p, pg, refpad, flags, total, ctrl, q, bkey,
                                           bdone, epoch, timeout,
                                           smem + gid * seq_group_words<N, M, T>(p, ng),
                                           tid - gid * ng, ng, 1 + gid, &s_gitem[gid], &s_gred[gid]);
  } else {
    // ---------------------------------------------------------------- search CTAs
    for (;;) {
      if (tid == 0) {
        const int slot = atomicAdd(&ctrl->fs_head, 1);
        // the queue holds at most total * S entries: a slot beyond can never
        // be filled, so the CTA is done without touching it
        const int qcap = total * S;
        s_slice = slot % S;
        const volatile unsigned long long* rd = q + (slot < qcap ? slot : 0);
        const volatile int* done = &ctrl->pbm_done;
        const volatile int* tail = &ctrl->fs_tail;
        const volatile int* err = &ctrl->error;
        const long long t0 = clock64(), lim = timeout;
        int got = -1;
        unsigned ns = 32;
        for (int it = 0;; it++) {
          if (slot >= qcap) break;
          const unsigned long long e = *rd;
          if (pub_epoch(e) == epoch) { got = (int)(uint32_t)e; break; }   // block | speculative bit
          // the end-of-run and error words are shared by every poller: read
          // them on every 8th round only
          if ((it & 7) == 7) {
            if (*done == total && *tail <= slot) break;   // no more blocks will come
            if (*err != 0) break;
            if (clock64() - t0 > lim) {
              atomicExch(&ctrl->error, (int)ME_ERR_TIMEOUT);
              break;
            }
          }
          __nanosleep(ns);
          if (ns < 64) ns *= 2;   // a queued search starts on the chain's clock
        }
        s_item = got;
      }
      __syncthreads();
      if (s_item == -1) break;
      const bool specj = (s_item & kSeqSpecBit) != 0;
      const int o = s_item & ~kSeqSpecBit;
      if (o >= total) {
        // not a block of this run: report it instead of touching memory
        if (tid == 0) atomicExch(&ctrl->error, (int)ME_ERR_CUDA);
        __syncthreads();
        continue;
      }
      const int k = o / nbf, b = o - k * nbf;
      // this CTA's slice of the mvx columns
      const int nc0 = (n + S - 1) / S, c0 = s_slice * nc0;
      const FsGeom g = fs_geom<N, M, T>(p, 1, blockDim.x, c0, min(nc0, n - c0));
      fs_group<N, M, T>(fr.f[k + 1], fr.f[k], W, H, (b % BW) * N, (b / BW) * M, g, a.lam, smem, keys,
                        nullptr, FsPad{refpad + (size_t)k * padsz, pg.pitch, pg.P, pg.rows});
      bool last = true;
      unsigned long long key = keys[0];
      if (S > 1 && tid == 0) {
        // slices meet in a 64-bit minimum (the key order is total, so the
        // order of arrival does not matter); the last slice publishes
        atomicMin(bkey + o, key);
        __threadfence();
        last = atomicAdd(bdone + o, 1) == S - 1;
        if (last) key = atomicMin(bkey + o, kNoKey);
      }
      if (tid == 0 && specj) {
        // a speculative search publishes only if its block has failed PBM;
        // else the PBM warp publishes this key when it decides (or the
        // block passed and the key is not used)
        bkey[o] = key;
        __threadfence();
        last = (atomicOr(bdone + o, kSeqSearched) & kSeqFailed) != 0;
      }
      if (tid == 0 && last) seq_publish_fs(a, flags, epoch, o, k, b, nbf, p, n, key);
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------ ACBM, one CTA per SM
//
// The same ACBM over K pairs with both roles in one CTA per SM (512 threads):
// warps 0..pw-1 run PBM exactly as the PBM CTAs of k_acbm_seq; the other
// warps form the SM's search group.  A PBM warp whose block fails both
// conditions has the block's whole search window and current pixels in its
// shared memory already (staged for PBM), so it copies them into a free
// hand-off slot of its own CTA and goes on to its next block; the search
// group builds its shifted words from that slot (no second trip to global
// memory) and searches the block with all its threads.  When both slots are
// taken the block goes to the global queue instead, which every search group
// drains when its own slots are empty (staging that window from the padded
// reference itself).  The search group synchronises with a named barrier, so
// the PBM warps never wait for it.
//
// Progress: a PBM warp only waits for blocks claimed before its own; such a
// block is either published, in some CTA's slot (that CTA's search group
// runs and takes its slots first), or in the global queue (whose entries a
// running PBM warp writes right after reserving them).  A search group exits
// once every block has been through PBM, the global queue is drained and its
// own slots are empty.  Every wait is also bounded in time.
constexpr int kSeq2Threads = 512;
constexpr int kSeq2Slots = 2;   // hand-off slots per CTA; slot kSeq2Slots: global jobs

__device__ __forceinline__ void seq2_bar(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

template <int N, int M, int T>
__global__ void __launch_bounds__(kSeq2Threads, 1) k_acbm_seq2(
    SeqFrames fr, SeqArgs a, int W, int H, int p, PadGeom pg, const uint8_t* __restrict__ refpad,
    const uint32_t* __restrict__ intra, unsigned long long* __restrict__ flags,
    const int* __restrict__ items, int total, SeqCtrl* ctrl, unsigned long long* __restrict__ q,
    int pbm_warps) {
  constexpr int NW = N / 4;
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ int s_state[kSeq2Slots];    // 0 free, 1 being filled, 2 full
  __shared__ int s_seq[kSeq2Slots];      // claim index (age) of the block in each full slot
  __shared__ int s_blk[kSeq2Slots + 1];  // block of each slot
  __shared__ int s_job;
  __shared__ unsigned long long s_red;
  const unsigned FULL = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int BW = W / N, BH = H / M, nbf = BW * BH;
  const int epoch = *reinterpret_cast<volatile int*>(&ctrl->epoch);
  const long long timeout = ctrl->timeout_cycles;
  const size_t padsz = (size_t)pg.pitch * pg.rows;
  const int n = 2 * p + 1;
  const int wwin = pbm_win_words(N, M, p);   // window words of a PBM warp / slot
  const int wwords = wwin + M * NW;          // + the current block
  uint32_t* slots = smem + pbm_warps * wwords;               // [kSeq2Slots + 1][wwords]
  const FsGeom g = fs_geom<N, M, T>(p, 1, blockDim.x - 32 * pbm_warps);
  uint32_t* sh = slots + (kSeq2Slots + 1) * wwords;          // [g.rows][g.sp]
  uint32_t* tabJ = sh + g.rows * g.sp;
  uint32_t* tabK = tabJ + g.rows;
  uint32_t* tabQ = tabK + g.rows;
  if (tid < kSeq2Slots) s_state[tid] = 0;
  if (tid == 0) s_red = kNoKey;
  __syncthreads();

  if (warp < pbm_warps) {
    // ---------------------------------------------------------------- PBM warps
    uint32_t* win = smem + warp * wwords;
    uint32_t* curs = win + wwin;
    int nxt = 0, onxt = 0;
    if (lane == 0) {
      nxt = atomicAdd(&ctrl->next, 1);
      if (nxt < total) onxt = items[nxt];
    }
    for (;;) {
      const int i = __shfl_sync(FULL, nxt, 0);
      if (i >= total) break;
      const int o = __shfl_sync(FULL, onxt, 0);
      const int k = o / nbf, b = o - k * nbf;
      const int bx = b % BW, by = b / BW;
      const PbmWin wg = pbm_stage<N, M>(fr.f[k + 1], refpad + (size_t)k * padsz, pg, W, p, bx * N,
                                        by * M, curs, win);
      const uint32_t ix = intra[o];
      int cx = 0, cy = 0, nidx = -1;
      bool valid = false;
      if (lane < 4) {
        const int dx = (lane < 2) ? -1 : (lane == 2 ? 0 : 1);
        const int dy = (lane == 0) ? 0 : -1;
        const int nx = bx + dx, ny = by + dy;
        if (nx >= 0 && nx < BW && ny >= 0) {
          nidx = k * nbf + ny * BW + nx;
          valid = true;
        }
      } else if (lane < 13) {
        const int t = lane - 4, nx = bx + t % 3 - 1, ny = by + t / 3 - 1;
        if (nx >= 0 && nx < BW && ny >= 0 && ny < BH) {
          valid = true;
          if (k > 0) {
            nidx = (k - 1) * nbf + ny * BW + nx;
          } else if (a.prev0) {
            cx = a.prev0[2 * (ny * BW + nx)];
            cy = a.prev0[2 * (ny * BW + nx) + 1];
          }
        }
      } else if (lane == 13) {
        valid = true;
      }
      {
        const unsigned long long w = warp_wait_flags(nidx >= 0 ? flags + nidx : nullptr, epoch,
                                                     &ctrl->error, &ctrl->err_item, timeout, i);
        if (nidx >= 0) {
          cx = pub_mvx(w);
          cy = pub_mvy(w);
        }
      }
      const PbmResult r = pbm_eval<N, M>(cx, cy, valid, wg, p, a.lam, ix, a.alpha, a.beta, a.gnum,
                                         a.gden, a.qp, a.refine, curs, win);
      if (r.pass) {
        if (lane == 0) {
          const Decoded d = decode_key(r.key, p, a.lam);
          atomicExch(flags + o, pub_word(epoch, d.mvx, d.mvy));
          int16_t* field = a.mv + (size_t)k * nbf * 2;
          field[2 * b] = (int16_t)d.mvx;
          field[2 * b + 1] = (int16_t)d.mvy;
          a.J[o] = d.J;
          a.mask[o] = 0;
          if (a.sad) a.sad[o] = d.sad;
          if (a.load) a.load[o] = (uint32_t)r.load;
        }
      } else {
        // hand the staged window to this SM's search group, or queue it
        int got = -1;
        if (lane == 0) {
          for (int s = 0; s < kSeq2Slots && got < 0; s++)
            if (atomicCAS(&s_state[s], 0, 1) == 0) got = s;
        }
        got = __shfl_sync(FULL, got, 0);
        if (got >= 0) {
          uint32_t* dst = slots + got * wwords;
          const int nw = wg.rows * wg.wp;
          for (int j = lane; j < nw; j += 32) dst[j] = win[j];
          for (int j = lane; j < M * NW; j += 32) dst[wwin + j] = curs[j];
          __syncwarp();
          if (lane == 0) {
            s_blk[got] = o;
            s_seq[got] = i;
            __threadfence_block();
            atomicExch(&s_state[got], 2);
          }
        } else if (lane == 0) {
          const int slot = atomicAdd(&ctrl->fs_tail, 1);
          atomicExch(q + slot, ((unsigned long long)(uint32_t)epoch << 32) | (uint32_t)i);
        }
      }
      if (lane == 0) {
        // the hand-off (slot state or queue entry) is ordered before the count
        __threadfence();
        atomicAdd(&ctrl->pbm_done, 1);
        nxt = atomicAdd(&ctrl->next, 1);
        onxt = nxt < total ? items[nxt] : 0;
      }
      __syncwarp();
    }
    return;
  }

  // ---------------------------------------------------------------- search group
  const int ns = blockDim.x - 32 * pbm_warps;   // search threads
  const int st = tid - 32 * pbm_warps;          // index within the group
  const int fast = key_mode(N, M, p, a.lam);
  const int rb = rank_bits(p);
  for (int r = st; r < g.rows; r += ns) {
    const int mvy = r - p;
    const int am = mvy < 0 ? -mvy : mvy;
    tabJ[r] = a.lam * (uint32_t)mv_bits(mvy);
    tabK[r] = ((uint32_t)am << 17) + (uint32_t)r * (uint32_t)n;
    tabQ[r] = tabq_value(fast, tabJ[r], mvy, p);
  }
  const volatile int* vstate = s_state;
  for (;;) {
    if (st == 0) {
      // next job: the oldest block (smallest claim index) in this CTA's full
      // slots, else the head of the global queue, else wait (bounded) for
      // either or for the end of the run.  (Serving an older global entry
      // before a full local slot measured twice as slow: the slots stay
      // taken, more blocks go to the queue and each costs a staging trip.)
      int job = -1;
      const long long t0 = clock64();
      unsigned nsl = 32;
      for (int it = 0;; it++) {
        int best = -1, bseq = 0;
        bool busy = false;
        for (int s = 0; s < kSeq2Slots; s++) {
          const int v = vstate[s];
          busy |= v != 0;
          if (v == 2) {
            __threadfence_block();
            const int sq = *reinterpret_cast<volatile int*>(&s_seq[s]);
            if (best < 0 || sq < bseq) { best = s; bseq = sq; }
          }
        }
        const int h = *reinterpret_cast<volatile int*>(&ctrl->fs_head);
        const int tl = *reinterpret_cast<volatile int*>(&ctrl->fs_tail);
        // this CTA's slots first (no staging); the global queue when they are empty
        const bool take_global = best < 0 && h < tl && h < total;
        if (!take_global && best >= 0) { job = best; break; }
        if (take_global) {
          if (atomicCAS(&ctrl->fs_head, h, h + 1) == h) {
            // reserved entry h: its writer has already counted it in fs_tail
            const volatile unsigned long long* rd = q + h;
            int ci = -1;
            for (;;) {
              const unsigned long long e = *rd;
              if (pub_epoch(e) == epoch) { ci = (int)(uint32_t)e; break; }
              if (*reinterpret_cast<volatile int*>(&ctrl->error) != 0) break;
              if (clock64() - t0 > timeout) {
                atomicExch(&ctrl->error, (int)ME_ERR_TIMEOUT);
                break;
              }
              __nanosleep(32);
            }
            if (ci >= 0 && ci < total) {
              s_blk[kSeq2Slots] = items[ci];
              job = kSeq2Slots;
            } else if (ci >= total) {
              atomicExch(&ctrl->error, (int)ME_ERR_CUDA);
            }
            break;
          }
          continue;
        }
        if (!busy && *reinterpret_cast<volatile int*>(&ctrl->pbm_done) == total &&
            *reinterpret_cast<volatile int*>(&ctrl->fs_head) >=
                *reinterpret_cast<volatile int*>(&ctrl->fs_tail))
          break;   // every block through PBM, the queue drained, no slot of ours in use
        if ((it & 7) == 7) {
          if (*reinterpret_cast<volatile int*>(&ctrl->error) != 0) break;
          if (clock64() - t0 > timeout) {
            atomicExch(&ctrl->error, (int)ME_ERR_TIMEOUT);
            break;
          }
        }
        __nanosleep(nsl);
        if (nsl < 256) nsl *= 2;
      }
      s_job = job;
    }
    seq2_bar(ns);
    const int job = s_job;
    if (job < 0) break;
    const int o = s_blk[job];
    const int k = o / nbf, b = o - k * nbf;
    const int x0 = (b % BW) * N, y0 = (b / BW) * M;
    uint32_t* raw = slots + job * wwords;
    const PbmWin wg = pbm_win(N, M, p, x0, pg.P);
    if (job == kSeq2Slots) {
      // a queued block: stage its window and current pixels as pbm_stage does
      const uint8_t* cur = fr.f[k + 1];
      for (int i = st; i < M * NW; i += ns) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(raw + wwin + i);
        const void* src = cur + (size_t)(y0 + i / NW) * W + x0 + 4 * (i % NW);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
      }
      const uint8_t* base = refpad + (size_t)k * padsz + (size_t)(y0 + pg.P - p) * pg.pitch +
                            ((x0 + pg.P - p) & ~15);
      for (int i = st; i < wg.rows * wg.chunks; i += ns) {
        const int r = i / wg.chunks, c = i - r * wg.chunks;
        const unsigned dst = (unsigned)__cvta_generic_to_shared(raw + r * wg.wp + 4 * c);
        const void* src = base + (size_t)r * pg.pitch + 16 * c;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      asm volatile("cp.async.wait_all;" ::: "memory");
      seq2_bar(ns);
    }
    // shifted words: sh[r][o] = window bytes s0+o .. s0+o+3 of row r (rows
    // past the window's last row only feed candidates beyond 2p: any row)
    {
      // a row per warp of the group, four consecutive words per lane
      const int gw = st >> 5, ngw = ns >> 5, quads = (g.pos + 3) >> 2;
      for (int r = gw; r < g.rows; r += ngw) {
        const uint32_t* row = raw + (r < wg.rows ? r : wg.rows - 1) * wg.wp;
        for (int qd = lane; qd < quads; qd += 32) {
          const int oo = 4 * qd;
          const uint32_t* rw = row + ((wg.s0 + oo) >> 2);
          const uint32_t w0 = rw[0], w1 = rw[1], w2 = rw[2];
          const int t0 = (wg.s0 + oo) & 3;
          uint32_t* dst = sh + r * g.sp + oo;
#pragma unroll
          for (int d = 0; d < 4; d++) {
            const int t = t0 + d;
            if (oo + d < g.pos)
              dst[d] = t < 4 ? __funnelshift_r(w0, w1, 8 * t) : __funnelshift_r(w1, w2, 8 * (t - 4));
          }
        }
      }
    }
    uint32_t c[M][NW];
#pragma unroll
    for (int j = 0; j < M; j++)
#pragma unroll
      for (int w = 0; w < NW; w++) c[j][w] = raw[wwin + j * NW + w];
    seq2_bar(ns);
    if (st == 0 && job < kSeq2Slots) atomicExch(&s_state[job], 0);   // slot read in full
    unsigned long long best = kNoKey;
    {
      const int nc = g.nc;
      int seg = st / nc, col = st - (st / nc) * nc;
      const int dseg = ns / nc, dcol = ns - (ns / nc) * nc;
      for (int t = st; t < g.tasks; t += ns) {
        const int row0 = seg * T;
        uint32_t acc[T];
        fs_run_sads<N, M, T>(c, sh + row0 * g.sp + col, g.sp, acc);
        best = umin64(best, fs_run_key<T>(acc, row0, col, p, n, a.lam, rb, fast, tabJ, tabK, tabQ));
        seg += dseg;
        col += dcol;
        if (col >= nc) { col -= nc; seg++; }
      }
    }
    best = warp_min64(best);
    if (lane == 0 && best != kNoKey) atomicMin(&s_red, best);
    seq2_bar(ns);
    if (st == 0) {
      const unsigned long long key = s_red;
      s_red = kNoKey;
      const Decoded d = decode_key(key, p, a.lam);
      atomicExch(flags + o, pub_word(epoch, d.mvx, d.mvy));
      int16_t* field = a.mv + (size_t)k * nbf * 2;
      field[2 * b] = (int16_t)d.mvx;
      field[2 * b + 1] = (int16_t)d.mvy;
      a.J[o] = d.J;
      a.mask[o] = 1;
      if (a.sad) a.sad[o] = d.sad;
      if (a.load) a.load[o] = (uint32_t)(n * n);
    }
  }
}

// ------------------------------------------------------------------ plans

struct SeqPlan {
  int dev, W, H, N, M, p, K;
  void* mem = nullptr;
  uint8_t* refpad = nullptr;
  uint32_t* intra = nullptr;
  unsigned long long* flags = nullptr;   // per block: epoch + final vector
  unsigned long long* q = nullptr;       // full-search queue: epoch + block, S per block
  unsigned long long* bkey = nullptr;    // per block: minimum key over the search slices
  int* bdone = nullptr;                  // per block: search slices finished
  int S = 1;                             // column slices per full search
  int* items = nullptr;                  // per lag: claim order -> block (pair * blocks + block)
  SeqCtrl* ctrl = nullptr;
  int total = 0;
  cudaEvent_t last = nullptr;   // end of the previous run (runs of one plan never overlap)
  bool ran = false;
  std::mutex mu;
  // launch candidates (same scratch, same results): the autotuner times them
  // on the plan's first call and keeps the fastest
  struct Cand {
    int ver;      // 1: k_acbm_seq (two CTA roles); 2: k_acbm_seq2 (one CTA per SM)
    int T;        // run length of the full searches
    int split;    // ver 1: every split-th SM hosts two search CTAs (0: none)
    int pw;       // ver 1: PBM warps per PBM CTA; ver 2: PBM warps per CTA
    int spec;     // ver 1: speculative full searches (single-slice searches only)
    int sgroups;  // ver 1: search groups per search CTA (named barriers); 0: one, fs_group
    int lag;      // claim-order table (index into kSeqLags)
    int lr;       // ver 1: the low-register build (registers for three CTAs per SM)
    int cps;      // ver 1: CTAs per SM the roles are dealt over (2 or 3)
    int ppsm;     // ver 1: PBM CTAs per SM
    int early;    // ver 1: the ring around part a's best evaluated during the spatial wait
    size_t smem;
    int grid;
    std::string name;
  };
  std::vector<Cand> cands;
  int model = 0;                // the cost model's candidate
  int chosen = -1;              // -1: not tuned yet
};

static std::mutex g_seq_mu;
static std::vector<SeqPlan*> g_seq_plans;

// PBM warps per CTA: as many windows as fit in about 100 KB (8 at p = 32).
static int seq_pbm_warps(int N, int M, int p) {
  const size_t per = (size_t)4 * (pbm_win_words(N, M, p) + M * (N / 4));
  return (int)std::max<size_t>(1, std::min<size_t>(kSeqThreads / 32, (100 * 1024) / per));
}

template <int N, int M, int T>
static size_t seq_smem(int p, int sgroups = 0) {
  const size_t pbm = (size_t)4 * seq_pbm_warps(N, M, p) * (pbm_win_words(N, M, p) + M * (N / 4));
  const size_t srch = sgroups > 0
                          ? 4 * (size_t)sgroups * seq_group_words<N, M, T>(p, kSeqThreads / sgroups)
                          : fs_smem_bytes<N, M, T>(fs_geom<N, M, T>(p, 1, kSeqThreads));
  return std::max(srch, pbm);
}

// Shared memory of k_acbm_seq2 with pw PBM warps.
template <int N, int M, int T>
static size_t seq2_smem(int p, int pw) {
  const size_t wwords = (size_t)pbm_win_words(N, M, p) + M * (N / 4);
  const FsGeom g = fs_geom<N, M, T>(p, 1, kSeq2Threads - 32 * pw);
  return 4 * ((pw + kSeq2Slots + 1) * wwords + (size_t)g.rows * g.sp + 3 * (size_t)g.rows);
}

#define ME_SEQ_NMT(X)                                                                          \
  X(16, 16, 8) X(16, 16, 11) X(16, 16, 13) X(16, 16, 16) X(16, 8, 8) X(16, 4, 8) X(8, 16, 8)   \
  X(8, 8, 8) X(8, 4, 8) X(4, 16, 8) X(4, 8, 8) X(4, 4, 8)

// The run lengths built for three CTAs per SM, and the shared memory each of
// those CTAs may take (three of them, plus the per-CTA reserve, fit the SM).
#define ME_SEQ3_NMT(X) X(16, 16, 8)
constexpr size_t kSeq3SmemCap = 74 * 1024;
template <int N, int M, int T>
constexpr bool seq3_built() {
  return N == 16 && M == 16 && T == 8;
}

// Modelled cost of a run length: staged rows per column and the per-run
// epilogue (16x16 has four instantiated run lengths, the other shapes one).
static double seq_T_cost(int M, int p, int T) {
  const int n = 2 * p + 1, nseg = (n + T - 1) / T;
  return (double)(nseg * T + M - 1) * (1.0 + 4.0 / T);
}

// Run lengths worth timing: the model's best and those within 10 % of it
// (model first).  ME_SEQ_T=8|11|13|16 fixes one (tile sweeps and tests).
static std::vector<int> seq_Ts(int N, int M, int p) {
  if (!(N == 16 && M == 16)) return {8};
  if (const char* e = std::getenv("ME_SEQ_T")) {
    const int t = std::atoi(e);
    if (t == 8 || t == 11 || t == 13 || t == 16) return {t};
  }
  static const int Ts[] = {8, 11, 13, 16};
  int bestT = 13;
  double best = 1e300;
  for (int T : Ts)
    if (seq_T_cost(M, p, T) < best * 0.999) { best = seq_T_cost(M, p, T); bestT = T; }
  std::vector<int> out{bestT};
  for (int T : Ts)
    if (T != bestT && seq_T_cost(M, p, T) <= 1.10 * best) out.push_back(T);
  return out;
}

// Adds the low-register form of k_acbm_seq (run length 8, the build for
// three CTAs per SM): one PBM and two search CTAs per SM, at claim-order lags
// of 5, 4 and 6 waves.  (Measured at 1080p
// p=32 over 59 pairs: 5.80-5.90 ms against 5.85-5.87 for the best two-CTA
// form; two PBM CTAs per SM 7.1, two search groups per search CTA 6.2-6.3.)
template <int N, int M>
static int seq_add_cands3(SeqPlan* pl, int nsm, int spec) {
  constexpr int T = 8;
  if constexpr (seq3_built<N, M, T>()) {
    const int p = pl->p;
    const size_t per = (size_t)4 * (pbm_win_words(N, M, p) + M * (N / 4));
    struct Form3 { int cps, ppsm, split, sg, lag; };
    const Form3 f3s[] = {{3, 1, 0, 1, 1}, {3, 1, 0, 1, 0}, {3, 1, 0, 1, 2}};
    for (const Form3& f : f3s) {
      const size_t srch = 4 * (size_t)f.sg * seq_group_words<N, M, T>(p, kSeqThreads / f.sg);
      const int pw = (int)std::min<size_t>(kSeqThreads / 32, kSeq3SmemCap / per);
      if (pw < 1 || srch > kSeq3SmemCap) continue;
      const size_t sm3 = std::max(srch, (size_t)pw * per);
      {
        const int e = ensure_dynamic_smem((const void*)k_acbm_seq<N, M, T, 3>, sm3);
        if (e) return e;
      }
      int per_sm = 0;
      ME_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_acbm_seq<N, M, T, 3>,
                                                            kSeqThreads, sm3));
      if (per_sm < f.cps) continue;
      char nm[80];
      std::snprintf(nm, sizeof(nm), "seq3 T=%d pbm=%d/%d split=%d spec=%d groups=%d lag=%d", T,
                    f.ppsm, f.cps, f.split, spec, f.sg, kSeqLags[f.lag]);
      pl->cands.push_back(SeqPlan::Cand{1, T, f.split, pw, spec, f.sg, f.lag, 1, f.cps, f.ppsm, 1,
                                        sm3, f.cps * nsm, nm});
      // and with the ring evaluated after the spatial predictors only
      if (f.lag == 1)
        pl->cands.push_back(SeqPlan::Cand{1, T, f.split, pw, spec, f.sg, f.lag, 1, f.cps, f.ppsm, 0,
                                          sm3, f.cps * nsm, std::string(nm) + " ring=late"});
    }
  }
  return ME_OK;
}

// Adds the launch candidates of run length T to the plan: k_acbm_seq with
// two search CTAs on every 3rd (the model), 2nd or 4th SM, and k_acbm_seq2
// with 4 or 5 PBM warps per CTA when its shared memory allows (single-slice
// searches only).
template <int N, int M, int T>
static int seq_add_cands(SeqPlan* pl, int nsm, bool model_T) {
  const int p = pl->p;
  // speculation on unless ME_SEQ_SPEC=0 (A/B sweeps); the model's form is
  // also timed without it
  const char* se = std::getenv("ME_SEQ_SPEC");
  const int spec = pl->S == 1 && !(se && se[0] == '0') ? 1 : 0;
  struct Form { int split, spec, sg, lag; };
  std::vector<Form> forms{{kSeqSearchEvery, spec, 0, 0}};
  if (pl->S == 1) {
    forms.push_back({2, spec, 0, 0});
    if (spec && model_T) forms.push_back({kSeqSearchEvery, 0, 0, 0});
    forms.push_back({kSeqSearchEvery, spec, 2, 0});
    forms.push_back({2, spec, 2, 0});
    if (pl->K > 1) {
      forms.push_back({kSeqSearchEvery, spec, 0, 1});
      forms.push_back({kSeqSearchEvery, spec, 2, 1});
      forms.push_back({kSeqSearchEvery, spec, 0, 2});
      forms.push_back({kSeqSearchEvery, spec, 2, 2});
    }
  }
  for (const Form& f : forms) {
    const size_t sm1 = seq_smem<N, M, T>(p, f.sg);
    if (sm1 > 220 * 1024) continue;
    {
      const int e = ensure_dynamic_smem((const void*)k_acbm_seq<N, M, T>, sm1);
      if (e) return e;
    }
    int per_sm = 0;
    ME_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_acbm_seq<N, M, T>, kSeqThreads,
                                                          sm1));
    // two CTAs per SM, one of each role (cta_role).  (A third CTA per SM with
    // the 8-row build at 85 registers measured 30 % slower.)
    if (per_sm < 2) continue;
    char nm[64];
    std::snprintf(nm, sizeof(nm), "seq T=%d split=%d spec=%d groups=%d lag=%d", T, f.split, f.spec,
                  f.sg > 0 ? f.sg : 1, kSeqLags[f.lag]);
    if (model_T && &f == &forms[0]) pl->model = (int)pl->cands.size();
    pl->cands.push_back(SeqPlan::Cand{1, T, f.split, seq_pbm_warps(N, M, p), f.spec, f.sg, f.lag, 0,
                                      2, 1, 1, sm1, 2 * nsm, nm});
    if (f.split == kSeqSearchEvery && f.sg == 2 && f.lag == 1)
      pl->cands.push_back(SeqPlan::Cand{1, T, f.split, seq_pbm_warps(N, M, p), f.spec, f.sg, f.lag,
                                        0, 2, 1, 0, sm1, 2 * nsm, std::string(nm) + " ring=late"});
  }
  if (pl->S == 1 && pl->K > 1 && model_T) {
    const int e = seq_add_cands3<N, M>(pl, nsm, spec);
    if (e) return e;
  }
  if (pl->S == 1 && model_T) {
    for (int pw = 5; pw <= 5; pw++) {
      const size_t sm2 = seq2_smem<N, M, T>(p, pw);
      if (sm2 > 220 * 1024) continue;
      const int e = ensure_dynamic_smem((const void*)k_acbm_seq2<N, M, T>, sm2);
      if (e) return e;
      int per2 = 0;
      ME_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, k_acbm_seq2<N, M, T>,
                                                            kSeq2Threads, sm2));
      if (per2 < 1) continue;
      char nm[64];
      std::snprintf(nm, sizeof(nm), "seq2 T=%d pw=%d", T, pw);
      pl->cands.push_back(SeqPlan::Cand{2, T, 0, pw, 0, 0, 0, 0, 1, 1, 1, sm2, nsm, nm});
    }
  }
  return ME_OK;
}

static int build_seq_plan(SeqPlan* pl) {
  const int N = pl->N, M = pl->M, BW = pl->W / N, BH = pl->H / M, nbf = BW * BH;
  // claim orders: all blocks of all pairs by w + L * k, then pair, then row,
  // one table per lag L (a block's spatial predecessors have keys one to
  // three smaller, its temporal ones key + 3 - L: claimed earlier for L >= 4)
  const Waves wv = make_waves(BW, BH);
  std::vector<int> items;
  items.reserve((size_t)nbf * pl->K * kSeqNLags);
  for (int li = 0; li < kSeqNLags; li++) {
    const int L = kSeqLags[li];
    const int maxkey = wv.n - 1 + L * (pl->K - 1);
    for (int key = 0; key <= maxkey; key++)
      for (int k = 0; k < pl->K; k++) {
        const int w = key - L * k;
        if (w < 0 || w >= wv.n) continue;
        for (int by = wv.ylo(w); by <= wv.yhi(w); by++) items.push_back(k * nbf + by * BW + (w - 2 * by));
      }
  }
  pl->total = (int)(items.size() / kSeqNLags);
  const PadGeom pg = pad_geom(pl->W, pl->H, pl->p);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
  const size_t o_ctrl = take(sizeof(SeqCtrl));
  const size_t o_items = take(sizeof(int) * items.size());
  const size_t o_pad = take((size_t)pg.pitch * pg.rows * pl->K);
  const size_t o_intra = take(4 * (size_t)nbf * pl->K);
  const size_t o_flags = take(8 * (size_t)nbf * pl->K);
  // column slices per full search
  // One slice by default: splitting a block's full search over CTAs (S > 1,
  // merged by an atomic minimum) measured slower at 1080p p=32 (a slice of
  // half the columns took 7 us against 10 us for the whole search, and the
  // queue carried twice the entries); ME_SEQ_S=2..8 selects it for sweeps.
  pl->S = 1;
  if (const char* e = std::getenv("ME_SEQ_S")) pl->S = std::min(8, std::max(1, std::atoi(e)));
  if ((long long)pl->total * pl->S >= (1ll << 31)) return ME_ERR_SHAPE;
  const size_t o_q = take(8 * (size_t)nbf * pl->K * pl->S);
  const size_t o_bkey = take(8 * (size_t)nbf * pl->K);
  const size_t o_bdone = take(4 * (size_t)nbf * pl->K);
  ME_CUDA(cudaMalloc(&pl->mem, off));
  ME_CUDA(cudaMemset(pl->mem, 0, off));
  uint8_t* m = static_cast<uint8_t*>(pl->mem);
  pl->ctrl = reinterpret_cast<SeqCtrl*>(m + o_ctrl);
  pl->items = reinterpret_cast<int*>(m + o_items);
  pl->refpad = m + o_pad;
  pl->intra = reinterpret_cast<uint32_t*>(m + o_intra);
  pl->flags = reinterpret_cast<unsigned long long*>(m + o_flags);
  pl->q = reinterpret_cast<unsigned long long*>(m + o_q);
  pl->bkey = reinterpret_cast<unsigned long long*>(m + o_bkey);
  pl->bdone = reinterpret_cast<int*>(m + o_bdone);
  ME_CUDA(cudaMemcpy(pl->items, items.data(), sizeof(int) * items.size(), cudaMemcpyHostToDevice));
  SeqCtrl c;
  std::memset(&c, 0, sizeof(c));
  c.timeout_cycles = wait_cycles(1000000000ll);     // 1 s
  ME_CUDA(cudaMemcpy(pl->ctrl, &c, sizeof(c), cudaMemcpyHostToDevice));
  int nsm = 1;
  {
    const int e = sm_count(&nsm);
    if (e) return e;
  }
  const std::vector<int> Ts = seq_Ts(N, M, pl->p);
  for (size_t ti = 0; ti < Ts.size(); ti++) {
    int st = ME_ERR_ARG;
#define X(n_, m_, t_)                                                                          \
    if (N == n_ && M == m_ && Ts[ti] == t_) st = seq_add_cands<n_, m_, t_>(pl, nsm, ti == 0);
    ME_SEQ_NMT(X)
#undef X
    if (st) return st;
  }
  if (pl->cands.empty()) return ME_ERR_CUDA;
  if (pl->cands[pl->model].ver != 1) pl->model = 0;
  ME_CUDA(cudaEventCreateWithFlags(&pl->last, cudaEventDisableTiming));
  return ME_OK;
}

static int get_seq_plan(int W, int H, int N, int M, int p, int K, SeqPlan** out) {
  int dev = 0;
  ME_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_seq_mu);
  for (SeqPlan* pl : g_seq_plans)
    if (pl->dev == dev && pl->W == W && pl->H == H && pl->N == N && pl->M == M && pl->p == p &&
        pl->K == K) {
      *out = pl;
      return ME_OK;
    }
  SeqPlan* pl = new SeqPlan();
  pl->dev = dev; pl->W = W; pl->H = H; pl->N = N; pl->M = M; pl->p = p; pl->K = K;
  const int st = build_seq_plan(pl);
  if (st) {
    if (pl->mem) cudaFree(pl->mem);
    delete pl;
    return st;
  }
  g_seq_plans.push_back(pl);
  *out = pl;
  return ME_OK;
}

bool fsbm_pipe_applies(int N, int M, int p) {
  // 16x16 blocks with windows of kPipeBpc blocks within the kSeqSP pitch
  // (ME_FSBM_PIPE=0 selects the one-launch-per-group kernels instead)
  const char* pe = std::getenv("ME_FSBM_PIPE");
  if (pe && pe[0] == '0') return false;
  return N == 16 && M == 16 && (kPipeBpc - 1) * N + 2 * p + 1 + N - 4 <= kSeqSP;
}

int launch_fsbm_pipe(const uint8_t* const* frames, int K, int W, int H, int p, uint32_t lam,
                     int16_t* mv_out, uint32_t* J_out, uint32_t* sad_out, cudaStream_t s) {
  PipeOut o;
  std::memset(&o, 0, sizeof(o));
  o.mv = mv_out;
  o.J = J_out;
  o.sad = sad_out;
  return launch_fsbm_pipe_mode(kPipeKeys, frames, K, W, H, p, lam, o, s);
}

int launch_fsbm_pipe_mode(int mode, const uint8_t* const* frames, int K, int W, int H, int p,
                          uint32_t lam, const PipeOut& out, cudaStream_t s, int T) {
  if (K < 1 || K > kSeqMax) return ME_ERR_ARG;
  if (mode == kPipeStats && (!out.smin || !out.sdev)) return ME_ERR_ARG;
  if (mode == kPipeVolume && !out.vol) return ME_ERR_ARG;
  SeqFrames fr;
  std::memset(&fr, 0, sizeof(fr));
  for (int k = 0; k <= K; k++) fr.f[k] = frames[k];
  const FsPlan pl{T > 0 ? T : fs_plan(16, 16, p, W / 16).T, 0, 0, 0, 1};
  int nsm = 1;
  { const int e = sm_count(&nsm); if (e) return e; }
  const int BW = W / 16, BH = H / 16;
  const int groups = K * BH * ((BW + kPipeBpc - 1) / kPipeBpc);
  const int pgrid = std::min(nsm, groups);
  const long long lim = wait_cycles(1000000000ll);
#define X(t_, m_)                                                                             \
  if (pl.T == t_ && mode == m_) {                                                             \
    auto kern = k_fsbm_pipe<16, 16, t_, m_>;                                                  \
    const size_t smem = pipe_smem_bytes<16, 16, t_>(p);                                       \
    const int st = ensure_dynamic_smem((const void*)kern, smem);                              \
    if (st) return st;                                                                        \
    kern<<<pgrid, kPipeThreads, smem, s>>>(fr, W, H, p, lam, groups, lim, out);               \
    ME_CUDA(cudaGetLastError());                                                              \
    return ME_OK;                                                                             \
  }
#define Y(m_) X(8, m_) X(11, m_) X(13, m_) X(16, m_)
  Y(kPipeKeys) Y(kPipeStats) Y(kPipeVolume)
#undef Y
#undef X
  return ME_ERR_ARG;
}

// ------------------------------------------------------------------ pipelined search, any p: launches
bool pipe_tab_applies(int N, int M, int p) {
  const char* pe = std::getenv("ME_FSBM_PIPE");
  if (pe && pe[0] == '0') return false;
  return (N == 4 || N == 8 || N == 16) && (M == 4 || M == 8 || M == 16) && p >= 1 && p <= kMaxP;
}

int pipe_tab_bpc(int N, int p) {
  return N == 16 ? tab_bpc<16>(p) : N == 8 ? tab_bpc<8>(p) : tab_bpc<4>(p);
}

int pipe_tab_T(int N, int M) { return N == 16 && M == 16 ? TabCfg<16, 16>::T : TabCfg<8, 8>::T; }

template <int N, int M>
static int launch_pipe_tab_t(const TabArgs& A, int grid, cudaStream_t s) {
  const size_t smem = tab_smem_bytes<N, M>();
  const int st = ensure_dynamic_smem((const void*)k_fsbm_pipe_tab<N, M>, smem);
  if (st) return st;
  if (grid < 1) return ME_OK;
  k_fsbm_pipe_tab<N, M><<<grid, kPipeThreads, smem, s>>>(A);
  ME_CUDA(cudaGetLastError());
  return ME_OK;
}

static int launch_pipe_tab(int N, int M, const TabArgs& A, int grid, cudaStream_t s) {
#define X(n_, m_) \
  if (N == n_ && M == m_) return launch_pipe_tab_t<n_, m_>(A, grid, s);
  X(16, 16) X(16, 8) X(16, 4) X(8, 16) X(8, 8) X(8, 4) X(4, 16) X(4, 8) X(4, 4)
#undef X
  return ME_ERR_ARG;
}

int launch_pipe_tab_seq(const uint8_t* const* frames, int K, int W, int H, int N, int M, int p,
                        uint32_t lam, int16_t* mv_out, uint32_t* J_out, uint32_t* sad_out,
                        cudaStream_t s) {
  if (K < 1 || K > kSeqMax || !pipe_tab_applies(N, M, p)) return ME_ERR_ARG;
  TabArgs A;
  std::memset(&A, 0, sizeof(A));
  for (int k = 0; k <= K; k++) A.fr.f[k] = frames[k];
  A.W = W; A.H = H; A.p = p; A.K = K; A.lam = lam;
  A.mv = mv_out; A.J = J_out; A.sad = sad_out;
  const int BW = W / N, BH = H / M, bpc = pipe_tab_bpc(N, p);
  A.ngroups = K * BH * ((BW + bpc - 1) / bpc);
  A.lim = wait_cycles(1000000000ll);
  int nsm = 1;
  { const int e = sm_count(&nsm); if (e) return e; }
  return launch_pipe_tab(N, M, A, std::min(nsm, A.ngroups), s);
}

int launch_pipe_tab_batch(int N, int M, const BShape* shp, const BStream* st, const BFsEntry* ent,
                          int nent, int* ctr, int* err, cudaStream_t s) {
  TabArgs A;
  std::memset(&A, 0, sizeof(A));
  A.shp = shp; A.st = st; A.ent = ent; A.ngroups = nent; A.ctr = ctr; A.err = err;
  A.lim = wait_cycles(1000000000ll);
  int nsm = 1;
  { const int e = sm_count(&nsm); if (e) return e; }
  return launch_pipe_tab(N, M, A, std::min(nsm, nent), s);
}

// ------------------------------------------------------------------ tuned full search
// Full search of K pairs (frames[k] -> frames[k+1]) in one launch, with the
// launch form chosen by the autotuner on the first call of each shape: the
// pipelined kernel at each run length within 10 % of the model's best (16x16
// blocks, windows within its compile-time pitch), and the per-group kernel
// with the two or three plans of lowest modelled cost.
struct FsTune {
  int dev, W, H, N, M, p, K;
  bool pipe;
  struct Cand {
    int pipeT;    // > 0: k_fsbm_pipe with this run length; 0: k_fsbm_seq with pl;
                  // -1: k_fsbm_pipe_tab (any p)
    FsPlan pl;
    std::string name;
  };
  std::vector<Cand> cands;
  int model = 0, chosen = -1;
  std::mutex mu;
};
static std::mutex g_fst_mu;
static std::vector<FsTune*> g_fst;

static FsTune* fs_tune_entry(int dev, int W, int H, int N, int M, int p, int K) {
  const bool pipe = fsbm_pipe_applies(N, M, p);
  std::lock_guard<std::mutex> lk(g_fst_mu);
  for (FsTune* t : g_fst)
    if (t->dev == dev && t->W == W && t->H == H && t->N == N && t->M == M && t->p == p &&
        t->K == K && t->pipe == pipe)
      return t;
  FsTune* t = new FsTune();
  t->dev = dev; t->W = W; t->H = H; t->N = N; t->M = M; t->p = p; t->K = K; t->pipe = pipe;
  char nm[64];
  if (pipe) {
    const int T0 = fs_plan(16, 16, p, W / 16).T;
    static const int Ts[] = {8, 11, 13, 16};
    std::snprintf(nm, sizeof(nm), "pipe T=%d", T0);
    t->cands.push_back(FsTune::Cand{T0, FsPlan{T0, 0, 0, 0, 1}, nm});
    for (int T : Ts)
      if (T != T0 && seq_T_cost(16, p, T) <= 1.10 * seq_T_cost(16, p, T0)) {
        std::snprintf(nm, sizeof(nm), "pipe T=%d", T);
        t->cands.push_back(FsTune::Cand{T, FsPlan{T, 0, 0, 0, 1}, nm});
      }
  }
  // the any-p pipeline: the model's form for 16x16 blocks past the other
  // pipeline's ranges; after the per-group plans for the other shapes (whose
  // short runs it feeds less well: 8x8 at 1080p p=32 measured 1.11 ms for 4
  // pairs against 0.95 ms for the best per-group plan)
  const bool tab = pipe_tab_applies(N, M, p), tab_first = tab && N == 16 && M == 16;
  std::snprintf(nm, sizeof(nm), "pipetab B=%d", pipe_tab_bpc(N, p));
  const FsTune::Cand tabc{-1, FsPlan{pipe_tab_T(N, M), 0, 0, 0, 1}, nm};
  if (tab_first) t->cands.push_back(tabc);
  for (const FsPlan& pl : fs_plans_ranked(N, M, p, W / N, pipe ? 2 : 3)) {
    std::snprintf(nm, sizeof(nm), "group T=%d G=%d thr=%d", pl.T, pl.G, pl.threads);
    t->cands.push_back(FsTune::Cand{0, pl, nm});
  }
  if (tab && !tab_first) t->cands.push_back(tabc);
  g_fst.push_back(t);
  return t;
}

static int fs_seq_enqueue(const FsTune::Cand& cd, const uint8_t* const* frames, int K, int W,
                          int H, int N, int M, int p, uint32_t lam, int16_t* mv_out,
                          uint32_t* J_out, uint32_t* sad_out, cudaStream_t s) {
  if (cd.pipeT < 0)
    return launch_pipe_tab_seq(frames, K, W, H, N, M, p, lam, mv_out, J_out, sad_out, s);
  if (cd.pipeT > 0) {
    PipeOut o;
    std::memset(&o, 0, sizeof(o));
    o.mv = mv_out;
    o.J = J_out;
    o.sad = sad_out;
    return launch_fsbm_pipe_mode(kPipeKeys, frames, K, W, H, p, lam, o, s, cd.pipeT);
  }
  const FsPlan& pl = cd.pl;
  SeqFrames fr;
  std::memset(&fr, 0, sizeof(fr));
  for (int k = 0; k <= K; k++) fr.f[k] = frames[k];
  const int BW = W / N, BH = H / M, bpc = pl.threads / pl.G;
  const dim3 grid(((BW + bpc - 1) / bpc) * BH, K);
  // the 16x16 run length 13 with shifted rows of at most kSeqSP words (p <= 34
  // at 8 blocks per CTA) uses the build with a compile-time row pitch
  if (N == 16 && M == 16 && pl.T == 13 && (bpc - 1) * N + 2 * p + 1 + N - 4 <= kSeqSP) {
    auto kern = k_fsbm_seq<16, 16, 13, kSeqSP>;
    const size_t smem = fs_smem_bytes<16, 16, 13>(fs_geom<16, 16, 13>(p, bpc, pl.G, 0, 0, kSeqSP));
    const int st = ensure_dynamic_smem((const void*)kern, smem);
    if (st) return st;
    kern<<<grid, pl.threads, smem, s>>>(fr, W, H, p, pl.G, lam, mv_out, J_out, sad_out);
    ME_CUDA(cudaGetLastError());
    return ME_OK;
  }
  int st = ME_ERR_ARG;
#define X(n_, m_, t_)                                                                          \
  if (N == n_ && M == m_ && pl.T == t_) {                                                      \
    { const int e_ = ensure_dynamic_smem((const void*)k_fsbm_seq<n_, m_, t_>, pl.smem);         \
      if (e_) return e_; }                                                                     \
    k_fsbm_seq<n_, m_, t_><<<grid, pl.threads, pl.smem, s>>>(fr, W, H, p, pl.G, lam, mv_out,   \
                                                            J_out, sad_out);                   \
    st = ME_OK;                                                                                \
  }
  ME_SEQ_NMT(X)
#undef X
  if (st) return st;
  ME_CUDA(cudaGetLastError());
  return ME_OK;
}

int fsbm_tuned(const uint8_t* const* frames, int K, int W, int H, int N, int M, int p,
               uint32_t lam, int16_t* mv_out, uint32_t* J_out, uint32_t* sad_out, cudaStream_t s) {
  int dev = 0;
  ME_CUDA(cudaGetDevice(&dev));
  FsTune* t = fs_tune_entry(dev, W, H, N, M, p, K);
  std::lock_guard<std::mutex> lk(t->mu);
  auto run = [&](int c) {
    return fs_seq_enqueue(t->cands[c], frames, K, W, H, N, M, p, lam, mv_out, J_out, sad_out, s);
  };
  int c = tune_forced((int)t->cands.size());
  if (c < 0) {
    if (t->chosen < 0) {
      char what[96];
      std::snprintf(what, sizeof(what), "fsbm %dx%d %dx%d p=%d K=%d", W, H, N, M, p, K);
      std::vector<std::string> names;
      for (const FsTune::Cand& cd : t->cands) names.push_back(cd.name);
      int ch = t->model;
      const int st = tune_select(what, names, t->model, s, run, &ch);
      if (st) return st;
      t->chosen = ch;
    }
    c = t->chosen;
  }
  return run(c);
}

static int check_seq_frames(const uint8_t* const* frames, int K) {
  if (!frames || K < 1 || K > kSeqMax) return ME_ERR_ARG;
  for (int k = 0; k <= K; k++)
    if (!frames[k] || !aligned4(frames[k])) return ME_ERR_ARG;
  return ME_OK;
}

}  // namespace me

using namespace me;

// Enqueues one whole ACBM sequence run of plan candidate c on s: the run's
// control reset, the padded references and Intra_SAD of all pairs, and the
// persistent search kernel.  Called with the plan's lock held.
static int seq_enqueue(SeqPlan* pl, int c, const SeqFrames& fr, const SeqArgs& a, cudaStream_t s) {
  const int W = pl->W, H = pl->H, N = pl->N, M = pl->M, p = pl->p, K = pl->K;
  const SeqPlan::Cand& cd = pl->cands[c];
  const PadGeom pg = pad_geom(W, H, p);
  if (pl->ran) ME_CUDA(cudaStreamWaitEvent(s, pl->last, 0));
  k_seq_begin<<<1, 256, 0, s>>>(pl->ctrl);
  ME_CUDA(cudaGetLastError());
  const long long work = std::max<long long>((long long)pg.rows * (pg.pitch / 16) * K,
                                             32LL * (W / N) * (H / M) * K);
  int nsm = 1;
  { const int e = sm_count(&nsm); if (e) return e; }
  const int gp = (int)std::min<long long>((work + 255) / 256, nsm * 8LL);
  int st = ME_ERR_ARG;
#define X(n_, m_)                                                                              \
  if (N == n_ && M == m_) {                                                                    \
    k_seq_prologue<n_, m_><<<gp, 256, 0, s>>>(fr, K, pg, W, H, pl->refpad, pl->intra, pl->bkey, \
                                               pl->bdone);                                     \
    st = ME_OK;                                                                                \
  }
  X(16, 16) X(16, 8) X(16, 4) X(8, 16) X(8, 8) X(8, 4) X(4, 16) X(4, 8) X(4, 4)
#undef X
  if (st) return st;
  ME_CUDA(cudaGetLastError());
  st = ME_ERR_ARG;
#define X(n_, m_, t_)                                                                          \
  if (N == n_ && M == m_ && cd.T == t_) {                                                      \
    if (cd.ver == 2)                                                                           \
      k_acbm_seq2<n_, m_, t_><<<cd.grid, kSeq2Threads, cd.smem, s>>>(                          \
          fr, a, W, H, p, pg, pl->refpad, pl->intra, pl->flags,                                \
          pl->items + (size_t)cd.lag * pl->total, pl->total, pl->ctrl,                         \
          pl->q, cd.pw);                                                                       \
    else if (!cd.lr)                                                                           \
      k_acbm_seq<n_, m_, t_><<<cd.grid, kSeqThreads, cd.smem, s>>>(                            \
          fr, a, W, H, p, pg, pl->refpad, pl->intra, pl->flags,                                \
          pl->items + (size_t)cd.lag * pl->total, pl->total, pl->ctrl, pl->q, pl->bkey,        \
          pl->bdone, pl->S, cd.pw, cd.split, cd.spec, cd.sgroups, 2, 1, cd.early);             \
    st = !cd.lr || cd.ver == 2 ? ME_OK : ME_ERR_ARG;                                           \
  }
  ME_SEQ_NMT(X)
#undef X
#define X(n_, m_, t_)                                                                          \
  if (N == n_ && M == m_ && cd.T == t_ && cd.ver == 1 && cd.lr) {                             \
    k_acbm_seq<n_, m_, t_, 3><<<cd.grid, kSeqThreads, cd.smem, s>>>(                           \
        fr, a, W, H, p, pg, pl->refpad, pl->intra, pl->flags,                                  \
        pl->items + (size_t)cd.lag * pl->total, pl->total, pl->ctrl, pl->q, pl->bkey,          \
        pl->bdone, pl->S, cd.pw, cd.split, cd.spec, cd.sgroups, cd.cps, cd.ppsm, cd.early);    \
    st = ME_OK;                                                                                \
  }
  ME_SEQ3_NMT(X)
#undef X
  if (st) return st;
  ME_CUDA(cudaGetLastError());
  ME_CUDA(cudaEventRecord(pl->last, s));
  pl->ran = true;
  return ME_OK;
}

extern "C" {

int me_fsbm_sequence(const uint8_t* const* frames, int K, int W, int H, int N, int M, int p,
                     uint32_t lambda_q8, int16_t* mv_out, uint32_t* J_out, uint32_t* sad_out,
                     me_stream_t stream) {
  int st = check_seq_frames(frames, K);
  if (st) return st;
  if (!mv_out || !J_out) return ME_ERR_ARG;
  st = check_frame_args(W, H, N, M, p, lambda_q8);
  if (st) return st;
  return fsbm_tuned(frames, K, W, H, N, M, p, lambda_q8, mv_out, J_out, sad_out,
                    reinterpret_cast<cudaStream_t>(stream));
}

int me_acbm_sequence(const uint8_t* const* frames, int K, int W, int H, int N, int M, int p,
                     uint32_t lambda_q8, const int16_t* prev_mv_field, const me_acbm_params* prm,
                     int16_t* mv_out, uint32_t* J_out, uint8_t* fullsearch_mask_out,
                     uint32_t* sad_out, uint32_t* load_out, me_stream_t stream) {
  int st = check_seq_frames(frames, K);
  if (st) return st;
  if (!mv_out || !J_out || !fullsearch_mask_out) return ME_ERR_ARG;
  st = check_frame_args(W, H, N, M, p, lambda_q8);
  if (st) return st;
  st = check_acbm_params(prm);
  if (st) return st;
  SeqPlan* pl = nullptr;
  st = get_seq_plan(W, H, N, M, p, K, &pl);
  if (st) return st;
  SeqFrames fr;
  std::memset(&fr, 0, sizeof(fr));
  for (int k = 0; k <= K; k++) fr.f[k] = frames[k];
  SeqArgs a;
  a.prev0 = prev_mv_field;
  a.mv = mv_out; a.J = J_out; a.mask = fullsearch_mask_out; a.sad = sad_out; a.load = load_out;
  a.lam = lambda_q8;
  a.alpha = prm->alpha; a.beta = prm->beta; a.gnum = prm->gamma_num; a.gden = prm->gamma_den;
  a.qp = prm->qp; a.refine = prm->refine;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // runs that share a plan's scratch are ordered on the GPU, whatever their streams
  std::lock_guard<std::mutex> lk(pl->mu);
  auto run = [&](int c) { return seq_enqueue(pl, c, fr, a, s); };
  int c = tune_forced((int)pl->cands.size());
  if (c < 0) {
    if (pl->chosen < 0) {
      char what[96];
      std::snprintf(what, sizeof(what), "acbm_sequence %dx%d %dx%d p=%d K=%d", W, H, N, M, p, K);
      std::vector<std::string> names;
      for (const SeqPlan::Cand& cd : pl->cands) names.push_back(cd.name);
      int ch = pl->model;
      st = tune_select(what, names, pl->model, s, run, &ch);
      if (st) return st;
      pl->chosen = ch;
    }
    c = pl->chosen;
  }
  return run(c);
}

int me_fsbm_sequence_status(me_stream_t stream) {
  ME_CUDA(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
  int e = 0;
  ME_CUDA(cudaMemcpyFromSymbol(&e, g_fsbm_pipe_error, sizeof(int)));
  if (e) {
    const int zero = 0;
    ME_CUDA(cudaMemcpyToSymbol(g_fsbm_pipe_error, &zero, sizeof(int)));
  }
  return e ? e : ME_OK;
}

int me_acbm_sequence_status(int W, int H, int N, int M, int p, int K, me_stream_t stream) {
  SeqPlan* pl = nullptr;
  int st = get_seq_plan(W, H, N, M, p, K, &pl);
  if (st) return st;
  ME_CUDA(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
  SeqCtrl c;
  ME_CUDA(cudaMemcpy(&c, pl->ctrl, sizeof(c), cudaMemcpyDeviceToHost));
  return c.error ? c.error : ME_OK;
}

}  // extern "C"

namespace me {

// Tuning record of me_acbm per (device, shape): the chosen candidate of
// acbm_pair_tuned's list.
struct AcbmPairTune {
  int dev, W, H, N, M, p;
  int chosen = -1;
  std::mutex mu;
};
static std::mutex g_apt_mu;
static std::vector<AcbmPairTune*> g_apt;

int acbm_pair_tuned(const AcbmArgs& a, int W, int H, int N, int M, int p, cudaStream_t s,
                    const std::function<int()>& waves) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  ME_CUDA(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone) return waves();
  int dev = 0;
  ME_CUDA(cudaGetDevice(&dev));
  AcbmPairTune* t = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_apt_mu);
    for (AcbmPairTune* e : g_apt)
      if (e->dev == dev && e->W == W && e->H == H && e->N == N && e->M == M && e->p == p) t = e;
    if (!t) {
      t = new AcbmPairTune;
      t->dev = dev; t->W = W; t->H = H; t->N = N; t->M = M; t->p = p;
      g_apt.push_back(t);
    }
  }
  SeqPlan* pl = nullptr;
  int st = get_seq_plan(W, H, N, M, p, 1, &pl);
  if (st) return st;
  SeqFrames fr;
  std::memset(&fr, 0, sizeof(fr));
  fr.f[0] = a.ref;
  fr.f[1] = a.cur;
  SeqArgs sa;
  sa.prev0 = a.prev;
  sa.mv = a.mv; sa.J = a.J; sa.mask = a.mask; sa.sad = a.sad; sa.load = a.load;
  sa.lam = a.lam;
  sa.alpha = a.alpha; sa.beta = a.beta; sa.gnum = a.gnum; sa.gden = a.gden;
  sa.qp = a.qp; sa.refine = a.refine;
  auto run = [&](int c) -> int {
    if (c == 0) return waves();
    // runs that share the plan's scratch are ordered on the GPU
    std::lock_guard<std::mutex> lk(pl->mu);
    return seq_enqueue(pl, c - 1, fr, sa, s);
  };
  std::lock_guard<std::mutex> lk(t->mu);
  const int n = 1 + (int)pl->cands.size();
  int c = tune_forced(n);
  if (c < 0) {
    if (t->chosen < 0) {
      char what[96];
      std::snprintf(what, sizeof(what), "acbm %dx%d %dx%d p=%d", W, H, N, M, p);
      std::vector<std::string> names{"waves"};
      for (const SeqPlan::Cand& cd : pl->cands) names.push_back("persistent " + cd.name);
      // model: the persistent kernel (one launch; the wave graph pays a
      // launch per wave on the chain)
      int ch = 1 + pl->model;
      st = tune_select(what, names, 1 + pl->model, s, run, &ch);
      if (st) return st;
      t->chosen = ch;
    }
    c = t->chosen;
  }
  return run(c);
}

}  // namespace me

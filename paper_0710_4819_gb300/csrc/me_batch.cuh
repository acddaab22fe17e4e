// me_batch.cuh -- device structures and kernels of the multi-stream
// persistent forms (the batch API and the server): stream tables, work
// segments, the prologue kernels and the persistent FSBM / ACBM kernels.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "me_device.cuh"
#include "me_host.h"
#include "me_search.cuh"
#include "me_batch_types.h"

namespace me {

constexpr int kBatchThreads = 256;

struct BSegment {  // ACBM: the blocks of one wave of one stream
  int stream, wave, ylo, count, item_base;
};

// Control block of a step.  Counters that many warps update or poll each sit
// on their own 128-byte line: an atomic on a line that 1000+ warps keep
// reading waits behind those reads for microseconds.
struct BCtrl {
  int epoch;
  int error;
  int err_item;
  int skip_stream, skip_block;  // fault injection: never publish this block
  long long timeout_ns;
  alignas(128) int next;        // work claims
  alignas(128) int fs_head;     // full-search queue of the ACBM step: claims
  alignas(128) int fs_tail;     //   appends
  alignas(128) int pbm_done;    //   blocks through PBM
  alignas(128) int started;     // CTA arrivals (roles)
  int sm_arr[kRoleSlots];       // CTA arrivals per SM (roles)
};


static __device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

static __global__ void k_batch_begin(BCtrl* c, int epoch) {
  for (int i = threadIdx.x; i < kRoleSlots; i += blockDim.x) c->sm_arr[i] = 0;
  if (threadIdx.x != 0) return;
  c->epoch = epoch > 0 ? epoch : c->epoch + 1;
  c->fs_head = 0;
  c->fs_tail = 0;
  c->pbm_done = 0;
  c->started = 0;
  c->next = 0;
  c->error = 0;
  c->err_item = -1;
}

static __global__ void k_batch_pad(const BShape* __restrict__ shp, const BStream* __restrict__ st,
                            int nstreams, long long total) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = nstreams - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (shp[mid].pad_base <= i) lo = mid; else hi = mid - 1;
    }
    const BShape& s = shp[lo];
    const long long k = i - s.pad_base;
    const int chunks = s.pg.pitch / 16;
    const int y = (int)(k / chunks), cx = (int)(k % chunks) * 16;
    const uint8_t* src = st[lo].ref + (size_t)clampi(y - s.pg.P, 0, s.H - 1) * s.W;
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      uint32_t v = 0;
#pragma unroll
      for (int b = 0; b < 4; b++)
        v |= (uint32_t)src[clampi(cx + 4 * q + b - s.pg.P, 0, s.W - 1)] << (8 * b);
      w[q] = v;
    }
    *reinterpret_cast<uint4*>(s.refpad + (size_t)y * s.pg.pitch + cx) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

template <int N, int M>
__global__ void __launch_bounds__(256) k_batch_intra(const BShape* __restrict__ shp,
                                                     const BStream* __restrict__ st, int nstreams,
                                                     int total_blocks) {
  const int lane = threadIdx.x & 31;
  for (int g = blockIdx.x * 8 + (threadIdx.x >> 5); g < total_blocks; g += gridDim.x * 8) {
    int lo = 0, hi = nstreams - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (shp[mid].blk_base <= g) lo = mid; else hi = mid - 1;
    }
    const BShape& s = shp[lo];
    const int b = g - s.blk_base, BW = s.W / N;
    const uint32_t v = warp_intra_sad<N, M>(st[lo].cur, s.W, (b % BW) * N, (b / BW) * M);
    if (lane == 0) {
      s.intra[b] = v;
      if (s.bstate) s.bstate[b] = 0;
    }
  }
}

template <int N, int M, int T>
__global__ void __launch_bounds__(256, 2) k_fsbm_persist(const BShape* __restrict__ shp,
                                                      const BStream* __restrict__ st,
                                                      const BFsEntry* __restrict__ ent, int nent,
                                                      BCtrl* ctrl) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ unsigned long long keys[16];
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&ctrl->next, 1);
    __syncthreads();
    const int i = s_item;
    __syncthreads();
    if (i >= nent) break;
    const BFsEntry e = ent[i];
    const BShape& s = shp[e.stream];
    const BStream& a = st[e.stream];
    const FsGeom g = fs_geom<N, M, T>(s.p, e.nb, e.G);
    fs_group<N, M, T>(a.cur, a.ref, s.W, s.H, e.bx0 * N, e.by * M, g, a.lam, smem, keys);
    if ((int)threadIdx.x < e.nb) {
      const Decoded d = decode_key(keys[threadIdx.x], s.p, a.lam);
      const int b = e.by * (s.W / N) + e.bx0 + threadIdx.x;
      a.mv[2 * b] = (int16_t)d.mvx;
      a.mv[2 * b + 1] = (int16_t)d.mvy;
      a.J[b] = d.J;
      if (a.sad) a.sad[b] = d.sad;
    }
  }
}

// Bounded wait until the flag word carries epoch `want` (gives up after the
// timeout, or at once after any other wait has given up, and then reports
// ME_ERR_TIMEOUT); returns the word, whose low half is the block's vector.
static __device__ __forceinline__ unsigned long long batch_wait(const unsigned long long* f, int want,
                                                                BCtrl* ctrl, long long timeout,
                                                                int item) {
  const volatile unsigned long long* vf = f;
  const volatile int* err = &ctrl->error;
  unsigned long long w = *vf;
  if (pub_epoch(w) == want) return w;
  const long long t0 = global_ns();
  while (*err == 0) {
    __nanosleep(32);
    w = *vf;
    if (pub_epoch(w) == want) break;
    if (global_ns() - t0 > timeout) {
      atomicExch(&ctrl->error, (int)ME_ERR_TIMEOUT);
      atomicExch(&ctrl->err_item, item);
      break;
    }
  }
  return w;
}

// Claim order of an ACBM step as a table: item i -> (stream << 32) | block,
// expanded from the wave segments by one thread per item.
static __global__ void k_batch_items(const BSegment* __restrict__ seg, int nseg, int total,
                                     const BShape* __restrict__ shp, int N,
                                     unsigned long long* __restrict__ items) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (seg[mid].item_base <= i) lo = mid; else hi = mid - 1;
    }
    const BSegment sg = seg[lo];
    const int by = sg.ylo + (i - sg.item_base);
    const int b = by * (shp[sg.stream].W / N) + (sg.wave - 2 * by);
    items[i] = ((unsigned long long)(uint32_t)sg.stream << 32) | (uint32_t)b;
  }
}

// PBM warps per CTA for a search range: as many windows as fit in about 100 KB.
__host__ __device__ inline int batch_pbm_warps(int N, int M, int p) {
  const int per = 4 * (pbm_win_words(N, M, p) + M * (N / 4));
  const int w = (100 * 1024) / per;
  return w < 1 ? 1 : (w > kBatchThreads / 32 ? kBatchThreads / 32 : w);
}

// Speculative full searches of the ACBM step: the queue word carries
// kBatchSpecBit beside the claim index; the block's state word (BShape
// bstate, cleared by the Intra_SAD prologue) collects kBatchSearched (the
// key is in bkey) and kBatchFailed (PBM failed): whichever comes second
// publishes the full-search result.
constexpr int kBatchSpecBit = 1 << 30;
constexpr int kBatchSearched = 1, kBatchFailed = 2;

// Publishes block b of stream si with a full-search key (flag first: it
// carries the vector; the host-chosen fault block never publishes its flag).
__device__ __forceinline__ void batch_publish_fs(const BShape& s, const BStream& a, BCtrl* ctrl,
                                                 int epoch, int si, int b, unsigned long long key) {
  const Decoded d = decode_key(key, s.p, a.lam);
  if (!(si == ctrl->skip_stream && b == ctrl->skip_block))
    atomicExch(s.flags + b, pub_word(epoch, d.mvx, d.mvy));
  a.mv[2 * b] = (int16_t)d.mvx;
  a.mv[2 * b + 1] = (int16_t)d.mvy;
  a.J[b] = d.J;
  a.mask[b] = 1;
  if (a.sad) a.sad[b] = d.sad;
  if (a.load) a.load[b] = (uint32_t)((2 * s.p + 1) * (2 * s.p + 1));
}

// ACBM step over many streams, two roles in one launch (cta_role: one CTA of
// each per SM).  PBM CTAs: every warp
// claims blocks on its own, in wave order across streams (the item table maps
// a claim to its stream and block), queues the block's current pixels and
// search window as asynchronous copies, waits for the block's left / up-left /
// up / up-right neighbours (whose flag words carry their final vectors), runs
// PBM and the two conditions, and publishes the block or appends its claim to
// the full-search queue.  A warp claims its next block before working on the
// current one.  Search CTAs take queued blocks in order and search each with
// the whole CTA.  The smallest unfinished block is always some warp's current
// block with all its predecessors finished, and search CTAs only wait for
// queue entries a running PBM warp will write (or the end of the step): every
// wait ends, and each is also bounded in time.
template <int N, int M, int T>
__global__ void __launch_bounds__(256, 2) k_acbm_persist(const BShape* __restrict__ shp,
                                                         const BStream* __restrict__ st,
                                                         const unsigned long long* __restrict__ items,
                                                         int total, BCtrl* ctrl,
                                                         unsigned long long* __restrict__ q,
                                                         int pbm_warps, int win_words, int nsm,
                                                         int nstreams, int spec) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ unsigned long long keys[16];
  __shared__ int s_role, s_spec;
  __shared__ unsigned long long s_item;
  const unsigned FULL = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int epoch = *reinterpret_cast<volatile int*>(&ctrl->epoch);
  const long long timeout = ctrl->timeout_ns;
  if (tid == 0) s_role = cta_role(&ctrl->started, ctrl->sm_arr);
  __syncthreads();

  if (s_role == 0) {
    // ---------------------------------------------------------------- PBM warps
    if (warp >= pbm_warps) return;
    uint32_t* win = smem + warp * (win_words + M * (N / 4));
    uint32_t* curs = win + win_words;
    // lane 0 holds the next claim (item index and its stream/block)
    int nxt = 0;
    unsigned long long inxt = 0;
    if (lane == 0) {
      nxt = atomicAdd(&ctrl->next, 1);
      if (nxt < total) inxt = items[nxt];
    }
    for (;;) {
      const int i = __shfl_sync(FULL, nxt, 0);
      if (i >= total) break;
      const unsigned long long it = __shfl_sync(FULL, inxt, 0);
      const int si = (int)(it >> 32), b = (int)(uint32_t)it;
      const BShape& s = shp[si];
      const BStream& a = st[si];
      const int BW = s.W / N, BH = s.H / M;
      const int bx = b % BW, by = b / BW;
      const PbmWin wg = pbm_stage<N, M>(a.cur, s.refpad, s.pg, s.W, s.p, bx * N, by * M, curs, win);
      const uint32_t ix = s.intra[b];
      // predictors: lanes 0-3 the spatial ones (final vectors of this step,
      // carried by their flags), lanes 4-12 the previous field's 3x3, lane 13
      // the zero vector
      int cx = 0, cy = 0;
      bool valid = false;
      int sflag = -1;   // spatial neighbour whose flag this lane waits for
      if (lane < 4) {
        const int dx = (lane < 2) ? -1 : (lane == 2 ? 0 : 1);
        const int dy = (lane == 0) ? 0 : -1;
        const int nx = bx + dx, ny = by + dy;
        if (nx >= 0 && nx < BW && ny >= 0) {
          sflag = ny * BW + nx;
          valid = true;
        }
      } else if (lane < 13) {
        const int t = lane - 4, nx = bx + t % 3 - 1, ny = by + t / 3 - 1;
        if (nx >= 0 && nx < BW && ny >= 0 && ny < BH) {
          if (a.prev) {
            cx = a.prev[2 * (ny * BW + nx)];
            cy = a.prev[2 * (ny * BW + nx) + 1];
          }
          valid = true;
        }
      } else if (lane == 13) {
        valid = true;
      }
      // the previous field's and the zero predictors first (no wait); a block
      // that fails both conditions with them alone has its full search queued
      // at once (speculatively), while the warp waits for its spatial
      // neighbours -- its result does not depend on the guess
      const PbmPart pa = pbm_part_a<N, M>(cx, cy, valid, wg, s.p, a.lam, curs, win);
      const bool sp = spec && s.bstate &&
                      pbm_would_fail<N, M>(pa.best, s.p, a.lam, ix, a.alpha, a.beta, a.gnum, a.gden,
                                           a.qp);
      if (sp && lane == 0) {
        const int slot = atomicAdd(&ctrl->fs_tail, 1);
        atomicExch(q + slot, ((unsigned long long)(uint32_t)epoch << 32) | (uint32_t)i |
                                 kBatchSpecBit);
      }
      // the ring around part a's best, evaluated now if a spatial neighbour
      // is still running (part b uses it when no spatial predictor beats
      // part a's best; the result never depends on it)
      PbmRing ring0 = pbm_no_ring();
      if (a.refine) {
        const bool ready = sflag < 0 ||
                           pub_epoch(*reinterpret_cast<const volatile unsigned long long*>(
                               s.flags + sflag)) == epoch;
        if (!__all_sync(0xffffffffu, ready))
          ring0 = pbm_ring_early<N, M>(cx, cy, valid, pa, wg, s.p, a.lam, curs, win);
      }
      if (sflag >= 0) {
        const unsigned long long w = batch_wait(s.flags + sflag, epoch, ctrl, timeout, i);
        cx = pub_mvx(w);
        cy = pub_mvy(w);
      }
      const PbmResult r = pbm_part_b<N, M>(cx, cy, valid, pa, wg, s.p, a.lam, ix, a.alpha, a.beta,
                                           a.gnum, a.gden, a.qp, a.refine, curs, win, nullptr,
                                           ring0);
      if (lane == 0) {
        if (r.pass) {
          // the flag word carries the vector: publish first, outputs after
          const Decoded d = decode_key(r.key, s.p, a.lam);
          if (!(si == ctrl->skip_stream && b == ctrl->skip_block))
            atomicExch(s.flags + b, pub_word(epoch, d.mvx, d.mvy));
          a.mv[2 * b] = (int16_t)d.mvx;
          a.mv[2 * b + 1] = (int16_t)d.mvy;
          a.J[b] = d.J;
          a.mask[b] = 0;
          if (a.sad) a.sad[b] = d.sad;
          if (a.load) a.load[b] = (uint32_t)r.load;
        } else if (sp) {
          // the speculative search publishes if it finishes after this
          // decision; if it finished before, its key is here to publish
          if (atomicOr(s.bstate + b, kBatchFailed) & kBatchSearched) {
            __threadfence();
            batch_publish_fs(s, a, ctrl, epoch, si, b,
                             *reinterpret_cast<volatile unsigned long long*>(s.bkey + b));
          }
        } else {
          // queue entry = epoch and claim index in one word; the tail count is
          // ordered before this warp's pbm_done increment
          const int slot = atomicAdd(&ctrl->fs_tail, 1);
          atomicExch(q + slot, ((unsigned long long)(uint32_t)epoch << 32) | (uint32_t)i);
        }
        __threadfence();
        atomicAdd(&ctrl->pbm_done, 1);
        // the next claim, once this block is out of the warp's hands
        nxt = atomicAdd(&ctrl->next, 1);
        inxt = nxt < total ? items[nxt] : 0;
      }
      __syncwarp();
    }
  } else {
    // ---------------------------------------------------------------- search CTAs
    for (;;) {
      if (tid == 0) {
        const int slot = atomicAdd(&ctrl->fs_head, 1);
        // the queue holds at most `total` entries: a slot beyond can never be
        // filled, so the CTA is done without touching it
        const volatile unsigned long long* rd = q + (slot < total ? slot : 0);
        const volatile int* done = &ctrl->pbm_done;
        const volatile int* tail = &ctrl->fs_tail;
        const volatile int* err = &ctrl->error;
        const long long t0 = global_ns();
        int got = -1;
        for (;;) {
          if (slot >= total) break;
          const unsigned long long e = *rd;
          if (pub_epoch(e) == epoch) { got = (int)(uint32_t)e; break; }
          if (*done == total && *tail <= slot) break;     // no more blocks will come
          if (*err != 0) break;
          if (global_ns() - t0 > timeout) {
            atomicExch(&ctrl->error, (int)ME_ERR_TIMEOUT);
            break;
          }
          __nanosleep(32);
        }
        // a claim index beyond the table is not an item of this step
        const int ci = got & ~kBatchSpecBit;
        s_item = got < 0 ? ~0ull : (ci < total ? items[ci] : ~1ull);
        s_spec = got >= 0 && (got & kBatchSpecBit) != 0;
      }
      __syncthreads();
      const unsigned long long it = s_item;
      const bool specj = s_spec != 0;
      if (it == ~0ull) break;
      const int si = (int)(it >> 32), b = (int)(uint32_t)it;
      if (it == ~1ull || si < 0 || si >= nstreams || b < 0 ||
          b >= (shp[si].W / N) * (shp[si].H / M)) {
        // not a block of this step: report it instead of touching memory
        if (tid == 0) atomicExch(&ctrl->error, (int)ME_ERR_CUDA);
        __syncthreads();
        continue;
      }
      const BShape& s = shp[si];
      const BStream& a = st[si];
      const int BW = s.W / N;
      const FsGeom g = fs_geom<N, M, T>(s.p, 1, blockDim.x);
      // window staged from the stream's padded reference (written by this
      // step's prologue) with one round of asynchronous copies
      fs_group<N, M, T>(a.cur, a.ref, s.W, s.H, (b % BW) * N, (b / BW) * M, g, a.lam, smem, keys,
                        nullptr, FsPad{s.refpad, s.pg.pitch, s.pg.P, s.pg.rows});
      if (tid == 0) {
        bool pub = true;
        if (specj) {
          // published by this CTA only if the block has failed PBM already
          s.bkey[b] = keys[0];
          __threadfence();
          pub = (atomicOr(s.bstate + b, kBatchSearched) & kBatchFailed) != 0;
        }
        if (pub) batch_publish_fs(s, a, ctrl, epoch, si, b, keys[0]);
      }
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------ host side


template <int N, int M, int T>
inline size_t smem_of(int p, int bpc) {
  return fs_smem_bytes<N, M, T>(fs_geom<N, M, T>(p, bpc, 32));
}

// Dispatch over the instantiated (N, M, T) of the persistent kernels.
#define ME_BATCH_NMT(X)                                                             \
  X(16, 16, 8) X(16, 16, 11) X(16, 16, 13) X(16, 16, 16) X(16, 8, 8) X(16, 4, 8)    \
  X(8, 16, 8) X(8, 8, 8) X(8, 4, 8) X(4, 16, 8) X(4, 8, 8) X(4, 4, 8)

inline size_t batch_smem(int N, int M, int T, int p, int bpc) {
#define X(n, m, t) if (N == n && M == m && T == t) return smem_of<n, m, t>(p, bpc);
  ME_BATCH_NMT(X)
#undef X
  return 0;
}


// Run length for a set of streams: fewest wasted candidate rows, weighted by
// each stream's block count (16x16 blocks choose among 8, 11, 13, 16).
int batch_choose_T(int N, int M, const std::vector<BShape>& shapes);

// Enqueues one ACBM step over the streams in the device tables: the begin
// kernel (epoch = `epoch`, or the previous epoch + 1 when epoch <= 0), the
// item table, the padding and Intra_SAD prologue, and the persistent kernel.
// items and q hold at least total_items entries (q: no entry may carry the
// step's epoch before the step); smem and the PBM warp count come from
// acbm_step_smem for the largest search range p_max.
int launch_acbm_step(int N, int M, int T, BCtrl* ctrl, int epoch, const BShape* shapes,
                     const BStream* streams, int nstreams, long long total_pad, int total_blocks,
                     const BSegment* segs, int nseg, int total_items, size_t smem, int p_max,
                     unsigned long long* items, unsigned long long* q, cudaStream_t s,
                     int spec = 0);

// Dynamic shared memory of the ACBM step kernel for search ranges up to p_max.
size_t acbm_step_smem(int N, int M, int T, int p_max);

// Enqueues one FSBM step (begin kernel + persistent kernel).
int launch_fsbm_step(int N, int M, int T, BCtrl* ctrl, int epoch, const BShape* shapes,
                     const BStream* streams, const BFsEntry* ent, int nent, size_t smem,
                     cudaStream_t s);

// Enqueues one FSBM step through the pipelined search at any p (begin kernel
// + k_fsbm_pipe_tab over the group table `ent`, groups of at most
// pipe_tab_bpc(N, p) blocks, claimed from ctrl->next).
int launch_fsbm_tab_step(int N, int M, BCtrl* ctrl, int epoch, const BShape* shapes,
                         const BStream* streams, const BFsEntry* ent, int nent, cudaStream_t s);

// Run lengths worth timing for a set of streams: batch_choose_T's and those
// whose modelled waste is within 10 % of it (model first).
std::vector<int> batch_Ts(int N, int M, const std::vector<BShape>& shapes);

}  // namespace me

// me_batch.cu -- many independent streams of uneven size in one persistent
// launch per step (FSBM or ACBM), captured once into a CUDA graph.
//
// A step is: k_batch_begin (new epoch, reset the work counter), k_batch_pad and
// k_batch_intra (padded references and scaled Intra_SAD of every stream), then
// one persistent kernel whose CTAs pull work items from a global counter:
//   FSBM: items are groups of adjacent blocks of one block row of one stream,
//         largest search ranges first;
//   ACBM: items are single blocks, ordered by anti-diagonal wave w = x + 2y
//         (all streams' wave 0, then wave 1, ...).  A block waits (bounded) until
//         its left, up-left, up and up-right neighbours are final, then runs
//         PBM and the Sec. 3.2 test with one warp and, if it fails, the full
//         search with the whole CTA, and publishes its vector.
// Items are claimed in an order in which every dependency comes first, and a
// CTA never waits for a later item, so the waits always end (each one is also
// bounded in time and reports ME_ERR_TIMEOUT instead of hanging).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "me_device.cuh"
#include "me_host.h"
#include "me_search.cuh"

namespace me {

struct BStream {  // per-run arguments of one stream (copied to the device each run)
  const uint8_t* cur;
  const uint8_t* ref;
  const int16_t* prev;
  int16_t* mv;
  uint32_t* J;
  uint8_t* mask;
  uint32_t* sad;
  uint32_t* load;
  uint32_t lam;
  int32_t alpha, beta, gnum, gden, qp, refine;
};

struct BShape {  // fixed per stream
  int W, H, p;
  PadGeom pg;
  uint8_t* refpad;
  uint32_t* intra;
  int* flags;
  long long pad_base;  // first 16-byte chunk of this stream in the flat pad index
  int blk_base;        // first block of this stream in the flat block index
};

struct BSegment {  // ACBM: the blocks of one wave of one stream
  int stream, wave, ylo, count, item_base;
};

struct BFsEntry {  // FSBM: one group of adjacent blocks, G threads per block
  int stream, by, bx0, nb, G;
};

struct BCtrl {
  int epoch;
  int next;
  int error;
  int err_item;
  long long timeout_ns;
  int skip_stream, skip_block;  // fault injection: never publish this block
};

__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void k_batch_begin(BCtrl* c) {
  c->epoch += 1;
  c->next = 0;
  c->error = 0;
  c->err_item = -1;
}

__global__ void k_batch_pad(const BShape* __restrict__ shp, const BStream* __restrict__ st,
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
    if (lane == 0) s.intra[b] = v;
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

template <int N, int M, int T>
__global__ void __launch_bounds__(256, 2) k_acbm_persist(const BShape* __restrict__ shp,
                                                      const BStream* __restrict__ st,
                                                      const BSegment* __restrict__ seg, int nseg,
                                                      int total, BCtrl* ctrl) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ unsigned long long keys[16];
  __shared__ uint32_t curs[M * (N / 4)];
  __shared__ int s_item, s_stream, s_b, s_pass, s_load;
  __shared__ unsigned long long s_key;
  const int tid = threadIdx.x, lane = tid & 31;
  const int epoch = *reinterpret_cast<volatile int*>(&ctrl->epoch);
  const long long timeout = ctrl->timeout_ns;
  for (;;) {
    if (tid == 0) {
      const int i = atomicAdd(&ctrl->next, 1);
      s_item = i;
      if (i < total) {
        int lo = 0, hi = nseg - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) / 2;
          if (seg[mid].item_base <= i) lo = mid; else hi = mid - 1;
        }
        const BSegment sg = seg[lo];
        const int by = sg.ylo + (i - sg.item_base);
        const int bx = sg.wave - 2 * by;
        s_stream = sg.stream;
        s_b = by * (shp[sg.stream].W / N) + bx;
      }
    }
    __syncthreads();
    if (s_item >= total) break;
    const int si = s_stream, b = s_b;
    const BShape& s = shp[si];
    const BStream& a = st[si];
    const int BW = s.W / N;
    const int bx = b % BW, by = b / BW;
    if (tid < 32) {
      // wait until the spatial predictors are final (bounded)
      if (lane < 4) {
        const int dx = (lane < 2) ? -1 : (lane == 2 ? 0 : 1);
        const int dy = (lane == 0) ? 0 : -1;
        const int nx = bx + dx, ny = by + dy;
        if (nx >= 0 && nx < BW && ny >= 0) {
          const volatile int* f = s.flags + ny * BW + nx;
          const volatile int* err = &ctrl->error;
          const long long t0 = global_ns();
          // after the first wait that gave up, no other wait starts: the step
          // finishes quickly and reports the error
          while (*f != epoch && *err == 0) {
            if (global_ns() - t0 > timeout) {
              atomicExch(&ctrl->error, (int)ME_ERR_TIMEOUT);
              atomicExch(&ctrl->err_item, s_item);
              break;
            }
            __nanosleep(64);
          }
        }
      }
      __syncwarp();
      __threadfence();
      const PbmResult r = warp_pbm<N, M>(a.cur, s.refpad, s.pg, s.W, s.H, s.p, a.lam, a.mv, a.prev,
                                         bx, by, s.intra[b], a.alpha, a.beta, a.gnum, a.gden, a.qp,
                                         a.refine, curs);
      if (lane == 0) {
        s_key = r.key;
        s_pass = r.pass ? 1 : 0;
        s_load = r.load;
      }
    }
    __syncthreads();
    const bool pass = s_pass != 0;
    unsigned long long key = s_key;
    if (!pass) {
      const FsGeom g = fs_geom<N, M, T>(s.p, 1, blockDim.x);
      fs_group<N, M, T>(a.cur, a.ref, s.W, s.H, bx * N, by * M, g, a.lam, smem, keys);
      key = keys[0];
    }
    if (tid == 0) {
      const Decoded d = decode_key(key, s.p, a.lam);
      a.mv[2 * b] = (int16_t)d.mvx;
      a.mv[2 * b + 1] = (int16_t)d.mvy;
      a.J[b] = d.J;
      a.mask[b] = pass ? 0 : 1;
      if (a.sad) a.sad[b] = d.sad;
      if (a.load) a.load[b] = pass ? (uint32_t)s_load : (uint32_t)((2 * s.p + 1) * (2 * s.p + 1));
      __threadfence();
      if (!(si == ctrl->skip_stream && b == ctrl->skip_block)) atomicExch(s.flags + b, epoch);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ host side

static const int kBatchThreads = 256;

template <int N, int M, int T>
static size_t smem_of(int p, int bpc) {
  return fs_smem_bytes<N, M, T>(fs_geom<N, M, T>(p, bpc, 32));
}

// Dispatch over the instantiated (N, M, T) of the persistent kernels.
#define ME_BATCH_NMT(X)                                                             \
  X(16, 16, 8) X(16, 16, 11) X(16, 16, 13) X(16, 16, 16) X(16, 8, 8) X(16, 4, 8)    \
  X(8, 16, 8) X(8, 8, 8) X(8, 4, 8) X(4, 16, 8) X(4, 8, 8) X(4, 4, 8)

static size_t batch_smem(int N, int M, int T, int p, int bpc) {
#define X(n, m, t) if (N == n && M == m && T == t) return smem_of<n, m, t>(p, bpc);
  ME_BATCH_NMT(X)
#undef X
  return 0;
}

}  // namespace me

struct me_batch {
  int device = -1;
  int N = 0, M = 0, T = 8;
  bool started = false;
  std::vector<me::BShape> shapes;       // host copy (device pointers inside)
  std::vector<me::BSegment> segs;
  std::vector<me::BFsEntry> fsent;
  int total_items = 0, total_blocks = 0;
  long long total_pad = 0;
  size_t smem_fs = 0, smem_acbm = 0;
  int grid_fs = 0, grid_acbm = 0;
  // device memory
  void* dmem = nullptr;
  me::BShape* d_shapes = nullptr;
  me::BStream* d_streams = nullptr;
  me::BSegment* d_segs = nullptr;
  me::BFsEntry* d_fsent = nullptr;
  me::BCtrl* d_ctrl = nullptr;
  static constexpr int kRing = 4;       // staging buffers in flight
  me::BStream* h_streams = nullptr;     // pinned staging of the per-run arguments [kRing][n]
  me::BCtrl* h_ctrl = nullptr;          // pinned read-back of the control block
  cudaEvent_t staged[kRing] = {};       // the staging copy from ring slot i is done
  int ring = 0;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaGraph_t graph[2] = {nullptr, nullptr};
  long long timeout_ns = 1000000000ll;  // 1 s per wait
  int skip_stream = -1, skip_block = -1;
};

namespace me {

static int batch_finalize(me_batch* b) {
  // T: the run length that wastes the fewest candidate rows, weighted by work
  static const int kT16b[] = {8, 11, 13, 16};
  if (b->N == 16 && b->M == 16) {
    double best = 1e300;
    for (int T : kT16b) {
      double waste = 0;
      for (const BShape& s : b->shapes) {
        const int n = 2 * s.p + 1, nseg = (n + T - 1) / T;
        const double blocks = (double)(s.W / b->N) * (s.H / b->M);
        waste += blocks * n * (nseg * T + b->M - 1) * (1.0 + 4.0 / T);
      }
      if (waste < best * 0.999) { best = waste; b->T = T; }
    }
  } else {
    b->T = 8;
  }
  // FSBM work entries: threads per block (and so blocks per CTA) per stream
  b->fsent.clear();
  size_t smem_fs = 0;
  for (int si = 0; si < (int)b->shapes.size(); si++) {
    const BShape& s = b->shapes[si];
    const int BW = s.W / b->N, BH = s.H / b->M;
    const FsPlan pl = fs_plan_fixed(b->N, b->M, b->T, s.p, kBatchThreads, BW, 110 * 1024);
    const int bpc = kBatchThreads / pl.G;
    smem_fs = std::max(smem_fs, pl.smem);
    for (int by = 0; by < BH; by++)
      for (int bx0 = 0; bx0 < BW; bx0 += bpc)
        b->fsent.push_back(BFsEntry{si, by, bx0, std::min(bpc, BW - bx0), pl.G});
  }
  // largest work first
  std::stable_sort(b->fsent.begin(), b->fsent.end(), [&](const BFsEntry& x, const BFsEntry& y) {
    const int px = b->shapes[x.stream].p, py = b->shapes[y.stream].p;
    return (long long)px * px * x.nb > (long long)py * py * y.nb;
  });
  b->smem_fs = smem_fs;
  // ACBM segments: wave-major across streams
  b->segs.clear();
  int maxw = 0;
  for (const BShape& s : b->shapes) maxw = std::max(maxw, make_waves(s.W / b->N, s.H / b->M).n);
  int base = 0;
  for (int w = 0; w < maxw; w++) {
    for (int si = 0; si < (int)b->shapes.size(); si++) {
      const BShape& s = b->shapes[si];
      const Waves wv = make_waves(s.W / b->N, s.H / b->M);
      if (w >= wv.n) continue;
      const int c = wv.count(w);
      if (c == 0) continue;
      b->segs.push_back(BSegment{si, w, wv.ylo(w), c, base});
      base += c;
    }
  }
  b->total_items = base;
  size_t smem_a = 0;
  for (const BShape& s : b->shapes) smem_a = std::max(smem_a, batch_smem(b->N, b->M, b->T, s.p, 1));
  b->smem_acbm = smem_a;
  // device memory: control, tables, per-stream scratch
  const size_t n = b->shapes.size();
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
  const size_t o_ctrl = take(sizeof(BCtrl));
  const size_t o_shapes = take(sizeof(BShape) * n);
  const size_t o_streams = take(sizeof(BStream) * n);
  const size_t o_segs = take(sizeof(BSegment) * b->segs.size());
  const size_t o_fsent = take(sizeof(BFsEntry) * b->fsent.size());
  std::vector<size_t> o_pad(n), o_intra(n), o_flags(n);
  b->total_pad = 0;
  b->total_blocks = 0;
  for (size_t i = 0; i < n; i++) {
    BShape& s = b->shapes[i];
    const int nb = (s.W / b->N) * (s.H / b->M);
    o_pad[i] = take((size_t)s.pg.pitch * s.pg.rows);
    o_intra[i] = take(4 * (size_t)nb);
    o_flags[i] = take(4 * (size_t)nb);
    s.pad_base = b->total_pad;
    s.blk_base = b->total_blocks;
    b->total_pad += (long long)s.pg.rows * (s.pg.pitch / 16);
    b->total_blocks += nb;
  }
  ME_CUDA(cudaMalloc(&b->dmem, off));
  ME_CUDA(cudaMemset(b->dmem, 0, off));
  uint8_t* base8 = static_cast<uint8_t*>(b->dmem);
  for (size_t i = 0; i < n; i++) {
    b->shapes[i].refpad = base8 + o_pad[i];
    b->shapes[i].intra = reinterpret_cast<uint32_t*>(base8 + o_intra[i]);
    b->shapes[i].flags = reinterpret_cast<int*>(base8 + o_flags[i]);
  }
  b->d_ctrl = reinterpret_cast<BCtrl*>(base8 + o_ctrl);
  b->d_shapes = reinterpret_cast<BShape*>(base8 + o_shapes);
  b->d_streams = reinterpret_cast<BStream*>(base8 + o_streams);
  b->d_segs = reinterpret_cast<BSegment*>(base8 + o_segs);
  b->d_fsent = reinterpret_cast<BFsEntry*>(base8 + o_fsent);
  ME_CUDA(cudaMemcpy(b->d_shapes, b->shapes.data(), sizeof(BShape) * n, cudaMemcpyHostToDevice));
  if (!b->segs.empty())
    ME_CUDA(cudaMemcpy(b->d_segs, b->segs.data(), sizeof(BSegment) * b->segs.size(),
                       cudaMemcpyHostToDevice));
  if (!b->fsent.empty())
    ME_CUDA(cudaMemcpy(b->d_fsent, b->fsent.data(), sizeof(BFsEntry) * b->fsent.size(),
                       cudaMemcpyHostToDevice));
  BCtrl c;
  std::memset(&c, 0, sizeof(c));
  c.timeout_ns = b->timeout_ns;
  c.skip_stream = b->skip_stream;
  c.skip_block = b->skip_block;
  ME_CUDA(cudaMemcpy(b->d_ctrl, &c, sizeof(c), cudaMemcpyHostToDevice));
  ME_CUDA(cudaMallocHost(&b->h_streams, sizeof(BStream) * n * me_batch::kRing));
  ME_CUDA(cudaMallocHost(&b->h_ctrl, sizeof(BCtrl)));
  for (int i = 0; i < me_batch::kRing; i++)
    ME_CUDA(cudaEventCreateWithFlags(&b->staged[i], cudaEventDisableTiming));
  // persistent grids: as many CTAs as fit on the device at once
  int dev = 0, nsm = 0;
  ME_CUDA(cudaGetDevice(&dev));
  ME_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  b->device = dev;
  auto occ_grid = [&](const void* fn, size_t smem, int* grid) -> int {
    ME_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    ME_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBatchThreads, smem));
    *grid = std::max(1, per_sm) * nsm;
    return ME_OK;
  };
  int st = ME_ERR_ARG;
#define X(n_, m_, t_)                                                                          \
  if (b->N == n_ && b->M == m_ && b->T == t_) {                                                \
    st = occ_grid((const void*)k_fsbm_persist<n_, m_, t_>, b->smem_fs, &b->grid_fs);           \
    if (st == ME_OK)                                                                           \
      st = occ_grid((const void*)k_acbm_persist<n_, m_, t_>, b->smem_acbm, &b->grid_acbm);     \
  }
  ME_BATCH_NMT(X)
#undef X
  return st;
}

// Enqueues one step of `mode` (no argument staging).
static int batch_enqueue(me_batch* b, int mode, cudaStream_t s) {
  const int ns = (int)b->shapes.size();
  k_batch_begin<<<1, 1, 0, s>>>(b->d_ctrl);
  ME_CUDA(cudaGetLastError());
  if (mode == ME_MODE_ACBM) {
    const long long chunks = b->total_pad;
    const int grid = (int)std::min<long long>((chunks + 255) / 256, 152 * 16);
    k_batch_pad<<<grid, 256, 0, s>>>(b->d_shapes, b->d_streams, ns, chunks);
    ME_CUDA(cudaGetLastError());
    const int gi = std::min((b->total_blocks + 7) / 8, 152 * 16);
#define X(n_, m_)                                                                              \
  if (b->N == n_ && b->M == m_)                                                                \
    k_batch_intra<n_, m_><<<gi, 256, 0, s>>>(b->d_shapes, b->d_streams, ns, b->total_blocks);
    X(16, 16) X(16, 8) X(16, 4) X(8, 16) X(8, 8) X(8, 4) X(4, 16) X(4, 8) X(4, 4)
#undef X
    ME_CUDA(cudaGetLastError());
  }
#define X(n_, m_, t_)                                                                          \
  if (b->N == n_ && b->M == m_ && b->T == t_) {                                                \
    if (mode == ME_MODE_FSBM)                                                                  \
      k_fsbm_persist<n_, m_, t_><<<b->grid_fs, kBatchThreads, b->smem_fs, s>>>(                \
          b->d_shapes, b->d_streams, b->d_fsent, (int)b->fsent.size(), b->d_ctrl);             \
    else                                                                                       \
      k_acbm_persist<n_, m_, t_><<<b->grid_acbm, kBatchThreads, b->smem_acbm, s>>>(            \
          b->d_shapes, b->d_streams, b->d_segs, (int)b->segs.size(), b->total_items,           \
          b->d_ctrl);                                                                          \
  }
  ME_BATCH_NMT(X)
#undef X
  ME_CUDA(cudaGetLastError());
  return ME_OK;
}

}  // namespace me

using namespace me;

extern "C" {

int me_batch_create(me_batch** out) {
  if (!out) return ME_ERR_ARG;
  *out = new (std::nothrow) me_batch();
  return *out ? ME_OK : ME_ERR_NOMEM;
}

int me_batch_add_stream(me_batch* b, int W, int H, int N, int M, int p, int* index) {
  if (!b || b->started) return ME_ERR_ARG;
  int st = check_frame_args(W, H, N, M, p, 0);
  if (st) return st;
  if (!b->shapes.empty() && (N != b->N || M != b->M)) return ME_ERR_ARG;
  b->N = N;
  b->M = M;
  BShape s;
  std::memset(&s, 0, sizeof(s));
  s.W = W;
  s.H = H;
  s.p = p;
  s.pg = pad_geom(W, H, p);
  b->shapes.push_back(s);
  if (index) *index = (int)b->shapes.size() - 1;
  return ME_OK;
}

int me_batch_run(me_batch* b, int mode, const me_batch_item* items, int n_items,
                 me_stream_t stream) {
  if (!b || !items || b->shapes.empty() || n_items != (int)b->shapes.size()) return ME_ERR_ARG;
  if (mode != ME_MODE_FSBM && mode != ME_MODE_ACBM) return ME_ERR_ARG;
  for (int i = 0; i < n_items; i++) {
    const me_batch_item& it = items[i];
    if (!it.cur || !it.ref || !it.mv_out || !it.J_out) return ME_ERR_ARG;
    if (!aligned4(it.cur) || !aligned4(it.ref)) return ME_ERR_ARG;
    if (it.lambda_q8 > (1u << 20)) return ME_ERR_ARG;
    if (mode == ME_MODE_ACBM) {
      if (!it.mask_out) return ME_ERR_ARG;
      int st = check_acbm_params(&it.prm);
      if (st) return st;
    }
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!b->started) {
    int st = batch_finalize(b);
    if (st) return st;
    b->started = true;
  }
  int dev = 0;
  ME_CUDA(cudaGetDevice(&dev));
  if (dev != b->device) return ME_ERR_ARG;
  // a ring slot is reused only after the copy that last read it has run
  const int slot = b->ring;
  b->ring = (b->ring + 1) % me_batch::kRing;
  ME_CUDA(cudaEventSynchronize(b->staged[slot]));
  BStream* hs = b->h_streams + (size_t)slot * b->shapes.size();
  for (int i = 0; i < n_items; i++) {
    const me_batch_item& it = items[i];
    BStream& a = hs[i];
    a.cur = it.cur; a.ref = it.ref; a.prev = it.prev_mv;
    a.mv = it.mv_out; a.J = it.J_out; a.mask = it.mask_out; a.sad = it.sad_out;
    a.load = it.load_out; a.lam = it.lambda_q8;
    a.alpha = it.prm.alpha; a.beta = it.prm.beta; a.gnum = it.prm.gamma_num;
    a.gden = it.prm.gamma_den; a.qp = it.prm.qp; a.refine = it.prm.refine;
  }
  ME_CUDA(cudaMemcpyAsync(b->d_streams, hs, sizeof(BStream) * n_items, cudaMemcpyHostToDevice, s));
  ME_CUDA(cudaEventRecord(b->staged[slot], s));
  const int gi = mode == ME_MODE_ACBM ? 1 : 0;
  if (!b->exec[gi]) {
    // capture the step once on a private stream, then replay it
    cudaStream_t cs;
    ME_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    ME_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int st = batch_enqueue(b, mode, cs);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (st) return st;
    ME_CUDA(e);
    b->graph[gi] = g;
    ME_CUDA(cudaGraphInstantiate(&b->exec[gi], g, 0));
  }
  ME_CUDA(cudaGraphLaunch(b->exec[gi], s));
  ME_CUDA(cudaMemcpyAsync(b->h_ctrl, b->d_ctrl, sizeof(BCtrl), cudaMemcpyDeviceToHost, s));
  return ME_OK;
}

int me_batch_sync(me_batch* b, me_stream_t stream) {
  if (!b) return ME_ERR_ARG;
  if (!b->started) return ME_OK;
  ME_CUDA(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
  return b->h_ctrl->error ? b->h_ctrl->error : ME_OK;
}

int me_batch_set_fault(me_batch* b, long long timeout_ns, int skip_stream, int skip_block) {
  if (!b || b->started || timeout_ns <= 0) return ME_ERR_ARG;
  b->timeout_ns = timeout_ns;
  b->skip_stream = skip_stream;
  b->skip_block = skip_block;
  return ME_OK;
}

void me_batch_destroy(me_batch* b) {
  if (!b) return;
  for (int i = 0; i < 2; i++) {
    if (b->exec[i]) cudaGraphExecDestroy(b->exec[i]);
    if (b->graph[i]) cudaGraphDestroy(b->graph[i]);
  }
  for (int i = 0; i < me_batch::kRing; i++)
    if (b->staged[i]) {
      cudaEventSynchronize(b->staged[i]);
      cudaEventDestroy(b->staged[i]);
    }
  if (b->dmem) {
    cudaDeviceSynchronize();
    cudaFree(b->dmem);
  }
  if (b->h_streams) cudaFreeHost(b->h_streams);
  if (b->h_ctrl) cudaFreeHost(b->h_ctrl);
  delete b;
}

}  // extern "C"

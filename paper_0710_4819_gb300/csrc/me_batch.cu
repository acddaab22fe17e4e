// me_batch.cu -- many independent streams of uneven size in one persistent
// launch per step (FSBM or ACBM), captured once into a CUDA graph.
//
// A step is: k_batch_begin (new epoch, reset the work counter), k_batch_pad and
// k_batch_intra (padded references and scaled Intra_SAD of every stream), then
// one persistent kernel whose CTAs pull work items from a global counter:
//   FSBM: items are groups of adjacent blocks of one block row of one stream,
//         largest search ranges first (the per-group kernel, or the table-
//         driven pipelined search of me_sequence.cu, whichever the tuner
//         measured faster);
//   ACBM: items are single blocks, ordered by anti-diagonal wave w = x + 2y
//         (all streams' wave 0, then wave 1, ...).  PBM warps claim blocks,
//         run part a of PBM, queue a likely fallback's full search at once,
//         wait (bounded) until the left, up-left, up and up-right neighbours
//         are final, finish PBM and the Sec. 3.2 test and publish; search
//         CTAs take queued blocks and search each in full.
// Items are claimed in an order in which every dependency comes first, and a
// CTA never waits for a later item, so the waits always end (each one is also
// bounded in time and reports ME_ERR_TIMEOUT instead of hanging).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "me_batch.cuh"


struct me_batch {
  int device = -1;
  int N = 0, M = 0, T = 8;
  bool started = false;
  std::vector<me::BShape> shapes;       // host copy (device pointers inside)
  std::vector<me::BSegment> segs;
  std::vector<me::BFsEntry> fsent;
  std::vector<me::BFsEntry> fsent_tab;  // groups of the pipelined search (16x16 only)
  // step forms the autotuner chooses among, per mode (0 FSBM, 1 ACBM)
  std::vector<int> acbm_Ts;             // ACBM: run lengths
  std::vector<size_t> acbm_smem;        //   and their shared memory
  int form[2] = {-1, -1};               // chosen candidate, -1: not yet
  int total_items = 0, total_blocks = 0;
  long long total_pad = 0;
  size_t smem_fs = 0, smem_acbm = 0;
  // device memory
  void* dmem = nullptr;
  me::BShape* d_shapes = nullptr;
  me::BStream* d_streams = nullptr;
  me::BSegment* d_segs = nullptr;
  me::BFsEntry* d_fsent = nullptr;
  me::BFsEntry* d_fsent_tab = nullptr;
  me::BCtrl* d_ctrl = nullptr;
  unsigned long long* d_items = nullptr;   // claim order of the ACBM step
  unsigned long long* d_q = nullptr;       // full-search queue of the ACBM step
  int p_max = 1;
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

// Occupancy-sized persistent grids, cached per kernel and dynamic smem size.
static std::mutex g_grid_mu;
struct GridKey {
  const void* fn;
  size_t smem;
  int dev, grid;
};
static std::vector<GridKey> g_grids;

static int persistent_grid(const void* fn, size_t smem, int* grid) {
  int dev = 0;
  ME_CUDA(cudaGetDevice(&dev));
  int st = ensure_dynamic_smem(fn, smem);   // every launch path raises, never lowers
  if (st) return st;
  std::lock_guard<std::mutex> lk(g_grid_mu);
  for (const GridKey& k : g_grids)
    if (k.fn == fn && k.smem == smem && k.dev == dev) {
      *grid = k.grid;
      return ME_OK;
    }
  int nsm = 0, per_sm = 0;
  ME_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  ME_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBatchThreads, smem));
  *grid = std::max(1, per_sm) * nsm;
  g_grids.push_back(GridKey{fn, smem, dev, *grid});
  return ME_OK;
}

static double batch_T_waste(int N, int M, const std::vector<BShape>& shapes, int T) {
  double waste = 0;
  for (const BShape& s : shapes) {
    const int n = 2 * s.p + 1, nseg = (n + T - 1) / T;
    const double blocks = (double)(s.W / N) * (s.H / M);
    waste += blocks * n * (nseg * T + M - 1) * (1.0 + 4.0 / T);
  }
  return waste;
}

int batch_choose_T(int N, int M, const std::vector<BShape>& shapes) {
  static const int kT16b[] = {8, 11, 13, 16};
  if (!(N == 16 && M == 16)) return 8;
  int bestT = 13;
  double best = 1e300;
  for (int T : kT16b) {
    const double waste = batch_T_waste(N, M, shapes, T);
    if (waste < best * 0.999) { best = waste; bestT = T; }
  }
  return bestT;
}

std::vector<int> batch_Ts(int N, int M, const std::vector<BShape>& shapes) {
  const int T0 = batch_choose_T(N, M, shapes);
  std::vector<int> out{T0};
  if (!(N == 16 && M == 16)) return out;
  static const int kT16b[] = {8, 11, 13, 16};
  const double w0 = batch_T_waste(N, M, shapes, T0);
  for (int T : kT16b)
    if (T != T0 && batch_T_waste(N, M, shapes, T) <= 1.10 * w0) out.push_back(T);
  return out;
}

size_t acbm_step_smem(int N, int M, int T, int p_max) {
  const size_t pbm =
      (size_t)4 * batch_pbm_warps(N, M, p_max) * (pbm_win_words(N, M, p_max) + M * (N / 4));
  return std::max(batch_smem(N, M, T, p_max, 1), pbm);
}

int launch_acbm_step(int N, int M, int T, BCtrl* ctrl, int epoch, const BShape* shapes,
                     const BStream* streams, int nstreams, long long total_pad, int total_blocks,
                     const BSegment* segs, int nseg, int total_items, size_t smem, int p_max,
                     unsigned long long* items, unsigned long long* q, cudaStream_t s, int spec) {
  int nsm = 1;
  { const int e = sm_count(&nsm); if (e) return e; }
  k_batch_begin<<<1, 256, 0, s>>>(ctrl, epoch);
  ME_CUDA(cudaGetLastError());
  if (total_items > 0) {
    const int gt = std::max(1, std::min((total_items + 255) / 256, nsm * 8));
    k_batch_items<<<gt, 256, 0, s>>>(segs, nseg, total_items, shapes, N, items);
    ME_CUDA(cudaGetLastError());
  }
  const int gp = (int)std::max<long long>(1, std::min<long long>((total_pad + 255) / 256, nsm * 16LL));
  k_batch_pad<<<gp, 256, 0, s>>>(shapes, streams, nstreams, total_pad);
  ME_CUDA(cudaGetLastError());
  const int gi = std::max(1, std::min((total_blocks + 7) / 8, nsm * 16));
  int st = ME_ERR_ARG;
#define X(n_, m_)                                                                              \
  if (N == n_ && M == m_) {                                                                    \
    k_batch_intra<n_, m_><<<gi, 256, 0, s>>>(shapes, streams, nstreams, total_blocks);         \
    st = ME_OK;                                                                                \
  }
  X(16, 16) X(16, 8) X(16, 4) X(8, 16) X(8, 8) X(8, 4) X(4, 16) X(4, 8) X(4, 4)
#undef X
  if (st) return st;
  ME_CUDA(cudaGetLastError());
  // half the CTAs run PBM warps, half the full searches: two per SM
  const int pw = batch_pbm_warps(N, M, p_max);
  const int ww = pbm_win_words(N, M, p_max);
  st = ME_ERR_ARG;
#define X(n_, m_, t_)                                                                          \
  if (N == n_ && M == m_ && T == t_) {                                                         \
    int grid = 0;                                                                              \
    st = persistent_grid((const void*)k_acbm_persist<n_, m_, t_>, smem, &grid);                \
    if (st == ME_OK && grid < 2 * nsm) st = ME_ERR_CUDA;  /* needs two CTAs per SM */         \
    if (st == ME_OK)                                                                           \
      k_acbm_persist<n_, m_, t_><<<2 * nsm, kBatchThreads, smem, s>>>(                         \
          shapes, streams, items, total_items, ctrl, q, pw, ww, nsm, nstreams, spec);          \
  }
  ME_BATCH_NMT(X)
#undef X
  if (st) return st;
  ME_CUDA(cudaGetLastError());
  return ME_OK;
}

int launch_fsbm_step(int N, int M, int T, BCtrl* ctrl, int epoch, const BShape* shapes,
                     const BStream* streams, const BFsEntry* ent, int nent, size_t smem,
                     cudaStream_t s) {
  k_batch_begin<<<1, 256, 0, s>>>(ctrl, epoch);
  ME_CUDA(cudaGetLastError());
  int st = ME_ERR_ARG;
#define X(n_, m_, t_)                                                                          \
  if (N == n_ && M == m_ && T == t_) {                                                         \
    int grid = 0;                                                                              \
    st = persistent_grid((const void*)k_fsbm_persist<n_, m_, t_>, smem, &grid);                \
    if (st == ME_OK)                                                                           \
      k_fsbm_persist<n_, m_, t_><<<grid, kBatchThreads, smem, s>>>(shapes, streams, ent, nent,  \
                                                                   ctrl);                      \
  }
  ME_BATCH_NMT(X)
#undef X
  if (st) return st;
  ME_CUDA(cudaGetLastError());
  return ME_OK;
}

int launch_fsbm_tab_step(int N, int M, BCtrl* ctrl, int epoch, const BShape* shapes,
                         const BStream* streams, const BFsEntry* ent, int nent, cudaStream_t s) {
  k_batch_begin<<<1, 256, 0, s>>>(ctrl, epoch);
  ME_CUDA(cudaGetLastError());
  return launch_pipe_tab_batch(N, M, shapes, streams, ent, nent, &ctrl->next, &ctrl->error, s);
}

static int batch_finalize(me_batch* b) {
  b->T = batch_choose_T(b->N, b->M, b->shapes);
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
  // groups of the pipelined search, largest work first
  b->fsent_tab.clear();
  if (pipe_tab_applies(b->N, b->M, 1)) {
    for (int si = 0; si < (int)b->shapes.size(); si++) {
      const BShape& s = b->shapes[si];
      const int BW = s.W / b->N, BH = s.H / b->M, bpc = pipe_tab_bpc(b->N, s.p);
      for (int by = 0; by < BH; by++)
        for (int bx0 = 0; bx0 < BW; bx0 += bpc)
          b->fsent_tab.push_back(BFsEntry{si, by, bx0, std::min(bpc, BW - bx0), 0});
    }
    std::stable_sort(b->fsent_tab.begin(), b->fsent_tab.end(),
                     [&](const BFsEntry& x, const BFsEntry& y) {
                       const long long nx = 2 * b->shapes[x.stream].p + 1;
                       const long long ny = 2 * b->shapes[y.stream].p + 1;
                       return nx * nx * x.nb > ny * ny * y.nb;
                     });
  }
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
  b->p_max = 1;
  for (const BShape& s : b->shapes) b->p_max = std::max(b->p_max, s.p);
  b->smem_acbm = acbm_step_smem(b->N, b->M, b->T, b->p_max);
  b->acbm_Ts = batch_Ts(b->N, b->M, b->shapes);
  b->acbm_smem.clear();
  for (int T : b->acbm_Ts) b->acbm_smem.push_back(acbm_step_smem(b->N, b->M, T, b->p_max));
  // device memory: control, tables, per-stream scratch
  const size_t n = b->shapes.size();
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
  const size_t o_ctrl = take(sizeof(BCtrl));
  const size_t o_shapes = take(sizeof(BShape) * n);
  const size_t o_streams = take(sizeof(BStream) * n);
  const size_t o_segs = take(sizeof(BSegment) * b->segs.size());
  const size_t o_fsent = take(sizeof(BFsEntry) * b->fsent.size());
  const size_t o_fsent_tab = take(sizeof(BFsEntry) * std::max<size_t>(1, b->fsent_tab.size()));
  const size_t o_items = take(8 * (size_t)std::max(1, b->total_items));
  const size_t o_q = take(8 * (size_t)std::max(1, b->total_items));
  std::vector<size_t> o_pad(n), o_intra(n), o_flags(n), o_bkey(n), o_bstate(n);
  b->total_pad = 0;
  b->total_blocks = 0;
  for (size_t i = 0; i < n; i++) {
    BShape& s = b->shapes[i];
    const int nb = (s.W / b->N) * (s.H / b->M);
    o_pad[i] = take((size_t)s.pg.pitch * s.pg.rows);
    o_intra[i] = take(4 * (size_t)nb);
    o_flags[i] = take(8 * (size_t)nb);
    o_bkey[i] = take(8 * (size_t)nb);
    o_bstate[i] = take(4 * (size_t)nb);
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
    b->shapes[i].flags = reinterpret_cast<unsigned long long*>(base8 + o_flags[i]);
    b->shapes[i].bkey = reinterpret_cast<unsigned long long*>(base8 + o_bkey[i]);
    b->shapes[i].bstate = reinterpret_cast<int*>(base8 + o_bstate[i]);
  }
  b->d_ctrl = reinterpret_cast<BCtrl*>(base8 + o_ctrl);
  b->d_shapes = reinterpret_cast<BShape*>(base8 + o_shapes);
  b->d_streams = reinterpret_cast<BStream*>(base8 + o_streams);
  b->d_segs = reinterpret_cast<BSegment*>(base8 + o_segs);
  b->d_fsent = reinterpret_cast<BFsEntry*>(base8 + o_fsent);
  b->d_fsent_tab = reinterpret_cast<BFsEntry*>(base8 + o_fsent_tab);
  b->d_items = reinterpret_cast<unsigned long long*>(base8 + o_items);
  b->d_q = reinterpret_cast<unsigned long long*>(base8 + o_q);
  ME_CUDA(cudaMemcpy(b->d_shapes, b->shapes.data(), sizeof(BShape) * n, cudaMemcpyHostToDevice));
  if (!b->segs.empty())
    ME_CUDA(cudaMemcpy(b->d_segs, b->segs.data(), sizeof(BSegment) * b->segs.size(),
                       cudaMemcpyHostToDevice));
  if (!b->fsent.empty())
    ME_CUDA(cudaMemcpy(b->d_fsent, b->fsent.data(), sizeof(BFsEntry) * b->fsent.size(),
                       cudaMemcpyHostToDevice));
  if (!b->fsent_tab.empty())
    ME_CUDA(cudaMemcpy(b->d_fsent_tab, b->fsent_tab.data(),
                       sizeof(BFsEntry) * b->fsent_tab.size(), cudaMemcpyHostToDevice));
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
  int dev = 0;
  ME_CUDA(cudaGetDevice(&dev));
  b->device = dev;
  // size the persistent grids now, outside any capture
  int st = ME_ERR_ARG, grid = 0;
#define X(n_, m_, t_)                                                                          \
  if (b->N == n_ && b->M == m_ && b->T == t_)                                                  \
    st = persistent_grid((const void*)k_fsbm_persist<n_, m_, t_>, b->smem_fs, &grid);
  ME_BATCH_NMT(X)
#undef X
  for (size_t i = 0; i < b->acbm_Ts.size() && st == ME_OK; i++) {
    st = ME_ERR_ARG;
#define X(n_, m_, t_)                                                                          \
    if (b->N == n_ && b->M == m_ && b->acbm_Ts[i] == t_)                                       \
      st = persistent_grid((const void*)k_acbm_persist<n_, m_, t_>, b->acbm_smem[i], &grid);
    ME_BATCH_NMT(X)
#undef X
  }
  return st;
}

// Candidate step forms of a mode: FSBM -- the per-group persistent kernel at
// the model's run length, then (16x16) the pipelined search; ACBM -- the
// persistent kernel at each run length of acbm_Ts.
static std::vector<std::string> batch_forms(const me_batch* b, int mode) {
  std::vector<std::string> names;
  char nm[64];
  if (mode == ME_MODE_FSBM) {
    std::snprintf(nm, sizeof(nm), "persist T=%d", b->T);
    names.push_back(nm);
    if (!b->fsent_tab.empty()) names.push_back("pipetab");
  } else {
    // each run length with speculative searches, then without
    for (int spec = 1; spec >= 0; spec--)
      for (int T : b->acbm_Ts) {
        std::snprintf(nm, sizeof(nm), "persist T=%d spec=%d", T, spec);
        names.push_back(nm);
      }
  }
  return names;
}

// Enqueues one step of `mode` in candidate form c (no argument staging).
static int batch_enqueue(me_batch* b, int mode, int c, cudaStream_t s) {
  if (mode == ME_MODE_FSBM) {
    if (c == 1)
      return launch_fsbm_tab_step(b->N, b->M, b->d_ctrl, 0, b->d_shapes, b->d_streams,
                                  b->d_fsent_tab, (int)b->fsent_tab.size(), s);
    return launch_fsbm_step(b->N, b->M, b->T, b->d_ctrl, 0, b->d_shapes, b->d_streams, b->d_fsent,
                            (int)b->fsent.size(), b->smem_fs, s);
  }
  const int nT = (int)b->acbm_Ts.size();
  const int ti = c % nT, spec = c < nT ? 1 : 0;
  return launch_acbm_step(b->N, b->M, b->acbm_Ts[ti], b->d_ctrl, 0, b->d_shapes, b->d_streams,
                          (int)b->shapes.size(), b->total_pad, b->total_blocks, b->d_segs,
                          (int)b->segs.size(), b->total_items, b->acbm_smem[ti], b->p_max,
                          b->d_items, b->d_q, s, spec);
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
    // the step's form: forced (tests), else timed on this step's inputs
    const std::vector<std::string> names = batch_forms(b, mode);
    int c = tune_forced((int)names.size());
    if (c < 0) {
      char what[64];
      std::snprintf(what, sizeof(what), "batch %s %d streams", mode == ME_MODE_FSBM ? "fsbm" : "acbm",
                    (int)b->shapes.size());
      int st = tune_select(what, names, 0, s, [&](int k) { return batch_enqueue(b, mode, k, s); }, &c);
      if (st) return st;
    }
    b->form[gi] = c;
    // capture the step once on a private stream, then replay it
    cudaStream_t cs;
    ME_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    ME_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int st = batch_enqueue(b, mode, c, cs);
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

// me_server.cu -- a request server with continuous batching over many
// streams: frame-pair requests arrive one frame at a time per stream, each
// stream's reference frame and previous motion field stay resident in device
// memory, and a worker thread keeps up to `max_inflight` batch steps on the
// GPU at once.  A step takes the oldest pending request of every stream that
// is not already on the GPU, so requests that arrive while a step runs join
// the next one as soon as a step slot frees up.  Streams are admitted against
// a device-memory budget.  Each step is one persistent launch (the same
// kernels as the batch API), so a stream's result is identical alone or in
// any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "me_batch.cuh"

namespace me {

static double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct SrvRequest {
  long long id = 0;
  int stream = -1;
  uint8_t* h_frame = nullptr;     // pinned copy of the submitted frame
  size_t frame_bytes = 0;
  double t_submit = 0, latency_ms = 0;
  bool done = false, has_result = false;
  int status = ME_OK;
  std::vector<int16_t> mv;
  std::vector<uint32_t> J, sad, load;
  std::vector<uint8_t> mask;
};

struct SrvStream {
  int id = -1, W = 0, H = 0, p = 0;
  uint32_t lam = 0;
  me_acbm_params prm{};
  size_t bytes = 0;               // device bytes charged to the budget
  void* dmem = nullptr;
  uint8_t* d_frame[2] = {nullptr, nullptr};
  int cur_slot = 0;               // the next frame goes to d_frame[cur_slot]
  int16_t* d_mv[2] = {nullptr, nullptr};
  int mv_slot = 0;                // the next field goes to d_mv[mv_slot]
  bool have_prev = false;
  uint32_t *d_J = nullptr, *d_sad = nullptr, *d_load = nullptr;
  uint8_t* d_mask = nullptr;
  uint8_t* refpad = nullptr;
  uint32_t* intra = nullptr;
  unsigned long long* flags = nullptr;  // per block: epoch + final vector
  void* hmem = nullptr;           // pinned result slot
  int16_t* h_mv = nullptr;
  uint32_t *h_J = nullptr, *h_sad = nullptr, *h_load = nullptr;
  uint8_t* h_mask = nullptr;
  std::deque<SrvRequest*> queue;
  bool inflight = false, closing = false;
  long long frames = 0;
};

struct SrvSlot {
  cudaStream_t cs = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  BCtrl* d_ctrl = nullptr;
  BCtrl* h_ctrl = nullptr;
  void* d_tab = nullptr;          // shapes | streams | segments/entries
  void* h_tab = nullptr;          // pinned staging of the same
  size_t tab_bytes = 0;
  std::vector<std::pair<int, SrvRequest*>> work;  // (stream id, request) in the step
};

}  // namespace me

struct me_server {
  me_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  int device = 0;
  size_t used = 0;
  int next_stream = 0;
  long long next_req = 1;
  std::map<int, me::SrvStream*> streams;
  std::unordered_map<long long, me::SrvRequest*> reqs;
  std::vector<me::SrvSlot> slots;
  std::multimap<size_t, uint8_t*> pinned_free;  // reusable pinned frame buffers by size
  int fatal = ME_OK;
  char fatal_text[256] = "";                     // the worker's error text, for callers
  char diag[256] = "";                           // control block of the last step that timed out
};

namespace me {

static size_t stream_bytes(int W, int H, int N, int M, int p) {
  const PadGeom pg = pad_geom(W, H, p);
  const size_t nb = (size_t)(W / N) * (H / M), fr = (size_t)W * H;
  return align_up(fr, 256) * 2 + align_up(4 * nb, 256) * 2 + align_up(4 * nb, 256) * 3 +
         align_up(nb, 256) + align_up((size_t)pg.pitch * pg.rows, 256) + align_up(4 * nb, 256) +
         align_up(8 * nb, 256);
}

static int alloc_stream(me_server* sv, SrvStream* s) {
  const int N = sv->cfg.N, M = sv->cfg.M;
  const size_t nb = (size_t)(s->W / N) * (s->H / M), fr = (size_t)s->W * s->H;
  ME_CUDA(cudaMalloc(&s->dmem, s->bytes));
  ME_CUDA(cudaMemset(s->dmem, 0, s->bytes));
  uint8_t* q = static_cast<uint8_t*>(s->dmem);
  auto take = [&](size_t b) { uint8_t* r = q; q += align_up(b, 256); return r; };
  s->d_frame[0] = take(fr);
  s->d_frame[1] = take(fr);
  s->d_mv[0] = reinterpret_cast<int16_t*>(take(4 * nb));
  s->d_mv[1] = reinterpret_cast<int16_t*>(take(4 * nb));
  s->d_J = reinterpret_cast<uint32_t*>(take(4 * nb));
  s->d_sad = reinterpret_cast<uint32_t*>(take(4 * nb));
  s->d_load = reinterpret_cast<uint32_t*>(take(4 * nb));
  s->d_mask = take(nb);
  const PadGeom pg = pad_geom(s->W, s->H, s->p);
  s->refpad = take((size_t)pg.pitch * pg.rows);
  s->intra = reinterpret_cast<uint32_t*>(take(4 * nb));
  s->flags = reinterpret_cast<unsigned long long*>(take(8 * nb));
  const size_t hb = 4 * nb * 4 + nb;
  ME_CUDA(cudaMallocHost(&s->hmem, hb));
  uint8_t* h = static_cast<uint8_t*>(s->hmem);
  s->h_mv = reinterpret_cast<int16_t*>(h);
  s->h_J = reinterpret_cast<uint32_t*>(h + 4 * nb);
  s->h_sad = reinterpret_cast<uint32_t*>(h + 8 * nb);
  s->h_load = reinterpret_cast<uint32_t*>(h + 12 * nb);
  s->h_mask = h + 16 * nb;
  return ME_OK;
}

static void free_stream(SrvStream* s) {
  if (s->dmem) cudaFree(s->dmem);
  if (s->hmem) cudaFreeHost(s->hmem);
  delete s;
}

// Grows a slot's table buffers (device and pinned) to at least `bytes`.
static int slot_reserve(SrvSlot& sl, size_t bytes) {
  if (bytes <= sl.tab_bytes) return ME_OK;
  const size_t nb = std::max(bytes, sl.tab_bytes * 2);
  if (sl.d_tab) {
    ME_CUDA(cudaStreamSynchronize(sl.cs));
    cudaFree(sl.d_tab);
    cudaFreeHost(sl.h_tab);
    sl.d_tab = sl.h_tab = nullptr;
  }
  ME_CUDA(cudaMalloc(&sl.d_tab, nb));
  // a fresh buffer may hold an earlier owner's queue flags: clear it
  ME_CUDA(cudaMemsetAsync(sl.d_tab, 0, nb, sl.cs));
  ME_CUDA(cudaMallocHost(&sl.h_tab, nb));
  sl.tab_bytes = nb;
  return ME_OK;
}

// Step epochs are unique within the process, so ready flags and queue flags
// left in reused memory by another server can never match a current step.
static std::atomic<int> g_epoch{0};

// Launches one step on slot `sl` with the head request of every ready stream.
// Called with sv->mu held.
static int launch_step(me_server* sv, SrvSlot& sl, std::vector<SrvStream*>& ready) {
  const int N = sv->cfg.N, M = sv->cfg.M;
  const bool acbm = sv->cfg.mode == ME_MODE_ACBM;
  sl.work.clear();
  std::vector<BShape> shapes;
  std::vector<BStream> args;
  std::vector<SrvStream*> searched;
  for (SrvStream* s : ready) {
    SrvRequest* r = s->queue.front();
    s->queue.pop_front();
    s->inflight = true;
    sl.work.push_back({s->id, r});
    ME_CUDA(cudaMemcpyAsync(s->d_frame[s->cur_slot], r->h_frame, r->frame_bytes,
                            cudaMemcpyHostToDevice, sl.cs));
    if (s->frames == 0) continue;  // first frame: it only becomes the reference
    BShape sh;
    std::memset(&sh, 0, sizeof(sh));
    sh.W = s->W; sh.H = s->H; sh.p = s->p; sh.pg = pad_geom(s->W, s->H, s->p);
    sh.refpad = s->refpad; sh.intra = s->intra; sh.flags = s->flags;
    BStream a;
    a.cur = s->d_frame[s->cur_slot];
    a.ref = s->d_frame[s->cur_slot ^ 1];
    a.prev = s->have_prev ? s->d_mv[s->mv_slot ^ 1] : nullptr;
    a.mv = s->d_mv[s->mv_slot];
    a.J = s->d_J; a.mask = s->d_mask; a.sad = s->d_sad; a.load = s->d_load;
    a.lam = s->lam;
    a.alpha = s->prm.alpha; a.beta = s->prm.beta; a.gnum = s->prm.gamma_num;
    a.gden = s->prm.gamma_den; a.qp = s->prm.qp; a.refine = s->prm.refine;
    shapes.push_back(sh);
    args.push_back(a);
    searched.push_back(s);
  }
  if (!searched.empty()) {
    const int ns = (int)shapes.size();
    long long total_pad = 0;
    int total_blocks = 0;
    for (BShape& sh : shapes) {
      sh.pad_base = total_pad;
      sh.blk_base = total_blocks;
      total_pad += (long long)sh.pg.rows * (sh.pg.pitch / 16);
      total_blocks += (sh.W / N) * (sh.H / M);
    }
    const int T = batch_choose_T(N, M, shapes);
    std::vector<BSegment> segs;
    std::vector<BFsEntry> ent;
    size_t smem = 0;
    int total_items = 0, p_max = 1;
    if (acbm) {
      int maxw = 0;
      for (const BShape& sh : shapes) maxw = std::max(maxw, make_waves(sh.W / N, sh.H / M).n);
      for (int w = 0; w < maxw; w++)
        for (int si = 0; si < ns; si++) {
          const Waves wv = make_waves(shapes[si].W / N, shapes[si].H / M);
          if (w >= wv.n || wv.count(w) == 0) continue;
          segs.push_back(BSegment{si, w, wv.ylo(w), wv.count(w), total_items});
          total_items += wv.count(w);
        }
      for (const BShape& sh : shapes) p_max = std::max(p_max, sh.p);
      smem = acbm_step_smem(N, M, T, p_max);
    } else {
      for (int si = 0; si < ns; si++) {
        const BShape& sh = shapes[si];
        const int BW = sh.W / N, BH = sh.H / M;
        const FsPlan pl = fs_plan_fixed(N, M, T, sh.p, kBatchThreads, BW, 110 * 1024);
        const int bpc = kBatchThreads / pl.G;
        smem = std::max(smem, pl.smem);
        for (int by = 0; by < BH; by++)
          for (int bx0 = 0; bx0 < BW; bx0 += bpc)
            ent.push_back(BFsEntry{si, by, bx0, std::min(bpc, BW - bx0), pl.G});
      }
    }
    const size_t o_sh = 0;
    const size_t o_st = align_up(o_sh + sizeof(BShape) * ns, 256);
    const size_t o_tab = align_up(o_st + sizeof(BStream) * ns, 256);
    const size_t tab = acbm ? sizeof(BSegment) * segs.size() : sizeof(BFsEntry) * ent.size();
    // item table and full-search queue (ACBM): 8 + 8 bytes per block of the step
    const size_t o_items = align_up(o_tab + tab, 256);
    const size_t o_q = align_up(o_items + 8 * (size_t)std::max(1, total_items), 256);
    int st = slot_reserve(sl, o_q + 8 * (size_t)std::max(1, total_items) + 256);
    if (st) return st;
    uint8_t* h = static_cast<uint8_t*>(sl.h_tab);
    uint8_t* d = static_cast<uint8_t*>(sl.d_tab);
    std::memcpy(h + o_sh, shapes.data(), sizeof(BShape) * ns);
    std::memcpy(h + o_st, args.data(), sizeof(BStream) * ns);
    if (acbm) std::memcpy(h + o_tab, segs.data(), tab);
    else std::memcpy(h + o_tab, ent.data(), tab);
    ME_CUDA(cudaMemcpyAsync(d, h, o_tab + tab, cudaMemcpyHostToDevice, sl.cs));
    // the queue sits where earlier steps kept their tables: clear its entries
    if (acbm) ME_CUDA(cudaMemsetAsync(d + o_q, 0, 8 * (size_t)std::max(1, total_items), sl.cs));
    const int epoch = ++g_epoch;
    if (acbm)
      st = launch_acbm_step(N, M, T, sl.d_ctrl, epoch, reinterpret_cast<BShape*>(d + o_sh),
                            reinterpret_cast<BStream*>(d + o_st), ns, total_pad, total_blocks,
                            reinterpret_cast<BSegment*>(d + o_tab), (int)segs.size(), total_items,
                            smem, p_max, reinterpret_cast<unsigned long long*>(d + o_items),
                            reinterpret_cast<unsigned long long*>(d + o_q), sl.cs);
    else
      st = launch_fsbm_step(N, M, T, sl.d_ctrl, epoch, reinterpret_cast<BShape*>(d + o_sh),
                            reinterpret_cast<BStream*>(d + o_st),
                            reinterpret_cast<BFsEntry*>(d + o_tab), (int)ent.size(), smem, sl.cs);
    if (st) return st;
    for (SrvStream* s : searched) {
      const size_t nb = (size_t)(s->W / N) * (s->H / M);
      ME_CUDA(cudaMemcpyAsync(s->h_mv, s->d_mv[s->mv_slot], 4 * nb, cudaMemcpyDeviceToHost, sl.cs));
      ME_CUDA(cudaMemcpyAsync(s->h_J, s->d_J, 4 * nb, cudaMemcpyDeviceToHost, sl.cs));
      ME_CUDA(cudaMemcpyAsync(s->h_sad, s->d_sad, 4 * nb, cudaMemcpyDeviceToHost, sl.cs));
      if (acbm) {
        ME_CUDA(cudaMemcpyAsync(s->h_load, s->d_load, 4 * nb, cudaMemcpyDeviceToHost, sl.cs));
        ME_CUDA(cudaMemcpyAsync(s->h_mask, s->d_mask, nb, cudaMemcpyDeviceToHost, sl.cs));
      }
    }
    ME_CUDA(cudaMemcpyAsync(sl.h_ctrl, sl.d_ctrl, sizeof(BCtrl), cudaMemcpyDeviceToHost, sl.cs));
  } else {
    sl.h_ctrl->error = 0;
  }
  ME_CUDA(cudaEventRecord(sl.done, sl.cs));
  sl.busy = true;
  return ME_OK;
}

// Results of a finished step go to their requests.  Called with sv->mu held.
static void complete_step(me_server* sv, SrvSlot& sl) {
  const int N = sv->cfg.N, M = sv->cfg.M;
  const bool acbm = sv->cfg.mode == ME_MODE_ACBM;
  const int err = sl.h_ctrl->error;
  const double t = now_ms();
  if (err) {
    const BCtrl& c = *sl.h_ctrl;
    std::snprintf(sv->diag, sizeof(sv->diag),
                  "step epoch %d: error %d at item %d; next %d, pbm_done %d, queue head %d tail %d; "
                  "%d requests in the step",
                  c.epoch, c.error, c.err_item, c.next, c.pbm_done, c.fs_head, c.fs_tail,
                  (int)sl.work.size());
  }
  for (auto& wr : sl.work) {
    SrvStream* s = sv->streams[wr.first];
    SrvRequest* r = wr.second;
    if (s->frames > 0) {
      const size_t nb = (size_t)(s->W / N) * (s->H / M);
      r->has_result = true;
      r->mv.assign(s->h_mv, s->h_mv + 2 * nb);
      r->J.assign(s->h_J, s->h_J + nb);
      r->sad.assign(s->h_sad, s->h_sad + nb);
      if (acbm) {
        r->load.assign(s->h_load, s->h_load + nb);
        r->mask.assign(s->h_mask, s->h_mask + nb);
        s->have_prev = true;
        s->mv_slot ^= 1;
      }
      r->status = err ? err : ME_OK;
    }
    s->cur_slot ^= 1;
    s->frames++;
    s->inflight = false;
    sv->pinned_free.insert({r->frame_bytes, r->h_frame});
    r->h_frame = nullptr;
    r->latency_ms = t - r->t_submit;
    r->done = true;
  }
  sl.work.clear();
  sl.busy = false;
  // streams closed while on the GPU are released now
  for (auto it = sv->streams.begin(); it != sv->streams.end();) {
    SrvStream* s = it->second;
    if (s->closing && !s->inflight && s->queue.empty()) {
      sv->used -= s->bytes;
      free_stream(s);
      it = sv->streams.erase(it);
    } else {
      ++it;
    }
  }
  sv->cv_done.notify_all();
}

static void worker_main(me_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (!sv->stop) {
    bool any_busy = false;
    for (SrvSlot& sl : sv->slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaSuccess) complete_step(sv, sl);
      else if (q == cudaErrorNotReady) any_busy = true;
      else {
        sv->fatal = cuda_status(q);
        std::snprintf(sv->fatal_text, sizeof(sv->fatal_text), "%s", me_last_error());
        sl.busy = false;
      }
    }
    SrvSlot* free_slot = nullptr;
    for (SrvSlot& sl : sv->slots)
      if (!sl.busy) { free_slot = &sl; break; }
    std::vector<SrvStream*> ready;
    if (free_slot)
      for (auto& kv : sv->streams)
        if (!kv.second->inflight && !kv.second->queue.empty()) ready.push_back(kv.second);
    if (free_slot && !ready.empty() && sv->fatal == ME_OK) {
      const int st = launch_step(sv, *free_slot, ready);
      if (st) {
        sv->fatal = st;
        std::snprintf(sv->fatal_text, sizeof(sv->fatal_text), "%s", me_last_error());
      }
      continue;
    }
    if (any_busy) sv->cv_work.wait_for(lk, std::chrono::microseconds(20));
    else sv->cv_work.wait(lk);
  }
}

}  // namespace me

using namespace me;

extern "C" {

int me_server_create(const me_server_config* cfg, me_server** out) {
  if (!cfg || !out) return ME_ERR_ARG;
  if (cfg->device_budget_bytes <= 0 || cfg->max_inflight < 1 || cfg->max_inflight > 8) return ME_ERR_ARG;
  if (cfg->mode != ME_MODE_FSBM && cfg->mode != ME_MODE_ACBM) return ME_ERR_ARG;
  if (!(cfg->N == 4 || cfg->N == 8 || cfg->N == 16) || !(cfg->M == 4 || cfg->M == 8 || cfg->M == 16))
    return ME_ERR_ARG;
  me_server* sv = new (std::nothrow) me_server();
  if (!sv) return ME_ERR_NOMEM;
  sv->cfg = *cfg;
  ME_CUDA(cudaGetDevice(&sv->device));
  sv->slots.resize(cfg->max_inflight);
  for (SrvSlot& sl : sv->slots) {
    ME_CUDA(cudaStreamCreateWithFlags(&sl.cs, cudaStreamNonBlocking));
    ME_CUDA(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
    ME_CUDA(cudaMalloc(&sl.d_ctrl, sizeof(BCtrl)));
    ME_CUDA(cudaMallocHost(&sl.h_ctrl, sizeof(BCtrl)));
    BCtrl c;
    std::memset(&c, 0, sizeof(c));
    c.timeout_ns = 1000000000ll;
    c.skip_stream = c.skip_block = -1;
    ME_CUDA(cudaMemcpy(sl.d_ctrl, &c, sizeof(c), cudaMemcpyHostToDevice));
    std::memset(sl.h_ctrl, 0, sizeof(BCtrl));
  }
  sv->worker = std::thread(worker_main, sv);
  *out = sv;
  return ME_OK;
}

int me_server_open_stream(me_server* sv, int W, int H, int p, const me_acbm_params* prm,
                          int32_t qp, int* stream_id) {
  if (!sv || !stream_id) return ME_ERR_ARG;
  int st = check_frame_args(W, H, sv->cfg.N, sv->cfg.M, p, 0);
  if (st) return st;
  me_acbm_params pr = prm ? *prm : me_acbm_default_params(qp);
  st = check_acbm_params(&pr);
  if (st) return st;
  SrvStream* s = new (std::nothrow) SrvStream();
  if (!s) return ME_ERR_NOMEM;
  s->W = W; s->H = H; s->p = p; s->prm = pr;
  s->lam = me_lambda_q8(pr.qp);
  s->bytes = stream_bytes(W, H, sv->cfg.N, sv->cfg.M, p);
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->used + s->bytes > (size_t)sv->cfg.device_budget_bytes) {
      delete s;
      return ME_ERR_NOMEM;   // not admitted: over the device-memory budget
    }
    sv->used += s->bytes;
  }
  st = alloc_stream(sv, s);
  std::lock_guard<std::mutex> lk(sv->mu);
  if (st) {
    sv->used -= s->bytes;
    free_stream(s);
    return st;
  }
  s->id = sv->next_stream++;
  sv->streams[s->id] = s;
  *stream_id = s->id;
  return ME_OK;
}

int me_server_submit(me_server* sv, int stream_id, const uint8_t* frame, long long* request_id) {
  if (!sv || !frame || !request_id) return ME_ERR_ARG;
  size_t bytes = 0;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->fatal) {
      set_last_error_text(sv->fatal_text);
      return sv->fatal;
    }
    auto it = sv->streams.find(stream_id);
    if (it == sv->streams.end() || it->second->closing) return ME_ERR_NOTFOUND;
    bytes = (size_t)it->second->W * it->second->H;
  }
  uint8_t* buf = nullptr;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->pinned_free.find(bytes);
    if (it != sv->pinned_free.end()) {
      buf = it->second;
      sv->pinned_free.erase(it);
    }
  }
  if (!buf) ME_CUDA(cudaMallocHost(&buf, bytes));
  std::memcpy(buf, frame, bytes);
  SrvRequest* r = new (std::nothrow) SrvRequest();
  if (!r) return ME_ERR_NOMEM;
  r->h_frame = buf;
  r->frame_bytes = bytes;
  r->stream = stream_id;
  r->t_submit = now_ms();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->streams.find(stream_id);
    if (it == sv->streams.end() || it->second->closing) {
      sv->pinned_free.insert({bytes, buf});
      delete r;
      return ME_ERR_NOTFOUND;
    }
    r->id = sv->next_req++;
    sv->reqs[r->id] = r;
    it->second->queue.push_back(r);
    *request_id = r->id;
  }
  sv->cv_work.notify_one();
  return ME_OK;
}

static int take_result(me_server* sv, SrvRequest* r, me_server_result* res) {
  if (res) {
    res->has_result = r->has_result ? 1 : 0;
    res->status = r->status;
    res->latency_ms = r->latency_ms;
    if (r->has_result) {
      if (res->mv) std::memcpy(res->mv, r->mv.data(), r->mv.size() * sizeof(int16_t));
      if (res->J) std::memcpy(res->J, r->J.data(), r->J.size() * sizeof(uint32_t));
      if (res->sad) std::memcpy(res->sad, r->sad.data(), r->sad.size() * sizeof(uint32_t));
      if (res->mask && !r->mask.empty()) std::memcpy(res->mask, r->mask.data(), r->mask.size());
      if (res->load && !r->load.empty())
        std::memcpy(res->load, r->load.data(), r->load.size() * sizeof(uint32_t));
    }
  }
  const int st = r->status;
  sv->reqs.erase(r->id);
  delete r;
  return st;
}

int me_server_poll(me_server* sv, long long request_id, me_server_result* res) {
  if (!sv) return ME_ERR_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(request_id);
  if (it == sv->reqs.end()) return ME_ERR_NOTFOUND;
  if (!it->second->done) {
    if (sv->fatal) set_last_error_text(sv->fatal_text);
    return sv->fatal ? sv->fatal : ME_ERR_BUSY;
  }
  return take_result(sv, it->second, res);
}

int me_server_wait(me_server* sv, long long request_id, int timeout_ms, me_server_result* res) {
  if (!sv) return ME_ERR_ARG;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(request_id);
  if (it == sv->reqs.end()) return ME_ERR_NOTFOUND;
  SrvRequest* r = it->second;
  const bool ok = sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                       [&] { return r->done || sv->fatal != ME_OK; });
  if (!r->done) {
    if (sv->fatal) set_last_error_text(sv->fatal_text);
    return ok ? sv->fatal : ME_ERR_BUSY;
  }
  return take_result(sv, r, res);
}

int me_server_close_stream(me_server* sv, int stream_id) {
  if (!sv) return ME_ERR_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->streams.find(stream_id);
  if (it == sv->streams.end() || it->second->closing) return ME_ERR_NOTFOUND;
  SrvStream* s = it->second;
  s->closing = true;
  if (!s->inflight && s->queue.empty()) {
    sv->used -= s->bytes;
    free_stream(s);
    sv->streams.erase(it);
  }
  return ME_OK;
}

int me_server_stats(me_server* sv, long long* used_bytes, int* open_streams, int* pending) {
  if (!sv) return ME_ERR_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (used_bytes) *used_bytes = (long long)sv->used;
  if (open_streams) *open_streams = (int)sv->streams.size();
  if (pending) {
    int n = 0;
    for (auto& kv : sv->reqs) n += kv.second->done ? 0 : 1;
    *pending = n;
  }
  return sv->fatal;
}

const char* me_server_diagnostics(me_server* sv) {
  if (!sv) return "";
  std::lock_guard<std::mutex> lk(sv->mu);
  static thread_local char buf[256];
  std::snprintf(buf, sizeof(buf), "%s", sv->diag);
  return buf;
}

void me_server_destroy(me_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  for (SrvSlot& sl : sv->slots) {
    if (sl.cs) cudaStreamSynchronize(sl.cs);
    if (sl.busy) complete_step(sv, sl);   // hand back the pinned frames of a last step
    if (sl.d_tab) cudaFree(sl.d_tab);
    if (sl.h_tab) cudaFreeHost(sl.h_tab);
    if (sl.d_ctrl) cudaFree(sl.d_ctrl);
    if (sl.h_ctrl) cudaFreeHost(sl.h_ctrl);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.cs) cudaStreamDestroy(sl.cs);
  }
  for (auto& kv : sv->streams) {
    for (SrvRequest* r : kv.second->queue) {
      if (r->h_frame) cudaFreeHost(r->h_frame);
    }
    free_stream(kv.second);
  }
  for (auto& kv : sv->reqs) {
    if (kv.second->h_frame && kv.second->done) cudaFreeHost(kv.second->h_frame);
    delete kv.second;
  }
  for (auto& kv : sv->pinned_free) cudaFreeHost(kv.second);
  delete sv;
}

}  // extern "C"

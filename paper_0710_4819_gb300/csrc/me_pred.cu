// me_pred.cu -- FSBM with the vector's rate coded against a predictor.
//
// Sec. 2.1 takes R(mvx, mvy) as the bits that transmit the vector, and
// Sec. 2.2 notes that the standards code vectors differentially.  This
// variant codes each vector against the H.263-style median predictor pm: the
// component-wise median of the final vectors of the left (MV1), upper (MV2)
// and upper-right (MV3) blocks, with MV1 = 0 on the left edge, MV3 = 0 on the
// right edge and MV2 = MV3 = MV1 in the top row; R = L(mvx - pmx) +
// L(mvy - pmy), L the signed Exp-Golomb length; J_q8 = 256*SAD + lambda_q8*R;
// ties as for FSBM (J, then |mv|_1, then mvy, then mvx).
//
// The predictor makes every block depend on its left, upper and upper-right
// neighbours' results, so the search becomes a wavefront (w = x + 2y: the
// left and upper-right neighbours lie on wave w-1, the upper one on w-2).
// Only the argmin depends on the predictor, not the SADs, so the work splits:
//
//   k_sad_volume : the FSBM engine (fs_group, VOL mode) stores every
//                  candidate's SAD of every block as uint16 -- fully
//                  parallel, the same ALU-bound packed-SAD work as FSBM
//                  (16x16 blocks: the pipelined search in its volume mode);
//   k_pred_wave  : a persistent kernel; each CTA claims blocks in (wave,
//                  frame, row) order, stages the block's SAD volume into
//                  shared memory and lists the candidates that can still win
//                  whatever the predictor, then warp 0 waits (bounded) for the
//                  three predecessors' published vectors, evaluates J over the
//                  list (or the CTA over all (2p+1)^2 candidates when the list
//                  is long) and publishes the vector.  A block only waits for
//                  blocks claimed before it, which are held by running CTAs,
//                  so the claims always make progress; the frames of a
//                  sequence are independent and overlap.
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

constexpr int kPredMaxK = 64;
constexpr int kPredThreads = 128;

struct PredFrames {
  const uint8_t* f[kPredMaxK + 1];  // pair k: reference f[k], current f[k+1]
};

struct PredCtrl {
  int epoch, error, err_item;
  long long timeout_cycles;  // bound of every spin-wait (SM clock cycles)
  alignas(128) int next;  // claims
};

// uint16 entries per block volume, rounded up to 16 bytes (16-byte copies)
__host__ __device__ inline int pred_vstride(int p) {
  const int n = 2 * p + 1;
  return (n * n + 7) & ~7;
}

// Shifted-word row pitch of the 16x16, run-length-13 build with immediate
// row offsets (the same pitch the FSBM sequence kernel uses): 193 words is odd,
// so rows fall on different banks.
constexpr int kVolSP = 193;

template <int N, int M, int T, int SP = 0>
__global__ void __launch_bounds__(kMaxThreads) k_sad_volume(PredFrames fr, int W, int H, int p,
                                                            int G, int vstride,
                                                            uint16_t* __restrict__ vol) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ unsigned long long keys[16];
  const int BW = W / N, nbf = BW * (H / M);
  const int bpc = blockDim.x / G;
  const int gpr = (BW + bpc - 1) / bpc;
  const int k = blockIdx.y;
  const int by = blockIdx.x / gpr, bx0 = (blockIdx.x % gpr) * bpc;
  const int nb = min(bpc, BW - bx0);
  const FsGeom g = fs_geom<N, M, T>(p, nb, G, 0, 0, SP);
  fs_group<N, M, T, SP, false, true>(fr.f[k + 1], fr.f[k], W, H, bx0 * N, by * M, g, 0u, smem, keys,
                                    nullptr, FsPad{nullptr, 0, 0, 0}, nullptr,
                                    vol + ((size_t)k * nbf + (size_t)by * BW + bx0) * vstride,
                                    vstride);
}

__global__ void k_pred_begin(PredCtrl* c) {
  c->epoch += 1;
  c->next = 0;
  c->error = 0;
  c->err_item = -1;
}

__device__ __forceinline__ int med3(int a, int b, int c) {
  return max(min(a, b), min(max(a, b), c));
}

// Candidates whose cost could still win once the predictor is known: with
// pm anywhere in [-p, p]^2 the rate of mv lies between 2 (mv = pm) and
// Rmax(mv) = L(|mvx| + p) + L(|mvy| + p) (L grows with |d|), so with
// UBmin = min_mv 256*SAD(mv) + lambda*Rmax(mv) -- a cost some candidate
// reaches whatever pm is -- the winner, and every candidate tying with it,
// has 256*SAD + 2*lambda <= UBmin.  The list is built before the wait; when
// it is short, one warp evaluates it as soon as the predictor is known.
constexpr int kPredList = 512;
constexpr int kPredPruneMaxK = 8;   // pairs per call up to which the list is built

__global__ void __launch_bounds__(kPredThreads) k_pred_wave(
    const int* __restrict__ items, int total, int BW, int nbf, int p, uint32_t lam,
    const uint16_t* __restrict__ vol, int vstride, unsigned long long* flags, PredCtrl* ctrl,
    int16_t* __restrict__ mv_out, uint32_t* __restrict__ J_out, uint32_t* __restrict__ sad_out,
    int prune) {
  extern __shared__ __align__(16) uint16_t vs[];   // [vstride] SADs, then [vstride] list
  uint16_t* list = vs + vstride;
  __shared__ unsigned long long red[kPredThreads / 32];
  __shared__ uint32_t ured[kPredThreads / 32];
  __shared__ int s_item, s_pmx, s_pmy, s_bad, s_cnt;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned FULL = 0xffffffffu;
  const int n = 2 * p + 1;
  constexpr int kCols = (2 * kMaxP + 1 + 31) / 32;
  const int epoch = *reinterpret_cast<volatile int*>(&ctrl->epoch);
  const volatile int* verr = &ctrl->error;
  const long long lim = ctrl->timeout_cycles;
  for (;;) {
    if (tid == 0) {
      s_item = atomicAdd(&ctrl->next, 1);
      s_bad = 0;
      s_cnt = 0;
    }
    __syncthreads();
    const int it = s_item;
    if (it >= total) break;
    const int gblk = items[it];                  // frame * nbf + block
    const int k = gblk / nbf, b = gblk - k * nbf, bx = b % BW, by = b / BW;
    // 1. the block's SAD volume
    {
      const uint16_t* src = vol + (size_t)gblk * vstride;
      for (int i = tid; i < vstride / 8; i += kPredThreads) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(vs + 8 * i);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src + 8 * i)
                     : "memory");
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      asm volatile("cp.async.wait_all;" ::: "memory");
    }
    __syncthreads();
    // 2. UBmin, then the list of candidates that can still win (before the
    // wait; only when pruning: it shortens the wait-to-publish step of the
    // dependency chain, which bounds one pair, at the price of two more
    // passes over the volume, which bound many pairs)
    uint32_t ax[kCols];
#pragma unroll
    for (int j = 0; j < kCols; j++) ax[j] = (uint32_t)abs(lane + 32 * j - p);
    if (prune) {
      uint32_t rx[kCols];
#pragma unroll
      for (int j = 0; j < kCols; j++) rx[j] = lam * (uint32_t)mv_bits((int)ax[j] + p);
      uint32_t ub = 0xffffffffu;
      for (int r = warp; r < n; r += kPredThreads / 32) {
        const uint32_t ry = lam * (uint32_t)mv_bits(abs(r - p) + p);
        const uint16_t* row = vs + r * n;
#pragma unroll
        for (int j = 0; j < kCols; j++) {
          const int c = lane + 32 * j;
          if (c < n) ub = min(ub, 256u * (uint32_t)row[c] + rx[j] + ry);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ub = min(ub, __shfl_xor_sync(FULL, ub, o));
      if (lane == 0) ured[warp] = ub;
      __syncthreads();
      uint32_t ubmin = ured[0];
#pragma unroll
      for (int i = 1; i < kPredThreads / 32; i++) ubmin = min(ubmin, ured[i]);
      const uint32_t two = 2u * lam;
      for (int r = warp; r < n; r += kPredThreads / 32) {
        const uint16_t* row = vs + r * n;
#pragma unroll
        for (int j = 0; j < kCols; j++) {
          const int c = lane + 32 * j;
          const bool in = c < n && 256u * (uint32_t)row[c] + two <= ubmin;
          const unsigned m = __ballot_sync(FULL, in);
          if (m) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&s_cnt, __popc(m));
            base = __shfl_sync(FULL, base, 0);
            if (in) list[base + __popc(m & ((1u << lane) - 1u))] = (uint16_t)((r << 8) | c);
          }
        }
      }
      __syncthreads();
    }
    const int cnt = prune ? s_cnt : kPredList + 1;   // without the list: the whole CTA
    // 3. the three predecessors (warp 0; bounded), then the predictor
    if (warp == 0) {
      // lane 0: left, lane 1: upper, lane 2: upper-right (when inside the grid)
      const unsigned long long* fl = flags + (size_t)k * nbf;
      const unsigned long long* f = nullptr;
      if (lane == 0 && bx > 0) f = fl + b - 1;
      if (lane == 1 && by > 0) f = fl + b - BW;
      if (lane == 2 && by > 0 && bx + 1 < BW) f = fl + b - BW + 1;
      unsigned long long w = 0;
      bool ready = f == nullptr;
      bool bad = false;
      const long long t0 = clock64();
      for (;;) {
        if (!ready) {
          w = *reinterpret_cast<const volatile unsigned long long*>(f);
          ready = pub_epoch(w) == epoch;
        }
        if (__all_sync(FULL, ready)) break;
        // the way out is decided by lane 0 and taken by the whole warp
        int stop = 0;
        if (lane == 0) stop = *verr != 0 ? 1 : (clock64() - t0 > lim ? 2 : 0);
        stop = __shfl_sync(FULL, stop, 0);
        if (stop) {
          if (stop == 2 && lane == 0) {
            atomicExch(&ctrl->error, (int)ME_ERR_TIMEOUT);
            atomicExch(&ctrl->err_item, it);
          }
          bad = true;
          break;
        }
        __nanosleep(20);
      }
      const int vx = f ? pub_mvx(w) : 0, vy = f ? pub_mvy(w) : 0;
      const int x1 = __shfl_sync(FULL, vx, 0), y1 = __shfl_sync(FULL, vy, 0);
      const int x2 = __shfl_sync(FULL, vx, 1), y2 = __shfl_sync(FULL, vy, 1);
      const int x3 = __shfl_sync(FULL, vx, 2), y3 = __shfl_sync(FULL, vy, 2);
      int pmx, pmy;
      if (by == 0) {          // top row: the left vector (zero at the left edge)
        pmx = x1;
        pmy = y1;
      } else {                // absent neighbours read as zero vectors
        pmx = med3(x1, x2, x3);
        pmy = med3(y1, y2, y3);
      }
      if (!bad && cnt <= kPredList) {
        // 4a. short list: this warp finishes the block and publishes at once
        unsigned long long best = kNoKey;
        for (int e = lane; e < cnt; e += 32) {
          const int rc = list[e];               // row << 8 | column (n <= 129)
          const int r = rc >> 8, c = rc & 255, i = r * n + c;
          const int mvx = c - p, mvy = r - p;
          const uint32_t J = 256u * (uint32_t)vs[i] +
                             lam * (uint32_t)(mv_bits(mvx - pmx) + mv_bits(mvy - pmy));
          const uint32_t lo = ((uint32_t)(abs(mvx) + abs(mvy)) << 17) + (uint32_t)i;
          best = umin64(best, ((unsigned long long)J << 32) | lo);
        }
        best = warp_min64(best);
        if (lane == 0) {
          const int i = (int)(best & 0x1ffffu);
          const int mvx = i % n - p, mvy = i / n - p;
          const size_t o = (size_t)gblk;
          // the flag carries the vector itself, so no fence orders the
          // outputs before it: dependants read nothing else of this block
          *reinterpret_cast<volatile unsigned long long*>(flags + o) = pub_word(epoch, mvx, mvy);
          mv_out[2 * o] = (int16_t)mvx;
          mv_out[2 * o + 1] = (int16_t)mvy;
          J_out[o] = (uint32_t)(best >> 32);
          if (sad_out) sad_out[o] = vs[i];
        }
      }
      if (lane == 0) {
        s_pmx = pmx;
        s_pmy = pmy;
        if (bad) s_bad = 1;
      }
    }
    __syncthreads();
    if (s_bad) break;   // a wait gave up: the run is abandoned (status reports it)
    if (cnt > kPredList) {
      // 4b. long list (flat SAD surfaces): the whole CTA evaluates every candidate
      const int pmx = s_pmx, pmy = s_pmy;
      uint32_t jx[kCols];
#pragma unroll
      for (int j = 0; j < kCols; j++) jx[j] = lam * (uint32_t)mv_bits(lane + 32 * j - p - pmx);
      unsigned long long best = kNoKey;
      for (int r = warp; r < n; r += kPredThreads / 32) {
        const int mvy = r - p;
        const uint32_t jy = lam * (uint32_t)mv_bits(mvy - pmy);
        const uint32_t lo_y = ((uint32_t)abs(mvy) << 17) + (uint32_t)(r * n);
        const uint16_t* row = vs + r * n;
#pragma unroll
        for (int j = 0; j < kCols; j++) {
          const int c = lane + 32 * j;
          if (c < n) {
            const uint32_t J = 256u * (uint32_t)row[c] + jx[j] + jy;
            const uint32_t lo = lo_y + (ax[j] << 17) + (uint32_t)c;
            best = umin64(best, ((unsigned long long)J << 32) | lo);
          }
        }
      }
      best = warp_min64(best);
      if (lane == 0) red[warp] = best;
      __syncthreads();
      if (tid == 0) {
        unsigned long long m = red[0];
#pragma unroll
        for (int i = 1; i < kPredThreads / 32; i++) m = umin64(m, red[i]);
        const int i = (int)(m & 0x1ffffu);
        const int mvx = i % n - p, mvy = i / n - p;
        const size_t o = (size_t)gblk;
        *reinterpret_cast<volatile unsigned long long*>(flags + o) = pub_word(epoch, mvx, mvy);
        mv_out[2 * o] = (int16_t)mvx;
        mv_out[2 * o + 1] = (int16_t)mvy;
        J_out[o] = (uint32_t)(m >> 32);
        if (sad_out) sad_out[o] = vs[i];
      }
    }
    __syncthreads();    // the shared buffers are reused by the next claim
  }
}

// ------------------------------------------------------------------ plans
struct PredPlan {
  int dev, W, H, N, M, p, K;
  void* mem = nullptr;
  uint16_t* vol = nullptr;
  unsigned long long* flags = nullptr;
  int* items = nullptr;
  PredCtrl* ctrl = nullptr;
  int total = 0, grid = 0, vstride = 0;
  size_t smem = 0;
  cudaEvent_t last = nullptr;
  bool ran = false;
  std::mutex mu;
};

static std::mutex g_pred_mu;
static std::vector<PredPlan*> g_pred_plans;

static int build_pred_plan(PredPlan* pl) {
  const int BW = pl->W / pl->N, BH = pl->H / pl->M, nbf = BW * BH;
  // claim order: wave, then frame, then row within the wave
  const Waves wv = make_waves(BW, BH);
  std::vector<int> items;
  items.reserve((size_t)nbf * pl->K);
  for (int w = 0; w < wv.n; w++)
    for (int k = 0; k < pl->K; k++)
      for (int by = wv.ylo(w); by <= wv.yhi(w); by++) items.push_back(k * nbf + by * BW + (w - 2 * by));
  pl->total = (int)items.size();
  pl->vstride = pred_vstride(pl->p);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
  const size_t o_ctrl = take(sizeof(PredCtrl));
  const size_t o_items = take(sizeof(int) * items.size());
  const size_t o_flags = take(8 * (size_t)nbf * pl->K);
  const size_t o_vol = take(2 * (size_t)pl->vstride * nbf * pl->K);
  ME_CUDA(cudaMalloc(&pl->mem, off));
  ME_CUDA(cudaMemset(pl->mem, 0, o_vol));
  uint8_t* m = static_cast<uint8_t*>(pl->mem);
  pl->ctrl = reinterpret_cast<PredCtrl*>(m + o_ctrl);
  pl->items = reinterpret_cast<int*>(m + o_items);
  pl->flags = reinterpret_cast<unsigned long long*>(m + o_flags);
  pl->vol = reinterpret_cast<uint16_t*>(m + o_vol);
  ME_CUDA(cudaMemcpy(pl->items, items.data(), sizeof(int) * items.size(), cudaMemcpyHostToDevice));
  PredCtrl c;
  std::memset(&c, 0, sizeof(c));
  c.timeout_cycles = wait_cycles(1000000000ll);     // 1 s
  ME_CUDA(cudaMemcpy(pl->ctrl, &c, sizeof(c), cudaMemcpyHostToDevice));
  pl->smem = 4 * (size_t)pl->vstride;   // SAD volume + candidate list
  {
    const int e = ensure_dynamic_smem((const void*)k_pred_wave, pl->smem);
    if (e) return e;
  }
  int nsm = 0, per_sm = 0;
  ME_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, pl->dev));
  ME_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pred_wave, kPredThreads, pl->smem));
  if (per_sm < 1) return ME_ERR_CUDA;
  pl->grid = std::max(1, std::min(pl->total, nsm * per_sm));
  ME_CUDA(cudaEventCreateWithFlags(&pl->last, cudaEventDisableTiming));
  return ME_OK;
}

static int get_pred_plan(int W, int H, int N, int M, int p, int K, PredPlan** out) {
  int dev = 0;
  ME_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_pred_mu);
  for (PredPlan* pl : g_pred_plans)
    if (pl->dev == dev && pl->W == W && pl->H == H && pl->N == N && pl->M == M && pl->p == p &&
        pl->K == K) {
      *out = pl;
      return ME_OK;
    }
  PredPlan* pl = new PredPlan();
  pl->dev = dev; pl->W = W; pl->H = H; pl->N = N; pl->M = M; pl->p = p; pl->K = K;
  const int st = build_pred_plan(pl);
  if (st) {
    if (pl->mem) cudaFree(pl->mem);
    delete pl;
    return st;
  }
  g_pred_plans.push_back(pl);
  *out = pl;
  return ME_OK;
}

template <int N, int M, int T>
static int launch_volume_t(const PredFrames& fr, int K, int W, int H, int p, int vstride,
                           uint16_t* vol, const FsPlan& pl, cudaStream_t s) {
  auto kern = k_sad_volume<N, M, T>;
  {
    const int st = ensure_dynamic_smem((const void*)kern, pl.smem);
    if (st) return st;
  }
  const int BW = W / N, BH = H / M;
  const int bpc = pl.threads / pl.G;
  const dim3 grid(((BW + bpc - 1) / bpc) * BH, K);
  kern<<<grid, pl.threads, pl.smem, s>>>(fr, W, H, p, pl.G, vstride, vol);
  ME_CUDA(cudaGetLastError());
  return ME_OK;
}

static int launch_volume(const PredFrames& fr, int K, int W, int H, int N, int M, int p,
                         int vstride, uint16_t* vol, cudaStream_t s) {
  if (fsbm_pipe_applies(N, M, p)) {
    // 16x16: the pipelined persistent search in its volume mode
    PipeOut po;
    std::memset(&po, 0, sizeof(po));
    po.vol = vol;
    po.vstride = vstride;
    return launch_fsbm_pipe_mode(kPipeVolume, fr.f, K, W, H, p, 0u, po, s);
  }
  const FsPlan pl = fs_plan(N, M, p, W / N);
  const int bpc = pl.threads / pl.G;
  if (N == 16 && M == 16 && pl.T == 13 && (bpc - 1) * N + 2 * p + 1 + N - 4 <= kVolSP) {
    auto kern = k_sad_volume<16, 16, 13, kVolSP>;
    const size_t smem = fs_smem_bytes<16, 16, 13>(fs_geom<16, 16, 13>(p, bpc, pl.G, 0, 0, kVolSP));
    const int st = ensure_dynamic_smem((const void*)kern, smem);
    if (st) return st;
    const int BW = W / N, BH = H / M;
    const dim3 grid(((BW + bpc - 1) / bpc) * BH, K);
    kern<<<grid, pl.threads, smem, s>>>(fr, W, H, p, pl.G, vstride, vol);
    ME_CUDA(cudaGetLastError());
    return ME_OK;
  }
  ME_DISPATCH_FS(launch_volume_t, fr, K, W, H, p, vstride, vol, pl, s);
}

static int run_pred(const PredFrames& fr, int K, int W, int H, int N, int M, int p, uint32_t lam,
                    int16_t* mv, uint32_t* J, uint32_t* sad, cudaStream_t s) {
  PredPlan* pl = nullptr;
  int st = get_pred_plan(W, H, N, M, p, K, &pl);
  if (st) return st;
  // runs that share a plan's scratch are ordered on the GPU, whatever their streams
  std::lock_guard<std::mutex> lk(pl->mu);
  if (pl->ran) ME_CUDA(cudaStreamWaitEvent(s, pl->last, 0));
  k_pred_begin<<<1, 1, 0, s>>>(pl->ctrl);
  ME_CUDA(cudaGetLastError());
  st = launch_volume(fr, K, W, H, N, M, p, pl->vstride, pl->vol, s);
  if (st) return st;
  const int BW = W / N, nbf = BW * (H / M);
  // prune (the pre-wait candidate list) for short runs, whose time is the
  // dependency chain; long runs are bound by the work per block
  int prune = K <= kPredPruneMaxK ? 1 : 0;
  if (const char* e = std::getenv("ME_PRED_PRUNE")) prune = e[0] == '1' ? 1 : 0;
  k_pred_wave<<<pl->grid, kPredThreads, pl->smem, s>>>(pl->items, pl->total, BW, nbf, p, lam,
                                                       pl->vol, pl->vstride, pl->flags, pl->ctrl,
                                                       mv, J, sad, prune);
  ME_CUDA(cudaGetLastError());
  ME_CUDA(cudaEventRecord(pl->last, s));
  pl->ran = true;
  return ME_OK;
}

}  // namespace me

using namespace me;

extern "C" {

int me_fsbm_pred(const uint8_t* cur, const uint8_t* ref, int W, int H, int N, int M, int p,
                 uint32_t lambda_q8, int16_t* mv_out, uint32_t* J_out, uint32_t* sad_out,
                 me_stream_t stream) {
  if (!cur || !ref || !mv_out || !J_out) return ME_ERR_ARG;
  if (!aligned4(cur) || !aligned4(ref)) return ME_ERR_ARG;
  int st = check_frame_args(W, H, N, M, p, lambda_q8);
  if (st) return st;
  PredFrames fr;
  std::memset(&fr, 0, sizeof(fr));
  fr.f[0] = ref;
  fr.f[1] = cur;
  return run_pred(fr, 1, W, H, N, M, p, lambda_q8, mv_out, J_out, sad_out,
                  reinterpret_cast<cudaStream_t>(stream));
}

int me_fsbm_pred_sequence(const uint8_t* const* frames, int K, int W, int H, int N, int M, int p,
                          uint32_t lambda_q8, int16_t* mv_out, uint32_t* J_out, uint32_t* sad_out,
                          me_stream_t stream) {
  if (!frames || K < 1 || K > kPredMaxK || !mv_out || !J_out) return ME_ERR_ARG;
  int st = check_frame_args(W, H, N, M, p, lambda_q8);
  if (st) return st;
  PredFrames fr;
  std::memset(&fr, 0, sizeof(fr));
  for (int k = 0; k <= K; k++) {
    if (!frames[k] || !aligned4(frames[k])) return ME_ERR_ARG;
    fr.f[k] = frames[k];
  }
  return run_pred(fr, K, W, H, N, M, p, lambda_q8, mv_out, J_out, sad_out,
                  reinterpret_cast<cudaStream_t>(stream));
}

int me_fsbm_pred_status(int W, int H, int N, int M, int p, int K, me_stream_t stream) {
  if (K < 1 || K > kPredMaxK) return ME_ERR_ARG;
  int st = check_frame_args(W, H, N, M, p, 0);
  if (st) return st;
  PredPlan* pl = nullptr;
  st = get_pred_plan(W, H, N, M, p, K, &pl);
  if (st) return st;
  ME_CUDA(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
  PredCtrl c;
  ME_CUDA(cudaMemcpy(&c, pl->ctrl, sizeof(c), cudaMemcpyDeviceToHost));
  return c.error ? c.error : ME_OK;
}

}  // extern "C"

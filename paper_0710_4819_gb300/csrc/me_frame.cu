// me_frame.cu -- the per-frame C ABI: padding, Intra_SAD, FSBM and ACBM for
// one frame pair, with their kernels.
//
//   me_fsbm : one launch; full search of every block (Sec. 2.3) in the form
//             the autotuner picked for the shape: the pipelined searches of
//             me_sequence.cu (k_fsbm_pipe, k_fsbm_pipe_tab) or the per-group
//             k_fsbm
//   me_acbm : tuned between the persistent kernel of me_sequence.cu over the
//             one pair and the wave graph here: k_acbm_prologue (padding,
//             Intra_SAD), k_acbm_spec (the likely fallbacks guessed from the
//             early predictors and searched in full, all at once), then one
//             k_pbm_wave per anti-diagonal wave w = x + 2y of the block grid
//             (PBM + the Sec. 3.2 test; a failing block takes its early
//             search's result).  Wave w+1 starts after wave w, so every
//             spatial predictor is final when it is read.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "me_device.cuh"
#include "me_host.h"
#include "me_search.cuh"

namespace me {

__global__ void k_pad_ref(const uint8_t* __restrict__ ref, int W, int H, PadGeom g,
                          uint8_t* __restrict__ out) {
  const int chunks = g.pitch / 16;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)g.rows * chunks) return;
  const int y = (int)(i / chunks), cx = (int)(i % chunks) * 16;
  const uint8_t* src = ref + (size_t)clampi(y - g.P, 0, H - 1) * W;
  uint32_t w[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    uint32_t v = 0;
#pragma unroll
    for (int b = 0; b < 4; b++) v |= (uint32_t)src[clampi(cx + 4 * k + b - g.P, 0, W - 1)] << (8 * b);
    w[k] = v;
  }
  *reinterpret_cast<uint4*>(out + (size_t)y * g.pitch + cx) = make_uint4(w[0], w[1], w[2], w[3]);
}

template <int N, int M>
__global__ void __launch_bounds__(256) k_intra_sad(const uint8_t* __restrict__ cur, int W, int H,
                                                   uint32_t* __restrict__ out) {
  const int BW = W / N, nb = BW * (H / M);
  const int b = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (b >= nb) return;
  const uint32_t v = warp_intra_sad<N, M>(cur, W, (b % BW) * N, (b / BW) * M);
  if ((threadIdx.x & 31) == 0) out[b] = v;
}

// FSBM over a whole frame: CTA = blockDim/G adjacent blocks of one block row,
// G threads per block.
template <int N, int M, int T>
__global__ void __launch_bounds__(kMaxThreads) k_fsbm(const uint8_t* __restrict__ cur,
                                                      const uint8_t* __restrict__ ref, int W, int H,
                                                      int p, int G, uint32_t lam,
                                                      int16_t* __restrict__ mv_out,
                                                      uint32_t* __restrict__ J_out,
                                                      uint32_t* __restrict__ sad_out) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ unsigned long long keys[16];
  const int BW = W / N;
  const int bpc = blockDim.x / G;
  const int gpr = (BW + bpc - 1) / bpc;
  const int by = blockIdx.x / gpr, bx0 = (blockIdx.x % gpr) * bpc;
  const int nb = min(bpc, BW - bx0);
  const FsGeom g = fs_geom<N, M, T>(p, nb, G);
  fs_group<N, M, T>(cur, ref, W, H, bx0 * N, by * M, g, lam, smem, keys);
  if ((int)threadIdx.x < nb) {
    const Decoded d = decode_key(keys[threadIdx.x], p, lam);
    const int b = by * BW + bx0 + threadIdx.x;
    mv_out[2 * b] = (int16_t)d.mvx;
    mv_out[2 * b + 1] = (int16_t)d.mvy;
    J_out[b] = d.J;
    if (sad_out) sad_out[b] = d.sad;
  }
}

// ACBM prologue of one frame, one launch: stores the call's arguments in the
// device slot the wave kernels read, pads the reference (a1), computes the
// scaled Intra_SAD of every block (a2) and clears the early-search states.
template <int N, int M>
__global__ void __launch_bounds__(256) k_acbm_prologue(AcbmArgs a, AcbmArgs* __restrict__ slot,
                                                       PadGeom pg, int W, int H,
                                                       uint8_t* __restrict__ refpad,
                                                       uint32_t* __restrict__ intra,
                                                       unsigned long long* __restrict__ keys,
                                                       int* __restrict__ done) {
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthr = (long long)gridDim.x * blockDim.x;
  if (gtid == 0) *slot = a;
  const int nblk = (W / N) * (H / M);
  for (long long i = gtid; i < nblk; i += nthr) {
    keys[i] = kNoKey;
    done[i] = 0;
  }
  const int chunks = pg.pitch / 16;
  for (long long i = gtid; i < (long long)pg.rows * chunks; i += nthr) {
    const int y = (int)(i / chunks), cx = (int)(i % chunks) * 16;
    const uint8_t* src = a.ref + (size_t)clampi(y - pg.P, 0, H - 1) * W;
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      uint32_t v = 0;
#pragma unroll
      for (int b = 0; b < 4; b++) v |= (uint32_t)src[clampi(cx + 4 * k + b - pg.P, 0, W - 1)] << (8 * b);
      w[k] = v;
    }
    *reinterpret_cast<uint4*>(refpad + (size_t)y * pg.pitch + cx) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  const int BW = W / N, nb = BW * (H / M);
  const long long warps = nthr / 32;
  for (long long b = gtid / 32; b < nb; b += warps) {
    const uint32_t v = warp_intra_sad<N, M>(a.cur, W, (int)(b % BW) * N, (int)(b / BW) * M);
    if ((threadIdx.x & 31) == 0) intra[b] = v;
  }
}

// The frame's likely fallbacks, searched before the wave chain: one CTA per
// block; warp 0 stages the block's window and evaluates the PBM predictors
// known before any wave runs (the previous field's 3x3 and the zero vector,
// pbm_part_a); a block that already fails both conditions with them (it
// nearly always fails with all of them) is searched in full by the whole CTA
// and its key left in bkeys[b] with bdone[b] = kSpecDone, for the PBM wave to
// publish if the block fails there.  The result never depends on the guess.
constexpr int kSpecDone = -1;

template <int N, int M, int T>
__global__ void __launch_bounds__(256) k_acbm_spec(const AcbmArgs* __restrict__ ap,
                                                   const uint8_t* __restrict__ refpad, PadGeom pg,
                                                   const uint32_t* __restrict__ intra, int W, int H,
                                                   int p, unsigned long long* __restrict__ bkeys,
                                                   int* __restrict__ bdone) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ unsigned long long keys[16];
  __shared__ int s_go;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const AcbmArgs a = *ap;
  const int BW = W / N, BH = H / M, b = blockIdx.x;
  const int bx = b % BW, by = b / BW;
  if (warp == 0) {
    uint32_t* win = smem;
    uint32_t* curs = smem + pbm_win_words(N, M, p);
    const PbmWin wg = pbm_stage<N, M>(a.cur, refpad, pg, W, p, bx * N, by * M, curs, win);
    int cx = 0, cy = 0;
    bool valid = false;
    if (lane >= 4 && lane < 13) {
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
    const PbmPart pa = pbm_part_a<N, M>(cx, cy, valid, wg, p, a.lam, curs, win);
    if (lane == 0)
      s_go = pbm_would_fail<N, M>(pa.best, p, a.lam, intra[b], a.alpha, a.beta, a.gnum, a.gden,
                                  a.qp) ? 1 : 0;
  }
  __syncthreads();
  if (!s_go) return;
  const FsGeom g = fs_geom<N, M, T>(p, 1, blockDim.x);
  fs_group<N, M, T>(a.cur, a.ref, W, H, bx * N, by * M, g, a.lam, smem, keys, nullptr,
                    FsPad{refpad, pg.pitch, pg.P, pg.rows});
  if (threadIdx.x == 0) {
    bkeys[b] = keys[0];
    bdone[b] = kSpecDone;
  }
}

// ACBM, PBM stage of wave w: one warp per block of the wave.  Passing blocks
// get their final outputs; failing ones take the result of their early full
// search (k_acbm_spec).  A failing block without one (its early predictors
// passed: about 4 in a million blocks on the 1080p sequence) is searched in
// full by its own warp from the window it has staged, so the wave needs no
// second launch.
template <int N, int M>
__global__ void __launch_bounds__(128) k_pbm_wave(const AcbmArgs* __restrict__ ap,
                                                  const uint8_t* __restrict__ refpad,
                                                  PadGeom pg, const uint32_t* __restrict__ intra,
                                                  int W, int H, int p, int w, int ylo, int count,
                                                  const unsigned long long* __restrict__ bkeys,
                                                  const int* __restrict__ bdone) {
  __shared__ uint32_t curs[4][M * (N / 4)];
  extern __shared__ __align__(16) uint32_t wins[];   // 4 x pbm_win_words
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int idx = blockIdx.x * 4 + warp;
  if (idx >= count) return;
  const AcbmArgs a = *ap;
  const int by = ylo + idx, bx = w - 2 * by;
  const int BW = W / N, b = by * BW + bx;
  const int n = 2 * p + 1;
  if (!ME_CHECK(bx >= 0 && bx < BW && by >= 0 && by < H / M, "ME_CHECK pbm_wave w %d bx %d by %d\n",
                w, bx, by))
    return;
  uint32_t* win = wins + warp * pbm_win_words(N, M, p);
  const PbmResult r = warp_pbm<N, M>(a.cur, refpad, pg, W, H, p, a.lam, a.mv, a.prev, bx, by,
                                     intra[b], a.alpha, a.beta, a.gnum, a.gden, a.qp, a.refine,
                                     curs[warp], win);
  unsigned long long key = r.key;
  bool full = false;
  if (!r.pass) {
    full = true;
    if (bdone[b] == kSpecDone) {
      key = bkeys[b];
    } else {
      // every position of the window, from the staged window (Sec. 2.3)
      const PbmWin wg = pbm_win(N, M, p, bx * N, pg.P);
      unsigned long long best = kNoKey;
      for (int c = lane; c < n * n; c += 32) {
        const int mvx = c % n - p, mvy = c / n - p;
        const uint32_t sad = lane_sad_rows<N, M>(curs[warp], win, wg, p, mvx, mvy, 0, M);
        best = umin64(best, make_key(256u * sad + a.lam * (uint32_t)(mv_bits(mvx) + mv_bits(mvy)),
                                     mvx, mvy, p));
      }
      key = warp_min64(best);
    }
  }
  if (lane == 0) {
    const Decoded d = decode_key(key, p, a.lam);
    a.mv[2 * b] = (int16_t)d.mvx;
    a.mv[2 * b + 1] = (int16_t)d.mvy;
    a.J[b] = d.J;
    a.mask[b] = full ? 1 : 0;
    if (a.sad) a.sad[b] = d.sad;
    if (a.load) a.load[b] = full ? (uint32_t)(n * n) : (uint32_t)r.load;
  }
}

// ------------------------------------------------------------------ plan

static const int kT16[] = {8, 11, 13, 16};  // run lengths instantiated for 16x16
static const int kTOther[] = {8};

template <int N, int M, int T>
static size_t smem_for(int p, int bpc) {
  FsGeom g = fs_geom<N, M, T>(p, bpc, 32);
  return fs_smem_bytes<N, M, T>(g);
}

static size_t smem_dispatch(int N, int M, int T, int p, int bpc) {
#define ME_SM(n, m, t) \
  if (N == n && M == m && T == t) return smem_for<n, m, t>(p, bpc);
  ME_SM(16, 16, 8) ME_SM(16, 16, 11) ME_SM(16, 16, 13) ME_SM(16, 16, 16)
  ME_SM(16, 8, 8) ME_SM(16, 4, 8) ME_SM(8, 16, 8) ME_SM(8, 8, 8) ME_SM(8, 4, 8)
  ME_SM(4, 16, 8) ME_SM(4, 8, 8) ME_SM(4, 4, 8)
#undef ME_SM
  return 0;
}

// Instructions one thread spends on one task (SAD steps, shifted-word loads,
// cost/key epilogue, loop overhead).
static double task_cost(int N, int M, int T) {
  const int NW = N / 4;
  return (double)T * M * NW + (double)(T + M - 1) * NW + 7.0 * T + 20.0;
}

// Staging instructions per CTA (raw words + shifted words + tables).
static double stage_cost(int N, int M, int T, int p, int bpc) {
  const int n = 2 * p + 1, rows = ((n + T - 1) / T) * T + M - 1;
  const int pos = (bpc - 1) * N + n + N - 4;
  return (double)rows * (pos * 6.0 + (pos / 4 + 2) * 4.0);
}

FsPlan fs_plan(int N, int M, int p, int bpc_max) {
  const int n = 2 * p + 1;
  const int* Ts = (N == 16 && M == 16) ? kT16 : kTOther;
  const int nT = (N == 16 && M == 16) ? 4 : 1;
  // fallback (always valid): the first run length, one block of 128 threads
  FsPlan best{Ts[0], 128, 128, smem_dispatch(N, M, Ts[0], p, 1), 1};
  double best_cost = 1e300;
  static const int kG[] = {8, 16, 32, 64, 128, 256, 512};
  static const int kThr[] = {64, 128, 256, 512};
  for (int ti = 0; ti < nT; ti++) {
    const int T = Ts[ti];
    const int tasks = n * ((n + T - 1) / T);
    for (int G : kG) {
      const int rounds = (tasks + G - 1) / G;
      for (int thr : kThr) {
        if (thr < G || thr % G) continue;
        const int bpc = thr / G;
        if (bpc > std::min(bpc_max, 16)) continue;
        const size_t smem = smem_dispatch(N, M, T, p, bpc);
        if (smem > 110 * 1024) continue;
        const double per_thread = rounds * task_cost(N, M, T) + stage_cost(N, M, T, p, bpc) / thr;
        // resident warps per SM at 128 registers per thread and 228 KB of
        // shared memory; fewer than 16 leave the SAD pipe under-fed
        const int warps = thr / 32;
        int ctas = std::min(64 / warps, 65536 / (thr * 128));
        ctas = std::min(ctas, (int)((228 * 1024) / (smem + 1024)));
        if (ctas < 1) continue;
        const double occ = std::min(1.0, (double)(ctas * warps) / 16.0);
        const double cost = per_thread * thr / ((double)bpc * n * n) / occ;
        if (cost < best_cost * 0.999) {
          best_cost = cost;
          best = FsPlan{T, G, thr, smem, 1};
        }
      }
    }
  }
  return best;
}

// The k plans of lowest modelled cost with distinct (T, G, threads), best
// first (the first equals fs_plan's): the candidates the autotuner times.
std::vector<FsPlan> fs_plans_ranked(int N, int M, int p, int bpc_max, int k) {
  const int n = 2 * p + 1;
  const int* Ts = (N == 16 && M == 16) ? kT16 : kTOther;
  const int nT = (N == 16 && M == 16) ? 4 : 1;
  std::vector<std::pair<double, FsPlan>> all;
  static const int kG[] = {8, 16, 32, 64, 128, 256, 512};
  static const int kThr[] = {64, 128, 256, 512};
  for (int ti = 0; ti < nT; ti++) {
    const int T = Ts[ti];
    const int tasks = n * ((n + T - 1) / T);
    for (int G : kG) {
      const int rounds = (tasks + G - 1) / G;
      for (int thr : kThr) {
        if (thr < G || thr % G) continue;
        const int bpc = thr / G;
        if (bpc > std::min(bpc_max, 16)) continue;
        const size_t smem = smem_dispatch(N, M, T, p, bpc);
        if (smem > 110 * 1024) continue;
        const double per_thread = rounds * task_cost(N, M, T) + stage_cost(N, M, T, p, bpc) / thr;
        const int warps = thr / 32;
        int ctas = std::min(64 / warps, 65536 / (thr * 128));
        ctas = std::min(ctas, (int)((228 * 1024) / (smem + 1024)));
        if (ctas < 1) continue;
        const double occ = std::min(1.0, (double)(ctas * warps) / 16.0);
        all.push_back({per_thread * thr / ((double)bpc * n * n) / occ, FsPlan{T, G, thr, smem, 1}});
      }
    }
  }
  std::stable_sort(all.begin(), all.end(), [](const std::pair<double, FsPlan>& x,
                                              const std::pair<double, FsPlan>& y) {
    return x.first < y.first * 0.999;
  });
  std::vector<FsPlan> out{fs_plan(N, M, p, bpc_max)};
  for (const auto& e : all) {
    if ((int)out.size() >= k) break;
    bool dup = false;
    for (const FsPlan& o : out) dup |= o.T == e.second.T && o.G == e.second.G && o.threads == e.second.threads;
    if (!dup) out.push_back(e.second);
  }
  return out;
}

// Threads per block for a fixed run length and CTA size (persistent kernels,
// whose launch fixes both): the G with the lowest modelled cost per candidate.
FsPlan fs_plan_fixed(int N, int M, int T, int p, int thr, int bpc_max, size_t smem_limit) {
  const int n = 2 * p + 1;
  const int tasks = n * ((n + T - 1) / T);
  FsPlan best{T, thr, thr, smem_dispatch(N, M, T, p, 1), 1};
  double best_cost = 1e300;
  static const int kG[] = {8, 16, 32, 64, 128, 256, 512};
  for (int G : kG) {
    if (thr < G || thr % G) continue;
    const int bpc = thr / G;
    if (bpc > std::min(bpc_max, 16)) continue;
    const size_t smem = smem_dispatch(N, M, T, p, bpc);
    if (smem > smem_limit) continue;
    const int rounds = (tasks + G - 1) / G;
    const double per_thread = rounds * task_cost(N, M, T) + stage_cost(N, M, T, p, bpc) / thr;
    const double cost = per_thread * thr / ((double)bpc * n * n);
    if (cost < best_cost * 0.999) {
      best_cost = cost;
      best = FsPlan{T, G, thr, smem, 1};
    }
  }
  return best;
}

// Plan for searching single blocks where latency matters (the early ACBM
// searches run before the wave chain starts): S CTAs per block, each over a slice of about n/S
// mvx columns with one task per thread (at most 512 threads), choosing the run
// length and S with the fewest instructions per thread, plus a per-slice
// charge for the merge and for the SMs the extra CTAs take.
FsPlan fs_plan_latency(int N, int M, int p) {
  const int n = 2 * p + 1;
  const int* Ts = (N == 16 && M == 16) ? kT16 : kTOther;
  const int nT = (N == 16 && M == 16) ? 4 : 1;
  FsPlan best{Ts[0], 128, 128, smem_dispatch(N, M, Ts[0], p, 1), 1};
  double best_lat = 1e300;
  for (int ti = 0; ti < nT; ti++) {
    const int T = Ts[ti];
    const size_t smem = smem_dispatch(N, M, T, p, 1);
    if (smem > 200 * 1024) continue;
    const int nseg = (n + T - 1) / T;
    for (int S = 1; S <= 8 && S <= n; S++) {
      const int nc = (n + S - 1) / S, tasks = nc * nseg;
      const int thr = std::min(kMaxThreads, std::max(64, (tasks + 31) / 32 * 32));
      const int rounds = (tasks + thr - 1) / thr;
      // clocks: warps per SM sub-partition x (SAD steps at 2 clocks each, or
      // the issue of all instructions), one global round trip for the window,
      // and the merge of S > 1 slices
      const int wps = (thr / 32 + 3) / 4;
      const double lat = wps * rounds * std::max(2.0 * T * M * (N / 4), task_cost(N, M, T)) +
                         1000.0 + (S > 1 ? 400.0 : 0.0) + 50.0 * S;
      if (lat < best_lat * 0.999) {
        best_lat = lat;
        best = FsPlan{T, thr, thr, smem, S};
      }
    }
  }
  return best;
}

// Optional plan override "T,G,threads" (for tile sweeps); ignored unless
// the run length is one instantiated for the block shape.
static bool plan_override(int N, int M, FsPlan* pl, int p, int bpc_max) {
  const char* e = std::getenv("ME_FS_PLAN");
  if (!e) return false;
  int T = 0, G = 0, thr = 0;
  if (std::sscanf(e, "%d,%d,%d", &T, &G, &thr) != 3) return false;
  if (!(G == 8 || G == 16 || (G >= 32 && G % 32 == 0)) || thr < 32 || thr > kMaxThreads ||
      thr % 32 || thr % G)
    return false;
  const int bpc = thr / G;
  const size_t smem = smem_dispatch(N, M, T, p, bpc);
  if (smem == 0 || bpc > std::min(bpc_max, 16) || smem > 200 * 1024) return false;
  *pl = FsPlan{T, G, thr, smem, 1};
  return true;
}

template <int N, int M, int T>
static int launch_fsbm_t(const uint8_t* cur, const uint8_t* ref, int W, int H, int p, uint32_t lam,
                         int16_t* mv, uint32_t* J, uint32_t* sad, const FsPlan& pl, cudaStream_t s) {
  auto kern = k_fsbm<N, M, T>;
  {
    const int st = ensure_dynamic_smem((const void*)kern, pl.smem);
    if (st) return st;
  }
  const int BW = W / N, BH = H / M;
  const int bpc = pl.threads / pl.G;
  const int grid = ((BW + bpc - 1) / bpc) * BH;
  kern<<<grid, pl.threads, pl.smem, s>>>(cur, ref, W, H, p, pl.G, lam, mv, J, sad);
  ME_CUDA(cudaGetLastError());
  return ME_OK;
}

int launch_fsbm(const uint8_t* cur, const uint8_t* ref, int W, int H, int N, int M, int p,
                uint32_t lam, int16_t* mv, uint32_t* J, uint32_t* sad, cudaStream_t s) {
  FsPlan pl = fs_plan(N, M, p, W / N);
  if (!plan_override(N, M, &pl, p, W / N)) {
    const uint8_t* frames[2] = {ref, cur};
    return fsbm_tuned(frames, 1, W, H, N, M, p, lam, mv, J, sad, s);
  }
  ME_DISPATCH_FS(launch_fsbm_t, cur, ref, W, H, p, lam, mv, J, sad, pl, s);
}

#define ME_DISPATCH_NM(FN, ...)                                  \
  do {                                                           \
    if (N == 16 && M == 16) return FN<16, 16>(__VA_ARGS__);      \
    if (N == 16 && M == 8) return FN<16, 8>(__VA_ARGS__);        \
    if (N == 16 && M == 4) return FN<16, 4>(__VA_ARGS__);        \
    if (N == 8 && M == 16) return FN<8, 16>(__VA_ARGS__);        \
    if (N == 8 && M == 8) return FN<8, 8>(__VA_ARGS__);          \
    if (N == 8 && M == 4) return FN<8, 4>(__VA_ARGS__);          \
    if (N == 4 && M == 16) return FN<4, 16>(__VA_ARGS__);        \
    if (N == 4 && M == 8) return FN<4, 8>(__VA_ARGS__);          \
    if (N == 4 && M == 4) return FN<4, 4>(__VA_ARGS__);          \
    return ME_ERR_ARG;                                           \
  } while (0)

template <int N, int M>
static int launch_intra_t(const uint8_t* cur, int W, int H, uint32_t* out, cudaStream_t s) {
  const int nb = (W / N) * (H / M);
  k_intra_sad<N, M><<<(nb + 7) / 8, 256, 0, s>>>(cur, W, H, out);
  ME_CUDA(cudaGetLastError());
  return ME_OK;
}

int launch_intra(const uint8_t* cur, int W, int H, int N, int M, uint32_t* out, cudaStream_t s) {
  ME_DISPATCH_NM(launch_intra_t, cur, W, H, out, s);
}

int launch_pad(const uint8_t* ref, int W, int H, int p, uint8_t* out, cudaStream_t s) {
  const PadGeom g = pad_geom(W, H, p);
  const long long n = (long long)g.rows * (g.pitch / 16);
  k_pad_ref<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ref, W, H, g, out);
  ME_CUDA(cudaGetLastError());
  return ME_OK;
}

template <int N, int M>
static int launch_pbm_wave_t(const AcbmArgs* ap, const uint8_t* refpad, const PadGeom& pg,
                             const uint32_t* intra, int W, int H, int p, int w, int ylo, int count,
                             const unsigned long long* bkeys, const int* bdone, cudaStream_t s) {
  const size_t smem = 4 * 4 * (size_t)pbm_win_words(N, M, p);
  {
    const int st = ensure_dynamic_smem((const void*)k_pbm_wave<N, M>, smem);
    if (st) return st;
  }
  k_pbm_wave<N, M><<<(count + 3) / 4, 128, smem, s>>>(ap, refpad, pg, intra, W, H, p, w, ylo,
                                                      count, bkeys, bdone);
  ME_CUDA(cudaGetLastError());
  return ME_OK;
}

static int launch_pbm_wave(int N, int M, const AcbmArgs* ap, const uint8_t* refpad,
                           const PadGeom& pg, const uint32_t* intra, int W, int H, int p, int w,
                           int ylo, int count, const unsigned long long* bkeys, const int* bdone,
                           cudaStream_t s) {
  ME_DISPATCH_NM(launch_pbm_wave_t, ap, refpad, pg, intra, W, H, p, w, ylo, count, bkeys, bdone, s);
}

template <int N, int M, int T>
static int launch_spec_t(const AcbmArgs* ap, const uint8_t* refpad, const PadGeom& pg,
                         const uint32_t* intra, int W, int H, int p, unsigned long long* bkeys,
                         int* bdone, cudaStream_t s) {
  const FsGeom g = fs_geom<N, M, T>(p, 1, 256);
  const size_t smem = std::max(fs_smem_bytes<N, M, T>(g),
                               4 * ((size_t)pbm_win_words(N, M, p) + M * (N / 4)));
  {
    const int st = ensure_dynamic_smem((const void*)k_acbm_spec<N, M, T>, smem);
    if (st) return st;
  }
  k_acbm_spec<N, M, T><<<(W / N) * (H / M), 256, smem, s>>>(ap, refpad, pg, intra, W, H, p, bkeys,
                                                           bdone);
  ME_CUDA(cudaGetLastError());
  return ME_OK;
}

static int launch_spec(int N, int M, const AcbmArgs* ap, const uint8_t* refpad, const PadGeom& pg,
                       const uint32_t* intra, int W, int H, int p, unsigned long long* bkeys,
                       int* bdone, cudaStream_t s) {
  const FsPlan pl = fs_plan_latency(N, M, p);
  ME_DISPATCH_FS(launch_spec_t, ap, refpad, pg, intra, W, H, p, bkeys, bdone, s);
}

template <int N, int M>
static int launch_prologue_t(const AcbmArgs& a, AcbmArgs* slot, const PadGeom& pg, int W, int H,
                             uint8_t* refpad, uint32_t* intra, unsigned long long* bkeys,
                             int* bdone, cudaStream_t s) {
  const long long work = std::max<long long>((long long)pg.rows * (pg.pitch / 16),
                                             32LL * (W / N) * (H / M));
  int nsm = 1;
  { const int e = sm_count(&nsm); if (e) return e; }
  const int grid = (int)std::min<long long>((work + 255) / 256, nsm * 8LL);
  k_acbm_prologue<N, M><<<grid, 256, 0, s>>>(a, slot, pg, W, H, refpad, intra, bkeys, bdone);
  ME_CUDA(cudaGetLastError());
  return ME_OK;
}

static int launch_prologue(int N, int M, const AcbmArgs& a, AcbmArgs* slot, const PadGeom& pg,
                           int W, int H, uint8_t* refpad, uint32_t* intra,
                           unsigned long long* bkeys, int* bdone, cudaStream_t s) {
  ME_DISPATCH_NM(launch_prologue_t, a, slot, pg, W, H, refpad, intra, bkeys, bdone, s);
}

AcbmScratch acbm_scratch_layout(int W, int H, int N, int M, int p) {
  const PadGeom pg = pad_geom(W, H, p);
  const int nb = (W / N) * (H / M);
  AcbmScratch l;
  l.off_args = 0;
  l.off_pad = align_up(sizeof(AcbmArgs), 256);
  l.off_intra = align_up(l.off_pad + (size_t)pg.pitch * pg.rows, 256);
  l.off_keys = align_up(l.off_intra + 4 * (size_t)nb, 256);
  l.off_done = align_up(l.off_keys + 8 * (size_t)nb, 256);
  l.total = align_up(l.off_done + 4 * (size_t)nb, 256);
  return l;
}

// Enqueues the whole ACBM frame given scratch memory of acbm_scratch_layout.
int enqueue_acbm(const AcbmArgs& a, int W, int H, int N, int M, int p, uint8_t* scratch,
                        cudaStream_t s) {
  const AcbmScratch l = acbm_scratch_layout(W, H, N, M, p);
  const PadGeom pg = pad_geom(W, H, p);
  AcbmArgs* slot = reinterpret_cast<AcbmArgs*>(scratch + l.off_args);
  uint8_t* refpad = scratch + l.off_pad;
  uint32_t* intra = reinterpret_cast<uint32_t*>(scratch + l.off_intra);
  unsigned long long* bkeys = reinterpret_cast<unsigned long long*>(scratch + l.off_keys);
  int* bdone = reinterpret_cast<int*>(scratch + l.off_done);
  const Waves wv = make_waves(W / N, H / M);
  int st = launch_prologue(N, M, a, slot, pg, W, H, refpad, intra, bkeys, bdone, s);
  if (st) return st;
  st = launch_spec(N, M, slot, refpad, pg, intra, W, H, p, bkeys, bdone, s);
  if (st) return st;
  for (int w = 0; w < wv.n; w++) {
    const int c = wv.count(w);
    if (c == 0) continue;
    st = launch_pbm_wave(N, M, slot, refpad, pg, intra, W, H, p, w, wv.ylo(w), c, bkeys, bdone, s);
    if (st) return st;
  }
  return ME_OK;
}

// ------------------------------------------------------------------ ACBM plans
// One cached plan per (device, W, H, N, M, p): scratch memory and a CUDA graph
// of the whole frame (prologue, early searches, one kernel per wave), captured once and
// replayed.  A call updates the prologue node's by-value arguments and
// launches the graph; CUDA orders launches of one executable graph, so calls
// that share a plan (even on different streams) never overlap on the GPU.
struct AcbmPlan {
  int dev, W, H, N, M, p;
  uint8_t* scratch = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t prologue = nullptr;
  cudaKernelNodeParams kp{};
  std::mutex mu;
};

static std::mutex g_plan_mu;
static std::vector<AcbmPlan*> g_plans;

static int build_plan(AcbmPlan* pl) {
  const AcbmScratch l = acbm_scratch_layout(pl->W, pl->H, pl->N, pl->M, pl->p);
  ME_CUDA(cudaMalloc(&pl->scratch, l.total));
  cudaStream_t cs;
  ME_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  AcbmArgs dummy;
  std::memset(&dummy, 0, sizeof(dummy));
  dummy.gden = 1;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  int st = ME_OK;
  if (e == cudaSuccess) {
    st = enqueue_acbm(dummy, pl->W, pl->H, pl->N, pl->M, pl->p, pl->scratch, cs);
    e = cudaStreamEndCapture(cs, &pl->graph);
  }
  cudaStreamDestroy(cs);
  if (st) return st;
  ME_CUDA(e);
  size_t nroot = 1;
  ME_CUDA(cudaGraphGetRootNodes(pl->graph, &pl->prologue, &nroot));
  if (nroot != 1) return ME_ERR_CUDA;
  ME_CUDA(cudaGraphKernelNodeGetParams(pl->prologue, &pl->kp));
  ME_CUDA(cudaGraphInstantiate(&pl->exec, pl->graph, 0));
  return ME_OK;
}

static int get_plan(int W, int H, int N, int M, int p, AcbmPlan** out) {
  int dev = 0;
  ME_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_plan_mu);
  for (AcbmPlan* pl : g_plans)
    if (pl->dev == dev && pl->W == W && pl->H == H && pl->N == N && pl->M == M && pl->p == p) {
      *out = pl;
      return ME_OK;
    }
  AcbmPlan* pl = new AcbmPlan();
  pl->dev = dev; pl->W = W; pl->H = H; pl->N = N; pl->M = M; pl->p = p;
  int st = build_plan(pl);
  if (st) {
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->scratch) cudaFree(pl->scratch);
    delete pl;
    return st;
  }
  g_plans.push_back(pl);
  *out = pl;
  return ME_OK;
}

static int launch_plan(AcbmPlan* pl, const AcbmArgs& a, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(pl->mu);
  // the prologue's first parameter is the AcbmArgs value; the rest stay
  void* argv[16];
  for (int i = 0; i < 11; i++) argv[i] = pl->kp.kernelParams[i];
  AcbmArgs val = a;
  argv[0] = &val;
  cudaKernelNodeParams kp = pl->kp;
  kp.kernelParams = argv;
  kp.extra = nullptr;
  ME_CUDA(cudaGraphExecKernelNodeSetParams(pl->exec, pl->prologue, &kp));
  ME_CUDA(cudaGraphLaunch(pl->exec, s));
  return ME_OK;
}

}  // namespace me

using namespace me;

extern "C" {

int me_padded_geometry(int W, int H, int p, int* pitch, int* rows, int* P) {
  if (W < 1 || H < 1 || W > 16384 || H > 16384) return ME_ERR_SHAPE;
  if (p < 1 || p > kMaxP) return ME_ERR_ARG;
  const PadGeom g = pad_geom(W, H, p);
  if (pitch) *pitch = g.pitch;
  if (rows) *rows = g.rows;
  if (P) *P = g.P;
  return ME_OK;
}

int me_pad_ref(const uint8_t* ref, int W, int H, int p, uint8_t* out, me_stream_t stream) {
  if (!ref || !out) return ME_ERR_ARG;
  if (W < 1 || H < 1 || W > 16384 || H > 16384) return ME_ERR_SHAPE;
  if (p < 1 || p > kMaxP || (reinterpret_cast<uintptr_t>(out) & 15u)) return ME_ERR_ARG;
  return launch_pad(ref, W, H, p, out, reinterpret_cast<cudaStream_t>(stream));
}

int me_intra_sad(const uint8_t* cur, int W, int H, int N, int M, uint32_t* out, me_stream_t stream) {
  if (!cur || !out) return ME_ERR_ARG;
  int st = check_frame_args(W, H, N, M, 1, 0);
  if (st) return st;
  return launch_intra(cur, W, H, N, M, out, reinterpret_cast<cudaStream_t>(stream));
}

int me_fsbm(const uint8_t* cur, const uint8_t* ref, int W, int H, int N, int M, int p,
            uint32_t lambda_q8, int16_t* mv_out, uint32_t* J_out, uint32_t* sad_out,
            me_stream_t stream) {
  if (!cur || !ref || !mv_out || !J_out) return ME_ERR_ARG;
  if (!aligned4(cur) || !aligned4(ref)) return ME_ERR_ARG;
  int st = check_frame_args(W, H, N, M, p, lambda_q8);
  if (st) return st;
  return launch_fsbm(cur, ref, W, H, N, M, p, lambda_q8, mv_out, J_out, sad_out,
                     reinterpret_cast<cudaStream_t>(stream));
}

int me_acbm(const uint8_t* cur, const uint8_t* ref, int W, int H, int N, int M, int p,
            uint32_t lambda_q8, const int16_t* prev_mv_field, const me_acbm_params* prm,
            int16_t* mv_out, uint32_t* J_out, uint8_t* fullsearch_mask_out, uint32_t* sad_out,
            uint32_t* load_out, me_stream_t stream) {
  if (!cur || !ref || !mv_out || !J_out || !fullsearch_mask_out) return ME_ERR_ARG;
  if (!aligned4(cur) || !aligned4(ref)) return ME_ERR_ARG;
  int st = check_frame_args(W, H, N, M, p, lambda_q8);
  if (st) return st;
  st = check_acbm_params(prm);
  if (st) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  AcbmArgs a;
  a.cur = cur; a.ref = ref; a.prev = prev_mv_field;
  a.mv = mv_out; a.J = J_out; a.mask = fullsearch_mask_out; a.sad = sad_out; a.load = load_out;
  a.lam = lambda_q8;
  a.alpha = prm->alpha; a.beta = prm->beta; a.gnum = prm->gamma_num; a.gden = prm->gamma_den;
  a.qp = prm->qp; a.refine = prm->refine;
  AcbmPlan* pl = nullptr;
  st = get_plan(W, H, N, M, p, &pl);
  if (st) return st;
  return acbm_pair_tuned(a, W, H, N, M, p, s, [&]() { return launch_plan(pl, a, s); });
}

}  // extern "C"

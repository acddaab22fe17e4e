// me_stats.cu -- the SAD-surface statistics of Sec. 3.1 and the known-motion
// experiment built on them (Fig. 3).
//
// For a block, the full search evaluates SAD(u, v) at all (2p+1)^2 integer
// positions.  Sec. 3.1 summarises that surface by SAD_min, its least value,
// and SAD_deviation = sum_{u,v} |SAD(u,v) - SAD_min|.  Every term is
// non-negative, so SAD_deviation = sum_{u,v} SAD(u,v) - (2p+1)^2 * SAD_min
// exactly: the kernel is the FSBM engine (fs_group) with two extra per-thread
// accumulators (the SAD sum and minimum of the runs it evaluates), reduced per
// block with the winning key.  The extra work is two integer operations per
// candidate against N*M/4 packed SAD steps, so the kernel keeps the FSBM
// kernel's SAD-rate roofline.
//
//   me_sad_deviation : one frame pair (K = 1, no vector error); for 16x16
//                      blocks the pipelined persistent search (statistics
//                      mode) instead
//   me_motion_study  : frames[1..K] each against frames[0] in one launch
//                      (blockIdx.y = k), with Intra_SAD and the L1 error
//                      against the known global vector of each frame
#include <cuda_runtime.h>

#include <cstring>

#include "me_device.cuh"
#include "me_host.h"
#include "me_search.cuh"

namespace me {

constexpr int kStudyMaxK = 64;

struct StudyFrames {
  const uint8_t* f[kStudyMaxK + 1];  // f[0] the original frame, f[1..K] the moved ones
};

template <int N, int M, int T>
__global__ void __launch_bounds__(kMaxThreads) k_fsbm_stats(
    StudyFrames fr, int W, int H, int p, int G, uint32_t lam, const int16_t* __restrict__ gmv,
    int16_t* __restrict__ mv_out, uint32_t* __restrict__ J_out, uint32_t* __restrict__ intra_out,
    uint32_t* __restrict__ smin_out, uint32_t* __restrict__ sdev_out,
    uint8_t* __restrict__ err_out) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ unsigned long long keys[16];
  __shared__ uint32_t st[32];
  const int BW = W / N, nbf = BW * (H / M);
  const int bpc = blockDim.x / G;
  const int gpr = (BW + bpc - 1) / bpc;
  const int k = blockIdx.y;
  const uint8_t* __restrict__ cur = fr.f[k + 1];
  const uint8_t* __restrict__ ref = fr.f[0];
  const int by = blockIdx.x / gpr, bx0 = (blockIdx.x % gpr) * bpc;
  const int nb = min(bpc, BW - bx0);
  const FsGeom g = fs_geom<N, M, T>(p, nb, G);
  fs_group<N, M, T, 0, true>(cur, ref, W, H, bx0 * N, by * M, g, lam, smem, keys, nullptr,
                             FsPad{nullptr, 0, 0, 0}, st);
  const size_t base = (size_t)k * nbf + (size_t)by * BW + bx0;
  if ((int)threadIdx.x < nb) {
    const int t = threadIdx.x;
    const Decoded d = decode_key(keys[t], p, lam);
    const size_t b = base + t;
    if (mv_out) {
      mv_out[2 * b] = (int16_t)d.mvx;
      mv_out[2 * b + 1] = (int16_t)d.mvy;
    }
    if (J_out) J_out[b] = d.J;
    const uint32_t mn = st[2 * t + 1];
    smin_out[b] = mn;
    sdev_out[b] = st[2 * t] - (uint32_t)(g.n * g.n) * mn;
    if (err_out) {
      const int e = abs(d.mvx - (int)gmv[2 * k]) + abs(d.mvy - (int)gmv[2 * k + 1]);
      err_out[b] = (uint8_t)min(e, 255);
    }
  }
  if (intra_out) {
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < nb; i += nw) {
      const uint32_t v = warp_intra_sad<N, M>(cur, W, (bx0 + i) * N, by * M);
      if ((threadIdx.x & 31) == 0) intra_out[base + i] = v;
    }
  }
}

struct StatsOut {
  const int16_t* gmv;
  int16_t* mv;
  uint32_t* J;
  uint32_t* intra;
  uint32_t* smin;
  uint32_t* sdev;
  uint8_t* err;
};

template <int N, int M, int T>
static int launch_stats_t(const StudyFrames& fr, int K, int W, int H, int p, uint32_t lam,
                          const StatsOut& o, const FsPlan& pl, cudaStream_t s) {
  auto kern = k_fsbm_stats<N, M, T>;
  {
    const int st = ensure_dynamic_smem((const void*)kern, pl.smem);
    if (st) return st;
  }
  const int BW = W / N, BH = H / M;
  const int bpc = pl.threads / pl.G;
  const dim3 grid(((BW + bpc - 1) / bpc) * BH, K);
  kern<<<grid, pl.threads, pl.smem, s>>>(fr, W, H, p, pl.G, lam, o.gmv, o.mv, o.J, o.intra, o.smin,
                                         o.sdev, o.err);
  ME_CUDA(cudaGetLastError());
  return ME_OK;
}

static int launch_stats(const StudyFrames& fr, int K, int W, int H, int N, int M, int p,
                        uint32_t lam, const StatsOut& o, cudaStream_t s) {
  const FsPlan pl = fs_plan(N, M, p, W / N);
  ME_DISPATCH_FS(launch_stats_t, fr, K, W, H, p, lam, o, pl, s);
}

}  // namespace me

using namespace me;

extern "C" {

int me_sad_deviation(const uint8_t* cur, const uint8_t* ref, int W, int H, int N, int M, int p,
                     uint32_t lambda_q8, int16_t* mv_out, uint32_t* J_out, uint32_t* sad_min_out,
                     uint32_t* sad_dev_out, me_stream_t stream) {
  if (!cur || !ref || !sad_min_out || !sad_dev_out) return ME_ERR_ARG;
  if (!aligned4(cur) || !aligned4(ref)) return ME_ERR_ARG;
  int st = check_frame_args(W, H, N, M, p, lambda_q8);
  if (st) return st;
  StudyFrames fr;
  std::memset(&fr, 0, sizeof(fr));
  fr.f[0] = ref;
  fr.f[1] = cur;
  if (fsbm_pipe_applies(N, M, p)) {
    // 16x16: the pipelined persistent search in its statistics mode
    PipeOut po;
    std::memset(&po, 0, sizeof(po));
    po.mv = mv_out;
    po.J = J_out;
    po.smin = sad_min_out;
    po.sdev = sad_dev_out;
    return launch_fsbm_pipe_mode(kPipeStats, fr.f, 1, W, H, p, lambda_q8, po,
                                 reinterpret_cast<cudaStream_t>(stream));
  }
  const StatsOut o{nullptr, mv_out, J_out, nullptr, sad_min_out, sad_dev_out, nullptr};
  return launch_stats(fr, 1, W, H, N, M, p, lambda_q8, o, reinterpret_cast<cudaStream_t>(stream));
}

int me_motion_study(const uint8_t* const* frames, int K, int W, int H, int N, int M, int p,
                    uint32_t lambda_q8, const int16_t* true_mv, int16_t* mv_out,
                    uint32_t* intra_out, uint32_t* sad_min_out, uint32_t* sad_dev_out,
                    uint8_t* err_out, me_stream_t stream) {
  if (!frames || K < 1 || K > kStudyMaxK || !sad_min_out || !sad_dev_out) return ME_ERR_ARG;
  if (err_out && !true_mv) return ME_ERR_ARG;
  int st = check_frame_args(W, H, N, M, p, lambda_q8);
  if (st) return st;
  StudyFrames fr;
  std::memset(&fr, 0, sizeof(fr));
  for (int k = 0; k <= K; k++) {
    if (!frames[k] || !aligned4(frames[k])) return ME_ERR_ARG;
    fr.f[k] = frames[k];
  }
  const StatsOut o{true_mv, mv_out, nullptr, intra_out, sad_min_out, sad_dev_out, err_out};
  return launch_stats(fr, K, W, H, N, M, p, lambda_q8, o, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"

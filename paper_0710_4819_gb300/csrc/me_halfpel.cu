// me_halfpel.cu -- half-pel refinement of an integer vector field (Sec. 2.2:
// the best predictor is normally refined to half-pel accuracy; Sec. 2.3: the
// 8 half-pel positions around the integer vector).
//
// For every block: with (mvx, mvy) the integer vector clipped to [-p, p],
// the positions (2*mvx + dx, 2*mvy + dy), dx, dy in {-1,0,1}, in half-pel
// units, each component clipped to [-2p, 2p], repeated positions once; the reference at a half-pel position is the bilinear
// average of the integer pixels around it with H.263 rounding ((A+B+1)>>1 for
// a half step along one axis, (A+B+C+D+2)>>2 along both), pixels outside the
// frame taking the nearest edge pixel; cost 256*SAD + lambda_q8*(L(hx)+L(hy))
// with L the Exp-Golomb length in half-pel units; ties by |h|_1, then hy,
// then hx.
//
// One warp per block.  Every candidate reads reference pixels at offsets
// -1..+1 around the integer vector, so the warp stages the (N+2)x(M+2)
// patch at (x0+mvx-1, y0+mvy-1) once (edge-clamped) and each lane
// accumulates the 9 candidates' SADs over its N*M/32 pixels.
#include <cuda_runtime.h>

#include <cstring>

#include "me_device.cuh"
#include "me_host.h"

namespace me {

constexpr int kHpWarps = 8;
constexpr int kHpMaxK = 64;

struct HpFrames {
  const uint8_t* f[kHpMaxK + 1];  // f[k] reference of pair k, f[k+1] its current frame
};

template <int N, int M>
__global__ void __launch_bounds__(32 * kHpWarps) k_halfpel(HpFrames fr, int K, int W, int H, int p,
                                                           uint32_t lam,
                                                           const int16_t* __restrict__ mv_int,
                                                           int16_t* __restrict__ mv_out,
                                                           uint32_t* __restrict__ J_out,
                                                           uint32_t* __restrict__ sad_out) {
  constexpr int PW = N + 2, PH = M + 2;
  constexpr int PIX = (N * M + 31) / 32;   // pixels per lane
  __shared__ uint8_t patch_s[kHpWarps][PH * PW];
  const unsigned FULL = 0xffffffffu;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int BW = W / N, nbf = BW * (H / M);
  const long long g = (long long)blockIdx.x * kHpWarps + warp;
  if (g >= (long long)nbf * K) return;
  const int k = (int)(g / nbf), b = (int)(g - (long long)k * nbf);
  const uint8_t* __restrict__ cur = fr.f[k + 1];
  const uint8_t* __restrict__ ref = fr.f[k];
  const int x0 = (b % BW) * N, y0 = (b / BW) * M;
  // the integer vector, taken inside the window (so every candidate lies
  // within one pixel of it and inside the patch)
  const int mx = clampi(mv_int[2 * g], -p, p), my = clampi(mv_int[2 * g + 1], -p, p);
  uint8_t* patch = patch_s[warp];
  // the reference patch: columns x0+mx-1 .. x0+mx+N, rows y0+my-1 .. y0+my+M
  for (int i = lane; i < PH * PW; i += 32) {
    const int r = i / PW, c = i - r * PW;
    const int yy = clampi(y0 + my - 1 + r, 0, H - 1), xx = clampi(x0 + mx - 1 + c, 0, W - 1);
    patch[i] = ref[(size_t)yy * W + xx];
  }
  int cv[PIX];
#pragma unroll
  for (int q = 0; q < PIX; q++) {
    const int i = lane + 32 * q;
    cv[q] = i < N * M ? (int)cur[(size_t)(y0 + i / N) * W + x0 + (i % N)] : 0;
  }
  __syncwarp();
  // the 9 candidates (in every lane), clipped; a repeat of a lower one is skipped
  int hxs[9], hys[9];
  bool live[9];
#pragma unroll
  for (int c = 0; c < 9; c++) {
    hxs[c] = clampi(2 * mx + c % 3 - 1, -2 * p, 2 * p);
    hys[c] = clampi(2 * my + c / 3 - 1, -2 * p, 2 * p);
    bool dup = false;
#pragma unroll
    for (int e = 0; e < c; e++) dup |= hxs[e] == hxs[c] && hys[e] == hys[c];
    live[c] = !dup;
  }
  uint32_t s[9];
#pragma unroll
  for (int c = 0; c < 9; c++) s[c] = 0;
#pragma unroll
  for (int q = 0; q < PIX; q++) {
    const int i = lane + 32 * q;
    if (i >= N * M) break;
    const int pi = i % N, pj = i / N;
#pragma unroll
    for (int c = 0; c < 9; c++) {
      if (!live[c]) continue;
      // integer part (floor) and half flag of the position, relative to the
      // patch origin (mx-1, my-1): offsets 0 or 1
      const int ax = hxs[c] >> 1, fx = hxs[c] & 1, ay = hys[c] >> 1, fy = hys[c] & 1;
      const uint8_t* pp = patch + (pj + ay - my + 1) * PW + (pi + ax - mx + 1);
      const int A = pp[0];
      int pred = A;
      if (fx && fy) pred = (A + pp[1] + pp[PW] + pp[PW + 1] + 2) >> 2;
      else if (fx) pred = (A + pp[1] + 1) >> 1;
      else if (fy) pred = (A + pp[PW] + 1) >> 1;
      const int d = cv[q] - pred;
      s[c] += (uint32_t)(d < 0 ? -d : d);
    }
  }
  // warp sums, then the best key (lanes agree after the butterflies)
  unsigned long long best = kNoKey;
  const int n2 = 4 * p + 1;
#pragma unroll
  for (int c = 0; c < 9; c++) {
    uint32_t t = s[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
    s[c] = t;
    if (live[c]) {
      const uint32_t J = 256u * t + lam * (uint32_t)(mv_bits(hxs[c]) + mv_bits(hys[c]));
      const uint32_t l1 = (uint32_t)((hxs[c] < 0 ? -hxs[c] : hxs[c]) + (hys[c] < 0 ? -hys[c] : hys[c]));
      const uint32_t raster = (uint32_t)((hys[c] + 2 * p) * n2 + (hxs[c] + 2 * p));
      const unsigned long long key = ((unsigned long long)J << 32) | (l1 << 17) | raster;
      best = key < best ? key : best;
    }
  }
  if (lane == 0) {
    const uint32_t raster = (uint32_t)(best & 0x1FFFFu);
    const int hy = (int)(raster / (uint32_t)n2) - 2 * p, hx = (int)(raster % (uint32_t)n2) - 2 * p;
    mv_out[2 * g] = (int16_t)hx;
    mv_out[2 * g + 1] = (int16_t)hy;
    J_out[g] = (uint32_t)(best >> 32);
    if (sad_out) sad_out[g] = ((uint32_t)(best >> 32) - lam * (uint32_t)(mv_bits(hx) + mv_bits(hy))) >> 8;
  }
}

template <int N, int M>
static int launch_halfpel_t(const HpFrames& fr, int K, int W, int H, int p, uint32_t lam,
                            const int16_t* mv_int, int16_t* mv_out, uint32_t* J_out,
                            uint32_t* sad_out, cudaStream_t s) {
  const long long warps = (long long)(W / N) * (H / M) * K;
  const long long grid = (warps + kHpWarps - 1) / kHpWarps;
  k_halfpel<N, M><<<(unsigned)grid, 32 * kHpWarps, 0, s>>>(fr, K, W, H, p, lam, mv_int, mv_out,
                                                          J_out, sad_out);
  ME_CUDA(cudaGetLastError());
  return ME_OK;
}

static int launch_halfpel(const HpFrames& fr, int K, int W, int H, int N, int M, int p,
                          uint32_t lam, const int16_t* mv_int, int16_t* mv_out, uint32_t* J_out,
                          uint32_t* sad_out, cudaStream_t s) {
#define X(n_, m_) \
  if (N == n_ && M == m_) return launch_halfpel_t<n_, m_>(fr, K, W, H, p, lam, mv_int, mv_out, J_out, sad_out, s);
  X(16, 16) X(16, 8) X(16, 4) X(8, 16) X(8, 8) X(8, 4) X(4, 16) X(4, 8) X(4, 4)
#undef X
  return ME_ERR_ARG;
}

}  // namespace me

using namespace me;

extern "C" {

int me_halfpel(const uint8_t* cur, const uint8_t* ref, int W, int H, int N, int M, int p,
               uint32_t lambda_q8, const int16_t* mv_int, int16_t* mv_half_out, uint32_t* J_out,
               uint32_t* sad_out, me_stream_t stream) {
  if (!cur || !ref || !mv_int || !mv_half_out || !J_out) return ME_ERR_ARG;
  int st = check_frame_args(W, H, N, M, p, lambda_q8);
  if (st) return st;
  HpFrames fr;
  std::memset(&fr, 0, sizeof(fr));
  fr.f[0] = ref;
  fr.f[1] = cur;
  return launch_halfpel(fr, 1, W, H, N, M, p, lambda_q8, mv_int, mv_half_out, J_out, sad_out,
                        reinterpret_cast<cudaStream_t>(stream));
}

int me_halfpel_sequence(const uint8_t* const* frames, int K, int W, int H, int N, int M, int p,
                        uint32_t lambda_q8, const int16_t* mv_int, int16_t* mv_half_out,
                        uint32_t* J_out, uint32_t* sad_out, me_stream_t stream) {
  if (!frames || K < 1 || K > kHpMaxK || !mv_int || !mv_half_out || !J_out) return ME_ERR_ARG;
  int st = check_frame_args(W, H, N, M, p, lambda_q8);
  if (st) return st;
  HpFrames fr;
  std::memset(&fr, 0, sizeof(fr));
  for (int k = 0; k <= K; k++) {
    if (!frames[k]) return ME_ERR_ARG;
    fr.f[k] = frames[k];
  }
  return launch_halfpel(fr, K, W, H, N, M, p, lambda_q8, mv_int, mv_half_out, J_out, sad_out,
                        reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"

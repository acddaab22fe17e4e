// me_host.h -- host-side helpers shared by the translation units of the
// library (argument checks, CUDA error capture, scratch pool).  Internal.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/me.h"

namespace me {

// Records the CUDA error text for me_last_error() and maps it to a status.
int cuda_status(cudaError_t e);
// Sets this thread's me_last_error() text (to hand a worker thread's error to
// the caller that observes it).
void set_last_error_text(const char* text);

#define ME_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return ::me::cuda_status(e_); \
  } while (0)

// Raises a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device; the limit only ever grows, so concurrent callers asking for
// different sizes never lower it under one another's launch.
int ensure_dynamic_smem(const void* kernel, size_t bytes);

// Frame/shape validation shared by the frame calls (see me.h conventions).
int check_frame_args(int W, int H, int N, int M, int p, uint32_t lambda_q8);
int check_acbm_params(const me_acbm_params* prm);
bool aligned4(const void* ptr);

// Stream-ordered scratch from a library-owned pool of the current device
// (kept cached between calls).  Returns ME_OK or ME_ERR_NOMEM / ME_ERR_CUDA.
int scratch_alloc(void** ptr, size_t bytes, cudaStream_t s);
int scratch_free(void* ptr, cudaStream_t s);

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Geometry of the anti-diagonal waves x + 2y = w of a BW x BH block grid.
struct Waves {
  int BW, BH, n;  // n waves
  int ylo(int w) const { int t = w - BW + 1; t = t > 0 ? (t + 1) / 2 : 0; return t; }
  int yhi(int w) const { int t = w / 2; return t < BH - 1 ? t : BH - 1; }
  int count(int w) const { int c = yhi(w) - ylo(w) + 1; return c > 0 ? c : 0; }
};
inline Waves make_waves(int BW, int BH) { return Waves{BW, BH, (BW - 1) + 2 * (BH - 1) + 1}; }

}  // namespace me

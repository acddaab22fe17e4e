// me_host.h -- host-side helpers shared by the translation units of the
// library (argument checks, CUDA error capture, scratch pool).  Internal.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <functional>
#include <string>
#include <vector>

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

// SM count of the current device (cached per device).
int sm_count(int* out);
// A spin-wait bound in SM clock cycles for `timeout_ns` at the current
// device's peak SM clock (cached per device): at lower clocks the wait lasts
// longer than the timeout, never shorter.
long long wait_cycles(long long timeout_ns);

// The autotuner (me_tune.cu).  tune_select times run(c) for every candidate
// c (names[c] describes it) on stream s with CUDA events -- one untimed run,
// then the best of two timed runs -- and sets *chosen to the fastest.  When
// tuning is off (ME_TUNE=0), the stream is being captured, or there is one
// candidate, it runs nothing and chooses `model` (the cost model's pick).
// Every call is recorded for me_tune_log.  tune_forced(n): a candidate index
// forced by ME_TUNE_FORCE (tests of every candidate), else -1.
bool tune_enabled();
int tune_forced(int n);
int tune_select(const std::string& what, const std::vector<std::string>& names, int model,
                cudaStream_t s, const std::function<int(int)>& run, int* chosen);

// Geometry of the anti-diagonal waves x + 2y = w of a BW x BH block grid.
struct Waves {
  int BW, BH, n;  // n waves
  int ylo(int w) const { int t = w - BW + 1; t = t > 0 ? (t + 1) / 2 : 0; return t; }
  int yhi(int w) const { int t = w / 2; return t < BH - 1 ? t : BH - 1; }
  int count(int w) const { int c = yhi(w) - ylo(w) + 1; return c > 0 ? c : 0; }
};
inline Waves make_waves(int BW, int BH) { return Waves{BW, BH, (BW - 1) + 2 * (BH - 1) + 1}; }

}  // namespace me

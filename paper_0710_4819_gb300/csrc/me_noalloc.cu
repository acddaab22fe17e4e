// me_noalloc.cu -- ACBM for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc or any allocating routine: code running
// inside a host that owns every device allocation itself (a media pipeline
// or game engine with a fixed memory budget, an embedded runtime, a plugin
// loaded into another process), or code that must not add allocations
// after start-up.  me_acbm_noalloc serves them: the scratch memory that me_acbm
// takes from its stream-ordered pool lives here in a fixed, statically
// allocated device array instead, and the entry point allocates nothing.
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "me_device.cuh"
#include "me_host.h"
#include "me_search.cuh"

namespace me {

// Maximum scratch of one no-alloc ACBM call.  A call needs the padded
// reference, (16*ceil(W/16) + 2P + 16) x (H + 2P) bytes with P = 16*ceil(p/16),
// plus 16 bytes per block and a few small tables.  That fits frames up to
// 1920x1088 at any p <= 64 for every block shape of 32 pixels or more (4x8
// and larger; 3.6 MB at worst), but not 4x4 blocks at 1920x1088 (4.3-4.6 MB):
// 4x4 blocks fit frames up to 1280x720.  Every GPU that loads the library
// holds this array until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

// In host code, g_noalloc_scratch names a host-side stand-in, not a device
// address; the device address is looked up once per device (with that device
// current) and cached.
static std::mutex g_noalloc_mu;
static std::vector<uint8_t*> g_noalloc_ptr;

static int noalloc_scratch(uint8_t** out) {
  int dev = 0;
  ME_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if ((int)g_noalloc_ptr.size() <= dev) g_noalloc_ptr.resize(dev + 1, nullptr);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    ME_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<uint8_t*>(ptr);
  }
  *out = g_noalloc_ptr[dev];
  return ME_OK;
}

}  // namespace me

extern "C" int me_acbm_noalloc(const uint8_t* cur, const uint8_t* ref, int W, int H, int N, int M,
                               int p, uint32_t lambda_q8, const int16_t* prev_mv_field,
                               const me_acbm_params* prm, int16_t* mv_out, uint32_t* J_out,
                               uint8_t* fullsearch_mask_out, uint32_t* sad_out,
                               uint32_t* load_out, me_stream_t stream) {
  using namespace me;
  if (!cur || !ref || !mv_out || !J_out || !fullsearch_mask_out) return ME_ERR_ARG;
  if (!aligned4(cur) || !aligned4(ref)) return ME_ERR_ARG;
  int st = check_frame_args(W, H, N, M, p, lambda_q8);
  if (st) return st;
  st = check_acbm_params(prm);
  if (st) return st;
  const AcbmScratch l = acbm_scratch_layout(W, H, N, M, p);
  if (l.total > kNoAllocScratchBytes) return ME_ERR_NOMEM;
  uint8_t* scratch = nullptr;
  st = noalloc_scratch(&scratch);
  if (st) return st;
  AcbmArgs a;
  a.cur = cur; a.ref = ref; a.prev = prev_mv_field;
  a.mv = mv_out; a.J = J_out; a.mask = fullsearch_mask_out; a.sad = sad_out; a.load = load_out;
  a.lam = lambda_q8;
  a.alpha = prm->alpha; a.beta = prm->beta; a.gnum = prm->gamma_num; a.gden = prm->gamma_den;
  a.qp = prm->qp; a.refine = prm->refine;
  return enqueue_acbm(a, W, H, N, M, p, scratch, reinterpret_cast<cudaStream_t>(stream));
}

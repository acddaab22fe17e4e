// me_host.cu -- status codes, argument checks, the cost helpers of the C ABI
// and the library's stream-ordered scratch pool.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "me_device.cuh"
#include "me_host.h"

namespace me {

static thread_local char g_last_error[256] = "";

int cuda_status(cudaError_t e) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s", cudaGetErrorName(e),
                cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return ME_ERR_NOMEM;
  return ME_ERR_CUDA;
}

int check_frame_args(int W, int H, int N, int M, int p, uint32_t lambda_q8) {
  if (!(N == 4 || N == 8 || N == 16) || !(M == 4 || M == 8 || M == 16)) return ME_ERR_ARG;
  if (p < 1 || p > kMaxP) return ME_ERR_ARG;
  if (lambda_q8 > (1u << 20)) return ME_ERR_ARG;
  if (W < N || H < M || W > 16384 || H > 16384) return ME_ERR_SHAPE;
  if (W % N != 0 || H % M != 0) return ME_ERR_SHAPE;
  return ME_OK;
}

int check_acbm_params(const me_acbm_params* prm) {
  if (!prm) return ME_ERR_ARG;
  if (prm->gamma_den < 1 || prm->gamma_num < 0) return ME_ERR_ARG;
  if (prm->qp < 0 || prm->qp > 1023) return ME_ERR_ARG;
  if (prm->refine != 0 && prm->refine != 1) return ME_ERR_ARG;
  return ME_OK;
}

void set_last_error_text(const char* text) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s", text ? text : "");
}

static std::mutex g_smem_mu;
struct SmemAttr {
  const void* fn;
  int dev;
  size_t bytes;
};
static std::vector<SmemAttr> g_smem;

int ensure_dynamic_smem(const void* kernel, size_t bytes) {
  int dev = 0;
  ME_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_smem_mu);
  for (SmemAttr& a : g_smem)
    if (a.fn == kernel && a.dev == dev) {
      if (bytes > a.bytes) {
        ME_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        a.bytes = bytes;
      }
      return ME_OK;
    }
  // the default limit is 48 KB minus the kernel's static shared memory: start
  // from the kernel's actual limit, not from 48 KB
  cudaFuncAttributes fa;
  ME_CUDA(cudaFuncGetAttributes(&fa, kernel));
  size_t have = (size_t)fa.maxDynamicSharedSizeBytes;
  if (bytes > have) {
    ME_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    have = bytes;
  }
  g_smem.push_back(SmemAttr{kernel, dev, have});
  return ME_OK;
}

bool aligned4(const void* ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 3u) == 0; }

// Per-device SM count and peak SM clock (kHz), read once per device.
struct DevInfo {
  int sms = 0, clock_khz = 0;
};
static std::mutex g_dev_mu;
static std::vector<DevInfo> g_dev;

static int dev_info(DevInfo* out) {
  int dev = 0;
  ME_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if ((int)g_dev.size() <= dev) g_dev.resize(dev + 1);
  DevInfo& d = g_dev[dev];
  if (d.sms == 0) {
    ME_CUDA(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
    ME_CUDA(cudaDeviceGetAttribute(&d.clock_khz, cudaDevAttrClockRate, dev));
  }
  *out = d;
  return ME_OK;
}

int sm_count(int* out) {
  DevInfo d;
  const int st = dev_info(&d);
  *out = st == ME_OK && d.sms > 0 ? d.sms : 1;
  return st;
}

long long wait_cycles(long long timeout_ns) {
  DevInfo d;
  // without the clock rate, assume 3 GHz (above any GB300 clock: the bound
  // stays at least the timeout)
  const long long khz = dev_info(&d) == ME_OK && d.clock_khz > 0 ? d.clock_khz : 3000000;
  return timeout_ns / 1000000 * khz + timeout_ns % 1000000 * khz / 1000000;
}

// One pool per device, created on first use, that keeps freed blocks cached
// (release threshold = max) so steady-state calls do not return memory to the
// driver between frames.
static std::mutex g_pool_mu;
static std::vector<cudaMemPool_t> g_pools;

static int pool_for_current_device(cudaMemPool_t* out) {
  int dev = 0;
  ME_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if ((int)g_pools.size() <= dev) g_pools.resize(dev + 1, nullptr);
  if (!g_pools[dev]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    ME_CUDA(cudaMemPoolCreate(&pool, &props));
    uint64_t thr = ~0ull;
    ME_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    g_pools[dev] = pool;
  }
  *out = g_pools[dev];
  return ME_OK;
}

int scratch_alloc(void** ptr, size_t bytes, cudaStream_t s) {
  cudaMemPool_t pool;
  int st = pool_for_current_device(&pool);
  if (st) return st;
  ME_CUDA(cudaMallocFromPoolAsync(ptr, bytes == 0 ? 16 : bytes, pool, s));
  return ME_OK;
}

int scratch_free(void* ptr, cudaStream_t s) {
  if (ptr) ME_CUDA(cudaFreeAsync(ptr, s));
  return ME_OK;
}

}  // namespace me

extern "C" {

const char* me_status_string(int status) {
  switch (status) {
    case ME_OK: return "ok";
    case ME_ERR_ARG: return "invalid argument";
    case ME_ERR_SHAPE: return "frame size not a multiple of the block size or out of range";
    case ME_ERR_CUDA: return "CUDA error";
    case ME_ERR_NOMEM: return "out of memory";
    case ME_ERR_TIMEOUT: return "bounded device wait timed out";
    case ME_ERR_BUSY: return "busy";
    case ME_ERR_NOTFOUND: return "not found";
    default: return "unknown status";
  }
}

const char* me_last_error(void) { return me::g_last_error; }

uint32_t me_lambda_q8(int32_t qp) {
  if (qp < 0 || qp > 1023) return 0;
  return (uint32_t)((23552LL * qp + 50) / 100);
}

int32_t me_mv_bits(int32_t v) { return me::mv_bits(v); }

me_acbm_params me_acbm_default_params(int32_t qp) {
  me_acbm_params p;
  p.alpha = 1000;
  p.beta = 8;
  p.gamma_num = 1;
  p.gamma_den = 4;
  p.qp = qp;
  p.refine = 1;
  return p;
}

}  // extern "C"

// me_tune.cu -- the library's tile autotuner: on the first call of a shape,
// every candidate launch configuration (run length, CTA roles, kernel form)
// is timed with CUDA events on the caller's stream and the fastest is kept
// for the rest of the process.  Every candidate computes the same bytes (the
// argmin is over a total order), so tuning only changes the time.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "me_host.h"

namespace me {

struct TuneRecord {
  std::string what;
  std::vector<std::string> names;
  std::vector<float> ms;   // best timed run per candidate (-1: failed)
  int model = 0, chosen = 0;
  bool measured = false;
};

static std::mutex g_tune_mu;
static std::vector<TuneRecord> g_tune_log;

bool tune_enabled() {
  const char* e = std::getenv("ME_TUNE");
  return !(e && e[0] == '0');
}

int tune_forced(int n) {
  const char* e = std::getenv("ME_TUNE_FORCE");
  if (!e || !*e) return -1;
  const int c = std::atoi(e);
  return c >= 0 && c < n ? c : -1;
}

int tune_select(const std::string& what, const std::vector<std::string>& names, int model,
                cudaStream_t s, const std::function<int(int)>& run, int* chosen) {
  const int n = (int)names.size();
  TuneRecord rec;
  rec.what = what;
  rec.names = names;
  rec.model = model;
  rec.chosen = model;
  rec.ms.assign(n, -1.f);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  ME_CUDA(cudaStreamIsCapturing(s, &cs));
  if (n > 1 && tune_enabled() && cs == cudaStreamCaptureStatusNone) {
    cudaEvent_t e0, e1;
    ME_CUDA(cudaEventCreate(&e0));
    ME_CUDA(cudaEventCreate(&e1));
    float best = 0.f;
    int bi = -1;
    for (int c = 0; c < n; c++) {
      // one untimed run (first launches pay for set-up), then the best of two
      int st = run(c);
      float mc = -1.f;
      for (int r = 0; r < 2 && st == ME_OK; r++) {
        cudaEventRecord(e0, s);
        st = run(c);
        cudaEventRecord(e1, s);
        if (st == ME_OK && cudaEventSynchronize(e1) == cudaSuccess) {
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (mc < 0.f || ms < mc) mc = ms;
        }
      }
      const cudaError_t ce = cudaStreamSynchronize(s);
      if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return cuda_status(ce);
      }
      if (st != ME_OK) continue;   // a candidate that cannot launch here is skipped
      rec.ms[c] = mc;
      if (bi < 0 || mc < best) { best = mc; bi = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (bi >= 0) {
      rec.chosen = bi;
      rec.measured = true;
    }
  }
  *chosen = rec.chosen;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_log.push_back(rec);
  return ME_OK;
}

}  // namespace me

extern "C" int me_tune_log(char* buf, int len) {
  using namespace me;
  std::string out;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const TuneRecord& r : g_tune_log) {
      out += r.what + (r.measured ? " tuned" : " modelled") + ": model=" + r.names[r.model] +
             " chosen=" + r.names[r.chosen];
      for (size_t c = 0; c < r.names.size(); c++) {
        char t[96];
        std::snprintf(t, sizeof(t), " | %s %.4f ms", r.names[c].c_str(), r.ms[c]);
        out += t;
      }
      out += "\n";
    }
  }
  const int need = (int)out.size() + 1;
  if (buf && len > 0) {
    const int m = need < len ? need : len;
    std::memcpy(buf, out.c_str(), (size_t)m - 1);
    buf[m - 1] = '\0';
  }
  return need;
}

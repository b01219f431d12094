// Live per-kernel timing and launch counting.
//
// Every kernel launch of the library is bracketed by wm_prof_begin/end with a
// category.  Launches are always counted; when timing is enabled a pair of
// CUDA events is recorded on the launching stream around each launch, and the
// elapsed times are summed per category when they are read.
#include <atomic>
#include <mutex>

#include "wm_internal.h"

namespace {

const char* kNames[WM_PC_COUNT] = {
    "apply_outer", "smooth_level0", "smooth_coarse", "residual_level0", "residual_coarse", "restrict",
    "prolong", "coarse_solve", "cg_vectors", "cg_scalars", "noise", "sinc_mass_copy", "setup_bounds_inverse",
    "layout", "assembly", "apply_component", "true_residual_f64", "coarse_tail"};

constexpr int kPool = 1 << 16;

struct Prof {
  std::mutex mu;
  bool on = false;
  std::atomic<int64_t> launches[WM_PC_COUNT];
  int64_t timed[WM_PC_COUNT] = {};
  double ms[WM_PC_COUNT] = {};
  double bytes[WM_PC_COUNT] = {};
  double flops[WM_PC_COUNT] = {};
  std::vector<cudaEvent_t> ev;  // 2 * kPool
  std::vector<int> cat;         // category of pending pair k
  int used = 0;
  int open = -1;
  bool overflow = false;
  Prof() {
    for (auto& l : launches) l = 0;
  }
};

Prof& P() {
  static Prof p;
  return p;
}

void drain(Prof& p) {
  for (int k = 0; k < p.used; ++k) {
    float t = 0.f;
    if (cudaEventSynchronize(p.ev[2 * k + 1]) == cudaSuccess &&
        cudaEventElapsedTime(&t, p.ev[2 * k], p.ev[2 * k + 1]) == cudaSuccess) {
      p.ms[p.cat[k]] += t;
      p.timed[p.cat[k]] += 1;
    } else {
      cudaGetLastError();
    }
  }
  p.used = 0;
}

}  // namespace

void wm_prof_begin(int c, cudaStream_t s) {
  Prof& p = P();
  if (!p.on) return;
  std::lock_guard<std::mutex> g(p.mu);
  if (p.used >= kPool) {
    p.overflow = true;
    p.open = -1;
    return;
  }
  cudaEventRecord(p.ev[2 * p.used], s);
  p.open = c;
}

void wm_prof_end(int c, cudaStream_t s) {
  Prof& p = P();
  p.launches[c]++;
  if (!p.on) return;
  std::lock_guard<std::mutex> g(p.mu);
  if (p.open != c || p.used >= kPool) return;
  cudaEventRecord(p.ev[2 * p.used + 1], s);
  p.cat[p.used] = c;
  p.used++;
  p.open = -1;
}

void wm_prof_units(int c, double bytes, double flops) {
  Prof& p = P();
  if (!p.on) return;
  std::lock_guard<std::mutex> g(p.mu);
  p.bytes[c] += bytes;
  p.flops[c] += flops;
}

extern "C" int wm_profile_enable(int on) {
  Prof& p = P();
  std::lock_guard<std::mutex> g(p.mu);
  if (on) {
    if (p.ev.empty()) {
      p.ev.resize(2 * kPool);
      p.cat.resize(kPool);
      for (auto& e : p.ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
          wm_set_error("cudaEventCreate failed");
          return WM_ERR_CUDA;
        }
    }
    drain(p);
    for (int c = 0; c < WM_PC_COUNT; ++c) {
      p.ms[c] = 0.0;
      p.timed[c] = 0;
      p.bytes[c] = 0.0;
      p.flops[c] = 0.0;
    }
    p.overflow = false;
    p.on = true;
  } else {
    drain(p);
    p.on = false;
  }
  return WM_OK;
}

extern "C" int wm_profile_read(int c, double* total_ms, int64_t* timed_launches, int64_t* all_launches,
                               double* alg_bytes, double* alg_flops, const char** name) {
  if (c < 0 || c >= WM_PC_COUNT) return WM_ERR_INVALID_ARG;
  Prof& p = P();
  std::lock_guard<std::mutex> g(p.mu);
  drain(p);
  if (total_ms) *total_ms = p.ms[c];
  if (timed_launches) *timed_launches = p.timed[c];
  if (all_launches) *all_launches = p.launches[c].load();
  if (alg_bytes) *alg_bytes = p.bytes[c];
  if (alg_flops) *alg_flops = p.flops[c];
  if (name) *name = kNames[c];
  return p.overflow ? 1 : WM_OK;
}

extern "C" int wm_profile_categories(void) { return WM_PC_COUNT; }

// Kernel accounting (see prof.h) and its C ABI (lyap_prof_* in lyap.h).
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "lyap_internal.h"
#include "prof.h"

namespace {

const char* kNames[PK_COUNT] = {"capmv64", "tc_gemm", "ortho", "precond", "gram", "tsmm",
                                "ritz",    "epi32",   "lsq",   "cycle",   "panel", "recstart", "capmv_ff", "cap_build", "oz_gemm",
                                "prec_gemm"};

struct Rec {
  int kernel;
  cudaEvent_t a, b;
  double fpu, bpu;
  int units_host;
  int slot;  // pinned slot for a device unit count, or -1
};

std::atomic<long long> g_launches{0};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
int* g_pinned = nullptr;
int g_pinned_cap = 0, g_pinned_used = 0;

}  // namespace

void lyap_count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int prof_begin(int kernel, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return -1;
  Rec r{};
  r.kernel = kernel;
  r.slot = -1;
  if (cudaEventCreate(&r.a) != cudaSuccess) return -1;
  if (cudaEventCreate(&r.b) != cudaSuccess) {
    cudaEventDestroy(r.a);
    return -1;
  }
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
  return (int)g_recs.size() - 1;
}

void prof_end(int h, cudaStream_t st, double fpu, double bpu, int units_host, const int* units_dev) {
  if (h < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on || h >= (int)g_recs.size()) return;
  Rec& r = g_recs[h];
  cudaEventRecord(r.b, st);
  r.fpu = fpu;
  r.bpu = bpu;
  r.units_host = units_host;
  if (units_dev && g_pinned_used < g_pinned_cap) {
    r.slot = g_pinned_used++;
    cudaMemcpyAsync(g_pinned + r.slot, units_dev, sizeof(int), cudaMemcpyDeviceToHost, st);
  }
}

extern "C" int lyap_prof_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (Rec& r : g_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_recs.clear();
  g_pinned_used = 0;
  g_on = on != 0;
  if (g_on && !g_pinned) {
    // one fixed pinned area for device-side unit counts (never reallocated,
    // so copies in flight always land in valid memory)
    if (cudaMallocHost(&g_pinned, sizeof(int) * (1 << 20)) == cudaSuccess) g_pinned_cap = 1 << 20;
    else g_pinned = nullptr;
  }
  g_launches.store(0);
  return LYAP_OK;
}

extern "C" int lyap_prof_read(lyap_prof_kernel* out, int max, int* count, long long* launches) {
  if (launches) *launches = g_launches.load();
  std::lock_guard<std::mutex> lk(g_mu);
  if (cudaDeviceSynchronize() != cudaSuccess) return LYAP_ECUDA;
  lyap_prof_kernel acc[PK_COUNT];
  std::memset(acc, 0, sizeof(acc));
  for (int k = 0; k < PK_COUNT; ++k) std::strncpy(acc[k].name, kNames[k], sizeof(acc[k].name) - 1);
  for (Rec& r : g_recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) continue;
    double units = r.slot >= 0 ? (double)g_pinned[r.slot] : (double)r.units_host;
    lyap_prof_kernel& a = acc[r.kernel];
    a.launches += 1;
    a.total_ms += ms;
    a.units += units;
    a.flops += units * r.fpu;
    a.bytes += units * r.bpu;
  }
  int n = 0;
  for (int k = 0; k < PK_COUNT && n < max; ++k)
    if (acc[k].launches > 0 && out) out[n++] = acc[k];
  if (count) *count = n;
  return LYAP_OK;
}

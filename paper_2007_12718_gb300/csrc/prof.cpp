// Event-based kernel timing for ls_profile_* (see prof.h).
#include "prof.h"

#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "../../include/ls.h"

namespace ls {
namespace {

const char* kNames[PR_COUNT] = {"matvec_rows_fwd", "matvec_cols",  "matvec_rows_inv", "spectrum_setup",
                                "cpqr_id",         "kernel_block", "leaf_build",      "merge_gemm",
                                "merge_inverse",   "hbs_apply",    "gmres_orth",      "hbs_apply_block",
                                "gmres_block"};

struct Pending {
  cudaEvent_t a, b;
  int slot;
  double bytes, flops;
};

// Optional timeline (environment variable LS_TRACE=1): every resolved event
// pair is also printed to stderr as "slot start end" in ms relative to the
// first event recorded after profiling was enabled.
bool trace_on() {
  static const bool on = [] {
    const char* v = getenv("LS_TRACE");
    return v && v[0] && v[0] != '0';
  }();
  return on;
}

struct State {
  bool on = false;
  std::vector<cudaEvent_t> pool;  // free events
  std::vector<cudaEvent_t> open;  // begin events by token
  std::vector<Pending> pending;
  cudaEvent_t base = nullptr;  // trace origin
  double ms[PR_COUNT] = {0};
  long long launches[PR_COUNT] = {0};
  double bytes[PR_COUNT] = {0}, flops[PR_COUNT] = {0};
};
State g;
std::mutex mu;

cudaEvent_t get_event() {
  if (!g.pool.empty()) {
    cudaEvent_t e = g.pool.back();
    g.pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

void resolve() {
  for (auto& p : g.pending) {
    cudaEventSynchronize(p.b);
    float t = 0.f;
    cudaEventElapsedTime(&t, p.a, p.b);
    if (trace_on() && g.base) {
      float t0 = 0.f;
      cudaEventElapsedTime(&t0, g.base, p.a);
      fprintf(stderr, "[ls trace] %-16s %10.3f %10.3f\n", kNames[p.slot], t0, t0 + t);
    }
    g.ms[p.slot] += t;
    g.launches[p.slot] += 1;
    g.bytes[p.slot] += p.bytes;
    g.flops[p.slot] += p.flops;
    g.pool.push_back(p.a);
    g.pool.push_back(p.b);
  }
  g.pending.clear();
}

}  // namespace

int prof_begin(cudaStream_t st) {
  std::lock_guard<std::mutex> lk(mu);
  if (!g.on) return -1;
  cudaEvent_t e = get_event();
  cudaEventRecord(e, st);
  if (trace_on() && !g.base) {
    cudaEventCreate(&g.base);
    cudaEventRecord(g.base, st);
  }
  g.open.push_back(e);
  return (int)g.open.size() - 1;
}

void prof_end(int token, int slot, cudaStream_t st, double bytes, double flops) {
  if (token < 0) return;
  std::lock_guard<std::mutex> lk(mu);
  if (token >= (int)g.open.size()) return;
  cudaEvent_t b = get_event();
  cudaEventRecord(b, st);
  g.pending.push_back({g.open[token], b, slot, bytes, flops});
  g.open[token] = nullptr;
  bool all_closed = true;
  for (auto e : g.open) all_closed &= (e == nullptr);
  if (all_closed) g.open.clear();
  if (g.pending.size() > 4096) resolve();
}

}  // namespace ls

extern "C" {

int ls_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(ls::mu);
  ls::resolve();
  ls::g.on = on != 0;
  return LS_OK;
}

int ls_profile_reset(void) {
  std::lock_guard<std::mutex> lk(ls::mu);
  ls::resolve();
  memset(ls::g.ms, 0, sizeof(ls::g.ms));
  memset(ls::g.launches, 0, sizeof(ls::g.launches));
  memset(ls::g.bytes, 0, sizeof(ls::g.bytes));
  memset(ls::g.flops, 0, sizeof(ls::g.flops));
  if (ls::g.base) {
    cudaEventDestroy(ls::g.base);
    ls::g.base = nullptr;
  }
  return LS_OK;
}

int ls_profile_get(ls_profile_entry* out, int max_entries) {
  std::lock_guard<std::mutex> lk(ls::mu);
  ls::resolve();
  int n = 0;
  for (int s = 0; s < ls::PR_COUNT && n < max_entries; ++s, ++n) {
    strncpy(out[n].name, ls::kNames[s], sizeof(out[n].name) - 1);
    out[n].name[sizeof(out[n].name) - 1] = 0;
    out[n].launches = ls::g.launches[s];
    out[n].total_ms = ls::g.ms[s];
    out[n].bytes = ls::g.bytes[s];
    out[n].flops = ls::g.flops[s];
  }
  return n;
}

}  // extern "C"

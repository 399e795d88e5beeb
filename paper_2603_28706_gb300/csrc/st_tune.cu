// Launch-shape autotuner (see st_tune.h).
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "st_internal.h"
#include "st_tune.h"

namespace st {

namespace {

struct TuneEntry {
  int choice = 0;
  std::vector<float> ms;
  std::vector<std::string> labels;
};

std::mutex g_tune_mu;
std::map<std::string, TuneEntry>& table() {
  static std::map<std::string, TuneEntry> t;
  return t;
}

bool tuning_enabled() {
  const char* v = getenv("ST_AUTOTUNE");
  return !(v && strcmp(v, "0") == 0);
}

constexpr int TUNE_REPS = 3;

}  // namespace

int tune_pick(const std::string& key, int ncand, const std::function<cudaError_t(int)>& run,
              const std::function<std::string(int)>& label, cudaStream_t s) {
  if (ncand <= 1 || !tuning_enabled()) return 0;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = table().find(key);
    if (it != table().end()) return it->second.choice;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = table().find(key);
  if (it != table().end()) return it->second.choice;
  TuneEntry ent;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ok = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  float best = -1.0f;
  for (int i = 0; i < ncand && ok; ++i) {
    ok = run(i) == cudaSuccess;  // warm-up
    if (ok) ok = cudaEventRecord(e0, s) == cudaSuccess;
    for (int r = 0; r < TUNE_REPS && ok; ++r) ok = run(i) == cudaSuccess;
    if (ok) ok = cudaEventRecord(e1, s) == cudaSuccess;
    if (ok) ok = cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0.0f;
    if (ok) ok = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    if (!ok) break;
    ms /= TUNE_REPS;
    ent.ms.push_back(ms);
    ent.labels.push_back(label(i));
    if (best < 0.0f || ms < best) {
      best = ms;
      ent.choice = i;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (!ok) {  // a candidate failed to launch: use the default and remember that
    cudaGetLastError();
    ent.choice = 0;
  }
  table()[key] = ent;
  return ent.choice;
}

}  // namespace st

extern "C" size_t st_autotune_report(char* buf, size_t len) {
  std::string out;
  {
    std::lock_guard<std::mutex> lock(st::g_tune_mu);
    for (const auto& kv : st::table()) {
      const st::TuneEntry& e = kv.second;
      out += kv.first + ": ";
      if (e.labels.empty()) {
        out += "default (trials failed)\n";
        continue;
      }
      out += e.labels[e.choice] + " |";
      char tmp[64];
      for (size_t i = 0; i < e.ms.size(); ++i) {
        snprintf(tmp, sizeof(tmp), " %s%s %.4f ms", i == (size_t)e.choice ? "*" : "", e.labels[i].c_str(), e.ms[i]);
        out += tmp;
      }
      out += "\n";
    }
  }
  if (buf && len > 0) {
    const size_t n = out.size() < len - 1 ? out.size() : len - 1;
    memcpy(buf, out.data(), n);
    buf[n] = '\0';
  }
  return out.size() + 1;
}

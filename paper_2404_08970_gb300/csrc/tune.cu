// Process-wide table of tuned row configurations (the gw_tune_* entry points).
//
// An entry maps (kernel, dtype, m_lo..m_hi) to a configuration id; lookups
// take the latest matching entry.  Entries are checked when they are added (a
// configuration must belong to the dtype and cover m_hi columns), so a lookup
// never yields a configuration that cannot run the row.  Host code only: no
// CUDA call is made here.
#include <dlfcn.h>

#include <algorithm>
#include <atomic>
#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <string>
#include <vector>

#include "gw_internal.h"

namespace gw {
namespace {

// Longest rows the solver accepts (gw_solve checks the same bound).
constexpr int kMaxTunedColumns = 16384;

struct TuneEntry {
  int kernel, dtype, m_lo, m_hi, config;
};

std::mutex g_mu;
std::vector<TuneEntry> g_table;
std::atomic<unsigned> g_generation{0};

bool known(int kernel, int dtype) { return kernel == GW_TUNE_SINKHORN && (dtype == GW_F32 || dtype == GW_F64); }

// Columns covered by `config` when it belongs to `dtype`, else -1.
int cover_of(int config, int dtype) {
  int dt = -1, nw = 0, vpt = 0, ng = 0;
  if (!sk_config_shape(config, &dt, &nw, &vpt, &ng) || dt != dtype) return -1;
  return 32 * nw * vpt;
}

gw_status add_entry(int kernel, int dtype, int m_lo, int m_hi, int config) {
  if (!known(kernel, dtype) || m_lo < 1 || m_hi < m_lo || m_hi > kMaxTunedColumns) return GW_ERR_INVALID;
  if (cover_of(config, dtype) < m_hi) return GW_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_mu);
  g_table.push_back({kernel, dtype, m_lo, m_hi, config});
  g_generation.fetch_add(1);
  return GW_OK;
}

// One table line: "<kernel> <dtype> <m_lo> <m_hi> <config>", '#' starts a
// comment.  Returns 1 for an entry, 0 for a blank or comment line, -1 if
// malformed.
int parse_line(const char* line, TuneEntry* e) {
  std::string s(line);
  const size_t hash = s.find('#');
  if (hash != std::string::npos) s.resize(hash);
  size_t i = 0;
  while (i < s.size() && std::isspace((unsigned char)s[i])) ++i;
  if (i == s.size()) return 0;
  char tail = 0;
  const int got = std::sscanf(s.c_str() + i, "%d %d %d %d %d %c", &e->kernel, &e->dtype, &e->m_lo, &e->m_hi,
                              &e->config, &tail);
  return got == 5 ? 1 : -1;
}

}  // namespace

int tune_lookup(int kernel, int dtype, int m) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto it = g_table.rbegin(); it != g_table.rend(); ++it)
    if (it->kernel == kernel && it->dtype == dtype && m >= it->m_lo && m <= it->m_hi) return it->config;
  return -1;
}

unsigned tune_generation() { return g_generation.load(); }

gw_status tune_load_file(const char* path) {
  FILE* f = std::fopen(path, "r");
  if (!f) return GW_ERR_INVALID;
  char buf[512];
  gw_status rc = GW_OK;
  while (std::fgets(buf, sizeof buf, f)) {
    TuneEntry e{};
    const int r = parse_line(buf, &e);
    if (r == 0) continue;
    if (r < 0 || add_entry(e.kernel, e.dtype, e.m_lo, e.m_hi, e.config) != GW_OK) {
      rc = GW_ERR_INVALID;
      break;
    }
  }
  std::fclose(f);
  return rc;
}

void tune_autoload() {
  static std::once_flag once;
  std::call_once(once, [] {
    std::string path;
    const char* env = std::getenv("GW_TUNE_TABLE");
    if (env && *env) {
      path = env;
    } else {
      Dl_info info;
      if (dladdr((const void*)&tune_lookup, &info) && info.dli_fname) {
        const std::string lib = info.dli_fname;
        const size_t slash = lib.rfind('/');
        path = (slash == std::string::npos ? std::string(".") : lib.substr(0, slash)) + "/tune_table.txt";
      }
    }
    if (path.empty()) return;
    FILE* f = std::fopen(path.c_str(), "r");
    if (!f) return;
    std::fclose(f);
    tune_load_file(path.c_str());
  });
}

}  // namespace gw

extern "C" {

gw_status gw_tune_set(int kernel, int dtype, int m_lo, int m_hi, int config) {
  return gw::add_entry(kernel, dtype, m_lo, m_hi, config);
}

gw_status gw_tune_clear(void) {
  std::lock_guard<std::mutex> lk(gw::g_mu);
  gw::g_table.clear();
  gw::g_generation.fetch_add(1);
  return GW_OK;
}

gw_status gw_tune_load(const char* path) {
  if (!path) return GW_ERR_INVALID;
  return gw::tune_load_file(path);
}

int gw_tune_config(int kernel, int dtype, int m) {
  if (!gw::known(kernel, dtype) || m < 1 || m > gw::kMaxTunedColumns) return -1;
  const int t = gw::tune_lookup(kernel, dtype, m);
  return t >= 0 ? t : gw::sk_default_config(m, dtype);
}

int gw_tune_candidates(int kernel, int dtype, int m, int* out, int cap) {
  if (!gw::known(kernel, dtype) || m < 1 || m > gw::kMaxTunedColumns || cap < 0 || (cap > 0 && !out)) return -1;
  int ids[64];
  const int total = gw::sk_config_ids(ids, 64);
  // Built-in choice first, then the other configurations that cover m but
  // at most four times the built-in choice's columns, in order of the columns
  // they cover.
  std::vector<std::pair<int, int>> rest;
  const int def = gw::sk_default_config(m, dtype);
  const int def_cover = gw::cover_of(def, dtype);
  for (int i = 0; i < total && i < 64; ++i) {
    const int cov = gw::cover_of(ids[i], dtype);
    if (ids[i] != def && cov >= m && cov <= 4 * def_cover) rest.push_back({cov, ids[i]});
  }
  std::sort(rest.begin(), rest.end());
  int count = 0;
  auto put = [&](int id) {
    if (count < cap) out[count] = id;
    ++count;
  };
  put(def);
  for (const auto& r : rest) put(r.second);
  return count;
}

gw_status gw_tune_shape(int kernel, int config, int* nw, int* vpt, int* ng) {
  if (kernel != GW_TUNE_SINKHORN) return GW_ERR_INVALID;
  return gw::sk_config_shape(config, nullptr, nw, vpt, ng) ? GW_OK : GW_ERR_INVALID;
}

}  // extern "C"

// Launch-shape table of the mixed path: the autotuner's results (k_mixed.cu times the
// candidate shapes of a call and stores the fastest here), kept for the whole process and
// optionally in a text file, one line per shape:
//   part dtype V3 n_r nt nrep  NH nsplit  microseconds
// Lines starting with '#' are comments.  The table is shared by every context, since the
// best shape depends only on the problem shape and the GPU.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "lhc_internal.h"

namespace lhc {

bool TuneKey::operator<(const TuneKey &o) const {
  const int a[6] = {part, dtype, V3, n_r, nt, nrep}, b[6] = {o.part, o.dtype, o.V3, o.n_r, o.nt, o.nrep};
  return std::lexicographical_compare(a, a + 6, b, b + 6);
}

namespace {
std::mutex g_mu;
std::map<TuneKey, TuneChoice> g_table;
std::string g_path;

bool valid(const TuneKey &k, const TuneChoice &c) {
  return k.part >= 0 && k.part <= 2 && (k.dtype == LHC_C128 || k.dtype == LHC_C64) && k.V3 > 0 && k.n_r > 0 &&
         k.nt > 0 && k.nrep > 0 && c.NH >= 8 && c.NH <= 48 && c.NH % 8 == 0 && c.nsplit >= 1 && c.nsplit <= 64;
}

// caller holds g_mu
int save_locked() {
  if (g_path.empty()) return LHC_OK;
  const std::string tmp = g_path + ".tmp";
  FILE *f = std::fopen(tmp.c_str(), "w");
  if (!f) {
    set_error("cannot write the tuning table %s", tmp.c_str());
    return LHC_EINVAL;
  }
  std::fprintf(f, "# liblhc launch shapes: part dtype V3 n_r nt nrep  NH nsplit  us\n");
  for (const auto &kv : g_table) {
    const TuneKey &k = kv.first;
    const TuneChoice &c = kv.second;
    std::fprintf(f, "%d %d %d %d %d %d  %d %d  %.1f\n", k.part, k.dtype, k.V3, k.n_r, k.nt, k.nrep, c.NH, c.nsplit,
                 c.us);
  }
  const bool ok = std::fclose(f) == 0 && std::rename(tmp.c_str(), g_path.c_str()) == 0;
  if (!ok) {
    set_error("cannot write the tuning table %s", g_path.c_str());
    return LHC_EINVAL;
  }
  return LHC_OK;
}

// caller holds g_mu; returns the number of entries read, or -1 on a malformed line
int load_locked(const char *path) {
  FILE *f = std::fopen(path, "r");
  if (!f) return 0;   // no table yet
  char line[256];
  int n = 0, lineno = 0;
  while (std::fgets(line, sizeof line, f)) {
    ++lineno;
    const char *p = line;
    while (*p == ' ' || *p == '\t') ++p;
    if (*p == '#' || *p == '\n' || *p == '\0') continue;
    TuneKey k;
    TuneChoice c;
    if (std::sscanf(p, "%d %d %d %d %d %d %d %d %f", &k.part, &k.dtype, &k.V3, &k.n_r, &k.nt, &k.nrep, &c.NH,
                    &c.nsplit, &c.us) != 9 ||
        !valid(k, c)) {
      std::fclose(f);
      set_error("tuning table %s: malformed line %d", path, lineno);
      return -1;
    }
    g_table[k] = c;
    ++n;
  }
  std::fclose(f);
  return n;
}
}  // namespace

bool tune_lookup(const TuneKey &key, TuneChoice *out) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_table.find(key);
  if (it == g_table.end()) return false;
  *out = it->second;
  return true;
}

void tune_store(const TuneKey &key, const TuneChoice &c) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_table[key] = c;
  save_locked();   // a table that cannot be written stays in memory (the error text says why)
}

}  // namespace lhc

extern "C" int lhc_set_tuning(lhc_ctx ctx, int mode, const char *path) {
  if (!ctx || (mode != LHC_TUNE_OFF && mode != LHC_TUNE_ON)) {
    lhc::set_error("lhc_set_tuning: null context or unknown mode %d", mode);
    return LHC_EINVAL;
  }
  if (path && *path) {
    std::lock_guard<std::mutex> lk(lhc::g_mu);
    if (lhc::load_locked(path) < 0) return LHC_EINVAL;
    lhc::g_path = path;
  }
  ctx->tune_mode = mode;
  return LHC_OK;
}

extern "C" int lhc_tuning_table(int *entries, int cap, int *count) {
  if (!count || cap < 0 || (cap > 0 && !entries)) {
    lhc::set_error("lhc_tuning_table: bad arguments");
    return LHC_EINVAL;
  }
  std::lock_guard<std::mutex> lk(lhc::g_mu);
  int n = 0;
  for (const auto &kv : lhc::g_table) {
    if (n < cap) {
      int *e = entries + 8 * n;
      const lhc::TuneKey &k = kv.first;
      e[0] = k.part, e[1] = k.dtype, e[2] = k.V3, e[3] = k.n_r, e[4] = k.nt, e[5] = k.nrep;
      e[6] = kv.second.NH, e[7] = kv.second.nsplit;
    }
    ++n;
  }
  *count = n;
  return LHC_OK;
}

extern "C" int lhc_tuning_load(const char *path, int *count) {
  if (!path || !count) {
    lhc::set_error("lhc_tuning_load: null argument");
    return LHC_EINVAL;
  }
  std::lock_guard<std::mutex> lk(lhc::g_mu);
  const int n = lhc::load_locked(path);
  if (n < 0) return LHC_EINVAL;
  *count = n;
  return LHC_OK;
}

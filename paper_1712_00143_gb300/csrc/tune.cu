// tune.cu -- the autotuner's cache of launch variants: keys, the
// process-wide table, its JSON file, and the C ABI calls that expose it.
//
// A key names one tuned launch: kernel family, storage format, Naik entries
// per hop, right-hand sides per launch and lattice extents, e.g.
// "dslash_mrhs/fp32/nl6/n4/32x32x32x32".  An entry holds the chosen variant
// and its time per application (us).  When the environment variable
// STAG_TUNE_CACHE names a file, the table is loaded from it on first use and
// the file is rewritten after every new entry, so later processes skip the
// timing.  The file is a JSON object:
//   {"version": 1, "entries": {"<key>": {"variant": 3, "us": 104.2}, ...}}
// Host code only; no CUDA call.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "internal.h"

namespace stag {

namespace {

struct TuneEntry {
  int variant;
  double us;
};

std::mutex g_tmu;
std::map<std::string, TuneEntry> g_table;
bool g_env_loaded = false;

const char* prec_name(int prec) {
  switch (prec) {
    case STAG_FP64: return "fp64";
    case STAG_FP32: return "fp32";
    case STAG_FP16: return "fp16";
    case STAG_FX16: return "fx16";
    case STAG_DF64: return "df64";
    case STAG_FX16L32: return "fx16l";
    default: return "p?";
  }
}

// ---- a small reader for the file's format: objects, strings (no escapes
// other than \" and \\), numbers; anything else is an error.
struct Reader {
  const char* p;
  const char* end;
  void ws() {
    while (p < end && (*p == ' ' || *p == '\n' || *p == '\r' || *p == '\t')) ++p;
  }
  bool lit(char c) {
    ws();
    if (p < end && *p == c) {
      ++p;
      return true;
    }
    return false;
  }
  bool str(std::string* out) {
    ws();
    if (p >= end || *p != '"') return false;
    ++p;
    out->clear();
    while (p < end && *p != '"') {
      if (*p == '\\') {
        if (p + 1 >= end || (p[1] != '"' && p[1] != '\\')) return false;
        ++p;
      }
      out->push_back(*p++);
    }
    if (p >= end) return false;
    ++p;
    return true;
  }
  bool num(double* out) {
    ws();
    char* q = nullptr;
    std::string tmp(p, (size_t)(end - p < 64 ? end - p : 64));
    const double v = std::strtod(tmp.c_str(), &q);
    if (q == tmp.c_str()) return false;
    p += q - tmp.c_str();
    *out = v;
    return true;
  }
};

// {"variant": int, "us": number} in any order
bool read_entry(Reader& r, TuneEntry* e) {
  if (!r.lit('{')) return false;
  bool hv = false, hu = false;
  if (r.lit('}')) return false;
  do {
    std::string k;
    double v = 0.0;
    if (!r.str(&k) || !r.lit(':') || !r.num(&v)) return false;
    if (k == "variant") {
      if (v != (double)(int)v) return false;
      e->variant = (int)v;
      hv = true;
    } else if (k == "us") {
      e->us = v;
      hu = true;
    }
  } while (r.lit(','));
  return r.lit('}') && hv && hu;
}

bool parse(const std::string& text, std::map<std::string, TuneEntry>* out) {
  Reader r{text.data(), text.data() + text.size()};
  if (!r.lit('{')) return false;
  bool have_entries = false;
  if (!r.lit('}')) {
    do {
      std::string k;
      if (!r.str(&k) || !r.lit(':')) return false;
      if (k == "version") {
        double v;
        if (!r.num(&v) || v != 1.0) return false;
      } else if (k == "entries") {
        have_entries = true;
        if (!r.lit('{')) return false;
        if (!r.lit('}')) {
          do {
            std::string key;
            TuneEntry e{};
            if (!r.str(&key) || !r.lit(':') || !read_entry(r, &e)) return false;
            (*out)[key] = e;
          } while (r.lit(','));
          if (!r.lit('}')) return false;
        }
      } else {
        return false;
      }
    } while (r.lit(','));
    if (!r.lit('}')) return false;
  }
  r.ws();
  return have_entries && r.p == r.end;
}

int load_locked(const char* path) {
  FILE* f = std::fopen(path, "rb");
  if (!f) return STAG_EINVAL;
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, n);
  std::fclose(f);
  std::map<std::string, TuneEntry> got;
  if (!parse(text, &got)) return STAG_EINVAL;
  for (auto& kv : got) g_table[kv.first] = kv.second;
  return STAG_OK;
}

int save_locked(const char* path) {
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return STAG_EINVAL;
  std::fprintf(f, "{\"version\": 1, \"entries\": {");
  bool first = true;
  for (auto& kv : g_table) {
    std::string k;
    for (char c : kv.first) {
      if (c == '"' || c == '\\') k.push_back('\\');
      k.push_back(c);
    }
    std::fprintf(f, "%s\n  \"%s\": {\"variant\": %d, \"us\": %.6g}", first ? "" : ",", k.c_str(), kv.second.variant,
                 kv.second.us);
    first = false;
  }
  std::fprintf(f, "\n}}\n");
  const bool ok = std::fclose(f) == 0;
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return STAG_EINVAL;
  }
  return STAG_OK;
}

void env_load_locked() {
  if (g_env_loaded) return;
  g_env_loaded = true;
  const char* path = std::getenv("STAG_TUNE_CACHE");
  if (path && *path) load_locked(path);  // a missing or unreadable file starts an empty table
}

}  // namespace

std::string tune_key(const char* kernel, int prec, int nl, int nrhs, const int dims[4]) {
  char buf[160];
  std::snprintf(buf, sizeof buf, "%s/%s/nl%d/n%d/%dx%dx%dx%d", kernel ? kernel : "?", prec_name(prec), nl, nrhs,
                dims[0], dims[1], dims[2], dims[3]);
  return buf;
}

bool tune_cache_get(const std::string& key, int* variant, double* us) {
  std::lock_guard<std::mutex> lk(g_tmu);
  env_load_locked();
  auto it = g_table.find(key);
  if (it == g_table.end()) return false;
  if (variant) *variant = it->second.variant;
  if (us) *us = it->second.us;
  return true;
}

void tune_cache_put(const std::string& key, int variant, double us) {
  std::lock_guard<std::mutex> lk(g_tmu);
  env_load_locked();
  g_table[key] = TuneEntry{variant, us};
  const char* path = std::getenv("STAG_TUNE_CACHE");
  if (path && *path) save_locked(path);
}

}  // namespace stag

using namespace stag;

extern "C" {

int stag_tune_key(char* buf, int len, const char* kernel, int prec, int nl, int nrhs, const int dims[4]) {
  if (!buf || len <= 0 || !kernel || !dims) return STAG_EINVAL;
  const std::string k = tune_key(kernel, prec, nl, nrhs, dims);
  if ((int)k.size() + 1 > len) return STAG_EINVAL;
  std::memcpy(buf, k.c_str(), k.size() + 1);
  return STAG_OK;
}

int stag_tune_cache_get(const char* key, int* variant, double* us) {
  if (!key || !variant) return STAG_EINVAL;
  *variant = -1;
  if (us) *us = 0.0;
  tune_cache_get(key, variant, us);
  return STAG_OK;
}

int stag_tune_cache_put(const char* key, int variant, double us) {
  if (!key || !*key || variant < 0) return STAG_EINVAL;
  tune_cache_put(key, variant, us);
  return STAG_OK;
}

int stag_tune_cache_clear(void) {
  std::lock_guard<std::mutex> lk(g_tmu);
  g_table.clear();
  g_env_loaded = true;  // an explicit clear also forgets the file named by the environment
  return STAG_OK;
}

int stag_tune_cache_load(const char* path) {
  if (!path) return STAG_EINVAL;
  std::lock_guard<std::mutex> lk(g_tmu);
  return load_locked(path);
}

int stag_tune_cache_save(const char* path) {
  if (!path) return STAG_EINVAL;
  std::lock_guard<std::mutex> lk(g_tmu);
  return save_locked(path);
}

long long stag_tune_cache_size(void) {
  std::lock_guard<std::mutex> lk(g_tmu);
  return (long long)g_table.size();
}

}  // extern "C"

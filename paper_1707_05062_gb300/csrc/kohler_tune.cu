// The autotuner's table: for each kind of launch group (the pass its images
// take by default, M, and the size class of the group), the launch parameters
// that measured fastest.  kohler_autotune (in the C ABI unit) fills it; every
// later launch of a matching group reads it.  The table can be written to and
// read back from a small JSON file, so that a tuning run carries over to
// later processes.
//
// File format (one object per entry; keys in any order; unknown keys ignored):
//   {"kohler_tune": 1, "entries": [
//     {"pass": "u16_fast", "M": 4096, "px_class": 26, "route": "u16_fast",
//      "warps": 8, "px": 8, "per_sm": 1, "upw": 16, "us": 251.3}, ...]}
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "kohler.h"
#include "kohler_internal.h"

namespace kohler {
namespace {
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;
}  // namespace

bool tune_find(const TuneKey& k, TuneVal* v) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(k);
  if (it == g_tune.end()) return false;
  *v = it->second;
  return true;
}

void tune_put(const TuneKey& k, const TuneVal& v) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[k] = v;
}
}  // namespace kohler

using namespace kohler;

namespace {

// A tiny reader for the file format above: finds the "entries" array and reads
// each flat object's "key": value members (strings without escapes, numbers).
struct Reader {
  const std::string& s;
  size_t i = 0;
  explicit Reader(const std::string& text) : s(text) {}
  void ws() {
    while (i < s.size() && (s[i] == ' ' || s[i] == '\n' || s[i] == '\r' || s[i] == '\t')) ++i;
  }
  bool eat(char c) {
    ws();
    if (i < s.size() && s[i] == c) {
      ++i;
      return true;
    }
    return false;
  }
  bool str(std::string* out) {
    ws();
    if (i >= s.size() || s[i] != '"') return false;
    const size_t e = s.find('"', i + 1);
    if (e == std::string::npos) return false;
    *out = s.substr(i + 1, e - i - 1);
    if (out->find('\\') != std::string::npos) return false;
    i = e + 1;
    return true;
  }
  bool num(double* out) {
    ws();
    const char* b = s.c_str() + i;
    char* end = nullptr;
    *out = std::strtod(b, &end);
    if (end == b) return false;
    i += (size_t)(end - b);
    return true;
  }
};

bool read_entry(Reader& r, TuneKey* k, TuneVal* v) {
  if (!r.eat('{')) return false;
  std::string pass, route;
  double M = -1, pxc = -1, warps = -1, px = -1, per_sm = -1, upw = -1, us = 0;
  if (!r.eat('}')) {
    do {
      std::string key;
      if (!r.str(&key) || !r.eat(':')) return false;
      if (key == "pass" || key == "route") {
        if (!r.str(key == "pass" ? &pass : &route)) return false;
      } else {
        double x;
        if (!r.num(&x)) return false;
        if (key == "M") M = x;
        else if (key == "px_class") pxc = x;
        else if (key == "warps") warps = x;
        else if (key == "px") px = x;
        else if (key == "per_sm") per_sm = x;
        else if (key == "upw") upw = x;
        else if (key == "us") us = x;
      }
    } while (r.eat(','));
    if (!r.eat('}')) return false;
  }
  k->pass = pass_from_name(pass.c_str());
  v->route = pass_from_name(route.c_str());
  if (k->pass < 0 || v->route < 0 || M < 2 || M > 65536 || pxc < 0 || pxc > 62) return false;
  k->M = (int)M;
  k->px_class = (int)pxc;
  v->warps = (int)warps;
  v->px = (int)px;
  v->per_sm = (int)per_sm;
  v->upw = (int)upw;
  v->us = us;
  return tune_valid(k->pass, *v);
}

}  // namespace

extern "C" {

int kohler_tune_save(const char* path) {
  if (!path) return KOHLER_ERR_ARG;
  std::map<TuneKey, TuneVal> copy;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    copy = g_tune;
  }
  FILE* f = std::fopen(path, "w");
  if (!f) return KOHLER_ERR_ARG;
  std::fprintf(f, "{\"kohler_tune\": 1, \"entries\": [");
  bool first = true;
  for (const auto& e : copy) {
    std::fprintf(f,
                 "%s\n  {\"pass\": \"%s\", \"M\": %d, \"px_class\": %d, \"route\": \"%s\", \"warps\": %d, \"px\": %d, "
                 "\"per_sm\": %d, \"upw\": %d, \"us\": %.3f}",
                 first ? "" : ",", pass_name(e.first.pass), e.first.M, e.first.px_class, pass_name(e.second.route),
                 e.second.warps, e.second.px, e.second.per_sm, e.second.upw, e.second.us);
    first = false;
  }
  std::fprintf(f, "\n]}\n");
  const bool ok = std::fclose(f) == 0;
  return ok ? KOHLER_OK : KOHLER_ERR_ARG;
}

int kohler_tune_load(const char* path) {
  if (!path) return KOHLER_ERR_ARG;
  FILE* f = std::fopen(path, "rb");
  if (!f) return KOHLER_ERR_ARG;
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0) {
    text.append(buf, got);
    if (text.size() > ((size_t)1 << 24)) break;
  }
  std::fclose(f);
  Reader r(text);
  std::string key;
  double version = 0;
  if (!r.eat('{') || !r.str(&key) || key != "kohler_tune" || !r.eat(':') || !r.num(&version) || version != 1.0 ||
      !r.eat(',') || !r.str(&key) || key != "entries" || !r.eat(':') || !r.eat('['))
    return KOHLER_ERR_ARG;
  std::map<TuneKey, TuneVal> entries;
  if (!r.eat(']')) {
    do {
      TuneKey k;
      TuneVal v;
      if (!read_entry(r, &k, &v)) return KOHLER_ERR_ARG;
      entries[k] = v;
    } while (r.eat(','));
    if (!r.eat(']')) return KOHLER_ERR_ARG;
  }
  if (!r.eat('}')) return KOHLER_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (const auto& e : entries) g_tune[e.first] = e.second;
  return KOHLER_OK;
}

int kohler_tune_clear(void) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune.clear();
  return KOHLER_OK;
}

int32_t kohler_tune_count(void) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  return (int32_t)g_tune.size();
}

}  // extern "C"

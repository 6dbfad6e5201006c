// Launch parameters of the tunable V-cycle passes: a table of tuned choices keyed by
// pass, dimension, level pitch, precision and Arnoldi step, read from a JSON file
// (written by helm_autotune, committed beside the library), with built-in defaults
// for every key the table does not hold.  Every choice is a function of the level
// and the device only, so a problem's reductions run in the same order alone and in
// any batch.
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <algorithm>
#include <atomic>
#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/helm.h"
#include "helm_internal.h"
#include "profiler.h"

namespace helm {

namespace {

struct Key {
  int pass, dim, P, prec, J;
  bool operator<(const Key& o) const {
    if (pass != o.pass) return pass < o.pass;
    if (dim != o.dim) return dim < o.dim;
    if (P != o.P) return P < o.P;
    if (prec != o.prec) return prec < o.prec;
    return J < o.J;
  }
};

std::mutex g_mu;
std::map<Key, TuneChoice> g_table;
std::string g_device;        // device the table was tuned on
std::string g_runs;          // the "runs" records of the loaded file (kept verbatim)
std::once_flag g_default_once;

const char* pass_name(int pass) {
  switch (pass) {
    case TP_ARNOLDI: return "arnoldi";
    case TP_RESTRICT: return "restrict";
    case TP_PROLONG: return "prolong";
    case TP_PERSIST: return "persist";
    case TP_ZPLANES: return "zplanes";
    default: return "?";
  }
}
int pass_of(const std::string& s) {
  if (s == "arnoldi") return TP_ARNOLDI;
  if (s == "restrict") return TP_RESTRICT;
  if (s == "prolong") return TP_PROLONG;
  if (s == "persist") return TP_PERSIST;
  if (s == "zplanes") return TP_ZPLANES;
  return -1;
}

// ---- a small reader for the table's JSON (objects, arrays, strings, integers, numbers)
struct Reader {
  const std::string& s;
  size_t i = 0;
  explicit Reader(const std::string& t) : s(t) {}
  void ws() { while (i < s.size() && std::isspace((unsigned char)s[i])) ++i; }
  bool eat(char c) {
    ws();
    if (i < s.size() && s[i] == c) { ++i; return true; }
    return false;
  }
  bool str(std::string* out) {
    ws();
    if (i >= s.size() || s[i] != '"') return false;
    ++i;
    std::string r;
    while (i < s.size() && s[i] != '"') {
      if (s[i] == '\\' && i + 1 < s.size()) ++i;
      r += s[i++];
    }
    if (i >= s.size()) return false;
    ++i;
    if (out) *out = r;
    return true;
  }
  bool num(double* out) {
    ws();
    const char* b = s.c_str() + i;
    char* e = nullptr;
    const double v = std::strtod(b, &e);
    if (e == b) return false;
    i += (size_t)(e - b);
    if (out) *out = v;
    return true;
  }
  // skip any value; `raw` gets its text
  bool skip(std::string* raw = nullptr) {
    ws();
    const size_t b = i;
    if (i >= s.size()) return false;
    if (s[i] == '"') {
      if (!str(nullptr)) return false;
    } else if (s[i] == '{' || s[i] == '[') {
      int depth = 0;
      bool in_str = false;
      for (; i < s.size(); ++i) {
        const char c = s[i];
        if (in_str) {
          if (c == '\\') ++i;
          else if (c == '"') in_str = false;
          continue;
        }
        if (c == '"') in_str = true;
        else if (c == '{' || c == '[') ++depth;
        else if (c == '}' || c == ']') {
          if (--depth == 0) { ++i; break; }
        }
      }
      if (depth != 0) return false;
    } else {
      while (i < s.size() && s[i] != ',' && s[i] != '}' && s[i] != ']') ++i;
    }
    if (raw) *raw = s.substr(b, i - b);
    return true;
  }
};

bool parse_entry(Reader& r, Key* k, TuneChoice* c) {
  if (!r.eat('{')) return false;
  std::string pass;
  int got = 0;
  *c = TuneChoice{};
  bool first = true;
  while (!r.eat('}')) {
    if (!first && !r.eat(',')) return false;
    first = false;
    std::string name;
    if (!r.str(&name) || !r.eat(':')) return false;
    double d = 0;
    if (name == "pass") {
      if (!r.str(&pass)) return false;
      got |= 1;
    } else if (name == "dim" || name == "P" || name == "prec" || name == "J") {
      if (!r.num(&d)) return false;
      if (name == "dim") k->dim = (int)d;
      if (name == "P") k->P = (int)d;
      if (name == "prec") k->prec = (int)d;
      if (name == "J") k->J = (int)d;
      got |= name == "dim" ? 2 : name == "P" ? 4 : name == "prec" ? 8 : 16;
    } else if (name == "v") {
      if (!r.eat('[')) return false;
      int m = 0;
      while (!r.eat(']')) {
        if (m > 0 && !r.eat(',')) return false;
        if (!r.num(&d)) return false;
        if (m < TUNE_NV) c->v[m] = (int)d;
        ++m;
      }
      got |= 32;
    } else if (!r.skip()) {
      return false;
    }
  }
  k->pass = pass_of(pass);
  return got == 63 && k->pass >= 0;
}

std::string current_device_name() {
  int dev = 0;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
    cudaGetLastError();
    return "";
  }
  return p.name;
}

std::string default_path() {
  if (const char* env = std::getenv("HELM_TUNING")) return env;
  Dl_info info;
  if (dladdr(reinterpret_cast<void*>(&tune_load_default), &info) && info.dli_fname) {
    std::string so = info.dli_fname;
    const size_t slash = so.rfind('/');
    return (slash == std::string::npos ? std::string(".") : so.substr(0, slash)) + "/tuning.json";
  }
  return "tuning.json";
}

}  // namespace

int tune_load(const char* path, std::string* err) {
  const std::string p = path ? path : default_path();
  std::ifstream f(p);
  if (!f) {
    if (err) *err = "cannot open " + p;
    return HELM_EINVAL;
  }
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string text = ss.str();
  Reader r(text);
  std::map<Key, TuneChoice> table;
  std::string device, runs;
  bool ok = r.eat('{');
  bool first = true;
  while (ok && !r.eat('}')) {
    if (!first && !r.eat(',')) { ok = false; break; }
    first = false;
    std::string name;
    if (!r.str(&name) || !r.eat(':')) { ok = false; break; }
    if (name == "device") {
      ok = r.str(&device);
    } else if (name == "entries") {
      if (!r.eat('[')) { ok = false; break; }
      bool f2 = true;
      while (ok && !r.eat(']')) {
        if (!f2 && !r.eat(',')) { ok = false; break; }
        f2 = false;
        Key k{};
        TuneChoice c{};
        ok = parse_entry(r, &k, &c);
        if (ok) table[k] = c;
      }
    } else if (name == "runs") {
      ok = r.skip(&runs);
    } else {
      ok = r.skip();
    }
  }
  if (!ok) {
    if (err) *err = "malformed tuning table " + p;
    return HELM_EINVAL;
  }
  // a table tuned on another kind of device is not used (no device here: accepted)
  const std::string here = current_device_name();
  if (!here.empty() && !device.empty() && here != device) table.clear();
  std::lock_guard<std::mutex> lk(g_mu);
  g_table.swap(table);
  g_device = device;
  g_runs = runs;
  bump_launch_generation();
  return HELM_OK;
}

void tune_load_default() {
  std::call_once(g_default_once, [] {
    std::string err;
    tune_load(nullptr, &err);  // an absent table leaves the defaults
  });
}

bool tune_get(int pass, int dim, int P, int prec_bytes, int J, TuneChoice* out) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_table.find(Key{pass, dim, P, prec_bytes, J});
  if (it == g_table.end()) return false;
  *out = it->second;
  return true;
}

void tune_set(int pass, int dim, int P, int prec_bytes, int J, const TuneChoice* c) {
  {
    std::lock_guard<std::mutex> lk(g_mu);
    const Key k{pass, dim, P, prec_bytes, J};
    if (c) g_table[k] = *c;
    else g_table.erase(k);
  }
  bump_launch_generation();
}

int tune_entries() {
  std::lock_guard<std::mutex> lk(g_mu);
  return (int)g_table.size();
}

int tune_write(const char* path, const std::string& run_record, std::string* err) {
  std::ostringstream os;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    std::string device = current_device_name();
    if (device.empty()) device = g_device;
    os << "{\n \"device\": \"" << device << "\",\n \"entries\": [";
    bool first = true;
    for (const auto& kv : g_table) {
      os << (first ? "\n" : ",\n") << "  {\"pass\": \"" << pass_name(kv.first.pass) << "\", \"dim\": " << kv.first.dim
         << ", \"P\": " << kv.first.P << ", \"prec\": " << kv.first.prec << ", \"J\": " << kv.first.J << ", \"v\": [";
      for (int i = 0; i < TUNE_NV; ++i) os << (i ? ", " : "") << kv.second.v[i];
      os << "]}";
      first = false;
    }
    os << "\n ],\n \"runs\": [";
    std::string runs = g_runs;
    // the kept records (without their brackets) and the new one
    std::string inner;
    if (runs.size() >= 2) inner = runs.substr(1, runs.size() - 2);
    while (!inner.empty() && std::isspace((unsigned char)inner.back())) inner.pop_back();
    if (!inner.empty() && !run_record.empty()) inner += ",";
    if (!run_record.empty()) inner += "\n  " + run_record;
    os << inner << "\n ]\n}\n";
    g_runs = "[" + inner + "\n ]";
  }
  std::ofstream f(path);
  if (!f) {
    if (err) *err = std::string("cannot write ") + path;
    return HELM_EINVAL;
  }
  f << os.str();
  return f ? HELM_OK : HELM_EINVAL;
}

// 3D TMA-fed passes (Arnoldi step J; the prolongation's residual and the restriction,
// J = 0): tuned (on, plane slots, z pieces per column, points per thread in y), else on
// with as many plane slots in flight as leave the kernel its CTAs per SM (Arnoldi: 3, 2,
// 2, 2 for J = 1..4; restriction of four raw vectors: 2), one equal share of the level
// per resident CTA, two points per thread (the restriction always takes two).
Tma3Params tma3_params(int pass, int J, int P) {
  Tma3Params p;
  TuneChoice c;
  const int maxj = pass == TP_PROLONG ? 1 : J;
  if (tune_get(pass, 3, P, 8, J, &c)) {
    p.enabled = c.v[0] != 0;
    p.stages = std::max(2, std::min(c.v[1], TM3_STAGES_MAX));
    p.pieces = std::max(0, c.v[2]);
    p.qy = c.v[3] == 4 && maxj <= 2 ? 4 : 2;
    return p;
  }
  p.enabled = true;
  p.stages = pass == TP_RESTRICT ? 3 : (maxj <= 2 ? 6 : (maxj == 3 ? 4 : 3));
  p.pieces = 0;
  p.qy = 2;
  return p;
}

bool persist_level(int dim, int P, int prec_bytes) {
  TuneChoice c;
  if (tune_get(TP_PERSIST, dim, P, prec_bytes, 0, &c)) return c.v[0] != 0 && P <= (dim == 2 ? 512 : 64);
  // off by default: on GB300 the launch-per-pass chain with programmatic dependent
  // launch measured faster (a 63^3 V-cycle 0.30 against 0.41 ms, 1023^2 0.48 against 0.58)
  return false;
}

namespace {
std::atomic<unsigned long long> g_barrier_ns{1000000000ull};
}
unsigned long long barrier_limit_ns() { return g_barrier_ns.load(); }
void set_barrier_limit_ns(unsigned long long ns) {
  g_barrier_ns.store(ns);
  bump_launch_generation();  // captured graphs carry the limit as an argument
}

int tuned_zchunk(int P, int prec_bytes) {
  TuneChoice c;
  if (tune_get(TP_ZPLANES, 3, P, prec_bytes, 0, &c)) {
    const int z = c.v[0];
    if ((z == 2 || z == 4 || z == 8 || z == 16) && z <= P) return z;
  }
  return zchunk(P);
}

int tuned_tpc(int pass, int P, int prec_bytes, int J, int heuristic) {
  TuneChoice c;
  if (tune_get(pass, 2, P, prec_bytes, J, &c) && c.v[0] >= 1) return std::min(c.v[0], 64);
  return heuristic;
}

}  // namespace helm

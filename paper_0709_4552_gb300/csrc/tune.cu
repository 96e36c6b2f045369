// tune.cu -- the autotuner's table: the fastest measured launch shape per
// workload bin, and its JSON file.
//
// Two kinds of entries: the force launch of the host-driven path (i per
// thread, threads per CTA, j-tile and split-j factor, binned by the particle
// count N and the active block n, each bin a factor sqrt(2) wide), and the
// item shape of the device-driven loops and ensembles (i-tile and the number
// of force items planned per resident CTA, which sets the split-j length,
// binned by the median cluster size and the cluster count, factors sqrt(2)
// and 2).  nb_autotune and nb_ensemble_autotune fill the table by timing the
// candidates on the context's own state; the force dispatcher and the graph
// builder look their workload up in it.
//
// File (nb_tune_save / nb_tune_load, or the path in NB_TUNE_FILE, read by
// nb_create and nb_ensemble_create):
//   {"format": "libnbody tuning table 1", "device": "...", "sm_count": 152,
//    "entries": [{"kind": "single" | "batched", "precision": "fp64" | "mixed",
//                 "N_lo": ., "N_hi": ., "n_lo": ., "n_hi": ., "i_per_thread": .,
//                 "threads": ., "j_tile": ., "n_split": ., "item_waves": ., "ms": .}, ...]}
// A table measured on a GPU with another SM count is refused (NB_EINVAL).
#include <ctype.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "nb_internal.cuh"

namespace {

bool in_bin(const nb_tune_entry& e, int64_t N, int64_t n) { return N >= e.N_lo && N < e.N_hi && n >= e.n_lo && n < e.n_hi; }

// ---- a small JSON reader: objects, arrays, strings, numbers, literals -------
struct JVal {
  enum Kind { Null, Num, Str, Arr, Obj } kind = Null;
  double num = 0.0;
  std::string str;
  std::vector<JVal> arr;
  std::vector<std::pair<std::string, JVal>> obj;
  const JVal* get(const char* k) const {
    for (const auto& kv : obj)
      if (kv.first == k) return &kv.second;
    return nullptr;
  }
};

struct JParser {
  const char* p;
  const char* end;
  int depth = 0;
  void ws() {
    while (p < end && isspace((unsigned char)*p)) ++p;
  }
  bool lit(const char* s) {
    const size_t n = strlen(s);
    if ((size_t)(end - p) < n || strncmp(p, s, n) != 0) return false;
    p += n;
    return true;
  }
  bool string(std::string& out) {
    if (p >= end || *p != '"') return false;
    ++p;
    while (p < end && *p != '"') {
      if (*p == '\\') {
        if (++p >= end) return false;
        out.push_back(*p == 'n' ? '\n' : *p);  // \" \\ \/ kept literally; no \u in this format
      } else {
        out.push_back(*p);
      }
      ++p;
    }
    if (p >= end) return false;
    ++p;
    return true;
  }
  bool value(JVal& v) {
    if (++depth > 16) return false;
    ws();
    if (p >= end) return false;
    bool ok = true;
    if (*p == '{') {
      v.kind = JVal::Obj;
      ++p;
      ws();
      if (p < end && *p == '}') {
        ++p;
      } else {
        for (;;) {
          ws();
          std::string k;
          JVal x;
          if (!string(k)) return false;
          ws();
          if (p >= end || *p != ':') return false;
          ++p;
          if (!value(x)) return false;
          v.obj.emplace_back(std::move(k), std::move(x));
          ws();
          if (p < end && *p == ',') { ++p; continue; }
          if (p < end && *p == '}') { ++p; break; }
          return false;
        }
      }
    } else if (*p == '[') {
      v.kind = JVal::Arr;
      ++p;
      ws();
      if (p < end && *p == ']') {
        ++p;
      } else {
        for (;;) {
          JVal x;
          if (!value(x)) return false;
          v.arr.push_back(std::move(x));
          ws();
          if (p < end && *p == ',') { ++p; continue; }
          if (p < end && *p == ']') { ++p; break; }
          return false;
        }
      }
    } else if (*p == '"') {
      v.kind = JVal::Str;
      ok = string(v.str);
    } else if (lit("null") || lit("true") || lit("false")) {
      v.kind = JVal::Null;
    } else {
      char* q = nullptr;
      std::string tok;
      while (p < end && (isdigit((unsigned char)*p) || strchr("+-.eE", *p))) tok.push_back(*p++);
      if (tok.empty()) return false;
      v.kind = JVal::Num;
      v.num = strtod(tok.c_str(), &q);
      ok = q && *q == '\0';
    }
    --depth;
    return ok;
  }
};

bool num_field(const JVal& o, const char* k, double* out) {
  const JVal* v = o.get(k);
  if (!v || v->kind != JVal::Num || !isfinite(v->num)) return false;
  *out = v->num;
  return true;
}

int sm_count_of(const nb_ctx* c) { return c->sm_count; }

}  // namespace

const nb_tune_entry* nb_tune_find(const nb_ctx* c, int kind, int64_t N, int64_t n) {
  for (int i = 0; i < c->tune_count; ++i) {
    const nb_tune_entry& e = c->tune_table[i];
    if (e.kind == kind && e.precision == c->precision && in_bin(e, N, n)) return &e;
  }
  return nullptr;
}

void nb_tune_store(nb_ctx* c, int kind, int64_t N, int64_t n, const nb_tuning& cfg, double ms) {
  // single: N and n within a factor sqrt(2); batched: median N_c within
  // sqrt(2), cluster count within 2
  const double fn = kind == NB_TUNE_SINGLE ? 1.41421356 : 2.0;
  nb_tune_entry e{};
  e.kind = kind;
  e.precision = c->precision;
  e.N_lo = (int64_t)(N / 1.41421356);
  e.N_hi = (int64_t)(N * 1.41421356) + 1;
  e.n_lo = (int64_t)(n / fn);
  e.n_hi = (int64_t)(n * fn) + 1;
  e.cfg = cfg;
  e.ms = ms;
  // an entry of the same workload bin (its own n inside the new bin) is
  // replaced; a neighbour whose bin merely overlaps keeps its range and the
  // new bin stops at its edge, so that every (N, n) has one entry
  int slot = -1;
  for (int i = 0; i < c->tune_count; ++i) {
    const nb_tune_entry& o = c->tune_table[i];
    if (o.kind != kind || o.precision != e.precision || o.N_hi <= e.N_lo || e.N_hi <= o.N_lo) continue;
    if (o.n_hi <= e.n_lo || e.n_hi <= o.n_lo) continue;
    const double oc = sqrt((double)o.n_lo * (double)o.n_hi);  // the n it was tuned at
    if (n >= o.n_lo && n < o.n_hi && oc >= e.n_lo && oc < e.n_hi) {
      slot = i;
    } else if (o.n_hi <= n) {
      e.n_lo = std::max(e.n_lo, o.n_hi);
    } else {
      e.n_hi = std::min(e.n_hi, o.n_lo);
    }
  }
  if (e.n_hi <= e.n_lo) return;  // squeezed out by its neighbours
  if (slot < 0) slot = c->tune_count < NB_TUNE_MAX ? c->tune_count++ : NB_TUNE_MAX - 1;
  c->tune_table[slot] = e;
}

extern "C" int nb_tune_save(nb_ctx* c, const char* path) {
  if (!c || !path) return NB_EINVAL;
  FILE* f = fopen(path, "w");
  if (!f) return NB_EINVAL;
  cudaDeviceProp prop;
  const char* name = cudaGetDeviceProperties(&prop, c->device) == cudaSuccess ? prop.name : "unknown";
  cudaGetLastError();
  fprintf(f, "{\"format\": \"libnbody tuning table 1\", \"device\": \"");
  for (const char* s = name; *s; ++s)
    if (*s != '"' && *s != '\\' && (unsigned char)*s >= 0x20) fputc(*s, f);
  fprintf(f, "\", \"sm_count\": %d,\n \"entries\": [", sm_count_of(c));
  for (int i = 0; i < c->tune_count; ++i) {
    const nb_tune_entry& e = c->tune_table[i];
    fprintf(f,
            "%s\n  {\"kind\": \"%s\", \"precision\": \"%s\", \"N_lo\": %lld, \"N_hi\": %lld, \"n_lo\": %lld, "
            "\"n_hi\": %lld, \"i_per_thread\": %d, \"threads\": %d, \"j_tile\": %d, \"n_split\": %d, "
            "\"item_waves\": %d, \"ms\": %.6g}",
            i ? "," : "", e.kind == NB_TUNE_BATCHED ? "batched" : "single", e.precision == NB_FP64 ? "fp64" : "mixed",
            (long long)e.N_lo, (long long)e.N_hi, (long long)e.n_lo, (long long)e.n_hi, e.cfg.ipt, e.cfg.threads,
            e.cfg.jtile, e.cfg.nsplit, e.cfg.waves, e.ms);
  }
  fprintf(f, "\n ]}\n");
  const bool ok = ferror(f) == 0;
  return (fclose(f) == 0 && ok) ? NB_OK : NB_EINVAL;
}

extern "C" int nb_tune_load(nb_ctx* c, const char* path) {
  if (!c || !path) return NB_EINVAL;
  FILE* f = fopen(path, "rb");
  if (!f) return NB_EINVAL;
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = fread(buf, 1, sizeof(buf), f)) > 0 && text.size() < (1u << 20)) text.append(buf, got);
  fclose(f);
  JParser ps{text.data(), text.data() + text.size()};
  JVal root;
  if (!ps.value(root) || root.kind != JVal::Obj) return NB_EINVAL;
  const JVal* fmt = root.get("format");
  const JVal* ents = root.get("entries");
  double sms = 0;
  if (!fmt || fmt->kind != JVal::Str || fmt->str != "libnbody tuning table 1" || !ents || ents->kind != JVal::Arr ||
      !num_field(root, "sm_count", &sms))
    return NB_EINVAL;
  if ((int)sms != sm_count_of(c)) return NB_EINVAL;  // measured on another GPU
  std::vector<nb_tune_entry> out;
  for (const JVal& o : ents->arr) {
    if (o.kind != JVal::Obj) return NB_EINVAL;
    const JVal* kind = o.get("kind");
    const JVal* prec = o.get("precision");
    double v[10];
    const char* keys[10] = {"N_lo", "N_hi", "n_lo", "n_hi", "i_per_thread", "threads", "j_tile", "n_split",
                            "item_waves", "ms"};
    for (int k = 0; k < 10; ++k)
      if (!num_field(o, keys[k], &v[k])) return NB_EINVAL;
    if (!kind || kind->kind != JVal::Str || !prec || prec->kind != JVal::Str) return NB_EINVAL;
    nb_tune_entry e{};
    if (kind->str == "single") e.kind = NB_TUNE_SINGLE;
    else if (kind->str == "batched") e.kind = NB_TUNE_BATCHED;
    else return NB_EINVAL;
    if (prec->str == "fp64") e.precision = NB_FP64;
    else if (prec->str == "mixed") e.precision = NB_MIXED;
    else return NB_EINVAL;
    e.N_lo = (int64_t)v[0];
    e.N_hi = (int64_t)v[1];
    e.n_lo = (int64_t)v[2];
    e.n_hi = (int64_t)v[3];
    e.cfg = nb_tuning{(int)v[4], (int)v[5], (int)v[6], (int)v[7], (int)v[8]};
    e.ms = v[9];
    if (e.N_lo < 0 || e.N_hi <= e.N_lo || e.n_lo < 0 || e.n_hi <= e.n_lo) return NB_EINVAL;
    if (e.kind == NB_TUNE_SINGLE && !nb_tuning_supported(e.precision, e.cfg)) return NB_EINVAL;
    if (e.kind == NB_TUNE_BATCHED && !((e.cfg.threads == 32 || e.cfg.threads == 64 || e.cfg.threads == 128) &&
                                       e.cfg.waves >= 1 && e.cfg.waves <= 64))
      return NB_EINVAL;
    out.push_back(e);
    if (out.size() > NB_TUNE_MAX) return NB_EINVAL;
  }
  c->tune_count = (int)out.size();
  for (size_t i = 0; i < out.size(); ++i) c->tune_table[i] = out[i];
  return NB_OK;
}

extern "C" int nb_tune_count(nb_ctx* c, int* count) {
  if (!c || !count) return NB_EINVAL;
  *count = c->tune_count;
  return NB_OK;
}

extern "C" int nb_tune_clear(nb_ctx* c) {
  if (!c) return NB_EINVAL;
  c->tune_count = 0;
  return NB_OK;
}

void nb_tune_load_env(nb_ctx* c) {
  const char* path = getenv("NB_TUNE_FILE");
  if (path && *path) nb_tune_load(c, path);  // best effort: a missing or foreign table leaves it empty
}

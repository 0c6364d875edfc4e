// The autotuner's persistent cache: a JSON file that maps a plan key -- frame size, window
// length, storage precision, device name and SM count -- to the picks of dh_plan_autotune,
// so that a process restart (or a second plan of the same shape) applies them without
// measuring again:
//   {"version": 1, "entries": {"<key>": {"render_schedule": 0, "render_ring": 8, ...}, ...}}
// Host code only: a small recursive-descent reader for the JSON subset the file uses (objects,
// strings, numbers; arrays, true, false and null are accepted and skipped) and a writer that
// keeps every other entry of the file.
#include "dh_internal.cuh"

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

struct dh_plan;

namespace dh {
Plan &plan_of(dh_plan *h);  // dh_api.cu

namespace {

// Options the cache records, in file order.
struct Field { const char *name; int option; };
constexpr Field kFields[] = {
    {"render_schedule", DH_OPT_RENDER_SCHEDULE}, {"render_ring", DH_OPT_RENDER_RING},
    {"render_lag", DH_OPT_RENDER_LAG},           {"render_fft", DH_OPT_RENDER_FFT},
    {"fft_radix", DH_OPT_FFT_RADIX},             {"gram_units", DH_OPT_GRAM_UNITS},
};

struct JVal {
  enum Kind { OBJ, STR, NUM, OTHER } kind = OTHER;
  std::vector<std::pair<std::string, JVal>> obj;
  std::string str;
  double num = 0;
  const JVal *get(const char *k) const {
    for (const auto &kv : obj)
      if (kv.first == k) return &kv.second;
    return nullptr;
  }
};

struct Reader {
  const char *p, *end;
  int depth = 0;
  void ws() { while (p < end && (*p == ' ' || *p == '\t' || *p == '\n' || *p == '\r')) ++p; }
  bool lit(const char *w) {
    const size_t n = strlen(w);
    if ((size_t)(end - p) < n || strncmp(p, w, n) != 0) return false;
    p += n;
    return true;
  }
  bool string(std::string &out) {
    if (p >= end || *p != '"') return false;
    ++p;
    while (p < end && *p != '"') {
      if (*p == '\\') {
        if (++p >= end) return false;
        switch (*p) {
          case '"': out += '"'; break;
          case '\\': out += '\\'; break;
          case '/': out += '/'; break;
          case 'b': out += '\b'; break;
          case 'f': out += '\f'; break;
          case 'n': out += '\n'; break;
          case 'r': out += '\r'; break;
          case 't': out += '\t'; break;
          case 'u':  // kept verbatim: keys written by this library are plain ASCII
            if (end - p < 5) return false;
            out.append(p - 1, 6);
            p += 4;
            break;
          default: return false;
        }
        ++p;
      } else {
        out += *p++;
      }
    }
    if (p >= end) return false;
    ++p;
    return true;
  }
  bool value(JVal &v) {
    if (++depth > 32) return false;
    ws();
    if (p >= end) return false;
    bool ok = true;
    if (*p == '{') {
      v.kind = JVal::OBJ;
      ++p;
      ws();
      if (p < end && *p == '}') {
        ++p;
      } else {
        for (;;) {
          ws();
          std::string k;
          JVal x;
          if (!string(k)) { ok = false; break; }
          ws();
          if (p >= end || *p != ':') { ok = false; break; }
          ++p;
          if (!value(x)) { ok = false; break; }
          v.obj.emplace_back(std::move(k), std::move(x));
          ws();
          if (p < end && *p == ',') { ++p; continue; }
          if (p < end && *p == '}') { ++p; break; }
          ok = false;
          break;
        }
      }
    } else if (*p == '[') {
      ++p;
      ws();
      if (p < end && *p == ']') {
        ++p;
      } else {
        for (;;) {
          JVal x;
          if (!value(x)) { ok = false; break; }
          ws();
          if (p < end && *p == ',') { ++p; continue; }
          if (p < end && *p == ']') { ++p; break; }
          ok = false;
          break;
        }
      }
    } else if (*p == '"') {
      v.kind = JVal::STR;
      ok = string(v.str);
    } else if (lit("true") || lit("false") || lit("null")) {
      v.kind = JVal::OTHER;
    } else {
      char *q = nullptr;
      v.num = strtod(p, &q);
      if (q == p) {
        ok = false;
      } else {
        v.kind = JVal::NUM;
        p = q;
      }
    }
    --depth;
    return ok;
  }
};

// The whole file, parsed; `exists` false when it cannot be opened (a new cache).
bool read_file(const char *path, JVal &root, bool &exists) {
  exists = false;
  FILE *f = fopen(path, "rb");
  if (!f) return true;
  exists = true;
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, n);
  fclose(f);
  Reader r{text.data(), text.data() + text.size()};
  if (!r.value(root) || root.kind != JVal::OBJ) return false;
  r.ws();
  return r.p == r.end;
}

// A JSON string: quotes and backslashes escaped, control characters (which the reader decodes
// from escapes in other entries' keys) written back as escapes, so the file stays readable.
void put_string(std::string &o, const std::string &s) {
  o += '"';
  for (char ch : s) {
    const unsigned char u = (unsigned char)ch;
    if (ch == '"' || ch == '\\') {
      o += '\\';
      o += ch;
    } else if (u < 0x20) {
      char esc[8];
      snprintf(esc, sizeof esc, "\\u%04x", (unsigned)u);
      o += esc;
    } else {
      o += ch;
    }
  }
  o += '"';
}

std::string plan_key(const Plan &p) {
  cudaDeviceProp prop;
  const char *dev = cudaGetDeviceProperties(&prop, p.device) == cudaSuccess ? prop.name : "unknown";
  const char *prec = p.prec == DH_PREC_FP32 ? "fp32" : p.prec == DH_PREC_FP16 ? "fp16" : "bf16";
  char key[512];
  snprintf(key, sizeof key, "nx=%d,ny=%d,T=%d,prec=%s,device=%s,sms=%d", p.nx, p.ny, p.T, prec, dev, p.num_sms);
  return key;
}

}  // namespace
}  // namespace dh

using namespace dh;

extern "C" dh_status dh_plan_tune_load(dh_plan_t h, const char *path, int *found) {
  if (!h || !path || !found) return DH_ERR_INVALID_ARG;
  *found = 0;
  JVal root;
  bool exists = false;
  if (!read_file(path, root, exists)) return DH_ERR_INVALID_ARG;
  if (!exists) return DH_OK;
  const JVal *entries = root.get("entries");
  if (!entries || entries->kind != JVal::OBJ) return DH_OK;
  const JVal *e = entries->get(plan_key(plan_of(h)).c_str());
  if (!e || e->kind != JVal::OBJ) return DH_OK;
  // every recorded field must be a number the option accepts; nothing is applied otherwise
  int vals[sizeof kFields / sizeof kFields[0]];
  int saved[sizeof kFields / sizeof kFields[0]];
  for (size_t i = 0; i < sizeof kFields / sizeof kFields[0]; ++i) {
    const JVal *v = e->get(kFields[i].name);
    dh_status st = dh_plan_get_option(h, kFields[i].option, &saved[i]);
    if (st != DH_OK) return st;
    vals[i] = saved[i];
    if (v) {
      if (v->kind != JVal::NUM || !(v->num >= -1e9 && v->num <= 1e9) || v->num != (double)(int)v->num)
        return DH_ERR_INVALID_ARG;
      vals[i] = (int)v->num;
    }
  }
  for (size_t i = 0; i < sizeof kFields / sizeof kFields[0]; ++i) {
    dh_status st = dh_plan_set_option(h, kFields[i].option, vals[i]);
    if (st == DH_ERR_STATE && vals[i] == saved[i]) continue;  // not applicable to this plan
    if (st != DH_OK) {
      for (size_t k = 0; k < i; ++k) dh_plan_set_option(h, kFields[k].option, saved[k]);
      return st;
    }
  }
  *found = 1;
  return DH_OK;
}

extern "C" dh_status dh_plan_tune_save(dh_plan_t h, const char *path) {
  if (!h || !path) return DH_ERR_INVALID_ARG;
  JVal root;
  bool exists = false;
  if (!read_file(path, root, exists)) return DH_ERR_INVALID_ARG;  // never overwrite what we cannot read
  const std::string key = plan_key(plan_of(h));
  std::string entry = "{";
  for (size_t i = 0; i < sizeof kFields / sizeof kFields[0]; ++i) {
    int v = 0;
    dh_status st = dh_plan_get_option(h, kFields[i].option, &v);
    if (st != DH_OK) return st;
    entry += (i ? ", \"" : "\"") + std::string(kFields[i].name) + "\": " + std::to_string(v);
  }
  entry += "}";
  // rewrite: version, then every entry (numbers of other entries written back as integers when
  // they are integral, as this writer produced them)
  std::string out = "{\"version\": 1, \"entries\": {";
  bool first = true;
  const JVal *entries = exists ? root.get("entries") : nullptr;
  if (entries && entries->kind == JVal::OBJ) {
    for (const auto &kv : entries->obj) {
      if (kv.first == key || kv.second.kind != JVal::OBJ) continue;
      out += first ? "\n  " : ",\n  ";
      first = false;
      put_string(out, kv.first);
      out += ": {";
      bool f2 = true;
      for (const auto &fv : kv.second.obj) {
        if (fv.second.kind != JVal::NUM) continue;
        char num[64];
        const double x = fv.second.num;
        if (!std::isfinite(x)) continue;  // not representable in JSON: the field is dropped
        if (std::fabs(x) < 9.0e15 && x == (double)(long long)x) snprintf(num, sizeof num, ": %lld", (long long)x);
        else snprintf(num, sizeof num, ": %.17g", x);
        out += f2 ? "" : ", ";
        f2 = false;
        put_string(out, fv.first);
        out += num;
      }
      out += "}";
    }
  }
  out += first ? "\n  " : ",\n  ";
  put_string(out, key);
  out += ": " + entry + "\n}}\n";
  const std::string tmp = std::string(path) + ".tmp";
  FILE *f = fopen(tmp.c_str(), "wb");
  if (!f) return DH_ERR_INVALID_ARG;
  const bool wrote = fwrite(out.data(), 1, out.size(), f) == out.size();
  if (fclose(f) != 0 || !wrote || rename(tmp.c_str(), path) != 0) {
    remove(tmp.c_str());
    return DH_ERR_INVALID_ARG;
  }
  return DH_OK;
}

// checkpoint.cu - a context's state to a file and back (checkpoint / resume).
//
// File layout (little-endian, fixed-width fields):
//   magic "MRTLBCK1" (8 bytes), version u32 (1), precision u32, nx u32,
//   ny u32, steps i64, parameter hash u64, data bytes u64,
//   data: the dense state [16][ny][nx] in the state's precision (what
//   mrtlb_get_f returns),
//   checksum u64 of the data.
// Hash and checksum are 64-bit FNV-1a (Fowler-Noll-Vo).  The parameter hash
// covers everything the next step depends on besides the state: grid,
// spacings, time step, the current relaxation rates, equilibrium version,
// modification switch, precision and every side's kind and values.  A state
// written after step n and loaded into a context with the same parameters
// continues bitwise as the run it came from would have.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mrtlb.h"
#include "ctx.h"

namespace {

constexpr char kMagic[8] = {'M', 'R', 'T', 'L', 'B', 'C', 'K', '1'};
constexpr uint32_t kVersion = 1;

struct Fnv {
  uint64_t h = 14695981039346656037ull;
  void add(const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  }
  template <typename T>
  void put(T v) { add(&v, sizeof(v)); }
};

uint64_t params_hash(const mrtlb_ctx* c) {
  Fnv f;
  f.put<int32_t>(c->p.nx);
  f.put<int32_t>(c->p.ny);
  f.put<int32_t>(c->prec);
  f.put<double>(c->p.dx);
  f.put<double>(c->p.dy);
  f.put<double>(c->p.dt);
  for (int k = 0; k < 16; ++k) f.put<double>(c->s[k]);
  f.put<int32_t>(c->p.eq_version);
  f.put<int32_t>(c->p.modified);
  for (int s = 0; s < 4; ++s) {
    f.put<int32_t>(c->p.bc[s].kind);
    f.put<double>(c->p.bc[s].ux);
    f.put<double>(c->p.bc[s].uy);
    f.put<double>(c->p.bc[s].T);
    f.put<double>(c->p.bc[s].rho);
  }
  return f.h;
}

int ck_fail(mrtlb_ctx* c, int code, const std::string& msg) {
  c->last_error = msg;
  return code;
}

template <typename T>
void append(std::vector<unsigned char>& out, T v) {
  const unsigned char* b = reinterpret_cast<const unsigned char*>(&v);
  out.insert(out.end(), b, b + sizeof(v));
}

template <typename T>
bool take(FILE* fh, T* v) {
  return std::fread(v, sizeof(T), 1, fh) == 1;
}

}  // namespace

extern "C" int mrtlb_save(mrtlb_ctx* c, const char* path) {
  TraceRange trace_("mrtlb_save");
  if (!c) return MRTLB_ERR_ARG;
  if (!path || !path[0]) return ck_fail(c, MRTLB_ERR_ARG, "no checkpoint path");
  const size_t bytes = (size_t)16 * c->L.nx * c->L.ny * c->esize;
  std::vector<unsigned char> data(bytes);
  const int rc = mrtlb_get_f(c, data.data(), 0);  // synchronises; reports latched errors
  if (rc) return rc;
  std::vector<unsigned char> head;
  head.insert(head.end(), kMagic, kMagic + 8);
  append<uint32_t>(head, kVersion);
  append<uint32_t>(head, (uint32_t)c->prec);
  append<uint32_t>(head, (uint32_t)c->L.nx);
  append<uint32_t>(head, (uint32_t)c->L.ny);
  append<int64_t>(head, (int64_t)c->steps);
  append<uint64_t>(head, params_hash(c));
  append<uint64_t>(head, (uint64_t)bytes);
  Fnv sum;
  sum.add(data.data(), bytes);
  // write a sibling file, then move it over the target in one step
  const std::string tmp = std::string(path) + ".part";
  FILE* fh = std::fopen(tmp.c_str(), "wb");
  if (!fh) return ck_fail(c, MRTLB_ERR_ARG, "cannot write " + tmp);
  bool ok = std::fwrite(head.data(), 1, head.size(), fh) == head.size();
  ok = ok && std::fwrite(data.data(), 1, bytes, fh) == bytes;
  ok = ok && std::fwrite(&sum.h, sizeof(sum.h), 1, fh) == 1;
  ok = (std::fclose(fh) == 0) && ok;
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return ck_fail(c, MRTLB_ERR_ARG, std::string("cannot write ") + path);
  }
  return MRTLB_OK;
}

extern "C" int mrtlb_load(mrtlb_ctx* c, const char* path) {
  TraceRange trace_("mrtlb_load");
  if (!c) return MRTLB_ERR_ARG;
  if (!path || !path[0]) return ck_fail(c, MRTLB_ERR_ARG, "no checkpoint path");
  FILE* fh = std::fopen(path, "rb");
  if (!fh) return ck_fail(c, MRTLB_ERR_ARG, std::string("cannot read ") + path);
  char magic[8];
  uint32_t version = 0, prec = 0, nx = 0, ny = 0;
  int64_t steps = 0;
  uint64_t hash = 0, bytes = 0, sum_file = 0;
  bool ok = std::fread(magic, 1, 8, fh) == 8 && take(fh, &version) && take(fh, &prec) && take(fh, &nx) &&
            take(fh, &ny) && take(fh, &steps) && take(fh, &hash) && take(fh, &bytes);
  std::string why;
  if (!ok || std::memcmp(magic, kMagic, 8) != 0) why = "not a checkpoint of this library";
  else if (version != kVersion) why = "checkpoint version " + std::to_string(version);
  else if ((int)prec != c->prec || (int)nx != c->L.nx || (int)ny != c->L.ny)
    why = "checkpoint of another grid or precision";
  else if (hash != params_hash(c)) why = "checkpoint written with other parameters";
  else if (bytes != (uint64_t)16 * c->L.nx * c->L.ny * c->esize) why = "checkpoint size mismatch";
  std::vector<unsigned char> data;
  if (why.empty()) {
    data.resize(bytes);
    if (std::fread(data.data(), 1, bytes, fh) != bytes || !take(fh, &sum_file)) why = "checkpoint truncated";
  }
  std::fclose(fh);
  if (why.empty()) {
    Fnv sum;
    sum.add(data.data(), bytes);
    if (sum.h != sum_file) why = "checkpoint checksum mismatch";
  }
  if (!why.empty()) return ck_fail(c, MRTLB_ERR_ARG, why + ": " + path);
  const int rc = mrtlb_set_f(c, data.data(), 0);
  if (rc) return rc;
  c->steps = (long)steps;  // (mrtlb_set_f advanced the generation)
  return MRTLB_OK;
}

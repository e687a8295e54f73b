// MD checkpoints: the state of a run (positions, velocities, forces, species,
// parameter table, box, list radius, precision, launch options, step counter
// and the phase of the fixed rebuild period) in one host file, and its restoration into a
// context. Layout: one line of JSON text, then raw little-endian arrays in a
// fixed order (species int32 n; table double n_species^3 x 14; x, v, f double
// n x 3 each). The header is written and read by this file only, so reading
// looks for its own keys rather than parsing general JSON.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "internal.cuh"

namespace tgb {
namespace {

constexpr const char* kFormat = "tersoff-gb300-checkpoint";
constexpr int kVersion = 1;
constexpr size_t kMaxHeader = 4096;

struct FileCloser {
  void operator()(FILE* f) const {
    if (f) std::fclose(f);
  }
};
using File = std::unique_ptr<FILE, FileCloser>;

bool little_endian() {
  const uint16_t probe = 1;
  unsigned char b;
  std::memcpy(&b, &probe, 1);
  return b == 1;
}

struct Header {
  long long n = -1;
  int ns = 0;
  int precision = -1;
  double box[3] = {0, 0, 0};
  double r_list = 0.0;
  long long step = 0;
  int ssb = 0;
  int cap = 32;  // neighbour-list capacity per atom
  // launch options: scatter mode, force grid waves, capacity-8 split, block,
  // four lanes, ablation flags, graphs
  int opt[7] = {0, 0, -1, 256, -1, 0, 1};
};

constexpr const char* kOptKeys[7] = {"scatter", "waves", "split", "block",
                                     "lanes",   "ablate", "graphs"};

// value after "key": in the header text (numbers only)
bool find_number(const std::string& h, const char* key, double* out) {
  const std::string k = std::string("\"") + key + "\":";
  const size_t p = h.find(k);
  if (p == std::string::npos) return false;
  const char* s = h.c_str() + p + k.size();
  char* end = nullptr;
  *out = std::strtod(s, &end);
  return end != s;
}

bool parse_header(const std::string& h, Header* hd) {
  const std::string fmt = std::string("{\"format\":\"") + kFormat + "\",\"version\":";
  if (h.compare(0, fmt.size(), fmt) != 0) return false;
  double v;
  if (!find_number(h, "version", &v) || v != kVersion) return false;
  if (!find_number(h, "n", &v)) return false;
  hd->n = (long long)v;
  if (!find_number(h, "n_species", &v)) return false;
  hd->ns = (int)v;
  if (!find_number(h, "precision", &v)) return false;
  hd->precision = (int)v;
  if (!find_number(h, "r_list", &hd->r_list)) return false;
  if (!find_number(h, "step", &v)) return false;
  hd->step = (long long)v;
  if (!find_number(h, "steps_since_build", &v)) return false;
  hd->ssb = (int)v;
  if (!find_number(h, "capacity", &v)) return false;
  hd->cap = (int)v;
  for (int k = 0; k < 7; ++k) {
    if (!find_number(h, kOptKeys[k], &v)) return false;
    hd->opt[k] = (int)v;
  }
  const size_t p = h.find("\"box\":[");
  if (p == std::string::npos) return false;
  const char* s = h.c_str() + p + 7;
  for (int a = 0; a < 3; ++a) {
    char* end = nullptr;
    hd->box[a] = std::strtod(s, &end);
    if (end == s) return false;
    s = end;
    if (a < 2) {
      if (*s != ',') return false;
      ++s;
    }
  }
  return hd->n >= 0 && hd->n < MAX_ATOMS && hd->ns >= 1 && hd->ns <= TERSOFF_MAX_SPECIES &&
         (hd->precision == TERSOFF_FP64 || hd->precision == TERSOFF_MIXED);
}

// reads the header line of an open checkpoint file
int read_header(Ctx* c, FILE* f, Header* hd) {
  std::string h;
  int ch;
  while ((ch = std::fgetc(f)) != EOF && ch != '\n') {
    h.push_back((char)ch);
    if (h.size() > kMaxHeader) break;
  }
  if (ch != '\n' || !parse_header(h, hd))
    return c ? fail(c, TERSOFF_E_INVALID_ARG, "not a checkpoint of this library (header)")
             : TERSOFF_E_INVALID_ARG;
  return TERSOFF_OK;
}

}  // namespace
}  // namespace tgb

using tgb::Ctx;

extern "C" {

int tersoff_checkpoint_save(tersoff_ctx* p, const char* path, const double* x, const double* v,
                            const double* f, int n, long long step, void* stream) {
  tgb::NvtxRange nvtx_range("tersoff_checkpoint_save");
  Ctx* c = p ? &p->impl : nullptr;
  if (!c) return TERSOFF_E_INVALID_ARG;
  TGB_CUDA(c, cudaSetDevice(c->device));
  if (!path || (n > 0 && (!x || !v || !f)))
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "checkpoint: null path or array");
  if (!tgb::little_endian())
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "checkpoint: big-endian hosts are not supported");
  if (c->ns == 0 || !c->have_list || c->n_sys > 0)
    return tgb::fail(c, TERSOFF_E_STATE,
                     "checkpoint: needs parameters and a single-system neighbour build");
  if (n != c->n) return tgb::fail(c, TERSOFF_E_INVALID_ARG, "atom count differs from the neighbour build");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t m = 3 * (size_t)n;
  std::vector<int> types((size_t)n);
  std::vector<double> state(3 * m);
  if (n > 0) {
    TGB_CUDA(c, cudaMemcpyAsync(types.data(), c->d_types, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
    TGB_CUDA(c, cudaMemcpyAsync(state.data(), x, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    TGB_CUDA(c, cudaMemcpyAsync(state.data() + m, v, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    TGB_CUDA(c, cudaMemcpyAsync(state.data() + 2 * m, f, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
  }
  TGB_CUDA(c, cudaStreamSynchronize(s));
  char hdr[tgb::kMaxHeader];
  const int len = std::snprintf(
      hdr, sizeof hdr,
      "{\"format\":\"%s\",\"version\":%d,\"n\":%d,\"n_species\":%d,\"precision\":%d,"
      "\"box\":[%.17g,%.17g,%.17g],\"r_list\":%.17g,\"step\":%lld,\"steps_since_build\":%d,"
      "\"capacity\":%d,"
      "\"scatter\":%d,\"waves\":%d,\"split\":%d,\"block\":%d,\"lanes\":%d,\"ablate\":%d,"
      "\"graphs\":%d,\"endian\":\"little\",\"arrays\":[\"types:int32[n]\","
      "\"table:float64[n_species^3*14]\",\"x:float64[n*3]\",\"v:float64[n*3]\","
      "\"f:float64[n*3]\"]}\n",
      tgb::kFormat, tgb::kVersion, n, c->ns, c->precision, c->grid.L[0], c->grid.L[1],
      c->grid.L[2], c->r_list, step, c->steps_since_build, c->cap, c->scatter_atomic ? 1 : 0,
      c->opt_waves, c->opt_split, c->opt_block, c->opt_quad, c->ablate, c->use_graphs ? 1 : 0);
  if (len <= 0 || len >= (int)sizeof hdr) return tgb::fail(c, TERSOFF_E_INVALID_ARG, "checkpoint header");
  tgb::File fh(std::fopen(path, "wb"));
  if (!fh) return tgb::fail(c, TERSOFF_E_INVALID_ARG, "checkpoint: cannot open the file for writing");
  bool ok = std::fwrite(hdr, 1, (size_t)len, fh.get()) == (size_t)len;
  ok = ok && std::fwrite(types.data(), sizeof(int), types.size(), fh.get()) == types.size();
  ok = ok && std::fwrite(c->table.data(), sizeof(double), c->table.size(), fh.get()) ==
                 c->table.size();
  ok = ok && std::fwrite(state.data(), sizeof(double), state.size(), fh.get()) == state.size();
  ok = ok && std::fflush(fh.get()) == 0;
  if (!ok) return tgb::fail(c, TERSOFF_E_INVALID_ARG, "checkpoint: write failed");
  return TERSOFF_OK;
}

int tersoff_checkpoint_info(const char* path, int* n, int* n_species) {
  if (!path) return TERSOFF_E_INVALID_ARG;
  tgb::File fh(std::fopen(path, "rb"));
  if (!fh) return TERSOFF_E_INVALID_ARG;
  tgb::Header hd;
  const int st = tgb::read_header(nullptr, fh.get(), &hd);
  if (st) return st;
  if (n) *n = (int)hd.n;
  if (n_species) *n_species = hd.ns;
  return TERSOFF_OK;
}

int tersoff_checkpoint_load(tersoff_ctx* p, const char* path, double* x, double* v, double* f,
                            int* types, int n, long long* step, void* stream) {
  tgb::NvtxRange nvtx_range("tersoff_checkpoint_load");
  Ctx* c = p ? &p->impl : nullptr;
  if (!c) return TERSOFF_E_INVALID_ARG;
  TGB_CUDA(c, cudaSetDevice(c->device));
  if (!path || (n > 0 && (!x || !v || !f || !types)))
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "checkpoint: null path or array");
  if (!tgb::little_endian())
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "checkpoint: big-endian hosts are not supported");
  tgb::File fh(std::fopen(path, "rb"));
  if (!fh) return tgb::fail(c, TERSOFF_E_INVALID_ARG, "checkpoint: cannot open the file");
  tgb::Header hd;
  int st = tgb::read_header(c, fh.get(), &hd);
  if (st) return st;
  if (hd.n != n) return tgb::fail(c, TERSOFF_E_INVALID_ARG, "checkpoint: atom count differs");
  const size_t m = 3 * (size_t)n;
  const size_t nt = (size_t)hd.ns * hd.ns * hd.ns * TERSOFF_NPARAM;
  std::vector<int> ht((size_t)n);
  std::vector<double> table(nt), state(3 * m);
  bool ok = std::fread(ht.data(), sizeof(int), ht.size(), fh.get()) == ht.size();
  ok = ok && std::fread(table.data(), sizeof(double), nt, fh.get()) == nt;
  ok = ok && std::fread(state.data(), sizeof(double), state.size(), fh.get()) == state.size();
  if (!ok) return tgb::fail(c, TERSOFF_E_INVALID_ARG, "checkpoint: file is truncated");
  if ((st = tersoff_set_precision(p, hd.precision))) return st;
  if ((st = tersoff_params(p, hd.ns, table.data()))) return st;
  // the saved launch options (they decide which kernel evaluates an atom and
  // the order of its sums)
  if ((st = tersoff_set_scatter(p, hd.opt[0]))) return st;
  if ((st = tersoff_set_launch(p, hd.opt[1], hd.opt[2], hd.opt[3]))) return st;
  if ((st = tersoff_set_lanes(p, hd.opt[4] == 1 ? 4 : (hd.opt[4] == 0 ? 1 : 0)))) return st;
  if ((st = tersoff_set_ablation(p, hd.opt[5]))) return st;
  if ((st = tersoff_set_graphs(p, hd.opt[6]))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (n > 0) {
    TGB_CUDA(c, cudaMemcpyAsync(types, ht.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
    TGB_CUDA(c, cudaMemcpyAsync(x, state.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s));
    TGB_CUDA(c, cudaMemcpyAsync(v, state.data() + m, sizeof(double) * m, cudaMemcpyHostToDevice, s));
    TGB_CUDA(c, cudaMemcpyAsync(f, state.data() + 2 * m, sizeof(double) * m, cudaMemcpyHostToDevice, s));
  }
  // the list of the saved positions with the saved capacity (grown if they
  // need more; synchronises s), then the saved phase of the fixed rebuild period
  if ((st = tersoff_set_neighbor_capacity(p, hd.cap))) return st;
  if ((st = tersoff_neighbor_build(p, x, types, n, hd.box, hd.r_list, stream))) return st;
  c->steps_since_build = hd.ssb;
  if (step) *step = hd.step;
  return TERSOFF_OK;
}

}  // extern "C"

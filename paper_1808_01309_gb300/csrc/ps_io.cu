// Checkpoint and resume of a plan's state (include/ps.h, ps_checkpoint_*).
// The state is the caller's device buffer in the ABI layout, so a checkpoint
// is that buffer written to a file behind a fixed little-endian header with
// the grid, box, precision, equations, coefficients, time and step, and an
// FNV-1a 64 checksum of the payload.  Host code only: the payload moves in
// 64 MB chunks through one host buffer (no second device copy of the state).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ps.h"
#include "ps_kernels.h"

namespace ps {
void set_last_error(const std::string& msg);
// plan internals (ps_plan.cu): configuration and bytes of the caller-layout state
ps_config plan_config(const struct ::ps_plan* p);
size_t plan_state_bytes(const struct ::ps_plan* p);
}

using namespace ps;

namespace {

constexpr char kMagic[8] = {'P', 'S', 'C', 'K', 'P', 'T', 0, 1};
constexpr uint32_t kVersion = 1;
constexpr size_t kHeader = 136;
constexpr size_t kChunk = 64ull << 20;

ps_status bad(ps_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

struct Header {
  int32_t nx, ny, nz, prec, eq, dealias, rk_order, ncomp;
  double lx, ly, lz, nu, eta, n_bv, kappa, t;
  int64_t step;
  uint64_t payload, checksum;
};

int ncomp_of(int eq) { return eq == PS_MHD ? 6 : eq == PS_BOUSSINESQ ? 4 : 3; }

// Field-by-field little-endian encoding (no struct padding in the file).
template <typename V>
void put(unsigned char*& p, V v) {
  unsigned char b[sizeof(V)];
  std::memcpy(b, &v, sizeof(V));
  for (size_t i = 0; i < sizeof(V); ++i) *p++ = b[i];  // hosts of this library are little-endian
}
template <typename V>
V get(const unsigned char*& p) {
  V v;
  std::memcpy(&v, p, sizeof(V));
  p += sizeof(V);
  return v;
}

void encode(const Header& h, unsigned char* buf) {
  unsigned char* p = buf;
  std::memcpy(p, kMagic, 8);
  p += 8;
  put<uint32_t>(p, kVersion);
  put<uint32_t>(p, (uint32_t)kHeader);
  for (int32_t v : {h.nx, h.ny, h.nz, h.prec, h.eq, h.dealias, h.rk_order, h.ncomp}) put<int32_t>(p, v);
  for (double v : {h.lx, h.ly, h.lz, h.nu, h.eta, h.n_bv, h.kappa, h.t}) put<double>(p, v);
  put<int64_t>(p, h.step);
  put<uint64_t>(p, h.payload);
  put<uint64_t>(p, h.checksum);
}

ps_status decode(const unsigned char* buf, Header& h) {
  if (std::memcmp(buf, kMagic, 8) != 0) return bad(PS_ERR_INVALID_ARG, "checkpoint: not a checkpoint file (magic)");
  const unsigned char* p = buf + 8;
  if (get<uint32_t>(p) != kVersion) return bad(PS_ERR_INVALID_ARG, "checkpoint: unknown version");
  if (get<uint32_t>(p) != kHeader) return bad(PS_ERR_INVALID_ARG, "checkpoint: unknown header size");
  int32_t* iv[] = {&h.nx, &h.ny, &h.nz, &h.prec, &h.eq, &h.dealias, &h.rk_order, &h.ncomp};
  for (int32_t* v : iv) *v = get<int32_t>(p);
  double* dv[] = {&h.lx, &h.ly, &h.lz, &h.nu, &h.eta, &h.n_bv, &h.kappa, &h.t};
  for (double* v : dv) *v = get<double>(p);
  h.step = get<int64_t>(p);
  h.payload = get<uint64_t>(p);
  h.checksum = get<uint64_t>(p);
  if (h.nx <= 0 || h.ny <= 0 || h.nz <= 0 || (h.prec != PS_FP32 && h.prec != PS_FP64) ||
      h.ncomp != ncomp_of(h.eq))
    return bad(PS_ERR_INVALID_ARG, "checkpoint: inconsistent header");
  const uint64_t want = (uint64_t)h.ncomp * h.nz * h.ny * (h.nx / 2 + 1) * (h.prec == PS_FP32 ? 8 : 16);
  if (h.payload != want) return bad(PS_ERR_INVALID_ARG, "checkpoint: payload size does not match the grid");
  return PS_OK;
}

// FNV-1a, 64 bit (Fowler, Noll, Vo): offset basis and prime of the published definition.
struct Fnv {
  uint64_t h = 14695981039346656037ull;
  void add(const unsigned char* p, size_t n) {
    for (size_t i = 0; i < n; ++i) {
      h ^= p[i];
      h *= 1099511628211ull;
    }
  }
};

ps_status read_header(std::FILE* f, Header& h) {
  unsigned char buf[kHeader];
  if (std::fread(buf, 1, kHeader, f) != kHeader) return bad(PS_ERR_INVALID_ARG, "checkpoint: truncated header");
  return decode(buf, h);
}

ps_status cuda_bad(cudaError_t e, const char* where) {
  return bad(PS_ERR_CUDA, std::string("checkpoint: ") + where + ": " + cudaGetErrorString(e));
}

struct FileCloser {
  std::FILE* f;
  ~FileCloser() {
    if (f) std::fclose(f);
  }
};

}  // namespace

extern "C" ps_status ps_checkpoint_info(const char* path, ps_config* cfg, double* t, long long* step) {
  if (!path) return bad(PS_ERR_INVALID_ARG, "checkpoint: NULL path");
  std::FILE* f = std::fopen(path, "rb");
  if (!f) return bad(PS_ERR_INVALID_ARG, std::string("checkpoint: cannot open ") + path);
  FileCloser fc{f};
  Header h{};
  ps_status s = read_header(f, h);
  if (s != PS_OK) return s;
  if (cfg) {
    *cfg = ps_config{};
    cfg->nx = h.nx;
    cfg->ny = h.ny;
    cfg->nz = h.nz;
    cfg->lx = h.lx;
    cfg->ly = h.ly;
    cfg->lz = h.lz;
    cfg->prec = (ps_precision)h.prec;
    cfg->eq = (ps_equations)h.eq;
    cfg->dealias = (ps_dealias)h.dealias;
    cfg->rk_order = h.rk_order;
    cfg->nu = h.nu;
    cfg->eta = h.eta;
    cfg->n_bv = h.n_bv;
    cfg->kappa = h.kappa;
    cfg->forcing = nullptr;
  }
  if (t) *t = h.t;
  if (step) *step = h.step;
  return PS_OK;
}

namespace {
ps_status save_to(ps_plan* plan, const void* uhat, double t, long long step, const std::string& tmp);
}

extern "C" ps_status ps_checkpoint_save(ps_plan* plan, const void* uhat, double t, long long step, const char* path) {
  if (!plan || !uhat || !path) return bad(PS_ERR_INVALID_ARG, "checkpoint: NULL plan, state or path");
  const std::string tmp = std::string(path) + ".part";
  const ps_status s = save_to(plan, uhat, t, step, tmp);
  if (s != PS_OK) {
    std::remove(tmp.c_str());  // no partial file is left behind
    return s;
  }
  if (std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return bad(PS_ERR_INVALID_ARG, std::string("checkpoint: cannot rename to ") + path);
  }
  return PS_OK;
}

namespace {
// Header (checksum written once the payload is known) and payload into tmp.
ps_status save_to(ps_plan* plan, const void* uhat, double t, long long step, const std::string& tmp) {
  const ps_config c = plan_config(plan);
  Header h{};
  h.nx = c.nx;
  h.ny = c.ny;
  h.nz = c.nz;
  h.prec = c.prec;
  h.eq = c.eq;
  h.dealias = c.dealias;
  h.rk_order = c.rk_order;
  h.ncomp = ncomp_of(c.eq);
  h.lx = c.lx;
  h.ly = c.ly;
  h.lz = c.lz;
  h.nu = c.nu;
  h.eta = c.eta;
  h.n_bv = c.n_bv;
  h.kappa = c.kappa;
  h.t = t;
  h.step = step;
  h.payload = plan_state_bytes(plan);
  std::FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return bad(PS_ERR_INVALID_ARG, std::string("checkpoint: cannot create ") + tmp);
  FileCloser fc{f};
  unsigned char hb[kHeader] = {0};
  encode(h, hb);  // checksum written once the payload is known
  if (std::fwrite(hb, 1, kHeader, f) != kHeader) return bad(PS_ERR_INVALID_ARG, "checkpoint: write failed");
  cudaStream_t st = plan_stream(plan);
  cudaError_t e = cudaStreamSynchronize(st);  // the state is final
  if (e != cudaSuccess) return cuda_bad(e, "synchronise");
  std::vector<unsigned char> buf(std::min<size_t>(kChunk, h.payload));
  Fnv fnv;
  for (uint64_t off = 0; off < h.payload; off += buf.size()) {
    const size_t n = (size_t)std::min<uint64_t>(buf.size(), h.payload - off);
    if ((e = cudaMemcpy(buf.data(), static_cast<const char*>(uhat) + off, n, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_bad(e, "device to host");
    fnv.add(buf.data(), n);
    if (std::fwrite(buf.data(), 1, n, f) != n) return bad(PS_ERR_INVALID_ARG, "checkpoint: write failed");
  }
  h.checksum = fnv.h;
  encode(h, hb);
  if (std::fseek(f, 0, SEEK_SET) != 0 || std::fwrite(hb, 1, kHeader, f) != kHeader)
    return bad(PS_ERR_INVALID_ARG, "checkpoint: write failed");
  const int cl = std::fclose(f);
  fc.f = nullptr;
  if (cl != 0) return bad(PS_ERR_INVALID_ARG, "checkpoint: close failed");
  return PS_OK;
}
}  // namespace

extern "C" ps_status ps_checkpoint_load(ps_plan* plan, void* uhat, double* t, long long* step, const char* path) {
  if (!plan || !uhat || !path) return bad(PS_ERR_INVALID_ARG, "checkpoint: NULL plan, state or path");
  std::FILE* f = std::fopen(path, "rb");
  if (!f) return bad(PS_ERR_INVALID_ARG, std::string("checkpoint: cannot open ") + path);
  FileCloser fc{f};
  Header h{};
  ps_status s = read_header(f, h);
  if (s != PS_OK) return s;
  const ps_config c = plan_config(plan);
  if (h.nx != c.nx || h.ny != c.ny || h.nz != c.nz || h.prec != (int)c.prec || h.eq != (int)c.eq ||
      h.lx != c.lx || h.ly != c.ly || h.lz != c.lz)
    return bad(PS_ERR_INVALID_ARG, "checkpoint: grid, box, precision or equations differ from the plan's");
  if (h.payload != plan_state_bytes(plan)) return bad(PS_ERR_INVALID_ARG, "checkpoint: payload size differs");
  std::vector<unsigned char> buf(std::min<size_t>(kChunk, h.payload));
  // first pass: verify the checksum before anything reaches the caller's state
  Fnv fnv;
  for (uint64_t off = 0; off < h.payload; off += buf.size()) {
    const size_t n = (size_t)std::min<uint64_t>(buf.size(), h.payload - off);
    if (std::fread(buf.data(), 1, n, f) != n) return bad(PS_ERR_INVALID_ARG, "checkpoint: truncated payload");
    fnv.add(buf.data(), n);
  }
  if (fnv.h != h.checksum) return bad(PS_ERR_INVALID_ARG, "checkpoint: checksum mismatch (corrupted file)");
  if (std::fseek(f, (long)kHeader, SEEK_SET) != 0) return bad(PS_ERR_INVALID_ARG, "checkpoint: seek failed");
  cudaError_t e = cudaStreamSynchronize(plan_stream(plan));  // earlier work on the state is done
  if (e != cudaSuccess) return cuda_bad(e, "synchronise");
  for (uint64_t off = 0; off < h.payload; off += buf.size()) {
    const size_t n = (size_t)std::min<uint64_t>(buf.size(), h.payload - off);
    if (std::fread(buf.data(), 1, n, f) != n) return bad(PS_ERR_INVALID_ARG, "checkpoint: truncated payload");
    if ((e = cudaMemcpy(static_cast<char*>(uhat) + off, buf.data(), n, cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_bad(e, "host to device");
  }
  if (t) *t = h.t;
  if (step) *step = h.step;
  return PS_OK;
}

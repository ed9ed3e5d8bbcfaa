// Allocation-free right-hand side: ps_rhs_noalloc (include/ps.h).
//
// Some callers cannot allocate device memory: a host program that has handed
// the whole device to its own pool allocator, a callback or plugin that must
// keep the process's memory footprint fixed, or code that cannot afford the
// device-wide synchronisation that cudaMalloc/cudaFree can imply.  For them
// this entry point runs the same right-hand-side kernels as ps_rhs, but all of
// its scratch (intermediate fields, twiddle tables, forcing box) lives in the
// file-scope device array below, whose size is fixed at build time.  The
// paper has no counterpart of this entry point.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <string>

#include "ps.h"
#include "ps_fft.cuh"
#include "ps_kernels.h"

namespace ps {
void set_last_error(const std::string& msg);
}

using namespace ps;

namespace {

// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PS_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch on the current device.  In host code the
// symbol is only a host-side stand-in, so the address is looked up with the
// device current.  The lookup is repeated on every call (it is cheap), so an
// address never outlives the context it belongs to (after cudaDeviceReset the
// next call finds the array of the new context).
cudaError_t scratch_address(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
}

// exp(-2 pi i m/n), m < n, for the three axes, from the FP64 sincospi.
template <typename V>
__global__ void k_twiddles(V* tw, int nx, int ny, int nz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int total = nx + ny + nz;
  if (i >= total) return;
  int m, n;
  if (i < nx) {
    m = i;
    n = nx;
  } else if (i < nx + ny) {
    m = i - nx;
    n = ny;
  } else {
    m = i - nx - ny;
    n = nz;
  }
  double s, c;
  sincospi(2.0 * m / n, &s, &c);
  V v;
  v.x = (decltype(v.x))c;
  v.y = (decltype(v.x))(-s);
  tw[i] = v;
}

size_t up256(size_t b) { return (b + 255) / 256 * 256; }

int halfwidth(int n, ps_dealias d) { return d == PS_DEALIAS_NONE ? n / 2 - 1 : (n + 2) / 3 - 1; }

// Supported line lengths: powers of two from 8 to 1024, and 48, 96, 192.
bool pow2_in_range(int n) {
  return (n >= 8 && n <= 1024 && (n & (n - 1)) == 0) || n == 48 || n == 96 || n == 192;
}

ps_status bad(ps_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

ps_status cuda_bad(cudaError_t e, const char* where) {
  set_last_error(std::string("ps_rhs_noalloc: ") + where + ": " + cudaGetErrorString(e));
  return PS_ERR_CUDA;
}

template <typename T>
ps_status run(const ps_config* c, cudaStream_t s, const void* uhat, void* out) {
  using V = typename cplx<T>::type;
  Geo g{};
  g.nx = c->nx;
  g.ny = c->ny;
  g.nz = c->nz;
  g.nh = c->nx / 2 + 1;
  g.Kx = halfwidth(c->nx, c->dealias);
  g.Ky = halfwidth(c->ny, c->dealias);
  g.Kz = halfwidth(c->nz, c->dealias);
  g.cx = g.Kx + 1;
  g.cy = 2 * g.Ky + 1;
  g.cz = 2 * g.Kz + 1;
  g.kxp = (g.cx + 15) / 16 * 16;
  g.sphere = c->dealias == PS_DEALIAS_SPHERICAL ? 1 : 0;
  set_scales(g, c->lx, c->ly, c->lz);

  const size_t vb = sizeof(V), kxp = g.kxp;
  const size_t a1 = 6ull * g.nz * g.cy * kxp, a2 = 3ull * g.nz * g.ny * kxp;
  const size_t b1 = 6ull * g.nz * g.ny * kxp, b2 = 3ull * g.nz * g.cy * kxp;
  const size_t a_b = up256((a1 > a2 ? a1 : a2) * vb);
  const size_t b_b = up256((b1 > b2 ? b1 : b2) * vb);
  const size_t tw_b = up256((size_t)(g.nx + g.ny + g.nz) * vb);
  const size_t box_b = c->forcing ? up256(3ull * g.cz * g.cy * g.cx * vb) : 0;
  const size_t err_b = 256;  // error word of the x pass's bounded waits, cleared by every call
  const size_t need = a_b + b_b + tw_b + box_b + err_b;
  if (need > (size_t)PS_NOALLOC_SCRATCH_BYTES) {
    char msg[256];
    std::snprintf(msg, sizeof msg,
                  "ps_rhs_noalloc: a %dx%dx%d grid needs %zu bytes of scratch, more than the %zu-byte "
                  "static array; use ps_plan_create/ps_rhs",
                  c->nx, c->ny, c->nz, need, (size_t)PS_NOALLOC_SCRATCH_BYTES);
    return bad(PS_ERR_INVALID_ARG, msg);
  }
  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return cuda_bad(e, "cudaGetSymbolAddress");
  char* p = static_cast<char*>(base);

  PassArgs a{};
  a.g = g;
  a.a6 = p;
  a.b6 = p + a_b;
  V* tw = reinterpret_cast<V*>(p + a_b + b_b);
  a.tw_x = tw;
  a.tw_y = tw + g.nx;
  a.tw_z = tw + g.nx + g.ny;
  a.nu = c->nu;
  a.ng = 1;  // velocity only (HD)
  a.nsc = 0;
  a.nfi = 6;
  a.nfo = 3;
  a.err = reinterpret_cast<int*>(p + a_b + b_b + tw_b + box_b);
  a.Fx = a.Fy = a.Fz = -1;
  Spec in;
  in.p = uhat;
  in.ys = g.nh;
  in.zs = (long long)g.ny * g.nh;
  in.cs = (long long)g.nz * g.ny * g.nh;
  in.zwrap = g.nz;
  in.ywrap = g.ny;
  a.in = in;
  a.u_n = in;
  a.out_full = out;
  a.mode = ZF_RHS;

  // the previous call's error word: a wait that gave up then must not turn
  // this call's output into NaN (the update kernel reads the word)
  if ((e = cudaMemsetAsync(a.err, 0, sizeof(int), s)) != cudaSuccess) return cuda_bad(e, "error word");
  const int ntw = g.nx + g.ny + g.nz;
  k_twiddles<V><<<(ntw + 255) / 256, 256, 0, s>>>(tw, g.nx, g.ny, g.nz);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_bad(e, "twiddles");
  if (c->forcing) {
    // the whole retained cube as the forcing box: no extent query, no sync
    Spec f = in;
    f.p = c->forcing;
    void* box = p + a_b + b_b + tw_b;
    if ((e = launch_forcing_gather<T>(g, f, g.Kx, g.Ky, g.Kz, box, s)) != cudaSuccess) return cuda_bad(e, "forcing");
    a.fbox = box;
    a.Fx = g.Kx;
    a.Fy = g.Ky;
    a.Fz = g.Kz;
  }
  if ((e = launch_zinv<T>(a, s, nullptr)) != cudaSuccess) return cuda_bad(e, "z-inverse pass");
  if ((e = launch_yinv<T>(a, s)) != cudaSuccess) return cuda_bad(e, "y-inverse pass");
  if ((e = launch_xpass<T>(a, s)) != cudaSuccess) return cuda_bad(e, "x pass");
  if ((e = launch_yfwd<T>(a, s)) != cudaSuccess) return cuda_bad(e, "y-forward pass");
  if ((e = launch_zfwd<T>(a, s)) != cudaSuccess) return cuda_bad(e, "z-forward pass");
  if ((e = launch_update<T>(a, s)) != cudaSuccess) return cuda_bad(e, "update");
  return PS_OK;
}

}  // namespace

extern "C" ps_status ps_rhs_noalloc(const ps_config* cfg, void* cuda_stream, const void* uhat, void* rhs_out,
                                    double t) {
  (void)t;
  if (!cfg || !uhat || !rhs_out) return bad(PS_ERR_INVALID_ARG, "ps_rhs_noalloc: NULL config or buffer");
  if (!pow2_in_range(cfg->nx) || !pow2_in_range(cfg->ny) || !pow2_in_range(cfg->nz))
    return bad(PS_ERR_INVALID_ARG, "ps_rhs_noalloc: nx, ny, nz must be powers of two in [8, 1024] or 48, 96, 192");
  if (!(std::isfinite(cfg->lx) && std::isfinite(cfg->ly) && std::isfinite(cfg->lz) && cfg->lx > 0 &&
        cfg->ly > 0 && cfg->lz > 0))
    return bad(PS_ERR_INVALID_ARG, "ps_rhs_noalloc: box lengths must be finite and positive");
  if (cfg->prec != PS_FP32 && cfg->prec != PS_FP64) return bad(PS_ERR_INVALID_ARG, "ps_rhs_noalloc: precision");
  if (cfg->eq != PS_HD) return bad(cfg->eq == PS_MHD || cfg->eq == PS_BOUSSINESQ ? PS_ERR_UNSUPPORTED : PS_ERR_INVALID_ARG,
                                   "ps_rhs_noalloc: only the HD equations are implemented");
  if (cfg->dealias != PS_DEALIAS_CUBIC && cfg->dealias != PS_DEALIAS_SPHERICAL && cfg->dealias != PS_DEALIAS_NONE)
    return bad(PS_ERR_INVALID_ARG, "ps_rhs_noalloc: unknown dealias rule");
  if (!(std::isfinite(cfg->nu) && cfg->nu >= 0)) return bad(PS_ERR_INVALID_ARG, "ps_rhs_noalloc: nu");
  const size_t bytes = 3ull * cfg->nz * cfg->ny * (cfg->nx / 2 + 1) * (cfg->prec == PS_FP32 ? 8 : 16);
  const size_t vb = cfg->prec == PS_FP32 ? 8 : 16;
  if (reinterpret_cast<uintptr_t>(uhat) % vb || reinterpret_cast<uintptr_t>(rhs_out) % vb ||
      (cfg->forcing && reinterpret_cast<uintptr_t>(cfg->forcing) % vb))
    return bad(PS_ERR_INVALID_ARG, "ps_rhs_noalloc: buffers must be aligned to the complex element size");
  const char* x = static_cast<const char*>(uhat);
  const char* y = static_cast<const char*>(rhs_out);
  if (x < y + bytes && y < x + bytes) return bad(PS_ERR_INVALID_ARG, "ps_rhs_noalloc: rhs_out overlaps uhat");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  return cfg->prec == PS_FP32 ? run<float>(cfg, s, uhat, rhs_out) : run<double>(cfg, s, uhat, rhs_out);
}

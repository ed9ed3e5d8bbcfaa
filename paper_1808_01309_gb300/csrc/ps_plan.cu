// Plan layer and C ABI (include/ps.h): validation, scratch ownership, twiddle
// tables, forcing box, and the launch sequence of one right-hand side and of
// one integrating-factor Runge-Kutta step.
#include <algorithm>
#include <cmath>
#include <new>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "ps.h"
#include "ps_kernels.h"

using namespace ps;

namespace {

thread_local std::string g_last_error;

ps_status fail(ps_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

ps_status cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? PS_ERR_OOM : PS_ERR_CUDA;
}

#define PS_CU(call, where)                      \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

// Supported line lengths: powers of two from 8 to 1024, and 48, 96, 192.
bool pow2_in_range(int n) {
  return (n >= 8 && n <= 1024 && (n & (n - 1)) == 0) || n == 48 || n == 96 || n == 192;
}

int halfwidth(int n, ps_dealias d) {
  if (d == PS_DEALIAS_NONE) return n / 2 - 1;
  return (n + 2) / 3 - 1;  // largest integer strictly below n/3
}

ps_status validate(const ps_config* c) {
  if (!c) return fail(PS_ERR_INVALID_ARG, "config is NULL");
  if (!pow2_in_range(c->nx) || !pow2_in_range(c->ny) || !pow2_in_range(c->nz))
    return fail(PS_ERR_INVALID_ARG, "nx, ny, nz must be powers of two in [8, 1024] or 48, 96, 192");
  if (!(std::isfinite(c->lx) && std::isfinite(c->ly) && std::isfinite(c->lz) && c->lx > 0 && c->ly > 0 && c->lz > 0))
    return fail(PS_ERR_INVALID_ARG, "box lengths must be finite and positive");
  if (c->prec != PS_FP32 && c->prec != PS_FP64) return fail(PS_ERR_INVALID_ARG, "unknown precision");
  if (c->eq != PS_HD && c->eq != PS_MHD && c->eq != PS_BOUSSINESQ)
    return fail(PS_ERR_INVALID_ARG, "unknown equation set");
  if (c->eq == PS_MHD && !(std::isfinite(c->eta) && c->eta >= 0))
    return fail(PS_ERR_INVALID_ARG, "eta must be finite and >= 0");
  if (c->eq == PS_BOUSSINESQ && !(std::isfinite(c->kappa) && c->kappa >= 0 && std::isfinite(c->n_bv)))
    return fail(PS_ERR_INVALID_ARG, "kappa must be finite and >= 0, n_bv finite");
  if (c->dealias != PS_DEALIAS_CUBIC && c->dealias != PS_DEALIAS_SPHERICAL && c->dealias != PS_DEALIAS_NONE)
    return fail(PS_ERR_INVALID_ARG, "unknown dealias rule");
  if (c->rk_order != 2 && c->rk_order != 4) return fail(PS_ERR_INVALID_ARG, "rk_order must be 2 or 4");
  if (c->forcing && reinterpret_cast<uintptr_t>(c->forcing) % (c->prec == PS_FP32 ? 8 : 16))
    return fail(PS_ERR_INVALID_ARG, "the forcing buffer must be aligned to the complex element size");
  if (!(std::isfinite(c->nu) && c->nu >= 0)) return fail(PS_ERR_INVALID_ARG, "nu must be finite and >= 0");
  return PS_OK;
}

Geo make_geo(const ps_config* c) {
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
  return g;
}

struct Sizes {
  size_t vb;       // bytes per complex element
  size_t a6, b6;   // intermediate buffers (elements)
  size_t cmp;      // compact 3-field buffer (elements)
  size_t state;    // caller-layout field (elements)
};

// Field counts of an equation set: ng 3-component groups with a curl (HD: u;
// MHD: u, B), nsc scalars (Boussinesq: theta), ncomp state components, nfi
// fields into the x pass (u, omega, (B, j,) (grad theta)) and nfo out of it
// (u x omega (+ j x B), (u x B), (u . grad theta)).
struct Counts {
  int ng, nsc, ncomp, nfi, nfo;
};
Counts counts_of(const ps_config* c) {
  if (c->eq == PS_MHD) return {2, 0, 6, 12, 6};
  if (c->eq == PS_BOUSSINESQ) return {1, 1, 4, 9, 4};
  return {1, 0, 3, 6, 3};
}

Sizes sizes(const Geo& g, ps_precision p, const Counts& n) {
  Sizes s{};
  s.vb = p == PS_FP32 ? 8 : 16;
  const size_t kxp = g.kxp;
  // a6: z-inverse out [nfi][nz][cy], x-pass out [nfo][nz][ny], z-forward out [nfo][cz][cy]
  const size_t a1 = (size_t)n.nfi * g.nz * g.cy * kxp, a2 = (size_t)n.nfo * g.nz * g.ny * kxp;
  // b6: y-inverse out [nfi][nz][ny], y-forward out [nfo][nz][cy]
  const size_t b1 = (size_t)n.nfi * g.nz * g.ny * kxp, b2 = (size_t)n.nfo * g.nz * g.cy * kxp;
  s.a6 = a1 > a2 ? a1 : a2;
  s.b6 = b1 > b2 ? b1 : b2;
  s.cmp = (size_t)n.ncomp * g.cz * g.cy * kxp;
  s.state = (size_t)n.ncomp * g.nz * g.ny * g.nh;
  return s;
}

int nshells_of(const Geo& g) {
  const double kx = g.Kx * g.sx, ky = g.Ky * g.sy, kz = g.Kz * g.sz;
  return (int)std::floor(std::sqrt(kx * kx + ky * ky + kz * kz) + 0.5) + 1;
}

struct TimedLaunch {
  int kind;
  cudaEvent_t a, b;
};

}  // namespace

namespace ps {
// Lets other translation units of the library report through ps_last_error().
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace ps

struct ps_plan {
  ps_config cfg{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int xrpc = 0;  // x-pass rows per CTA override (0 = automatic)
  int shape[3] = {0, 0, 0};  // shape variants of the z-inverse, y and z-forward passes
  int n_epart_run = 0;       // energy partials written by the last z-inverse launch
  unsigned wait_test_polls = 0;  // ps_plan_set_wait_test: 0 = off
  // learned LES closure (ps_plan_set_closure)
  bool les_on = false;
  ps::LesScratch les{};
  void* les_mem[9] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int ng = 1;    // 3-component groups: 1 HD and Boussinesq, 2 MHD
  Counts cn{1, 0, 3, 6, 3};
  Geo g{};
  Sizes sz{};
  void* a6 = nullptr;
  void* b6 = nullptr;
  void* nxt = nullptr;
  void* acc = nullptr;
  void* tw = nullptr;         // [nx | ny | nz] twiddles
  void* iftab = nullptr;      // [cx | cy | cz] integrating factors
  double if_dt = NAN;
  void* fbox = nullptr;
  int Fx = -1, Fy = -1, Fz = -1;
  double* e_part = nullptr;
  int n_epart = 0;
  double* stats = nullptr;                 // [energy]
  unsigned long long* umax2 = nullptr;     // max |u|^2 bits
  int* ext = nullptr;
  int* err = nullptr;                      // device error word of bounded waits
  int nshells = 0;
  double* dpart = nullptr;                 // diagnostics partials
  double* dout = nullptr;                  // diagnostics result (device)
  void* hstate = nullptr;                  // device state for ps_rk_step_host
  int host_mode = PS_HOST_AUTO;            // ps_plan_set_host_mode
  // ps_rk_steps: captured graph of nsteps steps, keyed by (state, dt, nsteps)
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const void* g_u = nullptr;
  double g_dt = NAN;
  int g_n = 0;
  long long g_launches = 0;
  cudaStream_t side = nullptr;             // zero fill of the host state's masked modes
  cudaEvent_t side_go = nullptr, side_done = nullptr;
  void* zbuf = nullptr;                    // zeros, ZBUF_BYTES
  double time = 0.0;
  long long launches = 0;
  bool timing = false;
  std::vector<TimedLaunch> tl;
  std::vector<cudaEvent_t> pool;
  double ms_acc[PS_NKINDS] = {0};
  long long n_acc[PS_NKINDS] = {0};
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

cudaEvent_t take_event(ps_plan* p) {
  if (!p->pool.empty()) {
    cudaEvent_t e = p->pool.back();
    p->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Wraps one kernel launch: counts it and, with timing on, brackets it with
// events on the plan stream.
template <class F>
ps_status launch(ps_plan* p, int kind, F&& f, const char* what) {
  TimedLaunch t{kind, nullptr, nullptr};
  if (p->timing) {
    t.a = take_event(p);
    t.b = take_event(p);
    cudaEventRecord(t.a, p->stream);
  }
  cudaError_t e = f();
  if (e != cudaSuccess) return cuda_fail(e, what);
  if (p->timing) {
    cudaEventRecord(t.b, p->stream);
    p->tl.push_back(t);
  }
  p->launches++;
  return PS_OK;
}

ps_status collect_timing(ps_plan* p) {
  if (p->tl.empty()) return PS_OK;
  PS_CU(cudaStreamSynchronize(p->stream), "timing sync");
  for (auto& t : p->tl) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t.a, t.b);
    p->ms_acc[t.kind] += ms;
    p->n_acc[t.kind] += 1;
    p->pool.push_back(t.a);
    p->pool.push_back(t.b);
  }
  p->tl.clear();
  return PS_OK;
}

Spec caller_spec(const Geo& g, const void* ptr) {
  Spec s;
  s.p = ptr;
  s.ys = g.nh;
  s.zs = (long long)g.ny * g.nh;
  s.cs = (long long)g.nz * g.ny * g.nh;
  s.zwrap = g.nz;
  s.ywrap = g.ny;
  return s;
}

Spec compact_spec(const Geo& g, const void* ptr) {
  Spec s;
  s.p = ptr;
  s.ys = g.kxp;
  s.zs = (long long)g.cy * g.kxp;
  s.cs = (long long)g.cz * g.cy * g.kxp;
  s.zwrap = g.cz;
  s.ywrap = g.cy;
  return s;
}

PassArgs base_args(ps_plan* p) {
  PassArgs a{};
  a.g = p->g;
  a.a6 = p->a6;
  a.b6 = p->b6;
  const size_t vb = p->sz.vb;
  a.tw_x = p->tw;
  a.tw_y = static_cast<char*>(p->tw) + vb * p->g.nx;
  a.tw_z = static_cast<char*>(p->tw) + vb * (p->g.nx + p->g.ny);
  a.nu = p->cfg.nu;
  a.fbox = p->fbox;
  a.Fx = p->Fx;
  a.Fy = p->Fy;
  a.Fz = p->Fz;
  const size_t tb = p->cfg.prec == PS_FP32 ? 4 : 8;
  a.ifx = p->iftab;
  a.ify = static_cast<char*>(p->iftab) + tb * p->g.cx;
  a.ifz = static_cast<char*>(p->iftab) + tb * (p->g.cx + p->g.cy);
  const size_t half = tb * (p->g.cx + p->g.cy + p->g.cz);
  a.jfx = static_cast<char*>(p->iftab) + half;
  a.jfy = static_cast<char*>(p->iftab) + half + tb * p->g.cx;
  a.jfz = static_cast<char*>(p->iftab) + half + tb * (p->g.cx + p->g.cy);
  a.ng = p->ng;
  a.nsc = p->cn.nsc;
  a.nfi = p->cn.nfi;
  a.nfo = p->cn.nfo;
  a.n_bv = p->cfg.eq == PS_BOUSSINESQ ? p->cfg.n_bv : 0.0;
  a.eta = p->cfg.eq == PS_BOUSSINESQ ? p->cfg.kappa : p->cfg.eta;
  a.nxt = p->nxt;
  a.acc = p->acc;
  a.err = p->err;
  a.xrpc = p->xrpc;
  for (int k = 0; k < 3; ++k) a.shape[k] = p->shape[k];
  a.wait_test = p->wait_test_polls ? 1 : 0;
  a.wait_polls = p->wait_test_polls;
  return a;
}

// Reads the device error word (after a stream synchronisation).
ps_status check_device_error(ps_plan* p) {
  int e = 0;
  PS_CU(cudaMemcpyAsync(&e, p->err, sizeof(int), cudaMemcpyDeviceToHost, p->stream), "error word");
  PS_CU(cudaStreamSynchronize(p->stream), "error word");
  if (e != 0) {
    // reported once: the word is cleared so that the plan's next calls start clean
    PS_CU(cudaMemsetAsync(p->err, 0, sizeof(int), p->stream), "error word");
    PS_CU(cudaStreamSynchronize(p->stream), "error word");
    return fail(PS_ERR_TIMEOUT, "a bounded device wait gave up (asynchronous copy never completed)");
  }
  return PS_OK;
}

template <typename T>
ps_status run_inverse_and_x(ps_plan* p, PassArgs& a) {
  ps_status s;
  int nb = 0;
  if ((s = launch(p, 0, [&] { return launch_zinv<T>(a, p->stream, &nb); }, "z-inverse pass")) != PS_OK) return s;
  p->n_epart_run = nb;
  if ((s = launch(p, 1, [&] { return launch_yinv<T>(a, p->stream); }, "y-inverse pass")) != PS_OK) return s;
  if ((s = launch(p, 2, [&] { return launch_xpass<T>(a, p->stream); }, "x pass")) != PS_OK) return s;
  return PS_OK;
}

// One evaluation of D P(N + f) followed by the selected output of the update
// kernel (right-hand side or RK stage update).
template <typename T>
ps_status run_rhs_passes(ps_plan* p, PassArgs& a) {
  ps_status s;
  if ((s = run_inverse_and_x<T>(p, a)) != PS_OK) return s;
  if (a.e_part) {
    if ((s = launch(p, 5, [&] { return launch_sum_partials(p->e_part, p->n_epart_run, p->stats, p->stream); },
                    "energy reduction")) != PS_OK)
      return s;
  }
  if ((s = launch(p, 3, [&] { return launch_yfwd<T>(a, p->stream); }, "y-forward pass")) != PS_OK) return s;
  if (p->les_on) {
    // closure term of the stage input, added by the z-forward pass
    if ((s = launch(p, 5, [&] { return les_closure_term(p->g, a.in, a.tw_x, a.tw_y, a.tw_z, p->les, p->stream); },
                    "LES closure")) != PS_OK)
      return s;
    p->launches += 10;  // the closure is 11 kernels
    a.extra = p->les.extra;
  }
  if ((s = launch(p, 4, [&] { return launch_zfwd<T>(a, p->stream); }, "z-forward pass")) != PS_OK) return s;
  if ((s = launch(p, 6, [&] { return launch_update<T>(a, p->stream); }, "update")) != PS_OK) return s;
  return PS_OK;
}

template <typename T>
ps_status do_rhs(ps_plan* p, const void* uhat, void* out) {
  PassArgs a = base_args(p);
  a.in = caller_spec(p->g, uhat);
  a.u_n = a.in;
  a.out_full = out;
  a.mode = ZF_RHS;
  return run_rhs_passes<T>(p, a);
}

// Arguments of RK stage st of one step on the caller's state uhat: stage 0
// reads the state, later stages the compact stage input; with stats stage 0
// also writes the energy partials and max |u|^2 of the step statistics.
PassArgs stage_args(ps_plan* p, void* uhat, double dt, int st, bool stats) {
  const int nst = p->cfg.rk_order == 4 ? 4 : 2;
  PassArgs a = base_args(p);
  a.in = st == 0 ? caller_spec(p->g, uhat) : compact_spec(p->g, p->nxt);
  a.u_n = caller_spec(p->g, uhat);
  a.out_full = uhat;
  a.dt = dt;
  a.e_part = st == 0 && stats ? p->e_part : nullptr;
  a.umax2 = st == 0 && stats ? p->umax2 : nullptr;
  a.mode = nst == 4 ? ZF_RK4_1 + st : ZF_RK2_1 + st;
  return a;
}

template <typename T>
ps_status do_rk_step(ps_plan* p, void* uhat, double dt) {
  ps_status s;
  if (!(p->if_dt == dt)) {
    if ((s = launch(p, 5, [&] { return launch_if_tables<T>(p->g, p->cfg.nu, dt, p->iftab, p->stream); },
                    "integrating-factor tables")) != PS_OK)
      return s;
    if (p->ng == 2 || p->cn.nsc) {
      void* jt = static_cast<char*>(p->iftab) + sizeof(T) * (p->g.cx + p->g.cy + p->g.cz);
      const double d2 = p->cfg.eq == PS_BOUSSINESQ ? p->cfg.kappa : p->cfg.eta;
      if ((s = launch(p, 5, [&] { return launch_if_tables<T>(p->g, d2, dt, jt, p->stream); },
                      "integrating-factor tables")) != PS_OK)
        return s;
    }
    p->if_dt = dt;
  }
  PS_CU(cudaMemsetAsync(p->umax2, 0, sizeof(unsigned long long), p->stream), "reset max|u|");
  const int nst = p->cfg.rk_order == 4 ? 4 : 2;
  for (int st = 0; st < nst; ++st) {
    PassArgs a = stage_args(p, uhat, dt, st, true);
    if ((s = run_rhs_passes<T>(p, a)) != PS_OK) return s;
  }
  return PS_OK;
}

template <typename T>
ps_status do_diag(ps_plan* p, const void* uhat, double* host_out) {
  ps_status s;
  const int w = DIAG_HEAD + p->nshells;
  PS_CU(cudaMemsetAsync(p->dpart, 0, sizeof(double) * (size_t)p->g.cz * w, p->stream), "diag reset");
  PS_CU(cudaMemsetAsync(p->umax2, 0, sizeof(unsigned long long), p->stream), "diag reset");
  const Spec u = caller_spec(p->g, uhat);
  if ((s = launch(p, 5, [&] { return launch_diag_spectral<T>(p->g, u, p->dpart, p->nshells, (int)p->cfg.eq, p->stream); },
                  "spectral diagnostics")) != PS_OK)
    return s;
  if ((s = launch(p, 5, [&] { return launch_diag_final(p->dpart, p->g.cz, p->nshells, p->dout, p->stream); },
                  "diagnostics reduction")) != PS_OK)
    return s;
  PassArgs a = base_args(p);
  a.in = u;
  a.umax2 = p->umax2;
  a.xdiag = 1;
  if ((s = run_inverse_and_x<T>(p, a)) != PS_OK) return s;
  PS_CU(cudaMemcpyAsync(host_out, p->dout, sizeof(double) * w, cudaMemcpyDeviceToHost, p->stream), "diag copy");
  unsigned long long bits = 0;
  PS_CU(cudaMemcpyAsync(&bits, p->umax2, sizeof(bits), cudaMemcpyDeviceToHost, p->stream), "diag copy");
  PS_CU(cudaStreamSynchronize(p->stream), "diag sync");
  double m2;
  std::memcpy(&m2, &bits, sizeof(m2));
  host_out[w] = std::sqrt(m2);
  return PS_OK;
}

// Device fields must start on a multiple of their complex element size (the
// passes copy whole elements, 16 bytes at a time in FP64).
bool misaligned(const void* ptr, size_t vb) { return (reinterpret_cast<uintptr_t>(ptr) % vb) != 0; }

bool ranges_overlap(const void* a, const void* b, size_t n) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + n && y < x + n;
}

// Twiddles exp(-2 pi i m/n), m < n, evaluated in long double and rounded.
template <typename V>
void fill_twiddles(std::vector<V>& out, int n) {
  const long double two_pi = 6.283185307179586476925286766559L;
  for (int m = 0; m < n; ++m) {
    const long double ang = two_pi * (long double)m / (long double)n;
    V v;
    v.x = (decltype(v.x))std::cos(ang);
    v.y = (decltype(v.x))(-std::sin(ang));
    out.push_back(v);
  }
}

template <typename V>
ps_status upload_twiddles(ps_plan* p) {
  std::vector<V> h;
  fill_twiddles(h, p->g.nx);
  fill_twiddles(h, p->g.ny);
  fill_twiddles(h, p->g.nz);
  PS_CU(cudaMemcpy(p->tw, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice), "twiddle upload");
  return PS_OK;
}

template <typename T>
ps_status setup_forcing(ps_plan* p) {
  const Spec f = caller_spec(p->g, p->cfg.forcing);
  PS_CU(cudaMemsetAsync(p->ext, 0xff, 3 * sizeof(int), p->stream), "forcing extent");
  PS_CU(launch_forcing_extent<T>(p->g, f, p->ext, p->stream), "forcing extent");
  int ext[3];
  PS_CU(cudaMemcpyAsync(ext, p->ext, sizeof(ext), cudaMemcpyDeviceToHost, p->stream), "forcing extent");
  PS_CU(cudaStreamSynchronize(p->stream), "forcing extent");
  if (ext[0] < 0) return PS_OK;  // no retained forcing mode
  p->Fx = ext[0];
  p->Fy = ext[1];
  p->Fz = ext[2];
  const size_t n = 3ull * (p->Fx + 1) * (2 * p->Fy + 1) * (2 * p->Fz + 1);
  PS_CU(cudaMalloc(&p->fbox, n * p->sz.vb), "forcing box");
  PS_CU(launch_forcing_gather<T>(p->g, f, p->Fx, p->Fy, p->Fz, p->fbox, p->stream), "forcing gather");
  PS_CU(cudaStreamSynchronize(p->stream), "forcing gather");
  return PS_OK;
}

// Forget the graph ps_rk_steps captured: the launch sequence or its
// arguments change with the closure, the wait test hook and the x-pass rows.
void drop_cached_graph(ps_plan* p) {
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->gexec = nullptr;
  p->graph = nullptr;
  p->g_n = 0;
}

void release(ps_plan* p) {
  void* bufs[] = {p->a6, p->b6, p->nxt, p->acc, p->tw, p->iftab, p->fbox, p->e_part, p->stats,
                  p->umax2, p->ext, p->err, p->dpart, p->dout, p->hstate, p->les_mem[0], p->les_mem[1],
                  p->les_mem[2], p->les_mem[3], p->les_mem[4], p->les_mem[5], p->les_mem[6], p->les_mem[7],
                  p->les_mem[8]};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (auto& t : p->tl) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (auto e : p->pool) cudaEventDestroy(e);
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->cap) cudaStreamDestroy(p->cap);
  if (p->zbuf) cudaFree(p->zbuf);
  if (p->side_go) cudaEventDestroy(p->side_go);
  if (p->side_done) cudaEventDestroy(p->side_done);
  if (p->side) cudaStreamDestroy(p->side);
}

}  // namespace

namespace ps {
void plan_set_stream(ps_plan* p, cudaStream_t s) { p->stream = s; }
cudaStream_t plan_stream(const ps_plan* p) { return p->stream; }
void plan_set_xrpc(ps_plan* p, int rpc) {
  if (p->xrpc != rpc) drop_cached_graph(p);
  p->xrpc = rpc;
}
void plan_invalidate_tables(ps_plan* p) { p->if_dt = NAN; }
bool plan_set_shape(ps_plan* p, int k, int var) {
  if (k < 0 || k > 2) return false;
  const int n = k == 1 ? p->g.ny : p->g.nz;
  int c = 0, e = 0;
  const bool ok = p->cfg.prec == PS_FP32 ? pass_shape<float>(k, n, var, &c, &e) : pass_shape<double>(k, n, var, &c, &e);
  if (!ok) return false;
  if (p->shape[k] != var) drop_cached_graph(p);
  p->shape[k] = var;
  return true;
}
int plan_shape(const ps_plan* p, int k) { return (k >= 0 && k < 3) ? p->shape[k] : 0; }
int plan_check_error(ps_plan* p) { return (int)check_device_error(p); }
void plan_set_time(ps_plan* p, double t) { p->time = t; }
PlanView plan_view(const ps_plan* p) {
  PlanView v{};
  v.g = p->g;
  v.prec = (int)p->cfg.prec;
  v.eq = (int)p->cfg.eq;
  v.rk_stages = p->cfg.rk_order == 4 ? 4 : 2;
  v.closure = p->les_on;
  v.e_part = p->e_part;
  v.n_epart = p->n_epart;
  v.stats = p->stats;
  v.umax2 = p->umax2;
  return v;
}
PassArgs plan_stage_args(ps_plan* p, void* uhat, double dt, int st, bool stats) {
  PassArgs a = stage_args(p, uhat, dt, st, stats);
  prepare_args(a);
  return a;
}
int plan_if_tables(ps_plan* p, double dt) {
  const bool f32 = p->cfg.prec == PS_FP32;
  const size_t tb = f32 ? 4 : 8;
  ps_status s = launch(p, 5, [&] {
    return f32 ? launch_if_tables<float>(p->g, p->cfg.nu, dt, p->iftab, p->stream)
               : launch_if_tables<double>(p->g, p->cfg.nu, dt, p->iftab, p->stream);
  }, "integrating-factor tables");
  if (s != PS_OK) return s;
  if (p->ng == 2 || p->cn.nsc) {
    void* jt = static_cast<char*>(p->iftab) + tb * (p->g.cx + p->g.cy + p->g.cz);
    const double d2 = p->cfg.eq == PS_BOUSSINESQ ? p->cfg.kappa : p->cfg.eta;
    s = launch(p, 5, [&] {
      return f32 ? launch_if_tables<float>(p->g, d2, dt, jt, p->stream) : launch_if_tables<double>(p->g, d2, dt, jt, p->stream);
    }, "integrating-factor tables");
    if (s != PS_OK) return s;
  }
  p->if_dt = dt;
  return PS_OK;
}
// used by the checkpoint layer (ps_io.cu)
ps_config plan_config(const ps_plan* p) { return p->cfg; }
size_t plan_state_bytes(const ps_plan* p) { return p->sz.state * p->sz.vb; }
}  // namespace ps

extern "C" {

const char* ps_status_string(ps_status s) {
  switch (s) {
    case PS_OK: return "ok";
    case PS_ERR_INVALID_ARG: return "invalid argument";
    case PS_ERR_UNSUPPORTED: return "unsupported";
    case PS_ERR_OOM: return "out of device memory";
    case PS_ERR_CUDA: return "CUDA error";
    case PS_ERR_NONFINITE: return "non-finite result";
    case PS_ERR_TIMEOUT: return "timeout";
  }
  return "unknown status";
}

const char* ps_last_error(void) { return g_last_error.c_str(); }

const char* ps_kind_name(int kind) {
  static const char* names[PS_NKINDS] = {"z_inverse", "y_inverse", "x_fused", "y_forward",
                                         "z_forward", "aux", "update"};
  return (kind >= 0 && kind < PS_NKINDS) ? names[kind] : "?";
}

ps_status ps_plan_workspace_bytes(const ps_config* cfg, size_t* bytes) {
  ps_status s = validate(cfg);
  if (s != PS_OK) return s;
  if (!bytes) return fail(PS_ERR_INVALID_ARG, "bytes is NULL");
  const Geo g = make_geo(cfg);
  const Sizes z = sizes(g, cfg->prec, counts_of(cfg));
  const size_t tb = cfg->prec == PS_FP32 ? 4 : 8;
  *bytes = z.vb * (z.a6 + z.b6 + 2 * z.cmp + (size_t)(g.nx + g.ny + g.nz)) + 2 * tb * (g.cx + g.cy + g.cz) +
           sizeof(double) * (size_t)(g.cz * (g.kxp + DIAG_HEAD + nshells_of(g)) + 16);
  return PS_OK;
}

ps_status ps_plan_create(const ps_config* cfg, void* cuda_stream, ps_plan** out) {
  if (!out) return fail(PS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  ps_status s = validate(cfg);
  if (s != PS_OK) return s;
  ps_plan* p = new (std::nothrow) ps_plan();
  if (!p) return fail(PS_ERR_OOM, "host allocation failed");
  p->cfg = *cfg;
  p->stream = static_cast<cudaStream_t>(cuda_stream);
  p->g = make_geo(cfg);
  p->cn = counts_of(cfg);
  p->ng = p->cn.ng;
  p->sz = sizes(p->g, cfg->prec, p->cn);
  p->nshells = nshells_of(p->g);
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "cudaGetDevice");
  }
  auto bail = [&](ps_status st) {
    release(p);
    delete p;
    return st;
  };
  const size_t vb = p->sz.vb, tb = cfg->prec == PS_FP32 ? 4 : 8;
#define ALLOC(ptr, bytes, what)                          \
  do {                                                   \
    cudaError_t e_ = cudaMalloc((void**)&(ptr), (bytes)); \
    if (e_ != cudaSuccess) return bail(cuda_fail(e_, what)); \
  } while (0)
  ALLOC(p->a6, p->sz.a6 * vb, "scratch a");
  ALLOC(p->b6, p->sz.b6 * vb, "scratch b");
  ALLOC(p->nxt, p->sz.cmp * vb, "stage input");
  ALLOC(p->acc, p->sz.cmp * vb, "stage accumulator");
  ALLOC(p->tw, vb * (size_t)(p->g.nx + p->g.ny + p->g.nz), "twiddles");
  ALLOC(p->iftab, 2 * tb * (size_t)(p->g.cx + p->g.cy + p->g.cz), "integrating factors");
  const bool f32 = cfg->prec == PS_FP32;
  p->n_epart = f32 ? zinv_blocks<float>(p->g, 0) : zinv_blocks<double>(p->g, 0);
  p->n_epart_run = p->n_epart;
  // room for the partials of every shape variant of the z-inverse pass
  const int nb = f32 ? zinv_blocks<float>(p->g, -1) : zinv_blocks<double>(p->g, -1);
  ALLOC(p->e_part, sizeof(double) * (size_t)(nb > 0 ? nb : 1), "energy partials");
  ALLOC(p->stats, sizeof(double) * 4, "stats");
  ALLOC(p->umax2, sizeof(unsigned long long), "max|u|");
  ALLOC(p->ext, sizeof(int) * 4, "forcing extent");
  ALLOC(p->err, sizeof(int), "error word");
  ALLOC(p->dpart, sizeof(double) * (size_t)p->g.cz * (DIAG_HEAD + p->nshells), "diagnostic partials");
  ALLOC(p->dout, sizeof(double) * (size_t)(DIAG_HEAD + p->nshells), "diagnostics");
#undef ALLOC
  // Clean scratch once so that padding columns never hold uninitialised bits.
  e = cudaMemsetAsync(p->a6, 0, p->sz.a6 * vb, p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->b6, 0, p->sz.b6 * vb, p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->nxt, 0, p->sz.cmp * vb, p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->acc, 0, p->sz.cmp * vb, p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->stats, 0, sizeof(double) * 4, p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->umax2, 0, sizeof(unsigned long long), p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->err, 0, sizeof(int), p->stream);
  if (e != cudaSuccess) return bail(cuda_fail(e, "scratch clear"));
  s = cfg->prec == PS_FP32 ? upload_twiddles<float2>(p) : upload_twiddles<double2>(p);
  if (s != PS_OK) return bail(s);
  if (cfg->forcing) {
    s = cfg->prec == PS_FP32 ? setup_forcing<float>(p) : setup_forcing<double>(p);
    if (s != PS_OK) return bail(s);
  }
  e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return bail(cuda_fail(e, "plan create sync"));
  *out = p;
  return PS_OK;
}

ps_status ps_plan_destroy(ps_plan* p) {
  if (!p) return PS_OK;
  DeviceGuard dg(p->device);
  cudaStreamSynchronize(p->stream);
  release(p);
  delete p;
  return PS_OK;
}

ps_status ps_rhs(ps_plan* p, const void* uhat, void* rhs_out, double t) {
  (void)t;
  if (!p || !uhat || !rhs_out) return fail(PS_ERR_INVALID_ARG, "NULL plan or buffer");
  if (misaligned(uhat, p->sz.vb) || misaligned(rhs_out, p->sz.vb))
    return fail(PS_ERR_INVALID_ARG, "uhat and rhs_out must be aligned to the complex element size");
  if (ranges_overlap(uhat, rhs_out, p->sz.state * p->sz.vb))
    return fail(PS_ERR_INVALID_ARG, "rhs_out overlaps uhat");
  DeviceGuard dg(p->device);
  return p->cfg.prec == PS_FP32 ? do_rhs<float>(p, uhat, rhs_out) : do_rhs<double>(p, uhat, rhs_out);
}

ps_status ps_rk_step(ps_plan* p, void* uhat, double dt, double t) {
  if (!p || !uhat) return fail(PS_ERR_INVALID_ARG, "NULL plan or state");
  if (misaligned(uhat, p->sz.vb)) return fail(PS_ERR_INVALID_ARG, "uhat must be aligned to the complex element size");
  if (!std::isfinite(dt) || !std::isfinite(t)) return fail(PS_ERR_INVALID_ARG, "dt and t must be finite");
  DeviceGuard dg(p->device);
  ps_status s = p->cfg.prec == PS_FP32 ? do_rk_step<float>(p, uhat, dt) : do_rk_step<double>(p, uhat, dt);
  if (s == PS_OK) p->time = t + dt;
  return s;
}

ps_status ps_plan_set_host_mode(ps_plan* p, int mode) {
  if (!p) return fail(PS_ERR_INVALID_ARG, "NULL plan");
  if (mode < PS_HOST_AUTO || mode > PS_HOST_CUBE_CE)
    return fail(PS_ERR_INVALID_ARG, "unknown host mode");
  p->host_mode = mode;
  return PS_OK;
}

namespace {

constexpr size_t ZBUF_BYTES = 32ull << 20;

// Zeros into the modes of the page-locked host state outside the retained
// cube, by copy-engine transfers from a zero buffer on the side stream:
// the planes |r| > Kz, in the other planes the rows |q| > Ky, and in the
// remaining rows the entries kx > Kx.
cudaError_t zero_outside_cube(ps_plan* p, char* host) {
  const ps::Geo& g = p->g;
  const size_t vb = p->sz.vb, row = (size_t)g.nh * vb, plane = (size_t)g.ny * row;
  const size_t fcs = (size_t)g.nz * plane;
  const int nc = p->cn.ncomp;
  cudaStream_t st = p->side;
  const cudaMemcpyKind k = cudaMemcpyDeviceToHost;
  cudaError_t e = cudaSuccess;
  const int zr0 = g.Kz + 1, nzr = g.nz - 2 * g.Kz - 1;  // masked planes
  const int yr0 = g.Ky + 1, nyr = g.ny - 2 * g.Ky - 1;  // masked rows
  const size_t xw = (size_t)(g.nh - g.cx) * vb;          // masked tail of a row
  const int zlo[2] = {0, g.nz - g.Kz}, zn[2] = {g.Kz + 1, g.Kz};
  const int ylo[2] = {0, g.ny - g.Ky}, yn[2] = {g.Ky + 1, g.Ky};
  for (int c = 0; c < nc && e == cudaSuccess; ++c) {
    char* base = host + c * fcs;
    // whole planes
    for (size_t off = 0, n = (size_t)nzr * plane; off < n && e == cudaSuccess; off += ZBUF_BYTES)
      e = cudaMemcpyAsync(base + zr0 * plane + off, p->zbuf, std::min(ZBUF_BYTES, n - off), k, st);
    for (int a = 0; a < 2 && e == cudaSuccess; ++a) {
      if (zn[a] <= 0) continue;
      // whole rows of the retained planes
      if (nyr > 0) {
        const size_t w = (size_t)nyr * row;
        const int hc = (int)std::max<size_t>(1, ZBUF_BYTES / w);
        for (int h0 = 0; h0 < zn[a] && e == cudaSuccess; h0 += hc)
          e = cudaMemcpy2DAsync(base + (size_t)(zlo[a] + h0) * plane + yr0 * row, plane, p->zbuf, w, w,
                                std::min(hc, zn[a] - h0), k, st);
      }
      // row tails of the retained rows
      for (int b = 0; b < 2 && e == cudaSuccess && xw > 0; ++b) {
        if (yn[b] <= 0) continue;
        const int dc = (int)std::max<size_t>(1, ZBUF_BYTES / (xw * yn[b]));
        for (int d0 = 0; d0 < zn[a] && e == cudaSuccess; d0 += dc) {
          cudaMemcpy3DParms m{};
          m.srcPtr = make_cudaPitchedPtr(p->zbuf, xw, xw, yn[b]);
          m.dstPtr = make_cudaPitchedPtr(base + (size_t)(zlo[a] + d0) * plane + (size_t)ylo[b] * row + g.cx * vb,
                                         row, row, g.ny);
          m.extent = make_cudaExtent(xw, yn[b], std::min(dc, zn[a] - d0));
          m.kind = k;
          e = cudaMemcpy3DAsync(&m, st);
        }
      }
    }
  }
  return e;
}

// The same zeros written by host threads: every (component, kz) plane of the
// host state is one task; a masked plane is cleared whole, a retained plane
// in its masked rows (one contiguous block) and in the tails kx > Kx of its
// retained rows.  Nothing crosses the host link.
void zero_outside_cube_host(const ps_plan* p, char* host) {
  const ps::Geo& g = p->g;
  const size_t vb = p->sz.vb, row = (size_t)g.nh * vb, plane = (size_t)g.ny * row;
  const int nc = p->cn.ncomp;
  const long long nplanes = (long long)nc * g.nz;
  auto work = [&](long long first, long long last) {
    for (long long i = first; i < last; ++i) {
      const int c = (int)(i / g.nz), z = (int)(i % g.nz);
      char* base = host + (size_t)c * g.nz * plane + (size_t)z * plane;
      const int r = z < (g.nz + 1) / 2 ? z : z - g.nz;
      if (r > g.Kz || r < -g.Kz) {
        std::memset(base, 0, plane);
        continue;
      }
      const int yr0 = g.Ky + 1, nyr = g.ny - 2 * g.Ky - 1;
      if (nyr > 0) std::memset(base + (size_t)yr0 * row, 0, (size_t)nyr * row);
      const size_t tail = (size_t)(g.nh - g.cx) * vb;
      if (tail == 0) continue;
      for (int y = 0; y < g.ny; ++y) {
        const int q = y < (g.ny + 1) / 2 ? y : y - g.ny;
        if (q > g.Ky || q < -g.Ky) continue;
        std::memset(base + (size_t)y * row + (size_t)g.cx * vb, 0, tail);
      }
    }
  };
  unsigned nt = std::thread::hardware_concurrency();
  nt = nt < 1 ? 1 : nt > 16 ? 16 : nt;
  std::vector<std::thread> pool;
  const long long per = (nplanes + nt - 1) / nt;
  for (unsigned t = 1; t < nt; ++t) {
    const long long a = t * per, b = std::min<long long>(nplanes, a + per);
    if (a < b) pool.emplace_back(work, a, b);
  }
  work(0, std::min<long long>(nplanes, per));
  for (auto& th : pool) th.join();
}

}  // namespace

ps_status ps_rk_steps(ps_plan* p, void* uhat, double dt, double t, int nsteps) {
  if (!p || !uhat) return fail(PS_ERR_INVALID_ARG, "NULL plan or state");
  if (misaligned(uhat, p->sz.vb)) return fail(PS_ERR_INVALID_ARG, "uhat must be aligned to the complex element size");
  if (nsteps < 0) return fail(PS_ERR_INVALID_ARG, "nsteps must be >= 0");
  if (!std::isfinite(dt) || !std::isfinite(t)) return fail(PS_ERR_INVALID_ARG, "dt and t must be finite");
  if (nsteps == 0) return PS_OK;
  DeviceGuard dg(p->device);
  if (p->timing) {  // per-kernel events: plain launches
    for (int i = 0; i < nsteps; ++i) {
      ps_status s = ps_rk_step(p, uhat, dt, t + i * dt);
      if (s != PS_OK) return s;
    }
    return PS_OK;
  }
  if (!(p->gexec && p->g_u == uhat && p->g_dt == dt && p->g_n == nsteps)) {
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->gexec = nullptr;
    p->graph = nullptr;
    if (!p->cap) PS_CU(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking), "capture stream");
    cudaStream_t home = p->stream;
    const long long l0 = p->launches;
    // work already queued on the plan stream comes first
    cudaEvent_t ready = nullptr;
    PS_CU(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming), "capture event");
    cudaEventRecord(ready, home);
    cudaStreamWaitEvent(p->cap, ready, 0);
    cudaEventDestroy(ready);
    PS_CU(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    p->stream = p->cap;
    p->if_dt = NAN;  // the factor tables are part of the graph
    ps_status st = PS_OK;
    for (int i = 0; i < nsteps && st == PS_OK; ++i) st = ps_rk_step(p, uhat, dt, t + i * dt);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(p->cap, &g);
    p->stream = home;
    if (st != PS_OK) {
      if (g) cudaGraphDestroy(g);
      p->if_dt = NAN;
      return st;
    }
    PS_CU(ce, "end capture");
    p->graph = g;
    PS_CU(cudaGraphInstantiate(&p->gexec, g, 0), "graph instantiate");
    p->g_u = uhat;
    p->g_dt = dt;
    p->g_n = nsteps;
    p->g_launches = p->launches - l0;
    p->launches = l0;
  }
  PS_CU(cudaGraphLaunch(p->gexec, p->stream), "graph launch");
  p->launches += p->g_launches;
  p->time = t + nsteps * dt;
  return PS_OK;
}

ps_status ps_rk_step_host(ps_plan* p, void* uhat_host, double dt, double t, int nsteps) {
  if (!p || !uhat_host) return fail(PS_ERR_INVALID_ARG, "NULL plan or state");
  if (nsteps < 0) return fail(PS_ERR_INVALID_ARG, "nsteps must be >= 0");
  if (!std::isfinite(dt) || !std::isfinite(t)) return fail(PS_ERR_INVALID_ARG, "dt and t must be finite");
  if (nsteps == 0) return PS_OK;
  DeviceGuard dg(p->device);
  const size_t bytes = p->sz.state * p->sz.vb;
  // device address of a page-locked host buffer (NVLink-C2C on Grace systems)
  void* mapped = nullptr;
  if (p->host_mode != PS_HOST_COPY) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, uhat_host) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer)
      mapped = at.devicePointer;
    else
      (void)cudaGetLastError();  // clear the error of an unregistered pointer
    if (!mapped && p->host_mode != PS_HOST_AUTO)
      return fail(PS_ERR_UNSUPPORTED, "this host mode needs page-locked (registered or cudaHostAlloc) memory");
  }
  if (mapped && p->host_mode == PS_HOST_MAPPED) {
    for (int i = 0; i < nsteps; ++i) {
      ps_status s = ps_rk_step(p, mapped, dt, t + i * dt);
      if (s != PS_OK) return s;
    }
    PS_CU(cudaStreamSynchronize(p->stream), "host-path sync");
    return check_device_error(p);
  }
  if (!p->hstate) PS_CU(cudaMalloc(&p->hstate, bytes), "host-path state");
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
  const bool cube = mapped && (p->host_mode == PS_HOST_AUTO || p->host_mode == PS_HOST_CUBE_CE);
  const bool host_zero = cube && p->host_mode == PS_HOST_AUTO;
  if (host_zero) {
    // only the retained modes cross the host link; host threads write the
    // zeros of the masked modes while the GPU runs the steps
    PS_CU(ps::launch_copy_cube(mapped, p->hstate, p->g, p->cn.ncomp, p->sz.vb, nsm, p->stream), "state upload");
    p->launches++;
  } else if (cube) {
    // only the retained modes cross the host link; the masked modes of the
    // host state are zeroed by copy engines while the steps run
    if (!p->side) {
      PS_CU(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking), "side stream");
      PS_CU(cudaEventCreateWithFlags(&p->side_go, cudaEventDisableTiming), "side event");
      PS_CU(cudaEventCreateWithFlags(&p->side_done, cudaEventDisableTiming), "side event");
      PS_CU(cudaMalloc(&p->zbuf, ZBUF_BYTES), "zero buffer");
      PS_CU(cudaMemsetAsync(p->zbuf, 0, ZBUF_BYTES, p->stream), "zero buffer");
    }
    PS_CU(cudaEventRecord(p->side_go, p->stream), "side event");
    PS_CU(cudaStreamWaitEvent(p->side, p->side_go, 0), "side event");
    PS_CU(zero_outside_cube(p, static_cast<char*>(uhat_host)), "zero fill of the masked modes");
    PS_CU(cudaEventRecord(p->side_done, p->side), "side event");
    PS_CU(ps::launch_copy_cube(mapped, p->hstate, p->g, p->cn.ncomp, p->sz.vb, nsm, p->stream), "state upload");
    p->launches++;
  } else if (mapped) {
    PS_CU(ps::launch_stream_copy(mapped, p->hstate, bytes, nsm, p->stream), "state upload");
    p->launches++;
  } else {
    PS_CU(cudaMemcpyAsync(p->hstate, uhat_host, bytes, cudaMemcpyHostToDevice, p->stream), "state upload");
  }
  for (int i = 0; i < nsteps; ++i) {
    ps_status s = ps_rk_step(p, p->hstate, dt, t + i * dt);
    if (s != PS_OK) {
      if (cube && !host_zero) cudaStreamSynchronize(p->side);
      if (host_zero) cudaStreamSynchronize(p->stream);
      return s;
    }
  }
  if (cube) {
    PS_CU(ps::launch_copy_cube(p->hstate, mapped, p->g, p->cn.ncomp, p->sz.vb, nsm, p->stream), "state download");
    p->launches++;
    if (!host_zero) PS_CU(cudaStreamWaitEvent(p->stream, p->side_done, 0), "side event");
  } else if (mapped) {
    PS_CU(ps::launch_stream_copy(p->hstate, mapped, bytes, nsm, p->stream), "state download");
    p->launches++;
  } else {
    PS_CU(cudaMemcpyAsync(uhat_host, p->hstate, bytes, cudaMemcpyDeviceToHost, p->stream), "state download");
  }
  // the host threads' zeros touch only masked modes, the kernels only
  // retained ones: both run while the steps are queued on the GPU
  if (host_zero) zero_outside_cube_host(p, static_cast<char*>(uhat_host));
  PS_CU(cudaStreamSynchronize(p->stream), "host-path sync");
  return check_device_error(p);
}

ps_status ps_step_stats(ps_plan* p, double* energy, double* max_u) {
  if (!p) return fail(PS_ERR_INVALID_ARG, "NULL plan");
  DeviceGuard dg(p->device);
  double e = 0;
  unsigned long long bits = 0;
  PS_CU(cudaMemcpyAsync(&e, p->stats, sizeof(e), cudaMemcpyDeviceToHost, p->stream), "stats copy");
  PS_CU(cudaMemcpyAsync(&bits, p->umax2, sizeof(bits), cudaMemcpyDeviceToHost, p->stream), "stats copy");
  PS_CU(cudaStreamSynchronize(p->stream), "stats sync");
  double m2;
  std::memcpy(&m2, &bits, sizeof(m2));
  if (energy) *energy = e;
  if (max_u) *max_u = std::sqrt(m2);
  return check_device_error(p);
}

ps_status ps_diagnostics(ps_plan* p, const void* uhat, double cfl, ps_diag* out) {
  if (!p || !uhat || !out) return fail(PS_ERR_INVALID_ARG, "NULL plan, state or output");
  if (misaligned(uhat, p->sz.vb)) return fail(PS_ERR_INVALID_ARG, "uhat must be aligned to the complex element size");
  if (!std::isfinite(cfl)) return fail(PS_ERR_INVALID_ARG, "cfl must be finite");
  if (out->spectrum && out->nshells < 0) return fail(PS_ERR_INVALID_ARG, "negative spectrum capacity");
  DeviceGuard dg(p->device);
  std::vector<double> h(DIAG_HEAD + 1 + p->nshells);
  ps_status s = p->cfg.prec == PS_FP32 ? do_diag<float>(p, uhat, h.data()) : do_diag<double>(p, uhat, h.data());
  if (s != PS_OK) return s;
  if ((s = check_device_error(p)) != PS_OK) return s;
  out->energy = h[0];
  out->enstrophy = h[1];
  out->helicity = h[2];
  out->max_div = h[3];
  out->max_u = h[DIAG_HEAD + p->nshells];
  out->magnetic_energy = h[4];
  out->cross_helicity = h[5];
  out->magnetic_helicity = h[6];
  out->potential_energy = h[7];
  const double dmin = std::fmin(p->cfg.lx / p->cfg.nx, std::fmin(p->cfg.ly / p->cfg.ny, p->cfg.lz / p->cfg.nz));
  out->cfl_dt = out->max_u > 0 ? cfl * dmin / out->max_u : INFINITY;
  out->time = p->time;
  if (out->spectrum) {
    const int n = out->nshells < p->nshells ? out->nshells : p->nshells;
    for (int i = 0; i < n; ++i) out->spectrum[i] = h[DIAG_HEAD + i];
  }
  out->nshells = p->nshells;
  for (int i = 0; i < DIAG_HEAD + 1 + p->nshells; ++i)
    if (!std::isfinite(h[i])) return fail(PS_ERR_NONFINITE, "non-finite diagnostic");
  return PS_OK;
}

ps_status ps_plan_set_timing(ps_plan* p, int enable) {
  if (!p) return fail(PS_ERR_INVALID_ARG, "NULL plan");
  DeviceGuard dg(p->device);
  ps_status s = collect_timing(p);
  if (s != PS_OK) return s;
  for (int k = 0; k < PS_NKINDS; ++k) {
    p->ms_acc[k] = 0;
    p->n_acc[k] = 0;
  }
  p->timing = enable != 0;
  return PS_OK;
}

ps_status ps_plan_set_pass_shape(ps_plan* p, int pass, int variant, int* cols, int* points) {
  if (!p) return fail(PS_ERR_INVALID_ARG, "NULL plan");
  if (pass < 0 || pass > 2) return fail(PS_ERR_INVALID_ARG, "pass must be 0 (z-inverse), 1 (y passes) or 2 (z-forward)");
  if (variant < 0 || variant > 2) return fail(PS_ERR_INVALID_ARG, "variant must be 0, 1 or 2");
  const bool slab = p->g.kx0 != 0 || p->g.ncx != 0 || p->g.rowlen != 0;
  if (variant != 0 && (p->ng != 1 || p->cn.nsc || slab || !plan_set_shape(p, pass, variant)))
    return fail(PS_ERR_UNSUPPORTED, "no such shape variant for this plan (FP32 hydrodynamic plans with lines of "
                                    "64, 96 or 128 points; variant 2 not for 96)");
  if (variant == 0) plan_set_shape(p, pass, 0);
  const int n = pass == 1 ? p->g.ny : p->g.nz;
  int c = 0, e = 0;
  if (p->cfg.prec == PS_FP32) pass_shape<float>(pass, n, variant, &c, &e);
  else pass_shape<double>(pass, n, variant, &c, &e);
  if (cols) *cols = c;
  if (points) *points = e;
  return PS_OK;
}

ps_status ps_plan_set_wait_test(ps_plan* p, int polls) {
  if (!p) return fail(PS_ERR_INVALID_ARG, "NULL plan");
  if (polls < 0 || polls > (1 << 20)) return fail(PS_ERR_INVALID_ARG, "polls must be in [0, 2^20]");
  if (p->wait_test_polls != (unsigned)polls) drop_cached_graph(p);
  p->wait_test_polls = (unsigned)polls;
  return PS_OK;
}

ps_status ps_plan_get_timing(ps_plan* p, ps_timing* out) {
  if (!p || !out) return fail(PS_ERR_INVALID_ARG, "NULL plan or output");
  DeviceGuard dg(p->device);
  ps_status s = collect_timing(p);
  if (s != PS_OK) return s;
  for (int k = 0; k < PS_NKINDS; ++k) {
    out->ms[k] = p->ms_acc[k];
    out->launches[k] = p->n_acc[k];
  }
  return PS_OK;
}

ps_status ps_plan_set_closure(ps_plan* p, const float* params, const double* norm12) {
  if (!p) return fail(PS_ERR_INVALID_ARG, "NULL plan");
  if (!params) {
    if (p->les_on) drop_cached_graph(p);
    p->les_on = false;
    return PS_OK;
  }
  if (!norm12) return fail(PS_ERR_INVALID_ARG, "NULL normalisation");
  for (int i = 0; i < 12; ++i)
    if (!std::isfinite(norm12[i]) || (i >= 5 && !(norm12[i] > 0)))
      return fail(PS_ERR_INVALID_ARG, "normalisation: finite values, positive std, s_tau and s_A required");
  if (p->cfg.prec != PS_FP32 || p->cfg.eq != PS_HD || p->cfg.dealias == PS_DEALIAS_SPHERICAL)
    return fail(PS_ERR_UNSUPPORTED, "the LES closure needs an FP32 HD plan with the cubic or no truncation");
  const auto les_n = [](int n) { return n >= 16 && n <= 512 && (n % 16 == 0) && ((n & (n - 1)) == 0 || n % 48 == 0); };
  if (!les_n(p->g.nx) || !les_n(p->g.ny) || !les_n(p->g.nz))
    return fail(PS_ERR_UNSUPPORTED, "the LES closure supports grid sizes 16..512");
  DeviceGuard dg(p->device);
  const ps::Geo& g = p->g;
  const size_t P = (size_t)g.nx * g.ny * g.nz, M = (size_t)g.nz * g.ny * g.nh;
  if (!p->les_mem[0]) {
    const size_t sizes[7] = {sizeof(float) * PS_MLP_NPARAM, sizeof(float) * 16, sizeof(float2) * 9 * M,
                             sizeof(float) * 9 * P, sizeof(float) * 5 * P, sizeof(float) * 6 * P,
                             sizeof(float2) * p->sz.cmp};
    for (int i = 0; i < 7; ++i) PS_CU(cudaMalloc(&p->les_mem[i], sizes[i]), "closure scratch");
    PS_CU(cudaMemsetAsync(p->les_mem[6], 0, sizes[6], p->stream), "closure scratch");
  }
  float h[12];
  for (int i = 0; i < 5; ++i) {
    h[i] = (float)norm12[i];
    h[5 + i] = (float)(1.0 / norm12[5 + i]);
  }
  h[10] = (float)norm12[10];
  h[11] = (float)(1.0 / norm12[11]);
  PS_CU(cudaMemcpyAsync(p->les_mem[0], params, sizeof(float) * PS_MLP_NPARAM, cudaMemcpyDeviceToDevice, p->stream),
        "closure parameters");
  PS_CU(cudaMemcpyAsync(p->les_mem[1], h, sizeof(h), cudaMemcpyHostToDevice, p->stream), "closure scales");
  PS_CU(cudaStreamSynchronize(p->stream), "closure setup");
  p->les.params = static_cast<const float*>(p->les_mem[0]);
  p->les.norm = static_cast<const float*>(p->les_mem[1]);
  p->les.spec = static_cast<float2*>(p->les_mem[2]);
  p->les.phys = static_cast<float*>(p->les_mem[3]);
  p->les.X = static_cast<float*>(p->les_mem[4]);
  p->les.Y = static_cast<float*>(p->les_mem[5]);
  p->les.extra = static_cast<float2*>(p->les_mem[6]);
  if (!p->les_on) drop_cached_graph(p);  // the closure launches join the step
  p->les_on = true;
  return PS_OK;
}

ps_status ps_plan_closure_grad(ps_plan* p, const float* params, const void* ubar, const void* force, float* grad,
                               double* loss, int accumulate) {
  if (!p || !params || !ubar || !force || !grad || !loss) return fail(PS_ERR_INVALID_ARG, "NULL plan or buffer");
  if (!p->les_on) return fail(PS_ERR_INVALID_ARG, "no closure attached (ps_plan_set_closure)");
  DeviceGuard dg(p->device);
  const ps::Geo& g = p->g;
  const size_t P = (size_t)g.nx * g.ny * g.nz;
  if (!p->les_mem[7]) PS_CU(cudaMalloc(&p->les_mem[7], sizeof(float) * 9 * P), "closure training scratch");
  p->les.Arows = static_cast<float*>(p->les_mem[7]);
  if (!accumulate) {
    PS_CU(cudaMemsetAsync(grad, 0, sizeof(float) * PS_MLP_NPARAM, p->stream), "gradient reset");
    PS_CU(cudaMemsetAsync(loss, 0, sizeof(double), p->stream), "loss reset");
  }
  const cudaError_t e = ps::les_closure_grad(g, caller_spec(g, ubar), caller_spec(g, force), p->tw,
                                             static_cast<char*>(p->tw) + sizeof(float2) * g.nx,
                                             static_cast<char*>(p->tw) + sizeof(float2) * (g.nx + g.ny), p->les,
                                             params, grad, loss, p->stream);
  PS_CU(e, "closure gradient");
  return PS_OK;
}

ps_status ps_plan_closure_grad_transfer(ps_plan* p, const float* params, const void* ubar, const double* t_exact,
                                        int nshells, float* grad, double* loss, int accumulate) {
  if (!p || !params || !ubar || !t_exact || !grad || !loss) return fail(PS_ERR_INVALID_ARG, "NULL plan or buffer");
  if (nshells < 1 || nshells > 1024) return fail(PS_ERR_INVALID_ARG, "nshells must be in 1..1024");
  if (!p->les_on) return fail(PS_ERR_INVALID_ARG, "no closure attached (ps_plan_set_closure)");
  DeviceGuard dg(p->device);
  const ps::Geo& g = p->g;
  const size_t P = (size_t)g.nx * g.ny * g.nz;
  if (!p->les_mem[7]) PS_CU(cudaMalloc(&p->les_mem[7], sizeof(float) * 9 * P), "closure training scratch");
  if (!p->les_mem[8]) PS_CU(cudaMalloc(&p->les_mem[8], sizeof(double) * 3 * 1024), "closure transfer scratch");
  p->les.Arows = static_cast<float*>(p->les_mem[7]);
  double* te = static_cast<double*>(p->les_mem[8]);
  PS_CU(cudaMemcpyAsync(te, t_exact, sizeof(double) * nshells, cudaMemcpyHostToDevice, p->stream), "transfer target");
  if (!accumulate) {
    PS_CU(cudaMemsetAsync(grad, 0, sizeof(float) * PS_MLP_NPARAM, p->stream), "gradient reset");
    PS_CU(cudaMemsetAsync(loss, 0, sizeof(double), p->stream), "loss reset");
  }
  const ps::Spec u = caller_spec(g, ubar);
  const cudaError_t e = ps::les_closure_grad(g, u, u, p->tw, static_cast<char*>(p->tw) + sizeof(float2) * g.nx,
                                             static_cast<char*>(p->tw) + sizeof(float2) * (g.nx + g.ny), p->les,
                                             params, grad, loss, p->stream, te, nshells, te + 1024);
  PS_CU(e, "closure transfer gradient");
  // the host target may be released once the copy has run
  PS_CU(cudaStreamSynchronize(p->stream), "transfer target");
  return PS_OK;
}

ps_status ps_plan_launch_count(ps_plan* p, long long* launches) {
  if (!p || !launches) return fail(PS_ERR_INVALID_ARG, "NULL plan or output");
  *launches = p->launches;
  return PS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Slab decomposition (include/ps.h, ps_slab_*): the passes of one right-hand
// side on a rank's kx columns and z planes; the exchanges between them are
// the caller's (paper Sec. 2 and Sec. 3.3: one all-to-all per 3D transform).
// ---------------------------------------------------------------------------
struct ps_slab {
  ps_config cfg{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int kx_lo = 0, kx_hi = 0, z_lo = 0, z_hi = 0;
  Geo gl{};  // the local kx columns (all z, y)
  Geo gx{};  // the x rows of the local z planes (all kx)
  size_t vb = 8;
  void* a6 = nullptr;  // z-backward output [6][nz][cy][kxp]; z-forward output [3][cz][cy][kxp]
  void* b6 = nullptr;  // y-forward output [3][nz][cy][kxp]
  void* tw = nullptr;  // [nx | ny | nz] twiddles
  void* fbox = nullptr;
  int* err = nullptr;
};

namespace {

void slab_release(ps_slab* s) {
  void* bufs[] = {s->a6, s->b6, s->tw, s->fbox, s->err};
  for (void* b : bufs)
    if (b) cudaFree(b);
}

PassArgs slab_args(const ps_slab* s, const Geo& g) {
  PassArgs a{};
  a.g = g;
  a.tw_x = s->tw;
  a.tw_y = static_cast<char*>(s->tw) + s->vb * g.nx;
  a.tw_z = static_cast<char*>(s->tw) + s->vb * (g.nx + g.ny);
  a.nu = s->cfg.nu;
  a.ng = 1;
  a.nsc = 0;
  a.nfi = 6;
  a.nfo = 3;
  a.err = s->err;
  a.fbox = s->fbox;
  a.Fx = s->fbox ? g.ncx - 1 : -1;
  a.Fy = s->fbox ? g.Ky : -1;
  a.Fz = s->fbox ? g.Kz : -1;
  return a;
}

Spec local_spec(const Geo& g, const void* ptr) {
  Spec sp;
  sp.p = ptr;
  sp.ys = g.rowlen;
  sp.zs = (long long)g.ny * g.rowlen;
  sp.cs = (long long)g.nz * g.ny * g.rowlen;
  sp.zwrap = g.nz;
  sp.ywrap = g.ny;
  return sp;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" {

ps_status ps_slab_create(const ps_config* cfg, int kx_lo, int kx_hi, int z_lo, int z_hi, void* cuda_stream,
                         ps_slab** out) {
  if (!out) return fail(PS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  ps_status st = validate(cfg);
  if (st != PS_OK) return st;
  if (cfg->eq != PS_HD) return fail(PS_ERR_UNSUPPORTED, "slab decomposition: HD equations only");
  const Geo g = make_geo(cfg);
  if (!(0 <= kx_lo && kx_lo < kx_hi && kx_hi <= g.cx))
    return fail(PS_ERR_INVALID_ARG, "kx range must satisfy 0 <= kx_lo < kx_hi <= Kx + 1");
  if (!(0 <= z_lo && z_lo < z_hi && z_hi <= g.nz))
    return fail(PS_ERR_INVALID_ARG, "z range must satisfy 0 <= z_lo < z_hi <= nz");
  ps_slab* s = new (std::nothrow) ps_slab();
  if (!s) return fail(PS_ERR_OOM, "host allocation failed");
  s->cfg = *cfg;
  s->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaGetDevice(&s->device);
  s->kx_lo = kx_lo;
  s->kx_hi = kx_hi;
  s->z_lo = z_lo;
  s->z_hi = z_hi;
  s->vb = cfg->prec == PS_FP32 ? 8 : 16;
  s->gl = g;
  s->gl.kx0 = kx_lo;
  s->gl.ncx = kx_hi - kx_lo;
  s->gl.rowlen = kx_hi - kx_lo;
  s->gl.kxp = (s->gl.ncx + 15) / 16 * 16;
  s->gx = g;
  s->gx.nz = z_hi - z_lo;  // the x pass sees only the rows of the local planes
  const size_t kxp = s->gl.kxp;
  auto bail = [&](ps_status r) {
    slab_release(s);
    delete s;
    return r;
  };
  cudaError_t e;
  const size_t a6 = std::max(6ull * g.nz * g.cy * kxp, 3ull * g.cz * g.cy * kxp);
  if ((e = cudaMalloc(&s->a6, a6 * s->vb)) != cudaSuccess) return bail(cuda_fail(e, "slab scratch"));
  if ((e = cudaMalloc(&s->b6, 3ull * g.nz * g.cy * kxp * s->vb)) != cudaSuccess)
    return bail(cuda_fail(e, "slab scratch"));
  if ((e = cudaMalloc(&s->tw, (size_t)(g.nx + g.ny + g.nz) * s->vb)) != cudaSuccess)
    return bail(cuda_fail(e, "slab twiddles"));
  if ((e = cudaMalloc(&s->err, sizeof(int))) != cudaSuccess) return bail(cuda_fail(e, "slab error word"));
  if ((e = cudaMemsetAsync(s->err, 0, sizeof(int), s->stream)) != cudaSuccess)
    return bail(cuda_fail(e, "slab error word"));
  if (cfg->prec == PS_FP32) {
    std::vector<float2> h;
    fill_twiddles(h, g.nx);
    fill_twiddles(h, g.ny);
    fill_twiddles(h, g.nz);
    e = cudaMemcpy(s->tw, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice);
  } else {
    std::vector<double2> h;
    fill_twiddles(h, g.nx);
    fill_twiddles(h, g.ny);
    fill_twiddles(h, g.nz);
    e = cudaMemcpy(s->tw, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return bail(cuda_fail(e, "slab twiddle upload"));
  if (cfg->forcing) {
    // the whole local retained block as the forcing box
    const size_t n = 3ull * s->gl.ncx * g.cy * g.cz;
    if ((e = cudaMalloc(&s->fbox, n * s->vb)) != cudaSuccess) return bail(cuda_fail(e, "slab forcing box"));
    const Spec f = local_spec(s->gl, cfg->forcing);
    e = cfg->prec == PS_FP32 ? launch_forcing_gather<float>(s->gl, f, s->gl.ncx - 1, g.Ky, g.Kz, s->fbox, s->stream)
                             : launch_forcing_gather<double>(s->gl, f, s->gl.ncx - 1, g.Ky, g.Kz, s->fbox, s->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "slab forcing gather"));
  }
  if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return bail(cuda_fail(e, "slab create sync"));
  *out = s;
  return PS_OK;
}

ps_status ps_slab_destroy(ps_slab* s) {
  if (!s) return PS_OK;
  DeviceGuard dg(s->device);
  cudaStreamSynchronize(s->stream);
  slab_release(s);
  delete s;
  return PS_OK;
}

ps_status ps_slab_info_get(const ps_slab* s, ps_slab_info* out) {
  if (!s || !out) return fail(PS_ERR_INVALID_ARG, "NULL slab or output");
  out->ncx = s->gl.ncx;
  out->kxp = s->gl.kxp;
  out->cxp = s->gx.kxp;
  out->rows = s->gx.nz * s->gx.ny;
  return PS_OK;
}

ps_status ps_slab_inverse(ps_slab* s, const void* uhat_local, void* out6) {
  if (!s || !uhat_local || !out6) return fail(PS_ERR_INVALID_ARG, "NULL slab or buffer");
  if (!aligned16(uhat_local) || !aligned16(out6)) return fail(PS_ERR_INVALID_ARG, "slab buffers must be 16-byte aligned");
  DeviceGuard dg(s->device);
  PassArgs a = slab_args(s, s->gl);
  a.in = local_spec(s->gl, uhat_local);
  a.a6 = s->a6;
  a.b6 = out6;
  const bool f32 = s->cfg.prec == PS_FP32;
  PS_CU(f32 ? launch_zinv<float>(a, s->stream, nullptr) : launch_zinv<double>(a, s->stream, nullptr), "slab z-inverse");
  PS_CU(f32 ? launch_yinv<float>(a, s->stream) : launch_yinv<double>(a, s->stream), "slab y-inverse");
  return PS_OK;
}

ps_status ps_slab_xpass(ps_slab* s, const void* xin, void* xout) {
  if (!s || !xin || !xout) return fail(PS_ERR_INVALID_ARG, "NULL slab or buffer");
  if (!aligned16(xin) || !aligned16(xout)) return fail(PS_ERR_INVALID_ARG, "slab buffers must be 16-byte aligned");
  DeviceGuard dg(s->device);
  PassArgs a = slab_args(s, s->gx);
  a.b6 = const_cast<void*>(xin);
  a.a6 = xout;
  PS_CU(s->cfg.prec == PS_FP32 ? launch_xpass<float>(a, s->stream) : launch_xpass<double>(a, s->stream), "slab x pass");
  return PS_OK;
}

ps_status ps_slab_forward(ps_slab* s, const void* yin, const void* uhat_local, void* rhs_local) {
  if (!s || !yin || !uhat_local || !rhs_local) return fail(PS_ERR_INVALID_ARG, "NULL slab or buffer");
  if (!aligned16(yin) || !aligned16(uhat_local) || !aligned16(rhs_local))
    return fail(PS_ERR_INVALID_ARG, "slab buffers must be 16-byte aligned");
  const size_t bytes = 3ull * s->gl.nz * s->gl.ny * s->gl.rowlen * s->vb;
  if (ranges_overlap(uhat_local, rhs_local, bytes)) return fail(PS_ERR_INVALID_ARG, "rhs_local overlaps uhat_local");
  DeviceGuard dg(s->device);
  const bool f32 = s->cfg.prec == PS_FP32;
  PassArgs a = slab_args(s, s->gl);
  a.a6 = const_cast<void*>(yin);
  a.b6 = s->b6;
  PS_CU(f32 ? launch_yfwd<float>(a, s->stream) : launch_yfwd<double>(a, s->stream), "slab y-forward");
  a.a6 = s->a6;
  PS_CU(f32 ? launch_zfwd<float>(a, s->stream) : launch_zfwd<double>(a, s->stream), "slab z-forward");
  a.in = local_spec(s->gl, uhat_local);
  a.u_n = a.in;
  a.out_full = rhs_local;
  a.mode = ZF_RHS;
  PS_CU(f32 ? launch_update<float>(a, s->stream) : launch_update<double>(a, s->stream), "slab update");
  return PS_OK;
}

ps_status ps_slab_check(ps_slab* s) {
  if (!s) return fail(PS_ERR_INVALID_ARG, "NULL slab");
  DeviceGuard dg(s->device);
  int e = 0;
  PS_CU(cudaMemcpyAsync(&e, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->stream), "slab error word");
  PS_CU(cudaStreamSynchronize(s->stream), "slab sync");
  if (e != 0) {
    PS_CU(cudaMemsetAsync(s->err, 0, sizeof(int), s->stream), "slab error word");
    PS_CU(cudaStreamSynchronize(s->stream), "slab sync");
    return fail(PS_ERR_TIMEOUT, "a bounded device wait gave up (asynchronous copy never completed)");
  }
  return PS_OK;
}

}  // extern "C"

// Ensemble of independent solves of uneven sizes (include/ps.h,
// ps_ensemble_*): one plan per member, stepped either member after member on
// one stream, or as a single CUDA graph in which the members' launch chains
// are independent branches that the GPU runs concurrently.  A small autotuner
// picks the number of concurrent branches and, per grid size, the x-pass row
// group (rows per CTA) by timing the candidates.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ps.h"
#include "ps_kernels.h"

namespace ps {
void set_last_error(const std::string& msg);
}

using namespace ps;

struct ps_ensemble {
  std::vector<ps_plan*> plans;
  std::vector<ps_config> cfgs;
  cudaStream_t main = nullptr;  // the caller's stream (may be the legacy default stream)
  cudaStream_t cap = nullptr;   // internal stream graphs are captured on
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  int nbranch = 1;  // tuned
  // cached graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<void*> key_states;
  double key_dt = NAN, key_t = NAN;
  int key_steps = -1, key_branches = -1;
};

namespace {

ps_status bad(ps_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

ps_status cu(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return PS_OK;
  set_last_error(std::string("ensemble: ") + where + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? PS_ERR_OOM : PS_ERR_CUDA;
}

#define ENS_CU(call, where)                 \
  do {                                      \
    ps_status s_ = cu((call), where);       \
    if (s_ != PS_OK) return s_;             \
  } while (0)

size_t state_bytes(const ps_config& c) {
  const size_t nc = c.eq == PS_MHD ? 6 : c.eq == PS_BOUSSINESQ ? 4 : 3;
  return nc * c.nz * c.ny * (c.nx / 2 + 1) * (c.prec == PS_FP32 ? 8 : 16);
}

void drop_graph(ps_ensemble* e) {
  if (e->exec) cudaGraphExecDestroy(e->exec);
  if (e->graph) cudaGraphDestroy(e->graph);
  e->exec = nullptr;
  e->graph = nullptr;
  e->key_steps = -1;
}

// Sequential: every member's steps on the ensemble stream, member by member.
ps_status run_sequential(ps_ensemble* e, void* const* u, double dt, double t, int nsteps) {
  for (size_t i = 0; i < e->plans.size(); ++i) plan_set_stream(e->plans[i], e->main);
  for (int s = 0; s < nsteps; ++s)
    for (size_t i = 0; i < e->plans.size(); ++i) {
      ps_status st = ps_rk_step(e->plans[i], u[i], dt, t + s * dt);
      if (st != PS_OK) return st;
    }
  return PS_OK;
}

// Captures nsteps steps of every member into one graph; member i runs on
// branch i mod B, the branches fork from and join back into the capture
// stream (a private non-blocking stream: the legacy default stream cannot be
// captured).  The graph is then launched on the caller's stream.
ps_status capture(ps_ensemble* e, void* const* u, double dt, double t, int nsteps, int B) {
  drop_graph(e);
  ENS_CU(cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
  ps_status st = PS_OK;
  cudaError_t ce = cudaEventRecord(e->fork, e->cap);
  for (int b = 0; b < B && ce == cudaSuccess; ++b) ce = cudaStreamWaitEvent(e->branch[b], e->fork, 0);
  if (ce != cudaSuccess) st = cu(ce, "fork");
  for (size_t i = 0; i < e->plans.size() && st == PS_OK; ++i) {
    plan_set_stream(e->plans[i], e->branch[i % B]);
    plan_invalidate_tables(e->plans[i]);
  }
  for (int s = 0; s < nsteps && st == PS_OK; ++s)
    for (size_t i = 0; i < e->plans.size() && st == PS_OK; ++i) st = ps_rk_step(e->plans[i], u[i], dt, t + s * dt);
  for (int b = 0; b < B && st == PS_OK; ++b) {
    ce = cudaEventRecord(e->join[b], e->branch[b]);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(e->cap, e->join[b], 0);
    if (ce != cudaSuccess) st = cu(ce, "join");
  }
  cudaGraph_t g = nullptr;
  ce = cudaStreamEndCapture(e->cap, &g);
  if (st != PS_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  ENS_CU(ce, "end capture");
  e->graph = g;
  ENS_CU(cudaGraphInstantiate(&e->exec, g, 0), "instantiate");
  e->key_states.assign(u, u + e->plans.size());
  e->key_dt = dt;
  e->key_t = t;
  e->key_steps = nsteps;
  e->key_branches = B;
  return PS_OK;
}

ps_status run_graph(ps_ensemble* e, void* const* u, double dt, double t, int nsteps) {
  // t is not part of the key: the right-hand side does not depend on it
  const bool same = e->exec && e->key_steps == nsteps && e->key_dt == dt &&
                    e->key_branches == e->nbranch &&
                    std::equal(e->key_states.begin(), e->key_states.end(), u);
  if (!same) {
    ps_status st = capture(e, u, dt, t, nsteps, e->nbranch);
    if (st != PS_OK) return st;
  }
  ENS_CU(cudaGraphLaunch(e->exec, e->main), "graph launch");
  for (ps_plan* p : e->plans) plan_set_time(p, t + nsteps * dt);
  return PS_OK;
}

// Average milliseconds of `reps` calls of f on the main stream.
template <class F>
ps_status time_ms(ps_ensemble* e, int reps, F&& f, double* ms) {
  cudaEvent_t a, b;
  ENS_CU(cudaEventCreate(&a), "event");
  ENS_CU(cudaEventCreate(&b), "event");
  ps_status st = f();  // warm-up (captures a graph if needed)
  if (st == PS_OK) st = cu(cudaStreamSynchronize(e->main), "sync");
  if (st == PS_OK) st = cu(cudaEventRecord(a, e->main), "event");
  for (int i = 0; i < reps && st == PS_OK; ++i) st = f();
  if (st == PS_OK) st = cu(cudaEventRecord(b, e->main), "event");
  if (st == PS_OK) st = cu(cudaEventSynchronize(b), "event");
  float t = 0.f;
  if (st == PS_OK) st = cu(cudaEventElapsedTime(&t, a, b), "event");
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = t / reps;
  return st;
}

}  // namespace

extern "C" {

ps_status ps_ensemble_create(const ps_config* cfgs, int count, void* cuda_stream, ps_ensemble** out) {
  if (!out) return bad(PS_ERR_INVALID_ARG, "ensemble: out is NULL");
  *out = nullptr;
  if (!cfgs || count <= 0 || count > PS_ENS_MAX_MEMBERS)
    return bad(PS_ERR_INVALID_ARG, "ensemble: need 1..PS_ENS_MAX_MEMBERS member configs");
  ps_ensemble* e = new ps_ensemble();
  e->main = static_cast<cudaStream_t>(cuda_stream);
  auto fail = [&](ps_status s) {
    ps_ensemble_destroy(e);
    return s;
  };
  for (int i = 0; i < count; ++i) {
    ps_plan* p = nullptr;
    ps_status s = ps_plan_create(&cfgs[i], cuda_stream, &p);
    if (s != PS_OK) return fail(s);
    e->plans.push_back(p);
    e->cfgs.push_back(cfgs[i]);
  }
  const int nb = count;
  e->branch.resize(nb, nullptr);
  e->join.resize(nb, nullptr);
  for (int b = 0; b < nb; ++b) {
    ps_status s = cu(cudaStreamCreateWithFlags(&e->branch[b], cudaStreamNonBlocking), "branch stream");
    if (s == PS_OK) s = cu(cudaEventCreateWithFlags(&e->join[b], cudaEventDisableTiming), "event");
    if (s != PS_OK) return fail(s);
  }
  ps_status s = cu(cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming), "event");
  if (s == PS_OK) s = cu(cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking), "capture stream");
  if (s != PS_OK) return fail(s);
  e->nbranch = std::min(count, 16);
  *out = e;
  return PS_OK;
}

ps_status ps_ensemble_destroy(ps_ensemble* e) {
  if (!e) return PS_OK;
  cudaStreamSynchronize(e->main);
  drop_graph(e);
  for (auto p : e->plans) ps_plan_destroy(p);
  for (auto s : e->branch)
    if (s) cudaStreamDestroy(s);
  for (auto v : e->join)
    if (v) cudaEventDestroy(v);
  if (e->fork) cudaEventDestroy(e->fork);
  if (e->cap) cudaStreamDestroy(e->cap);
  delete e;
  return PS_OK;
}

ps_status ps_ensemble_rk_steps(ps_ensemble* e, void* const* uhats, double dt, double t, int nsteps,
                               ps_ens_mode mode) {
  if (!e || !uhats) return bad(PS_ERR_INVALID_ARG, "ensemble: NULL ensemble or states");
  if (nsteps < 0 || !std::isfinite(dt) || !std::isfinite(t))
    return bad(PS_ERR_INVALID_ARG, "ensemble: nsteps >= 0, finite dt and t required");
  for (size_t i = 0; i < e->plans.size(); ++i)
    if (!uhats[i]) return bad(PS_ERR_INVALID_ARG, "ensemble: NULL member state");
  if (nsteps == 0) return PS_OK;
  if (mode == PS_ENS_SEQUENTIAL) return run_sequential(e, uhats, dt, t, nsteps);
  if (mode == PS_ENS_GRAPH) return run_graph(e, uhats, dt, t, nsteps);
  return bad(PS_ERR_INVALID_ARG, "ensemble: unknown mode");
}

ps_status ps_ensemble_tune(ps_ensemble* e, const void* const* uhats, double dt, ps_ens_tuning* out) {
  if (!e || !uhats || !out) return bad(PS_ERR_INVALID_ARG, "ensemble: NULL argument");
  if (!std::isfinite(dt)) return bad(PS_ERR_INVALID_ARG, "ensemble: dt must be finite");
  const size_t m = e->plans.size();
  // scratch copies: tuning steps them, the caller's states are left untouched
  std::vector<void*> work(m, nullptr);
  ps_status st = PS_OK;
  for (size_t i = 0; i < m && st == PS_OK; ++i) {
    st = cu(cudaMalloc(&work[i], state_bytes(e->cfgs[i])), "tuning copy");
    if (st == PS_OK)
      st = cu(cudaMemcpyAsync(work[i], uhats[i], state_bytes(e->cfgs[i]), cudaMemcpyDeviceToDevice, e->main),
              "tuning copy");
  }
  *out = ps_ens_tuning{};
  // 1. x-pass rows per CTA, per distinct grid (timed on its first member)
  std::vector<int> done;
  for (size_t i = 0; i < m && st == PS_OK; ++i) {
    const ps_config& c = e->cfgs[i];
    bool seen = false;
    for (int j : done) {
      const ps_config& d = e->cfgs[j];
      seen |= d.nx == c.nx && d.ny == c.ny && d.nz == c.nz && d.prec == c.prec;
    }
    if (seen) continue;
    done.push_back((int)i);
    const int cand[] = {0, 16, 8, 4, 2, 1};
    double best = 1e30;
    int best_r = 0;
    plan_set_stream(e->plans[i], e->main);
    for (int r : cand) {
      plan_set_xrpc(e->plans[i], r);
      double ms = 0;
      st = time_ms(e, 3, [&] { return ps_rk_step(e->plans[i], work[i], dt, 0.0); }, &ms);
      if (st != PS_OK) break;
      if (ms < best * 0.98) {
        best = ms;
        best_r = r;
      }
    }
    for (size_t j = i; j < m; ++j) {
      const ps_config& d = e->cfgs[j];
      if (d.nx == c.nx && d.ny == c.ny && d.nz == c.nz && d.prec == c.prec) plan_set_xrpc(e->plans[j], best_r);
    }
    if (out->nsizes < PS_ENS_MAX_SIZES) {
      out->n[out->nsizes] = c.nx;
      out->xrpc[out->nsizes] = best_r;
      out->nsizes++;
    }
  }
  // 2. number of concurrent graph branches, timed on one step of all members
  if (st == PS_OK) {
    const int cand[] = {1, 2, 4, 8, 16, 24, 32, 48, 64};
    double best = 1e30;
    int best_b = 1;
    for (int b : cand) {
      if (b > (int)m) break;
      e->nbranch = b;
      double ms = 0;
      st = time_ms(e, 3, [&] { return run_graph(e, work.data(), dt, 0.0, 1); }, &ms);
      if (st != PS_OK) break;
      if (ms < best * 0.98) {
        best = ms;
        best_b = b;
      }
    }
    e->nbranch = best_b;
    out->branches = best_b;
    out->step_ms = best;
  }
  drop_graph(e);
  cudaStreamSynchronize(e->main);
  for (void* w : work)
    if (w) cudaFree(w);
  return st;
}

}  // extern "C"

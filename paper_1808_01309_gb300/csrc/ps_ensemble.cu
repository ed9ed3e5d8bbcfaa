// Ensemble of independent solves of uneven sizes (include/ps.h,
// ps_ensemble_*): one plan per member, stepped member after member on one
// stream, as a single CUDA graph in which the members' launch chains are
// independent branches that the GPU runs concurrently, or as one persistent
// kernel launch over a device work queue of (member, pass, tile) items
// (ps_persist.cuh), itself captured in a CUDA graph.  An autotuner times the
// graph's branch count and x-pass row groups, and the persistent launch's
// tiles per work item, CTAs per SM and member order, and picks the faster
// mode for PS_ENS_AUTO.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "ps.h"
#include "ps_kernels.h"
#include "ps_batch.cuh"
#include "ps_persist.cuh"
#include "ps_worklist.h"

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
  // persistent launch: work list, counters and its captured graph
  EnsPass* d_passes = nullptr;
  PassArgs* d_args = nullptr;
  unsigned* d_done = nullptr;
  unsigned long long* d_head = nullptr;
  int* d_err = nullptr;
  size_t cap_passes = 0, cap_args = 0;
  int npass = 0;
  long long tickets = 0;
  size_t smem = 0;
  int grid = 0;
  cudaGraph_t pgraph = nullptr;
  cudaGraphExec_t pexec = nullptr;
  std::vector<void*> pkey_states;
  double pkey_dt = NAN;
  int pkey_steps = -1;
  // persistent tuning knobs: tiles per ticket per pass kind, CTAs per SM
  // (0 = as many as fit), member order (0 = as created, 1 = largest first)
  int per[7] = {1, 2, 1, 2, 1, 8, 1};
  int ctas_per_sm = 0;
  int order = 0;
  unsigned wait_test = 0;  // > 0: test hook (one dependency never completes; polls limit)
  // batched mode: members of one grid size share each pass's launch
  struct BatchClass {
    std::vector<int> members;     // at most BATCH_MAX
    std::vector<PassArgs> args;   // [stage][member]
    double** d_sum = nullptr;     // stats word of each member
    int nst = 0;
  };
  std::vector<BatchClass> bclasses;
  int bsize = 4;  // members per batched launch (tuned): classes split into sub-batches
  cudaGraph_t bgraph = nullptr;
  cudaGraphExec_t bexec = nullptr;
  std::vector<void*> bkey_states;
  double bkey_dt = NAN;
  int bkey_steps = -1;
  ps_ens_mode auto_mode = PS_ENS_GRAPH;
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

void drop_pgraph(ps_ensemble* e) {
  if (e->pexec) cudaGraphExecDestroy(e->pexec);
  if (e->pgraph) cudaGraphDestroy(e->pgraph);
  e->pexec = nullptr;
  e->pgraph = nullptr;
  e->pkey_steps = -1;
}

// Why the members cannot share one persistent launch ("" if they can).
std::string persist_unsupported(const ps_ensemble* e) {
  auto ok_n = [](int n) { return n == 32 || n == 48 || n == 64 || n == 96 || n == 128; };
  for (size_t i = 0; i < e->plans.size(); ++i) {
    const PlanView v = plan_view(e->plans[i]);
    if (v.prec != plan_view(e->plans[0]).prec) return "members of both precisions";
    if (v.eq != PS_HD) return "only the hydrodynamic system";
    if (v.closure) return "a member has a learned closure attached";
    if (!ok_n(v.g.nx) || !ok_n(v.g.ny) || !ok_n(v.g.nz)) return "axis lengths outside {32, 48, 64, 96, 128}";
  }
  return "";
}

// Builds the work list of nsteps steps of every member on the states u and
// uploads it with the stage arguments.
ps_status persist_build(ps_ensemble* e, void* const* u, double dt, int nsteps) {
  const std::string why = persist_unsupported(e);
  if (!why.empty()) return bad(PS_ERR_UNSUPPORTED, "ensemble: persistent mode: " + why);
  const size_t m = e->plans.size();
  const bool f32 = plan_view(e->plans[0]).prec == PS_FP32;
  std::vector<PassArgs> args;
  std::vector<int> base(m), nst(m);
  for (size_t i = 0; i < m; ++i) {
    const PlanView v = plan_view(e->plans[i]);
    nst[i] = v.rk_stages;
    base[i] = (int)args.size();
    for (int st = 0; st < nst[i]; ++st) args.push_back(plan_stage_args(e->plans[i], u[i], dt, st, false));
    args.push_back(plan_stage_args(e->plans[i], u[i], dt, 0, true));  // stage 0 with the step statistics
  }
  if (!e->d_err) ENS_CU(cudaMalloc(&e->d_err, sizeof(int)), "error word");
  for (auto& a : args) a.err = e->d_err;
  // each member's pass sequence: per step and stage z-inverse, (energy sum,)
  // y-inverse, x, y-forward, z-forward, update
  std::vector<std::vector<EnsPass>> mp(m);  // without ticket and dependency
  std::vector<std::vector<WlItem>> seq(m);
  const int kinds[] = {EK_ZINV, EK_SUM, EK_YINV, EK_XPASS, EK_YFWD, EK_ZFWD, EK_UPDATE};
  size_t smem = 0;
  for (size_t i = 0; i < m; ++i) {
    const PlanView v = plan_view(e->plans[i]);
    const Geo& g = v.g;
    for (int s = 0; s < nsteps; ++s)
      for (int st = 0; st < nst[i]; ++st)
        for (int kind : kinds) {
          const bool stats = s == nsteps - 1 && st == 0;
          if (kind == EK_SUM && !stats) continue;
          EnsPass P{};
          P.args = base[i] + (stats ? nst[i] : st);
          P.kind = kind;
          P.per = e->per[kind] > 0 ? e->per[kind] : 1;
          EnsShape sh;
          if (kind == EK_UPDATE) {
            P.full = (st == nst[i] - 1) ? 1 : 0;
            const long long n = P.full ? (long long)g.nz * g.ny * g.nh : (long long)g.cz * g.cy * g.cx;
            sh.ntiles = (int)((n + ENS_UPDATE_MODES - 1) / ENS_UPDATE_MODES);
          } else if (kind == EK_SUM) {
            sh.ntiles = 1;
            sh.gx = v.n_epart;
            P.sum_out = v.stats;
            P.per = 1;
          } else {
            const int n = kind == EK_XPASS ? g.nx : (kind == EK_YINV || kind == EK_YFWD) ? g.ny : g.nz;
            const int nf = kind == EK_YINV ? 6 : 3;
            sh = f32 ? ens_shape<float>(kind, n, g, nf) : ens_shape<double>(kind, n, g, nf);
            P.n = n;
          }
          if (sh.ntiles <= 0) return bad(PS_ERR_UNSUPPORTED, "ensemble: persistent mode: no tiles for a pass");
          P.ntiles = sh.ntiles;
          P.gx = sh.gx;
          P.gy = sh.gy;
          smem = std::max(smem, sh.smem);
          mp[i].push_back(P);
          seq[i].push_back(WlItem{P.ntiles, P.per, kind != EK_SUM});
        }
  }
  // member order: as created, or largest grid first (orders 1 and 2); order 2
  // also staggers the members' sequences (ps_worklist.h)
  std::vector<int> ord(m);
  std::iota(ord.begin(), ord.end(), 0);
  if (e->order >= 1)
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
      const Geo ga = plan_view(e->plans[a]).g, gb = plan_view(e->plans[b]).g;
      return (long long)ga.nx * ga.ny * ga.nz > (long long)gb.nx * gb.ny * gb.nz;
    });
  std::vector<WlSlot> slots;
  const long long tick = wl_schedule(seq, ord, wl_skew(ord, e->order), &slots);
  std::vector<EnsPass> passes;
  passes.reserve(slots.size());
  for (const WlSlot& sl : slots) {
    EnsPass P = mp[sl.member][sl.item];
    P.tick0 = sl.tick0;
    P.dep = sl.dep;
    P.need = sl.need;
    passes.push_back(P);
  }
  if (e->wait_test) {
    // test hook: the first pass that waits for another waits for one tile too many
    for (auto& P : passes)
      if (P.dep >= 0) {
        P.need += 1;
        break;
      }
  }
  if (passes.size() > e->cap_passes) {
    if (e->d_passes) cudaFree(e->d_passes);
    if (e->d_done) cudaFree(e->d_done);
    e->d_passes = nullptr;
    e->d_done = nullptr;
    ENS_CU(cudaMalloc(&e->d_passes, passes.size() * sizeof(EnsPass)), "work list");
    ENS_CU(cudaMalloc(&e->d_done, passes.size() * sizeof(unsigned)), "work counters");
    e->cap_passes = passes.size();
  }
  if (args.size() > e->cap_args) {
    if (e->d_args) cudaFree(e->d_args);
    e->d_args = nullptr;
    ENS_CU(cudaMalloc(&e->d_args, args.size() * sizeof(PassArgs)), "stage arguments");
    e->cap_args = args.size();
  }
  if (!e->d_head) ENS_CU(cudaMalloc(&e->d_head, sizeof(unsigned long long)), "ticket counter");
  ENS_CU(cudaMemcpy(e->d_passes, passes.data(), passes.size() * sizeof(EnsPass), cudaMemcpyHostToDevice), "work list");
  ENS_CU(cudaMemcpy(e->d_args, args.data(), args.size() * sizeof(PassArgs), cudaMemcpyHostToDevice), "stage arguments");
  e->npass = (int)passes.size();
  e->tickets = tick;
  e->smem = smem;
  int dev = 0, nsm = 0, per_sm = 0;
  ENS_CU(cudaGetDevice(&dev), "device");
  ENS_CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "SM count");
  ENS_CU(f32 ? ens_blocks_per_sm_f32(smem, &per_sm) : ens_blocks_per_sm_f64(smem, &per_sm), "occupancy");
  if (per_sm < 1) return bad(PS_ERR_UNSUPPORTED, "ensemble: persistent kernel does not fit an SM");
  if (e->ctas_per_sm > 0) per_sm = std::min(per_sm, e->ctas_per_sm);
  e->grid = nsm * per_sm;
  return PS_OK;
}

// Captures, on the capture stream: the members' integrating-factor tables,
// the reset of the step-statistics maximum, of the work counters and of the
// error word, then the persistent launch.
ps_status persist_capture(ps_ensemble* e, void* const* u, double dt, int nsteps) {
  drop_pgraph(e);
  ps_status st = persist_build(e, u, dt, nsteps);
  if (st != PS_OK) return st;
  const bool f32 = plan_view(e->plans[0]).prec == PS_FP32;
  ENS_CU(cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaError_t ce = cudaSuccess;
  for (size_t i = 0; i < e->plans.size() && st == PS_OK; ++i) {
    plan_set_stream(e->plans[i], e->cap);
    st = (ps_status)plan_if_tables(e->plans[i], dt);
    if (st == PS_OK) {
      ce = cudaMemsetAsync(plan_view(e->plans[i]).umax2, 0, sizeof(unsigned long long), e->cap);
      if (ce != cudaSuccess) st = cu(ce, "reset max|u|");
    }
  }
  if (st == PS_OK) {
    ce = cudaMemsetAsync(e->d_done, 0, (size_t)e->npass * sizeof(unsigned), e->cap);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(e->d_head, 0, sizeof(unsigned long long), e->cap);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(e->d_err, 0, sizeof(int), e->cap);
    EnsLaunch L{e->d_passes, e->npass, e->d_args, e->d_done, e->d_head, e->tickets, e->d_err,
                e->wait_test ? e->wait_test : (1u << 24)};
    if (ce == cudaSuccess) ce = f32 ? ens_launch_f32(L, e->grid, e->smem, e->cap) : ens_launch_f64(L, e->grid, e->smem, e->cap);
    if (ce != cudaSuccess) st = cu(ce, "persistent launch");
  }
  cudaGraph_t g = nullptr;
  ce = cudaStreamEndCapture(e->cap, &g);
  if (st != PS_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  ENS_CU(ce, "end capture");
  e->pgraph = g;
  ENS_CU(cudaGraphInstantiate(&e->pexec, g, 0), "instantiate");
  e->pkey_states.assign(u, u + e->plans.size());
  e->pkey_dt = dt;
  e->pkey_steps = nsteps;
  return PS_OK;
}

ps_status run_persistent(ps_ensemble* e, void* const* u, double dt, double t, int nsteps) {
  const bool same = e->pexec && e->pkey_steps == nsteps && e->pkey_dt == dt &&
                    std::equal(e->pkey_states.begin(), e->pkey_states.end(), u);
  if (!same) {
    ps_status st = persist_capture(e, u, dt, nsteps);
    if (st != PS_OK) return st;
  }
  ENS_CU(cudaGraphLaunch(e->pexec, e->main), "graph launch");
  for (ps_plan* p : e->plans) plan_set_time(p, t + nsteps * dt);
  return PS_OK;
}

void drop_bgraph(ps_ensemble* e) {
  if (e->bexec) cudaGraphExecDestroy(e->bexec);
  if (e->bgraph) cudaGraphDestroy(e->bgraph);
  e->bexec = nullptr;
  e->bgraph = nullptr;
  e->bkey_steps = -1;
  for (auto& c : e->bclasses)
    if (c.d_sum) cudaFree(c.d_sum);
  e->bclasses.clear();
}

// Why the members cannot run batched ("" if they can): the batched passes
// cover the hydrodynamic system without a closure, lines of 32..128 points.
std::string batch_unsupported(const ps_ensemble* e) {
  auto ok_n = [](int n) { return n == 32 || n == 48 || n == 64 || n == 96 || n == 128; };
  for (size_t i = 0; i < e->plans.size(); ++i) {
    const PlanView v = plan_view(e->plans[i]);
    if (v.eq != PS_HD) return "only the hydrodynamic system";
    if (v.closure) return "a member has a learned closure attached";
    if (!ok_n(v.g.nx) || !ok_n(v.g.ny) || !ok_n(v.g.nz)) return "axis lengths outside {32, 48, 64, 96, 128}";
  }
  return "";
}

// Members that can share launches: same grid, box, precision, dealiasing and
// RK order (viscosity, forcing and state are per member).
bool same_class(const ps_config& a, const ps_config& b) {
  return a.nx == b.nx && a.ny == b.ny && a.nz == b.nz && a.lx == b.lx && a.ly == b.ly && a.lz == b.lz &&
         a.prec == b.prec && a.dealias == b.dealias && a.rk_order == b.rk_order;
}

// Captures nsteps steps of all members as batched launches: one graph branch
// per grid class; on it, per member the integrating-factor tables, then per
// step and RK stage one launch per pass for all members of the class.
ps_status batch_capture(ps_ensemble* e, void* const* u, double dt, int nsteps) {
  drop_bgraph(e);
  const std::string why = batch_unsupported(e);
  if (!why.empty()) return bad(PS_ERR_UNSUPPORTED, "ensemble: batched mode: " + why);
  const size_t m = e->plans.size();
  // class id of each member: the first member of the same class
  std::vector<int> cls(m);
  for (size_t i = 0; i < m; ++i) {
    cls[i] = (int)i;
    for (size_t j = 0; j < i; ++j)
      if (same_class(e->cfgs[j], e->cfgs[i])) {
        cls[i] = (int)j;
        break;
      }
  }
  for (const std::vector<int>& group : wl_batches(cls, std::min(e->bsize, BATCH_MAX))) {
    ps_ensemble::BatchClass c;
    c.members = group;
    c.nst = plan_view(e->plans[group[0]]).rk_stages;
    const int M = (int)c.members.size();
    c.args.resize((size_t)c.nst * M);
    std::vector<double*> sums(M);
    for (int st = 0; st < c.nst; ++st)
      for (int k = 0; k < M; ++k)
        c.args[(size_t)st * M + k] = plan_stage_args(e->plans[c.members[k]], u[c.members[k]], dt, st, true);
    for (int k = 0; k < M; ++k) sums[k] = plan_view(e->plans[c.members[k]]).stats;
    e->bclasses.push_back(c);  // owned by the ensemble from here (freed by drop_bgraph)
    auto& cc = e->bclasses.back();
    ENS_CU(cudaMalloc(&cc.d_sum, sums.size() * sizeof(double*)), "batched arguments");
    ENS_CU(cudaMemcpy(cc.d_sum, sums.data(), sums.size() * sizeof(double*), cudaMemcpyHostToDevice), "batched arguments");
  }
  const int B = (int)e->bclasses.size();
  if (B > (int)e->branch.size()) return bad(PS_ERR_UNSUPPORTED, "ensemble: too many grid classes");
  std::vector<BatchArgs> bav(1);  // the launches' parameter image (about 14 KB)
  ENS_CU(cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
  ps_status st = PS_OK;
  cudaError_t ce = cudaEventRecord(e->fork, e->cap);
  for (int b = 0; b < B && ce == cudaSuccess; ++b) ce = cudaStreamWaitEvent(e->branch[b], e->fork, 0);
  if (ce != cudaSuccess) st = cu(ce, "fork");
  for (int b = 0; b < B && st == PS_OK; ++b) {
    const auto& c = e->bclasses[b];
    cudaStream_t s = e->branch[b];
    const int M = (int)c.members.size();
    for (int k = 0; k < M && st == PS_OK; ++k) {
      plan_set_stream(e->plans[c.members[k]], s);
      st = (ps_status)plan_if_tables(e->plans[c.members[k]], dt);
    }
    const PlanView v = plan_view(e->plans[c.members[0]]);
    const Geo& g = v.g;
    const bool f32 = v.prec == PS_FP32;
    const int lens[5] = {g.nz, g.ny, g.nx, g.ny, g.nz};
    for (int step = 0; step < nsteps && st == PS_OK; ++step)
      for (int k = 0; k < c.nst && st == PS_OK; ++k) {
        BatchArgs& ba = bav[0];
        ba = BatchArgs{};
        for (int j = 0; j < M; ++j) ba.args[j] = c.args[(size_t)k * M + j];
        for (int pass = 0; pass < 5 && ce == cudaSuccess; ++pass) {
          ce = f32 ? batch_pass_f32(pass, lens[pass], ba, g, M, s) : batch_pass_f64(pass, lens[pass], ba, g, M, s);
          if (ce == cudaSuccess && pass == 0 && k == 0) ce = batch_sum(ba, v.n_epart, c.d_sum, M, s);
        }
        if (ce == cudaSuccess)
          ce = f32 ? batch_update_f32(ba, g, M, k == c.nst - 1, s) : batch_update_f64(ba, g, M, k == c.nst - 1, s);
        if (ce != cudaSuccess) st = cu(ce, "batched pass");
      }
  }
  for (int b = 0; b < B && st == PS_OK; ++b) {
    ce = cudaEventRecord(e->join[b], e->branch[b]);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(e->cap, e->join[b], 0);
    if (ce != cudaSuccess) st = cu(ce, "join");
  }
  cudaGraph_t gr = nullptr;
  ce = cudaStreamEndCapture(e->cap, &gr);
  if (st != PS_OK) {
    if (gr) cudaGraphDestroy(gr);
    return st;
  }
  ENS_CU(ce, "end capture");
  e->bgraph = gr;
  ENS_CU(cudaGraphInstantiate(&e->bexec, gr, 0), "instantiate");
  e->bkey_states.assign(u, u + m);
  e->bkey_dt = dt;
  e->bkey_steps = nsteps;
  return PS_OK;
}

ps_status run_batched(ps_ensemble* e, void* const* u, double dt, double t, int nsteps) {
  const bool same = e->bexec && e->bkey_steps == nsteps && e->bkey_dt == dt &&
                    std::equal(e->bkey_states.begin(), e->bkey_states.end(), u);
  if (!same) {
    ps_status st = batch_capture(e, u, dt, nsteps);
    if (st != PS_OK) return st;
  }
  ENS_CU(cudaGraphLaunch(e->bexec, e->main), "graph launch");
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
  drop_pgraph(e);
  drop_bgraph(e);
  for (void* d : {(void*)e->d_passes, (void*)e->d_args, (void*)e->d_done, (void*)e->d_head, (void*)e->d_err})
    if (d) cudaFree(d);
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
  if (mode == PS_ENS_AUTO) mode = e->auto_mode;
  if (mode == PS_ENS_SEQUENTIAL) return run_sequential(e, uhats, dt, t, nsteps);
  if (mode == PS_ENS_GRAPH) return run_graph(e, uhats, dt, t, nsteps);
  if (mode == PS_ENS_PERSISTENT) return run_persistent(e, uhats, dt, t, nsteps);
  if (mode == PS_ENS_BATCHED) return run_batched(e, uhats, dt, t, nsteps);
  return bad(PS_ERR_INVALID_ARG, "ensemble: unknown mode");
}

ps_status ps_ensemble_check(ps_ensemble* e) {
  if (!e) return bad(PS_ERR_INVALID_ARG, "ensemble: NULL ensemble");
  ENS_CU(cudaStreamSynchronize(e->main), "sync");
  ps_status result = PS_OK;
  if (e->d_err) {
    int w = 0;
    ENS_CU(cudaMemcpy(&w, e->d_err, sizeof(int), cudaMemcpyDeviceToHost), "error word");
    if (w != 0) {
      ENS_CU(cudaMemset(e->d_err, 0, sizeof(int)), "error word");
      result = bad(PS_ERR_TIMEOUT, "ensemble: a bounded wait of the persistent launch gave up");
    }
  }
  // the members' own words (x-pass waits of the graph, batched and
  // sequential modes); every word is read and cleared
  for (ps_plan* p : e->plans) {
    plan_set_stream(p, e->main);
    const ps_status s = (ps_status)plan_check_error(p);
    if (result == PS_OK) result = s;
  }
  return result;
}

ps_status ps_ensemble_set_wait_test(ps_ensemble* e, unsigned polls) {
  if (!e) return bad(PS_ERR_INVALID_ARG, "ensemble: NULL ensemble");
  if (e->wait_test != polls) drop_pgraph(e);
  e->wait_test = polls;
  return PS_OK;
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
    plan_set_xrpc(e->plans[i], best_r);
    // tile shape of the column passes (columns per CTA, radix schedule), one
    // pass at a time on top of the choices so far
    int best_var[3] = {0, 0, 0};
    for (int k = 0; k < 3 && st == PS_OK; ++k)
      for (int var = 1; var <= 2 && st == PS_OK; ++var) {
        if (!plan_set_shape(e->plans[i], k, var)) continue;
        double ms = 0;
        st = time_ms(e, 3, [&] { return ps_rk_step(e->plans[i], work[i], dt, 0.0); }, &ms);
        if (st == PS_OK && ms < best * 0.98) {
          best = ms;
          best_var[k] = var;
        }
        plan_set_shape(e->plans[i], k, best_var[k]);
      }
    for (size_t j = i; j < m; ++j) {
      const ps_config& d = e->cfgs[j];
      if (d.nx == c.nx && d.ny == c.ny && d.nz == c.nz && d.prec == c.prec) {
        plan_set_xrpc(e->plans[j], best_r);
        for (int k = 0; k < 3; ++k) plan_set_shape(e->plans[j], k, best_var[k]);
      }
    }
    if (out->nsizes < PS_ENS_MAX_SIZES) {
      const int z = out->nsizes;
      out->n[z] = c.nx;
      out->xrpc[z] = best_r;
      for (int k = 0; k < 3; ++k) {
        const int len = k == 1 ? c.ny : c.nz;
        int cols = 0, pts = 0;
        if (c.prec == PS_FP32) pass_shape<float>(k, len, best_var[k], &cols, &pts);
        else pass_shape<double>(k, len, best_var[k], &cols, &pts);
        out->pass_cols[z][k] = cols;
        out->pass_points[z][k] = pts;
      }
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
  // 3. persistent launch: CTAs per SM, member order and tiles per work item
  //    per pass kind, one knob at a time (coordinate descent), each candidate
  //    timed on one step of all members
  out->persistent_step_ms = -1.0;
  out->best_mode = PS_ENS_GRAPH;
  e->auto_mode = PS_ENS_GRAPH;
  if (st == PS_OK && persist_unsupported(e).empty()) {
    auto timed = [&](double* ms) {
      drop_pgraph(e);
      return time_ms(e, 3, [&] { return run_persistent(e, work.data(), dt, 0.0, 1); }, ms);
    };
    double best = 1e30;
    st = timed(&best);
    auto knob = [&](int* k, std::initializer_list<int> cand) {
      const int keep = *k;
      int best_v = keep;
      for (int v : cand) {
        if (v == keep || st != PS_OK) continue;
        *k = v;
        double ms = 0;
        st = timed(&ms);
        if (st == PS_OK && ms < best * 0.98) {
          best = ms;
          best_v = v;
        }
      }
      *k = best_v;
    };
    knob(&e->ctas_per_sm, {0, 1});
    knob(&e->order, {0, 1, 2});
    knob(&e->per[EK_ZINV], {1, 2, 4});
    knob(&e->per[EK_YINV], {1, 2, 4, 8});
    knob(&e->per[EK_XPASS], {1, 2, 4});
    knob(&e->per[EK_YFWD], {1, 2, 4, 8});
    knob(&e->per[EK_ZFWD], {1, 2, 4});
    knob(&e->per[EK_UPDATE], {4, 8, 16, 32});
    drop_pgraph(e);
    if (st == PS_OK) {
      out->persistent_step_ms = best;
      out->persistent_ctas_per_sm = e->ctas_per_sm;
      out->persistent_order = e->order;
      for (int k = 0; k < 6; ++k) out->persistent_tiles_per_item[k] = e->per[k];
      if (best < out->step_ms) e->auto_mode = PS_ENS_PERSISTENT;
      out->best_mode = e->auto_mode;
    }
  }
  // 4. batched launches (one per pass and sub-batch of a grid class; the
  //    sub-batches are concurrent graph branches): members per launch
  out->batched_step_ms = -1.0;
  if (st == PS_OK && batch_unsupported(e).empty()) {
    double ms = 1e30;
    int best_bs = e->bsize;
    for (int bs : {BATCH_MAX, 16, 8, 4, 2}) {
      if (st != PS_OK) break;
      e->bsize = bs;
      double t_bs = 0;
      drop_bgraph(e);
      st = time_ms(e, 3, [&] { return run_batched(e, work.data(), dt, 0.0, 1); }, &t_bs);
      if (st == PS_OK && t_bs < ms * 0.98) {
        ms = t_bs;
        best_bs = bs;
      }
    }
    e->bsize = best_bs;
    drop_bgraph(e);
    if (st == PS_OK) {
      out->batched_step_ms = ms;
      out->batched_members_per_launch = best_bs;
      const double cur = e->auto_mode == PS_ENS_PERSISTENT ? out->persistent_step_ms : out->step_ms;
      if (ms < cur) e->auto_mode = PS_ENS_BATCHED;
      out->best_mode = e->auto_mode;
    }
  }
  cudaStreamSynchronize(e->main);
  for (void* w : work)
    if (w) cudaFree(w);
  return st;
}

}  // extern "C"

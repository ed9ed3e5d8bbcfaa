// Internal interface between the plan (ps_plan.cu) and the pass kernels.
// Not part of the public C ABI (include/ps.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct ps_plan;

namespace ps {

// Grid geometry and the retained (2/3-rule) cube.
struct Geo {
  int nx, ny, nz, nh;
  int Kx, Ky, Kz;   // largest retained |index| per axis
  int cx, cy, cz;   // retained counts: Kx+1, 2Ky+1, 2Kz+1
  int kxp;          // padded kx extent of the compact buffers (multiple of 16)
  int sphere;       // spherical truncation on top of the cube
  double sx, sy, sz;  // 2 pi / L per axis
  float sxf, syf, szf;  // the same in FP32 (set_scales), for FP32 kernels
  // kx slab of a decomposed problem (zero for a whole problem): local column
  // c is the global kx0 + c; ncx local retained columns (0: cx); caller rows
  // of rowlen entries (0: nh)
  int kx0, ncx, rowlen;
};
// Sets the wavenumber scales 2 pi / L (and their FP32 copies) of g.
inline void set_scales(Geo& g, double lx, double ly, double lz) {
  const double two_pi = 6.283185307179586476925286766559;
  g.sx = two_pi / lx;
  g.sy = two_pi / ly;
  g.sz = two_pi / lz;
  g.sxf = (float)g.sx;
  g.syf = (float)g.sy;
  g.szf = (float)g.sz;
}
__host__ __device__ inline int ncols(const Geo& g) { return g.ncx ? g.ncx : g.cx; }
__host__ __device__ inline int rowlen(const Geo& g) { return g.rowlen ? g.rowlen : g.nh; }

// A spectral vector field in HBM: element (c, r, q, p) at
// p + ys*row_y(q) + zs*row_z(r) + cs*c, with row(s) = s >= 0 ? s : s + wrap.
// The caller's layout has wrap = n (FFT order), the compact layout wrap = 2K+1.
struct Spec {
  const void* p;
  long long cs, zs, ys;
  int zwrap, ywrap;
};

enum ZfwdMode : int {
  ZF_RHS = 0,   // out_full = D P(N + f) - nu k^2 u_in
  ZF_RK4_1 = 1, ZF_RK4_2 = 2, ZF_RK4_3 = 3, ZF_RK4_4 = 4,
  ZF_RK2_1 = 5, ZF_RK2_2 = 6,
};

struct PassArgs {
  Geo g;
  // inverse z pass input (state or stage buffer)
  Spec in;
  // intermediate buffers
  void* a6;   // [6 ng][nz][cy][kxp]  (z-inverse out) / [3 ng][nz][ny][kxp] (x out)
  void* b6;   // [6 ng][nz][ny][kxp]  (y-inverse out) / [3 ng][nz][cy][kxp] (y-forward out)
  const void* tw_x;  // exp(-2 pi i m/nx), m < nx
  const void* tw_y;
  const void* tw_z;
  // fused reductions
  double* e_part;              // per-CTA energy partials of the z-inverse pass, or null
  unsigned long long* umax2;   // max |u|^2 (as ordered bits) from the x pass, or null
  // forward z pass
  int mode;
  Spec u_n;          // state at the start of the step (RK) / RHS input (ZF_RHS)
  void* out_full;    // caller-layout output: RHS or the new state
  void* nxt;         // compact next-stage input [3][cz][cy][kxp]
  void* acc;         // compact accumulator        [3][cz][cy][kxp]
  const void* ifx;   // exp(-nu kx^2 dt/2) for p <= Kx
  const void* ify;   // ... per retained ky index
  const void* ifz;   // ... per retained kz index
  double dt, nu, eta;  // eta: diffusivity of the second field (MHD: eta, Boussinesq: kappa)
  int ng;            // 3-component groups: 1 (HD: u; Boussinesq: u) or 2 (MHD: u, B)
  int nsc;           // scalar components after the groups: 1 (Boussinesq: theta) or 0
  int nfi;           // fields into the x pass: 6 ng + 3 nsc (u, omega, (B, j,) (grad theta))
  int nfo;           // fields out of the x pass: 3 ng + nsc (u x omega (+ j x B), (u x B), (u . grad theta))
  double n_bv;       // Boussinesq: Brunt-Vaisala frequency (the jf* tables hold kappa)
  const void* jfx;   // exp(-eta k^2 dt/2) tables of the magnetic group
  const void* jfy;
  const void* jfz;
  const void* fbox;  // forcing box [3][2Fz+1][2Fy+1][Fx+1] or null
  int Fx, Fy, Fz;
  int xdiag;         // x pass: only the max |u| reduction (no product, no output)
  int xrpc;          // x pass rows per CTA (0 = largest that keeps two CTAs per SM)
  int shape[3];      // shape variant of the z-inverse, y and z-forward passes (ColShape; 0 = default)
  int* err;          // device error word (bounded waits that gave up), never null
  unsigned wait_polls;  // x pass: polls before a wait gives up (0 = PS_WAIT_LIMIT)
  int wait_test;     // x pass: test hook, the first copy of every CTA is never issued
  const void* extra; // compact closure term added to the velocity group before projection, or null
  // Constants in the working precision, set by prepare_args() on the host so
  // that FP32 kernels convert or divide no double on the GPU's slow FP64 pipe
  float dtf, nuf, etaf, nbvf, inv_n3f;
  double inv_n3;     // 1/(nx ny nz)
};

// Fills the derived constants of a (every launcher calls it on its copy).
inline void prepare_args(PassArgs& a) {
  a.dtf = (float)a.dt;
  a.nuf = (float)a.nu;
  a.etaf = (float)a.eta;
  a.nbvf = (float)a.n_bv;
  a.inv_n3 = 1.0 / ((double)a.g.nx * a.g.ny * a.g.nz);
  a.inv_n3f = (float)a.inv_n3;
}

// The FP64 value in an FP64 kernel, its FP32 copy in an FP32 kernel.
template <typename T>
__host__ __device__ inline T pick(double d, float f) {
  if constexpr (sizeof(T) == 4) return f;
  else return d;
}

// Launchers (one per pass and precision); return the launch error.
template <typename T> cudaError_t launch_zinv(const PassArgs& a, cudaStream_t s, int* nblocks_out);
template <typename T> cudaError_t launch_yinv(const PassArgs& a, cudaStream_t s);
template <typename T> cudaError_t launch_xpass(const PassArgs& a, cudaStream_t s);
template <typename T> cudaError_t launch_yfwd(const PassArgs& a, cudaStream_t s);
template <typename T> cudaError_t launch_zfwd(const PassArgs& a, cudaStream_t s);
// projection, forcing, closure and the ZfwdMode output from the z-forward pass's a6
template <typename T> cudaError_t launch_update(const PassArgs& a, cudaStream_t s);
// number of CTAs (energy partials) the z-inverse pass uses for this geometry
// in shape variant var (-1: the largest over the variants)
template <typename T> int zinv_blocks(const Geo& g, int var = 0);
// Columns per CTA and points per thread of column pass k (0 z-inverse, 1 y
// passes, 2 z-forward) on lines of n points in shape variant var; false if
// the length has no such variant.
template <typename T> bool pass_shape(int k, int n, int var, int* cols, int* points);

// Auxiliary kernels (ps_aux.cu)
template <typename T>
cudaError_t launch_if_tables(const Geo& g, double nu, double dt, void* tab, cudaStream_t s);
cudaError_t launch_sum_partials(const double* part, int n, double* out, cudaStream_t s);
template <typename T>
cudaError_t launch_forcing_extent(const Geo& g, Spec f, int* ext, cudaStream_t s);
template <typename T>
cudaError_t launch_forcing_gather(const Geo& g, Spec f, int Fx, int Fy, int Fz, void* box, cudaStream_t s);
// Head of one diagnostics row: E, Omega, H, max|k.u|, E_B, H_c, H_m, E_P.
constexpr int DIAG_HEAD = 8;
template <typename T>
cudaError_t launch_diag_spectral(const Geo& g, Spec u, double* part, int nshells, int eq, cudaStream_t s);
cudaError_t launch_diag_final(const double* part, int nblk, int nshells, double* out, cudaStream_t s);

// LES closure (ps_les.cu): -i k_j tau_hat_ij of the model stress of the state
// `in`, written to the compact buffer s.extra ([3][cz][cy][kxp], FP32).
struct LesScratch {
  const float* params;  // MLP parameters (PS_MLP_NPARAM)
  const float* norm;    // mean[5], 1/std[5], s_tau, 1/s_A (device)
  float2* spec;         // [9][nz][ny][nh]
  float* phys;          // [9][nz][ny][nx]
  float* X;             // [P][5]
  float* Y;             // [P][6]
  float2* extra;        // compact closure term
  float* Arows;         // [P][9] gradient rows (training only)
};
cudaError_t launch_stream_copy(const void* src, void* dst, size_t bytes, int nsm, cudaStream_t s);
cudaError_t launch_copy_cube(const void* src, void* dst, const Geo& g, int nc, size_t vb, int nsm, cudaStream_t s);
cudaError_t les_closure_term(const Geo& g, Spec in, const void* twx, const void* twy, const void* twz,
                             const LesScratch& s, cudaStream_t st);
// Force loss (sum over the half spectrum of w |D P(closure) - f|^2) of the
// state `in` against the subgrid force f (full layout), added to *loss, and
// its parameter gradient added to grad; params replaces s.params.
// With t_exact (device, nsh shells) the loss is instead sum_K (T(K) - t_exact[K])^2
// of the shell energy transfer of the projected closure term; bins holds 2 nsh doubles.
cudaError_t les_closure_grad(const Geo& g, Spec in, Spec f, const void* twx, const void* twy, const void* twz,
                             const LesScratch& s, const float* params, float* grad, double* loss, cudaStream_t st,
                             const double* t_exact = nullptr, int nsh = 0, double* bins = nullptr);

// Plan internals used by the ensemble layer (ps_plan.cu).
void plan_set_stream(struct ::ps_plan* p, cudaStream_t s);
cudaStream_t plan_stream(const struct ::ps_plan* p);
void plan_set_xrpc(struct ::ps_plan* p, int rpc);
// Forget the cached integrating-factor tables so the next step recomputes them
// (a captured graph must contain that launch).
void plan_invalidate_tables(struct ::ps_plan* p);
// Shape variant (ColShape) of column pass k of p; false if it has none such.
bool plan_set_shape(struct ::ps_plan* p, int k, int var);
int plan_shape(const struct ::ps_plan* p, int k);
// Reads and clears the plan's device error word (synchronises its stream);
// a ps_status value, PS_ERR_TIMEOUT if a bounded wait gave up.
int plan_check_error(struct ::ps_plan* p);
void plan_set_time(struct ::ps_plan* p, double t);
// What the persistent ensemble launch (ps_persist.cu) needs of a member plan.
struct PlanView {
  Geo g;
  int prec, eq, rk_stages;
  bool closure;                 // a learned closure is attached
  double* e_part;               // energy partials of the z-inverse pass
  int n_epart;
  double* stats;                // [energy] of the step statistics
  unsigned long long* umax2;    // max |u|^2 bits of the step statistics
};
PlanView plan_view(const struct ::ps_plan* p);
// Arguments of RK stage st of one step on the caller's state uhat, exactly as
// ps_rk_step passes them to its kernels (derived constants prepared).
PassArgs plan_stage_args(struct ::ps_plan* p, void* uhat, double dt, int st, bool stats);
// Launches the integrating-factor tables for dt on the plan stream.
int plan_if_tables(struct ::ps_plan* p, double dt);  // a ps_status value

}  // namespace ps

// C ABI of the filtered SELBM library (include/selbm.h): handle creation,
// upload of the FP64 setup, the step loop, state import/export, diagnostics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/selbm.h"
#include "selbm_kernels.cuh"
#include "selbm_learn.cuh"
#include "selbm_setup.h"

using namespace slb;

namespace {
std::string g_create_error;
std::once_flag g_const_once;

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &src) {
  *dst = nullptr;
  if (src.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc((void **)dst, src.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

template <typename R>
std::vector<R> cast_vec(const std::vector<double> &v) {
  return std::vector<R>(v.begin(), v.end());
}
}  // namespace

struct selbm {
  Setup S;
  selbm_params P{};
  cudaStream_t stream = nullptr;
  int lat = 0, Q = 0, prec = 0, rsz = 8;
  double dt = 0, tau = 0, lam = 0, omega = 0, time = 0;
  int64_t steps = 0;
  bool initialized = false, filter_pending = false, filter_on = false, has_force = false;
  bool use_fast = true;   // SELBM_GENERIC_KERNEL=1 in the environment selects the generic stage kernel
  // population-split step (prologue + split stages); default for hexahedral meshes at the
  // compiled orders, SELBM_SPLIT=1 / 0 in the environment forces it on / off where compiled
  bool use_split = false;
  std::vector<double> Vm_h, Vinv_h;   // modal <-> nodal matrices
  // learned per-element filter control
  bool learned = false;
  int nin = 0;
  double mass_bound = 1e-6, ke_bound = 1e-6;
  void *d_Vm = nullptr, *d_Vinv = nullptr, *d_sigma_e = nullptr, *d_lo = nullptr, *d_hi = nullptr, *d_fixsig = nullptr;
  __nv_bfloat16 *d_W = nullptr;
  double *d_acc = nullptr;
  void *d_nq = nullptr;          // [2][Gs] rho - rho0 and |u| on unique nodes (learned control, split form)
  void *d_X = nullptr;           // [E][2n] element features (learned control, split form)
  int *d_flag = nullptr, *d_nfb = nullptr;
  int wall_max = 0;
  int n_wallpts = 0;             // wall points (element, node) over all elements
  double *d_xg = nullptr;        // [G][dim] coordinates of unique nodes (uploaded on first use)
  // per-node acceleration field A(t) S_g added to g (allocated on first use)
  bool field_on = false;
  double f_period = 0.0, f_tend = 0.0, ft_host = 0.0;
  void *d_fS = nullptr, *d_famp = nullptr;   // [3][G] S; [1] A(t) of the current step
  double *d_ft = nullptr;                    // [1] time at the start of the next step
  // time scheme: 0 Shu-Osher SSPRK3, 1 the printed four-stage form (extra stage buffers)
  int scheme = 0;
  void *S1 = nullptr, *S2 = nullptr, *SG = nullptr, *SB = nullptr;
  // captured steps (slot 0: no pending filter, slot 1: filter pending), launched with
  // cudaGraphLaunch on the handle's stream
  bool graph_enabled = true;   // SELBM_NO_GRAPH=1 in the environment disables capture
  int64_t eager_steps[2] = {0, 0};
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  cudaStream_t cap_stream = nullptr;
  void invalidate_graph() {
    for (int k = 0; k < 2; ++k) {
      if (gexec[k]) cudaGraphExecDestroy(gexec[k]);
      gexec[k] = nullptr;
    }
  }
  std::string err;
  std::vector<double> Fmat, sigma, FU, FW;
  int Fr = 0;
  // device buffers (Real = double or float by precision)
  void *FA = nullptr, *F0 = nullptr, *F2 = nullptr, *T = nullptr, *RHO = nullptr, *BUF = nullptr;
  void *d_el_drdx = nullptr, *d_el_J = nullptr, *d_drdx = nullptr, *d_wJ = nullptr, *d_gllw = nullptr;
  void *d_D = nullptr, *d_F = nullptr, *d_wall_u = nullptr, *d_walls = nullptr, *d_minv = nullptr;
  void *d_wall_u0 = nullptr;   // walls at rest (the source-free operator of time scheme 2)
  int32_t *d_l2g = nullptr, *d_bslot = nullptr, *d_bnode_g = nullptr, *d_bnode_off = nullptr, *d_bnode_slot = nullptr;
  int32_t *d_wall_off = nullptr, *d_first = nullptr;
  uint8_t *d_owner = nullptr;
  double *d_mass = nullptr, *d_partial = nullptr, *d_diag = nullptr;
  double *d_io = nullptr;  // staging for host <-> device FP64 arrays
  size_t io_bytes = 0;
  std::vector<void *> allocs;
  // tracing: event pairs around hot-path launches
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
  cudaEvent_t take_event() {
    if (!ev_pool.empty()) { cudaEvent_t e = ev_pool.back(); ev_pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  cudaEvent_t mark_begin() {
    if (!timing) return nullptr;
    cudaEvent_t e = take_event();
    cudaEventRecord(e, stream);
    return e;
  }
  void mark_end(int kind, cudaEvent_t b) {
    if (!timing || !b) return;
    cudaEvent_t e = take_event();
    cudaEventRecord(e, stream);
    ev_used.push_back({kind, {b, e}});
  }

  int fail(int code, const std::string &m) { err = m; return code; }
  int cuda_fail(cudaError_t e, const char *where) {
    err = std::string(where) + ": " + cudaGetErrorString(e);
    return SELBM_ERR_CUDA;
  }
  size_t nloc() const { return (size_t)S.E * S.Np; }
  // population stride of the state arrays: G rounded up to a multiple of 8, so that every
  // population row (and every element's interior block at N = 7) starts 16-byte aligned
  int Gs() const { return (S.G + 7) & ~7; }
};

namespace {

template <typename Real>
cudaError_t upload_real(selbm *h) {
  const Setup &S = h->S;
  cudaError_t e;
  const size_t G = S.G, GS = h->Gs(), Q = h->Q;
  auto alloc = [&](void **p, size_t bytes) {
    cudaError_t r = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (r == cudaSuccess) { h->allocs.push_back(*p); cudaMemsetAsync(*p, 0, std::max<size_t>(bytes, 16), h->stream); }
    return r;
  };
  if ((e = alloc(&h->FA, Q * GS * sizeof(Real)))) return e;
  if ((e = alloc(&h->F0, Q * GS * sizeof(Real)))) return e;
  if ((e = alloc(&h->F2, Q * GS * sizeof(Real)))) return e;
  if ((e = alloc(&h->BUF, Q * GS * sizeof(Real)))) return e;
  if ((e = alloc(&h->T, Q * (size_t)S.E * S.Nb * sizeof(Real)))) return e;
  if ((e = alloc(&h->RHO, G * sizeof(Real)))) return e;
  Real *p;
  if (S.affine) {
    std::vector<double> em = S.el_drdx;
    // exact zeros for metric entries that vanish up to rounding (axis-aligned elements)
    const int d = S.dim;
    for (int el = 0; el < S.E; ++el) {
      double mx = 0;
      for (int c = 0; c < d * d; ++c) mx = std::max(mx, std::fabs(em[(size_t)el * d * d + c]));
      for (int c = 0; c < d * d; ++c)
        if (std::fabs(em[(size_t)el * d * d + c]) < 1e-13 * mx) em[(size_t)el * d * d + c] = 0.0;
    }
    if ((e = upload(&p, cast_vec<Real>(em)))) return e; h->d_el_drdx = p; h->allocs.push_back(p);
    if ((e = upload(&p, cast_vec<Real>(S.el_J)))) return e; h->d_el_J = p; h->allocs.push_back(p);
  } else {
    if ((e = upload(&p, cast_vec<Real>(S.drdx)))) return e; h->d_drdx = p; h->allocs.push_back(p);
    if ((e = upload(&p, cast_vec<Real>(S.wJ)))) return e; h->d_wJ = p; h->allocs.push_back(p);
  }
  if ((e = upload(&p, cast_vec<Real>(S.gll.w)))) return e; h->d_gllw = p; h->allocs.push_back(p);
  if ((e = upload(&p, cast_vec<Real>(S.gll.D)))) return e; h->d_D = p; h->allocs.push_back(p);
  if ((e = alloc(&h->d_F, S.n1 * S.n1 * sizeof(Real)))) return e;
  {
    std::vector<double> V, Vi;
    build_modal(S.gll, &V, &Vi);
    h->Vm_h = V;
    h->Vinv_h = Vi;
    if ((e = upload(&p, cast_vec<Real>(V)))) return e; h->d_Vm = p; h->allocs.push_back(p);
    if ((e = upload(&p, cast_vec<Real>(Vi)))) return e; h->d_Vinv = p; h->allocs.push_back(p);
  }
  if ((e = alloc(&h->d_sigma_e, (size_t)S.E * S.n1 * sizeof(Real)))) return e;
  if ((e = alloc(&h->d_fixsig, S.n1 * sizeof(Real)))) return e;
  if ((e = alloc(&h->d_lo, 2 * S.n1 * sizeof(Real)))) return e;
  if ((e = alloc(&h->d_hi, 2 * S.n1 * sizeof(Real)))) return e;
  if ((e = alloc((void **)&h->d_acc, 8 * sizeof(double)))) return e;
  if ((e = alloc(&h->d_nq, 2 * (size_t)h->Gs() * sizeof(Real)))) return e;
  if ((e = alloc(&h->d_X, 2 * (size_t)S.n1 * S.E * sizeof(Real)))) return e;
  if ((e = alloc((void **)&h->d_flag, 2 * sizeof(int)))) return e;
  if ((e = alloc((void **)&h->d_nfb, 2 * sizeof(int)))) return e;
  if ((e = alloc((void **)&h->d_W, (size_t)mlp_nparams(2 * S.n1) * sizeof(__nv_bfloat16)))) return e;
  std::vector<double> wu = S.wall_u;
  if (wu.empty()) wu.assign(3, 0.0);
  if ((e = upload(&p, cast_vec<Real>(wu)))) return e; h->d_wall_u = p; h->allocs.push_back(p);
  std::vector<double> wz(wu.size(), 0.0);
  if ((e = upload(&p, cast_vec<Real>(wz)))) return e; h->d_wall_u0 = p; h->allocs.push_back(p);
  std::vector<double> minv(S.Gb);
  for (int u = 0; u < S.Gb; ++u) minv[u] = 1.0 / S.mass[S.bnode_g[u]];
  if ((e = upload(&p, cast_vec<Real>(minv)))) return e; h->d_minv = p; h->allocs.push_back(p);
  // wall nodes grouped per (element, node)
  std::vector<WallPt<Real>> wp;
  std::vector<int32_t> woff(S.E + 1, 0);
  for (int el = 0; el < S.E; ++el) {
    std::vector<const WallNode *> nodes;
    for (int k = S.wall_off[el]; k < S.wall_off[el + 1]; ++k) nodes.push_back(&S.walls[k]);
    std::stable_sort(nodes.begin(), nodes.end(), [](const WallNode *a, const WallNode *b) { return a->i < b->i; });
    for (size_t k = 0; k < nodes.size();) {
      WallPt<Real> w{};
      w.i = nodes[k]->i; w.b = nodes[k]->b; w.nf = 0;
      while (k < nodes.size() && nodes[k]->i == w.i) {
        if (w.nf < 3) {
          for (int c = 0; c < 3; ++c) w.n[w.nf][c] = (Real)nodes[k]->n[c];
          w.wsJs[w.nf] = (Real)nodes[k]->wsJs;
          w.wid[w.nf] = nodes[k]->wid;
          w.nf++;
        }
        ++k;
      }
      wp.push_back(w);
    }
    woff[el + 1] = (int32_t)wp.size();
    h->wall_max = std::max(h->wall_max, woff[el + 1] - woff[el]);
  }
  h->n_wallpts = (int)wp.size();
  WallPt<Real> *dw;
  if ((e = upload(&dw, wp))) return e; h->d_walls = dw; if (dw) h->allocs.push_back(dw);
  int32_t *q;
  if ((e = upload(&q, woff))) return e; h->d_wall_off = q; h->allocs.push_back(q);
  return cudaSuccess;
}

template <typename Real>
KParams<Real> base_params(selbm *h) {
  const Setup &S = h->S;
  KParams<Real> p{};
  p.E = S.E; p.Np = S.Np; p.Nb = S.Nb; p.N = S.N; p.n = S.n1; p.G = S.G; p.Gs = h->Gs(); p.Gb = S.Gb;
  p.dt = (Real)h->dt; p.half_dt = (Real)(0.5 * h->dt); p.omega = (Real)h->omega; p.rho0 = (Real)h->P.rho0;
  for (int k = 0; k < 3; ++k) p.g[k] = (Real)(k < S.dim ? h->P.body_accel[k] : 0.0);
  p.has_force = h->has_force;
  p.wall_max = h->wall_max;
  p.l2g = h->d_l2g; p.owner = h->d_owner; p.bslot = h->d_bslot;
  p.el_drdx = (const Real *)h->d_el_drdx; p.el_J = (const Real *)h->d_el_J;
  p.drdx = (const Real *)h->d_drdx; p.wJ = (const Real *)h->d_wJ; p.gllw = (const Real *)h->d_gllw;
  p.Dm = (const Real *)h->d_D; p.Fm = (const Real *)h->d_F;
  p.walls = (const WallPt<Real> *)h->d_walls; p.wall_off = h->d_wall_off; p.wall_u = (const Real *)h->d_wall_u;
  p.bnode_g = h->d_bnode_g; p.bnode_off = h->d_bnode_off; p.bnode_slot = h->d_bnode_slot;
  p.bnode_minv = (const Real *)h->d_minv;
  p.T = (Real *)h->T; p.rho = (Real *)h->RHO;
  p.fS = h->field_on ? (const Real *)h->d_fS : nullptr;
  p.famp = (const Real *)h->d_famp;
  return p;
}

// learned filter pass: per-element transfer functions from the features of `f`
// (the state the pending filter acts on), filtered interior nodes into `out`,
// weighted shares of boundary nodes into the trace, then their mass-weighted
// assembly into `out` (the drift check runs after the pass when requested)
template <typename Real>
cudaError_t enqueue_learned_filter(selbm *h, const Real *f, Real *out, bool with_drift) {
  const Setup &S = h->S;
  ControlArgs<Real> c{};
  c.E = S.E; c.Np = S.Np; c.n = S.n1; c.N = S.N; c.G = S.G; c.Gs = h->Gs(); c.Nb = S.Nb;
  c.l2g = h->d_l2g; c.bslot = h->d_bslot; c.f = f; c.rho0 = h->P.rho0; c.affine = S.affine ? 1 : 0;
  c.el_J = (const Real *)h->d_el_J; c.wJ = (const Real *)h->d_wJ; c.gllw = (const Real *)h->d_gllw;
  c.Vm = (const Real *)h->d_Vm; c.Vinv = (const Real *)h->d_Vinv; c.W = h->d_W;
  c.lo = (const Real *)h->d_lo; c.hi = (const Real *)h->d_hi; c.fixed_sigma = (const Real *)h->d_fixsig;
  c.flag = h->d_flag; c.acc = with_drift ? h->d_acc : nullptr;
  c.sigma_out = (Real *)h->d_sigma_e; c.feat_out = nullptr; c.n_fallback = with_drift ? h->d_nfb : nullptr;
  c.fout = out; c.T = (Real *)h->T;
  cudaError_t e = launch_control<Real>(h->lat, c, h->stream);
  if (e == cudaSuccess && with_drift)
    e = launch_drift_check(h->d_acc, h->d_flag, h->mass_bound, h->ke_bound, h->has_force ? 0 : 1, h->stream);
  if (e == cudaSuccess) {
    KParams<Real> q = base_params<Real>(h);
    q.A = Real(0); q.B = Real(0); q.has_force = 0; q.dt = Real(0);
    q.fin = out; q.f0 = out; q.fout = out;
    e = launch_dss<Real>(h->lat, q, h->stream);
  }
  return e;
}

// register-blocked kernel when compiled for (lattice, N); generic kernel otherwise
template <typename Real>
cudaError_t launch_stage_any(selbm *h, const KParams<Real> &p) {
  if (h->use_fast) {
    FastHost fh{h->S.gll.D.data(), h->FU.data(), h->FW.data(), h->S.gll.w.data(), h->Fr};
    cudaError_t err = cudaSuccess;
    bool done = false;
    if (h->lat == SELBM_D2Q9) done = launch_fast_d2q9<Real>(h->S.N, h->S.affine, p, fh, h->stream, &err);
    else if (h->lat == SELBM_D3Q19) done = launch_fast_d3q19<Real>(h->S.N, h->S.affine, p, fh, h->stream, &err);
    else done = launch_fast_d3q27<Real>(h->S.N, h->S.affine, p, fh, h->stream, &err);
    if (done) return err;
  }
  return launch_stage<Real>(h->lat, h->S.affine, p, h->stream);
}

SplitHost split_host(selbm *h) {
  return SplitHost{h->S.gll.D.data(), h->FU.data(), h->FW.data(), h->S.gll.w.data(), h->Fr,
                   h->Vm_h.data(), h->Vinv_h.data(), h->sigma.data()};
}

template <typename Real>
cudaError_t launch_split_stage(selbm *h, const KParams<Real> &p) {
  const SplitHost sh = split_host(h);
  cudaError_t err = cudaErrorInvalidValue;
  if (h->lat == SELBM_D3Q19) split_stage_d3q19<Real>(h->S.N, h->S.affine, p, sh, h->stream, &err);
  else if (h->lat == SELBM_D3Q27) split_stage_d3q27<Real>(h->S.N, h->S.affine, p, sh, h->stream, &err);
  return err;
}

template <typename Real>
cudaError_t launch_split_prologue(selbm *h, int mode, const KParams<Real> &p, const LearnedPtrs<Real> &lp) {
  const SplitHost sh = split_host(h);
  cudaError_t err = cudaErrorInvalidValue;
  if (h->lat == SELBM_D3Q19) split_prologue_d3q19<Real>(h->S.N, h->S.affine, mode, p, sh, lp, h->stream, &err);
  else if (h->lat == SELBM_D3Q27) split_prologue_d3q27<Real>(h->S.N, h->S.affine, mode, p, sh, lp, h->stream, &err);
  return err;
}

// the learned step prologue of the split form: the control (node features + network per
// element -> sigma_e), the filter with each element's sigma_e + collision of interior nodes +
// weighted shares of boundary nodes, the drift check, the assembly + collision of shared nodes
template <typename Real>
cudaError_t launch_split_learned(selbm *h, const KParams<Real> &p);

template <typename Real>
cudaError_t launch_split_collide(selbm *h, int which, const KParams<Real> &p) {
  if (h->lat == SELBM_D3Q19) return split_collide_d3q19<Real>(which, p, h->stream);
  if (h->lat == SELBM_D3Q27) return split_collide_d3q27<Real>(which, p, h->stream);
  return cudaErrorInvalidValue;
}

template <typename Real>
LearnedPtrs<Real> learned_ptrs(selbm *h, bool with_drift) {
  LearnedPtrs<Real> lp{};
  lp.W = h->d_W; lp.lo = (const Real *)h->d_lo; lp.hi = (const Real *)h->d_hi;
  lp.flag = h->d_flag; lp.acc = with_drift ? h->d_acc : nullptr;
  lp.sigma_out = (Real *)h->d_sigma_e; lp.feat_out = nullptr; lp.n_fallback = with_drift ? h->d_nfb : nullptr;
  lp.outputs = 1;
  return lp;
}

template <typename Real>
cudaError_t launch_split_learned(selbm *h, const KParams<Real> &p) {
  const SplitHost sh = split_host(h);
  const LearnedPtrs<Real> lp = learned_ptrs<Real>(h, true);
  cudaError_t e = cudaErrorInvalidValue;
  if (h->lat == SELBM_D3Q19) split_control_d3q19<Real>(h->S.N, p, sh, lp, (Real *)h->d_nq, (Real *)h->d_X, h->d_mass, h->stream, &e);
  else if (h->lat == SELBM_D3Q27) split_control_d3q27<Real>(h->S.N, p, sh, lp, (Real *)h->d_nq, (Real *)h->d_X, h->d_mass, h->stream, &e);
  if (e) return e;
  if ((e = launch_split_prologue<Real>(h, PRO_LEARNED, p, lp))) return e;
  if ((e = launch_drift_check(h->d_acc, h->d_flag, h->mass_bound, h->ke_bound, h->has_force ? 0 : 1, h->stream))) return e;
  return launch_split_collide<Real>(h, 1, p);
}

// one time step of the population-split form: prologue (pending filter + collision,
// f^0 on unique nodes), then three advection stages, each = split kernel + assembly
template <typename Real>
cudaError_t enqueue_step_split(selbm *h, bool apply_filter) {
  KParams<Real> p = base_params<Real>(h);
  Real *FA = (Real *)h->FA, *F0 = (Real *)h->F0, *F2 = (Real *)h->F2;
  cudaError_t e;
  p.fin = FA; p.f0out = F0;
  p.stage = 1; p.A = Real(0); p.B = Real(1);
  if (apply_filter && h->learned) {
    cudaEvent_t t0 = h->mark_begin();
    if ((e = launch_split_learned<Real>(h, p))) return e;
    h->mark_end(3, t0);
  } else {
    cudaEvent_t t0 = h->mark_begin();
    if (apply_filter) e = launch_split_prologue<Real>(h, PRO_FIXED, p, LearnedPtrs<Real>{});
    else e = launch_split_collide<Real>(h, 0, p);
    if (e) return e;
    h->mark_end(4, t0);
  }
  // Shu-Osher weights with A = 1 - B formed in the working precision: A + B = 1 exactly, so a
  // stage combination A f0 + B f' of the deviations carries no systematic scale error (with
  // A = fl(1/3), B = fl(2/3) in FP32 the sum is 1 + 3e-8 and the state drifts by that every step)
  const Real B[3] = {Real(1), Real(0.25), Real(2.0 / 3.0)};
  const Real A[3] = {Real(0), Real(1) - B[1], Real(1) - B[2]};
  const Real *fin[3] = {F0, FA, F2};   // f^{s-1}: stage 1 advects f^0
  Real *fout[3] = {FA, F2, FA};
  for (int s = 0; s < 3; ++s) {
    p.stage = s + 1; p.A = A[s]; p.B = B[s]; p.apply_filter = 0;
    p.fin = fin[s]; p.f0 = F0; p.fout = fout[s]; p.f0out = nullptr;
    cudaEvent_t t0 = h->mark_begin();
    if ((e = launch_split_stage<Real>(h, p))) return e;
    h->mark_end(s == 0 ? 0 : 1, t0);
    t0 = h->mark_begin();
    if ((e = launch_dss<Real>(h->lat, p, h->stream))) return e;
    h->mark_end(2, t0);
  }
  return cudaSuccess;
}

// one time step of the printed four-stage scheme (Sec. 2.2.2, taken literally):
//   f1 = f0 + dt/3 L f0,  f2 = f1 - 3 dt/4 L(f0 - f1),  f3 = f2 + 2 dt/3 L(f0 - f1 + f2),
//   f  = f3 - dt/4 L(f0 - f1 + f2 - f3),
// f0 the collided state.  The stage and assembly kernels form A b + B (g + dt L g); a stage
// f^s = f^{s-1} + c dt L(g) runs them with g the stage argument, B = c, A = 1 and
// b = f^{s-1} - c g (both written by one combination pass).  Stage 1 (g = f0, c = 1/3) takes
// b = 2/3 f0 where the kernel adds A b, and the whole-element kernel's first stage keeps f0
// with weight 1 by itself.
template <typename Real>
cudaError_t enqueue_step_printed(selbm *h, bool apply_filter) {
  KParams<Real> p = base_params<Real>(h);
  Real *FA = (Real *)h->FA, *F0 = (Real *)h->F0, *F1 = (Real *)h->F2;
  Real *F2 = (Real *)h->S1, *F3 = (Real *)h->S2, *GS = (Real *)h->SG, *BS = (Real *)h->SB;
  const size_t nv = (size_t)h->Q * h->Gs();
  const double third[4] = {2.0 / 3.0, 0, 0, 0};
  cudaError_t e;
  // stage 1 (collision and pending filter included): f1 = f0 + dt/3 L f0
  if (h->use_split) {
    p.stage = 1; p.A = Real(0); p.B = Real(1);
    p.fin = FA; p.f0out = F0;
    if (apply_filter && h->learned) {
      if ((e = launch_split_learned<Real>(h, p))) return e;
    } else {
      e = apply_filter ? launch_split_prologue<Real>(h, PRO_FIXED, p, LearnedPtrs<Real>{}) : launch_split_collide<Real>(h, 0, p);
      if (e) return e;
    }
    // b = 2/3 f0 (GS unused here), then A b + 1/3 (f0 + dt L f0)
    if ((e = launch_combine<Real>(nv, F0, F0, F0, F0, 1, third, F0, 0.0, BS, GS, h->stream))) return e;
    p.stage = 2; p.A = Real(1); p.B = Real(1.0 / 3.0); p.apply_filter = 0;
    p.fin = F0; p.f0 = BS; p.fout = F1; p.f0out = nullptr;
    if ((e = launch_split_stage<Real>(h, p))) return e;
    if ((e = launch_dss<Real>(h->lat, p, h->stream))) return e;
  } else {
    if (apply_filter && h->learned) {
      if ((e = enqueue_learned_filter<Real>(h, FA, FA, true))) return e;
      apply_filter = false;
    }
    // the first stage of the whole-element kernel writes f0 + B dt L f0 at interior nodes
    p.stage = 1; p.A = Real(0); p.B = Real(1.0 / 3.0);
    p.apply_filter = apply_filter ? 1 : 0;
    p.fin = FA; p.f0 = F0; p.fout = F1; p.f0out = F0;
    if ((e = launch_stage_any<Real>(h, p))) return e;
    // shared nodes: A b + B (f0 + ...) with b = 2/3 f0
    if ((e = launch_combine<Real>(nv, F0, F0, F0, F0, 1, third, F0, 0.0, BS, GS, h->stream))) return e;
    KParams<Real> q = p;
    q.A = Real(1); q.fin = F0; q.f0 = BS;
    if ((e = launch_dss<Real>(h->lat, q, h->stream))) return e;
  }
  // stages 2-4; with scheme 2 the difference arguments (stages 2 and 4) take L without its
  // source terms: no F*, walls at rest
  const KParams<Real> full = p;
  const double cs[3] = {-0.75, 2.0 / 3.0, -0.25};
  const double comb[3][4] = {{1, -1, 0, 0}, {1, -1, 1, 0}, {1, -1, 1, -1}};
  Real *base[3] = {F1, F2, F3};
  Real *outs[3] = {F2, F3, FA};
  for (int s = 0; s < 3; ++s) {
    if ((e = launch_combine<Real>(nv, F0, F1, F2, F3, s + 2, comb[s], base[s], cs[s], GS, BS, h->stream))) return e;
    p.stage = 2; p.A = Real(1); p.B = Real(cs[s]); p.apply_filter = 0;
    p.fin = GS; p.f0 = BS; p.fout = outs[s]; p.f0out = nullptr;
    const bool diff = h->scheme == 2 && s != 1;
    p.has_force = diff ? 0 : full.has_force;
    p.fS = diff ? nullptr : full.fS;
    p.wall_u = diff ? (const Real *)h->d_wall_u0 : full.wall_u;
    if (h->use_split) e = launch_split_stage<Real>(h, p);
    else e = launch_stage_any<Real>(h, p);
    if (e) return e;
    if ((e = launch_dss<Real>(h->lat, p, h->stream))) return e;
  }
  return cudaSuccess;
}

// one time step: three stages, each = element kernel + assembly kernel
template <typename Real>
cudaError_t enqueue_step(selbm *h, bool apply_filter) {
  if (h->field_on) {
    // time factor of the acceleration field for this step (device clock, so that graph
    // replays advance it)
    cudaError_t e = launch_force_amp<Real>(h->d_ft, (Real *)h->d_famp, h->dt, h->f_period, h->f_tend, h->stream);
    if (e != cudaSuccess) return e;
  }
  if (h->scheme != 0) return enqueue_step_printed<Real>(h, apply_filter);
  KParams<Real> p = base_params<Real>(h);
  if (h->use_split) return enqueue_step_split<Real>(h, apply_filter);
  Real *FA = (Real *)h->FA, *F0 = (Real *)h->F0, *F2 = (Real *)h->F2;
  // Shu-Osher weights with A = 1 - B formed in the working precision: A + B = 1 exactly, so a
  // stage combination A f0 + B f' of the deviations carries no systematic scale error (with
  // A = fl(1/3), B = fl(2/3) in FP32 the sum is 1 + 3e-8 and the state drifts by that every step)
  const Real B[3] = {Real(1), Real(0.25), Real(2.0 / 3.0)};
  const Real A[3] = {Real(0), Real(1) - B[1], Real(1) - B[2]};
  const Real *fin[3] = {FA, FA, F2};   // element-kernel input f^{s-1} (stage 1: f^3 of the last step)
  Real *fout[3] = {FA, F2, FA};
  cudaError_t e;
  if (apply_filter && h->learned) {
    // the learned control filters the pending state in its own pass; stage 1 then skips the filter
    cudaEvent_t t0 = h->mark_begin();
    if ((e = enqueue_learned_filter<Real>(h, FA, FA, true))) return e;
    h->mark_end(3, t0);
    apply_filter = false;
  }
  for (int s = 0; s < 3; ++s) {
    p.stage = s + 1; p.A = A[s]; p.B = B[s];
    p.apply_filter = (s == 0 && apply_filter) ? 1 : 0;
    p.fin = fin[s]; p.f0 = F0; p.fout = fout[s]; p.f0out = F0;
    cudaEvent_t t0 = h->mark_begin();
    if ((e = launch_stage_any<Real>(h, p))) return e;
    h->mark_end(s == 0 ? 0 : 1, t0);
    KParams<Real> q = p;
    q.fin = (s == 0) ? F0 : fin[s];      // assembly: f^{s-1} on shared nodes (stage 1: f^0)
    t0 = h->mark_begin();
    if ((e = launch_dss<Real>(h->lat, q, h->stream))) return e;
    h->mark_end(2, t0);
  }
  return cudaSuccess;
}

template <typename Real>
cudaError_t enqueue_finalize(selbm *h) {
  KParams<Real> p = base_params<Real>(h);
  p.fin = (const Real *)h->FA;
  p.fout = (Real *)h->BUF;
  if (h->filter_pending && h->learned) return enqueue_learned_filter<Real>(h, (const Real *)h->FA, (Real *)h->BUF, false);
  p.apply_filter = (h->filter_pending && h->filter_on) ? 1 : 0;
  return launch_finalize<Real>(h->lat, p, h->stream);
}

int set_filter_internal(selbm *h, const selbm_filter &f) {
  h->invalidate_graph();
  if (f.gamma != 0.0 && !(f.kc >= 1.0 && f.kc < h->S.N)) return h->fail(SELBM_ERR_ARG, "filter kc must satisfy 1 <= kc < N");
  if (f.gamma < 0.0 || f.gamma > 1.0) return h->fail(SELBM_ERR_ARG, "filter gamma must be in [0, 1]");
  h->P.filter = f;
  build_filter(h->S.gll, f, &h->Fmat, &h->sigma);
  build_filter_lowrank(h->S.gll, f, &h->FU, &h->FW, &h->Fr);
  h->filter_on = f.gamma != 0.0;
  cudaError_t e;
  if (h->prec == SELBM_FP64)
    e = cudaMemcpyAsync(h->d_F, h->Fmat.data(), h->Fmat.size() * 8, cudaMemcpyHostToDevice, h->stream);
  else {
    std::vector<float> ff(h->Fmat.begin(), h->Fmat.end());
    e = cudaMemcpyAsync(h->d_F, ff.data(), ff.size() * 4, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) {
    if (h->prec == SELBM_FP64) e = cudaMemcpy(h->d_fixsig, h->sigma.data(), h->sigma.size() * 8, cudaMemcpyHostToDevice);
    else {
      std::vector<float> sg(h->sigma.begin(), h->sigma.end());
      e = cudaMemcpy(h->d_fixsig, sg.data(), sg.size() * 4, cudaMemcpyHostToDevice);
    }
  }
  if (e != cudaSuccess) return h->cuda_fail(e, "set_filter");
  return SELBM_OK;
}

// SELBM_OK_FALLBACK when the learned control is on and its drift fallback has tripped (reads
// the device flag: the caller has synchronised the stream), else SELBM_OK
int fallback_status(selbm *h) {
  if (!h->learned) return SELBM_OK;
  int flag = 0;
  cudaError_t e = cudaMemcpy(&flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return h->cuda_fail(e, "fallback flag");
  return flag ? SELBM_OK_FALLBACK : SELBM_OK;
}

int ensure_io(selbm *h, size_t bytes) {
  if (h->io_bytes >= bytes) return SELBM_OK;
  if (h->d_io) cudaFree(h->d_io);
  h->d_io = nullptr; h->io_bytes = 0;
  cudaError_t e = cudaMalloc((void **)&h->d_io, bytes);
  if (e != cudaSuccess) return h->cuda_fail(e, "io buffer");
  h->io_bytes = bytes;
  return SELBM_OK;
}

}  // namespace

// shared body of selbm_create / selbm_create_nodes: `setup` fills the handle's Setup
template <typename SetupFn>
static int create_impl(SetupFn setup, const selbm_params *params, void *cuda_stream, selbm_t **out) {
  if (out) *out = nullptr;
  if (!params || !out) { g_create_error = "NULL argument"; return SELBM_ERR_ARG; }
  if (params->precision != SELBM_FP64 && params->precision != SELBM_FP32DEV) { g_create_error = "unknown precision"; return SELBM_ERR_ARG; }
  if (!(params->nu > 0.0)) { g_create_error = "nu must be positive"; return SELBM_ERR_ARG; }
  selbm *h = new selbm();
  h->P = *params;
  h->stream = (cudaStream_t)cuda_stream;
  h->lat = params->lattice;
  h->prec = params->precision;
  h->rsz = h->prec == SELBM_FP64 ? 8 : 4;
  {
    const char *gk = std::getenv("SELBM_GENERIC_KERNEL");
    h->use_fast = !(gk && gk[0] == '1');
    const char *ng = std::getenv("SELBM_NO_GRAPH");
    h->graph_enabled = !(ng && ng[0] == '1');
  }
  std::string err;
  int rc = setup(&h->S, &err);
  if (rc != SELBM_OK) { g_create_error = err; delete h; return rc; }
  Setup &S = h->S;
  h->Q = S.lat.Q;
  {
    const char *sp = std::getenv("SELBM_SPLIT");
    const bool ok = h->use_fast && S.dim == 3 && split_compiled(h->lat, S.N);
    h->use_split = ok && (sp && sp[0] ? sp[0] == '1' : true);
  }
  const size_t smem = stage_smem_bytes(h->lat, S.Np, S.n1, h->rsz);
  if (smem > 227 * 1024) { g_create_error = "element tile does not fit in shared memory (use FP32 or a lower order)"; delete h; return SELBM_ERR_ARG; }
  h->dt = params->dt > 0.0 ? params->dt : params->cfl * S.min_spacing;
  if (!(h->dt > 0.0)) { g_create_error = "time step must be positive"; delete h; return SELBM_ERR_ARG; }
  h->lam = params->nu / kCs2;
  h->tau = h->lam / h->dt;
  h->omega = 1.0 / (h->tau + 0.5);
  h->has_force = params->body_accel[0] != 0.0 || params->body_accel[1] != 0.0 || params->body_accel[2] != 0.0;
  std::call_once(g_const_once, upload_lattice_constants);
  cudaError_t e = cudaSuccess;
#define CK(x) do { if ((e = (x)) != cudaSuccess) { g_create_error = std::string(#x) + ": " + cudaGetErrorString(e); selbm_destroy(h); return SELBM_ERR_CUDA; } } while (0)
  CK(upload(&h->d_l2g, S.l2g));
  CK(upload(&h->d_owner, S.owner));
  CK(upload(&h->d_bslot, S.bslot));
  CK(upload(&h->d_bnode_g, S.bnode_g));
  CK(upload(&h->d_bnode_off, S.bnode_off));
  CK(upload(&h->d_bnode_slot, S.bnode_slot));
  CK(upload(&h->d_first, S.first_copy));
  CK(upload(&h->d_mass, S.mass));
  CK(cudaMalloc((void **)&h->d_partial, diag_blocks() * 6 * sizeof(double)));
  CK(cudaMalloc((void **)&h->d_diag, 8 * sizeof(double)));
  CK(cudaMemset(h->d_diag, 0, 8 * sizeof(double)));
  if (h->prec == SELBM_FP64) CK(upload_real<double>(h)); else CK(upload_real<float>(h));
#undef CK
  rc = set_filter_internal(h, params->filter);
  if (rc != SELBM_OK) { g_create_error = h->err; selbm_destroy(h); return rc; }
  *out = h;
  return SELBM_OK;
}

static int mesh_check_out(const Setup &S, int64_t out_i[6], double out_d[4]) {
  if (out_i) {
    out_i[0] = S.E; out_i[1] = S.Np; out_i[2] = S.lat.Q; out_i[3] = S.G; out_i[4] = S.Gb; out_i[5] = S.affine ? 1 : 0;
  }
  if (out_d) {
    double m = 0.0, ws = 0.0;
    for (double v : S.mass) m += v;
    for (const WallNode &w : S.walls) ws += w.wsJs;
    out_d[0] = S.min_spacing; out_d[1] = m; out_d[2] = (double)S.walls.size(); out_d[3] = ws;
  }
  return SELBM_OK;
}

// ===========================================================================
extern "C" {

int selbm_create(const selbm_mesh *mesh, const selbm_params *params, void *cuda_stream, selbm_t **out) {
  if (out) *out = nullptr;
  if (!mesh) { g_create_error = "NULL argument"; return SELBM_ERR_ARG; }
  return create_impl([&](Setup *S, std::string *err) { return build_setup(*mesh, params->lattice, params->order, S, err); },
                     params, cuda_stream, out);
}

int selbm_create_nodes(const selbm_mesh_nodes *mesh, const selbm_params *params, void *cuda_stream, selbm_t **out) {
  if (out) *out = nullptr;
  if (!mesh) { g_create_error = "NULL argument"; return SELBM_ERR_ARG; }
  return create_impl(
      [&](Setup *S, std::string *err) { return build_setup_nodes(*mesh, params->lattice, params->order, S, err); },
      params, cuda_stream, out);
}

void selbm_destroy(selbm_t *h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  h->invalidate_graph();
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (auto &u : h->ev_used) { cudaEventDestroy(u.second.first); cudaEventDestroy(u.second.second); }
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  for (void *p : h->allocs) cudaFree(p);
  void *own[] = {h->d_l2g, h->d_owner, h->d_bslot, h->d_bnode_g, h->d_bnode_off, h->d_bnode_slot, h->d_first,
                 h->d_mass, h->d_partial, h->d_diag, h->d_io, h->d_xg};
  for (void *p : own)
    if (p) cudaFree(p);
  delete h;
}

const char *selbm_last_error(const selbm_t *h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int selbm_info(const selbm_t *h, int64_t out_i[9], double out_d[4]) {
  if (!h) return SELBM_ERR_ARG;
  if (out_i) {
    out_i[0] = h->S.E; out_i[1] = h->S.Np; out_i[2] = h->Q; out_i[3] = h->S.G;
    out_i[4] = h->S.dim; out_i[5] = h->S.N; out_i[6] = h->prec; out_i[7] = h->steps;
    out_i[8] = h->use_split ? 1 : 0;
  }
  if (out_d) { out_d[0] = h->dt; out_d[1] = h->tau; out_d[2] = h->lam; out_d[3] = h->time; }
  return SELBM_OK;
}

int selbm_lattice_table(const selbm_t *h, int32_t *e, double *t, int32_t *opp) {
  if (!h) return SELBM_ERR_ARG;
  for (int a = 0; a < h->Q; ++a) {
    if (e) for (int k = 0; k < 3; ++k) e[3 * a + k] = h->S.lat.e[3 * a + k];
    if (t) t[a] = h->S.lat.t[a];
    if (opp) opp[a] = h->S.lat.opp[a];
  }
  return SELBM_OK;
}

int selbm_node_coords(const selbm_t *h, double *xyz) {
  if (!h || !xyz) return SELBM_ERR_ARG;
  std::memcpy(xyz, h->S.X.data(), h->S.X.size() * sizeof(double));
  return SELBM_OK;
}

int selbm_init(selbm_t *h, const double *rho, const double *u, int on_device) {
  if (!h || !rho || !u) return SELBM_ERR_ARG;
  const size_t nl = h->nloc(), d = h->S.dim;
  const double *drho = rho, *du = u;
  if (!on_device) {
    int rc = ensure_io(h, nl * (1 + d) * sizeof(double));
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(h->d_io, rho, nl * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_io + nl, u, nl * d * 8, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "init copy");
    drho = h->d_io; du = h->d_io + nl;
  }
  double g[3] = {h->P.body_accel[0], h->P.body_accel[1], h->P.body_accel[2]};
  // the acceleration field enters the initial state with its time factor at t = 0
  const double amp0 = !h->field_on || !(0.0 < h->f_tend) ? 0.0 : (h->f_period > 0.0 ? 0.0 : 1.0);
  cudaError_t e = h->prec == SELBM_FP64
                      ? launch_init<double>(h->lat, drho, du, h->d_first, h->S.G, h->Gs(), h->P.rho0, 0.5 * h->dt, g, h->has_force,
                                            h->field_on ? (const double *)h->d_fS : nullptr, amp0, (double *)h->FA, h->stream)
                      : launch_init<float>(h->lat, drho, du, h->d_first, h->S.G, h->Gs(), h->P.rho0, 0.5 * h->dt, g, h->has_force,
                                           h->field_on ? (const float *)h->d_fS : nullptr, amp0, (float *)h->FA, h->stream);
  if (e == cudaSuccess && h->d_ft) {
    h->ft_host = 0.0;
    e = cudaMemcpyAsync(h->d_ft, &h->ft_host, sizeof(double), cudaMemcpyHostToDevice, h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "init");
  h->initialized = true; h->filter_pending = false; h->steps = 0; h->time = 0.0;
  return SELBM_OK;
}

int selbm_set_state(selbm_t *h, const double *f, int on_device) {
  if (!h || !f) return SELBM_ERR_ARG;
  const size_t nl = h->nloc(), bytes = (size_t)h->Q * nl * 8;
  const double *df = f;
  if (!on_device) {
    int rc = ensure_io(h, bytes);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(h->d_io, f, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "set_state copy");
    df = h->d_io;
  }
  cudaError_t e = h->prec == SELBM_FP64
                      ? launch_set_state<double>(h->lat, df, h->d_first, h->S.G, h->Gs(), nl, h->P.rho0, (double *)h->FA, h->stream)
                      : launch_set_state<float>(h->lat, df, h->d_first, h->S.G, h->Gs(), nl, h->P.rho0, (float *)h->FA, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "set_state");
  h->initialized = true; h->filter_pending = false;
  return SELBM_OK;
}

static int finalize(selbm *h) {
  cudaError_t e = h->prec == SELBM_FP64 ? enqueue_finalize<double>(h) : enqueue_finalize<float>(h);
  if (e != cudaSuccess) return h->cuda_fail(e, "finalize");
  return SELBM_OK;
}

int selbm_get_state(selbm_t *h, double *f, int on_device) {
  if (!h || !f) return SELBM_ERR_ARG;
  if (!h->initialized) return h->fail(SELBM_ERR_STATE, "state not initialised");
  int rc = finalize(h);
  if (rc) return rc;
  const size_t nl = h->nloc(), bytes = (size_t)h->Q * nl * 8;
  double *df = f;
  if (!on_device) {
    if ((rc = ensure_io(h, bytes))) return rc;
    df = h->d_io;
  }
  cudaError_t e = h->prec == SELBM_FP64
                      ? launch_get_state<double>(h->lat, (const double *)h->BUF, h->d_l2g, h->Gs(), nl, h->P.rho0, df, h->stream)
                      : launch_get_state<float>(h->lat, (const float *)h->BUF, h->d_l2g, h->Gs(), nl, h->P.rho0, df, h->stream);
  if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(f, df, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "get_state");
  return SELBM_OK;
}

// capture one step of the given variant into a graph (after one eager step of that
// variant has set the kernels' attributes); any failure leaves the handle on eager launches
static void build_step_graph(selbm *h, int slot) {
  if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    h->graph_enabled = false;
    return;
  }
  cudaGraph_t g = nullptr;
  cudaStream_t user = h->stream;
  h->stream = h->cap_stream;
  cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
  cudaError_t e2 = cudaSuccess;
  if (e == cudaSuccess) {
    e2 = h->prec == SELBM_FP64 ? enqueue_step<double>(h, slot == 1) : enqueue_step<float>(h, slot == 1);
    e = cudaStreamEndCapture(h->cap_stream, &g);
  }
  h->stream = user;
  if (e == cudaSuccess && e2 == cudaSuccess && g) e = cudaGraphInstantiate(&h->gexec[slot], g, 0);
  else e = cudaErrorUnknown;
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->gexec[slot] = nullptr;
    h->graph_enabled = false;
    cudaGetLastError();
  }
}

int selbm_step(selbm_t *h, int64_t nsteps) {
  if (!h) return SELBM_ERR_ARG;
  if (!h->initialized) return h->fail(SELBM_ERR_STATE, "state not initialised");
  if (nsteps < 0) return h->fail(SELBM_ERR_ARG, "nsteps < 0");
  for (int64_t k = 0; k < nsteps; ++k) {
    const bool filt = h->filter_pending && (h->filter_on || h->learned);
    const int slot = filt ? 1 : 0;
    cudaError_t e = cudaSuccess;
    const bool graphable = h->graph_enabled && !h->timing;
    if (graphable && !h->gexec[slot] && h->eager_steps[slot] > 0) build_step_graph(h, slot);
    if (graphable && h->gexec[slot]) {
      e = cudaGraphLaunch(h->gexec[slot], h->stream);
    } else {
      e = h->prec == SELBM_FP64 ? enqueue_step<double>(h, filt) : enqueue_step<float>(h, filt);
      h->eager_steps[slot]++;
    }
    if (e != cudaSuccess) return h->cuda_fail(e, "step");
    h->filter_pending = true;
    h->steps++;
    h->time += h->dt;
  }
  return SELBM_OK;
}

int selbm_moments(selbm_t *h, double *rho, double *u, int on_device) {
  if (!h || !rho || !u) return SELBM_ERR_ARG;
  if (!h->initialized) return h->fail(SELBM_ERR_STATE, "state not initialised");
  int rc = finalize(h);
  if (rc) return rc;
  const size_t nl = h->nloc(), d = h->S.dim;
  double *dr = rho, *du = u;
  if (!on_device) {
    if ((rc = ensure_io(h, nl * (1 + d) * 8))) return rc;
    dr = h->d_io; du = h->d_io + nl;
  }
  cudaError_t e = h->prec == SELBM_FP64
                      ? launch_moments<double>(h->lat, (const double *)h->BUF, h->d_l2g, h->Gs(), nl, h->P.rho0, dr, du, h->stream)
                      : launch_moments<float>(h->lat, (const float *)h->BUF, h->d_l2g, h->Gs(), nl, h->P.rho0, dr, du, h->stream);
  if (e == cudaSuccess && !on_device) {
    e = cudaMemcpyAsync(rho, dr, nl * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(u, du, nl * d * 8, cudaMemcpyDeviceToHost, h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "moments");
  return SELBM_OK;
}

int selbm_stress(selbm_t *h, double *pi, int on_device) {
  if (!h || !pi) return SELBM_ERR_ARG;
  if (!h->initialized) return h->fail(SELBM_ERR_STATE, "state not initialised");
  int rc = finalize(h);
  if (rc) return rc;
  const size_t nl = h->nloc(), d = h->S.dim, n = nl * d * d;
  double *dp = pi;
  if (!on_device) {
    if ((rc = ensure_io(h, n * 8))) return rc;
    dp = h->d_io;
  }
  // the acceleration field's time factor at the read-back time
  const double t = h->time;
  const double amp = !h->field_on || !(t < h->f_tend)
                         ? 0.0
                         : (h->f_period > 0.0 ? std::sin(2.0 * 3.14159265358979323846 * t / h->f_period) : 1.0);
  const double factor = h->tau / (h->tau + 0.5);
  const double *g = h->P.body_accel;
  cudaError_t e = h->prec == SELBM_FP64
                      ? launch_stress<double>(h->lat, (const double *)h->BUF, h->d_l2g, h->S.G, h->Gs(), nl, h->P.rho0, 0.5 * h->dt,
                                              factor, g, h->has_force, h->field_on ? (const double *)h->d_fS : nullptr,
                                              amp, dp, h->stream)
                      : launch_stress<float>(h->lat, (const float *)h->BUF, h->d_l2g, h->S.G, h->Gs(), nl, h->P.rho0, 0.5 * h->dt,
                                             factor, g, h->has_force, h->field_on ? (const float *)h->d_fS : nullptr,
                                             amp, dp, h->stream);
  if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(pi, dp, n * 8, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "stress");
  return SELBM_OK;
}

int selbm_set_filter(selbm_t *h, const selbm_filter *f) {
  if (!h || !f) return SELBM_ERR_ARG;
  if (h->filter_pending && (h->filter_on || h->learned)) {
    // the last step's filter (old settings) must be applied before switching
    int rc = finalize(h);
    if (rc) return rc;
    size_t bytes = (size_t)h->Q * h->Gs() * h->rsz;
    cudaError_t e = cudaMemcpyAsync(h->FA, h->BUF, bytes, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "set_filter");
    h->filter_pending = false;
  }
  return set_filter_internal(h, *f);
}

int selbm_set_body_force(selbm_t *h, const double g[3]) {
  if (!h || !g) return SELBM_ERR_ARG;
  for (int k = 0; k < 3; ++k) h->P.body_accel[k] = g[k];
  h->has_force = g[0] != 0.0 || g[1] != 0.0 || g[2] != 0.0 || h->field_on;
  h->invalidate_graph();
  return SELBM_OK;
}

int selbm_set_time_scheme(selbm_t *h, int scheme) {
  if (!h) return SELBM_ERR_ARG;
  if (scheme < 0 || scheme > 2) return h->fail(SELBM_ERR_ARG, "time scheme must be 0, 1 or 2");
  if (scheme != 0) {
    // allocate whichever stage buffers are still missing (a failed call leaves the rest for
    // the next one)
    const size_t bytes = (size_t)h->Q * h->Gs() * h->rsz;
    void **bufs[4] = {&h->S1, &h->S2, &h->SG, &h->SB};
    for (void **b : bufs) {
      if (*b) continue;
      cudaError_t e = cudaMalloc(b, bytes);
      if (e != cudaSuccess) {
        *b = nullptr;
        return h->cuda_fail(e, "time scheme buffers");
      }
      h->allocs.push_back(*b);
    }
  }
  h->scheme = scheme;
  h->invalidate_graph();
  return SELBM_OK;
}

int selbm_set_force_field(selbm_t *h, const double *S, double period, double t_end) {
  if (!h) return SELBM_ERR_ARG;
  const double *ga = h->P.body_accel;
  if (!S) {
    h->field_on = false;
    h->has_force = ga[0] != 0.0 || ga[1] != 0.0 || ga[2] != 0.0;
    h->invalidate_graph();
    return SELBM_OK;
  }
  if (std::isnan(period) || std::isnan(t_end)) return h->fail(SELBM_ERR_ARG, "force field period / t_end is NaN");
  const size_t G = (size_t)h->S.G, nl = h->nloc(), d = h->S.dim;
  cudaError_t e = cudaSuccess;
  // allocate whichever of the field buffers are still missing
  struct { void **ptr; size_t bytes; } need[3] = {{&h->d_fS, 3 * G * h->rsz}, {&h->d_famp, 16},
                                                  {(void **)&h->d_ft, sizeof(double)}};
  for (auto &b : need) {
    if (*b.ptr) continue;
    if ((e = cudaMalloc(b.ptr, b.bytes)) != cudaSuccess) {
      *b.ptr = nullptr;
      return h->cuda_fail(e, "force field alloc");
    }
    h->allocs.push_back(*b.ptr);
  }
  int rc = ensure_io(h, nl * d * sizeof(double));
  if (rc) return rc;
  e = cudaMemcpyAsync(h->d_io, S, nl * d * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = h->prec == SELBM_FP64 ? launch_force_field<double>(h->d_io, h->d_first, (int)G, (int)d, (double *)h->d_fS, h->stream)
                              : launch_force_field<float>(h->d_io, h->d_first, (int)G, (int)d, (float *)h->d_fS, h->stream);
  h->ft_host = h->time;
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_ft, &h->ft_host, sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "force field");
  h->f_period = period;
  h->f_tend = t_end;
  h->field_on = true;
  h->has_force = true;
  h->invalidate_graph();
  return SELBM_OK;
}

int selbm_diagnostics(selbm_t *h, double out[8]) {
  if (!h || !out) return SELBM_ERR_ARG;
  if (!h->initialized) return h->fail(SELBM_ERR_STATE, "state not initialised");
  int rc = finalize(h);
  if (rc) return rc;
  cudaError_t e = h->prec == SELBM_FP64
                      ? launch_diag<double>(h->lat, (const double *)h->BUF, h->d_mass, h->S.G, h->Gs(), h->P.rho0, h->d_partial, h->d_diag, h->stream)
                      : launch_diag<float>(h->lat, (const float *)h->BUF, h->d_mass, h->S.G, h->Gs(), h->P.rho0, h->d_partial, h->d_diag, h->stream);
  // dissipation: velocity at local nodes, then per-element gradient integrals
  const size_t nl = h->nloc(), dim = h->S.dim;
  double *d_eps = nullptr;
  if (e == cudaSuccess && ensure_io(h, nl * (1 + dim) * 8 + (h->S.E + 1) * 8) != SELBM_OK) e = cudaErrorMemoryAllocation;
  if (e == cudaSuccess) {
    double *rho_l = h->d_io, *u_l = h->d_io + nl, *part = h->d_io + nl * (1 + dim);
    d_eps = h->d_diag + 6;
    const double mu = h->P.rho0 * h->P.nu;
    e = h->prec == SELBM_FP64
            ? launch_moments<double>(h->lat, (const double *)h->BUF, h->d_l2g, h->Gs(), nl, h->P.rho0, rho_l, u_l, h->stream)
            : launch_moments<float>(h->lat, (const float *)h->BUF, h->d_l2g, h->Gs(), nl, h->P.rho0, rho_l, u_l, h->stream);
    if (e == cudaSuccess)
      e = h->prec == SELBM_FP64
              ? launch_eps<double>(u_l, (int)dim, h->S.n1, h->S.Np, h->S.E, h->S.affine, (const double *)h->d_el_drdx,
                                   (const double *)h->d_drdx, (const double *)h->d_el_J, (const double *)h->d_wJ,
                                   (const double *)h->d_gllw, (const double *)h->d_D, mu, part, d_eps, h->stream)
              : launch_eps<float>(u_l, (int)dim, h->S.n1, h->S.Np, h->S.E, h->S.affine, (const float *)h->d_el_drdx,
                                  (const float *)h->d_drdx, (const float *)h->d_el_J, (const float *)h->d_wJ,
                                  (const float *)h->d_gllw, (const float *)h->d_D, mu, part, d_eps, h->stream);
  }
  double tmp[7];
  if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, h->d_diag, 7 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "diagnostics");
  out[0] = tmp[0];
  for (int k = 0; k < 3; ++k) out[1 + k] = tmp[1 + k];
  out[4] = tmp[4]; out[5] = tmp[6]; out[6] = h->dt; out[7] = h->time;
  if (tmp[5] > 0) return h->fail(SELBM_ERR_NONFINITE, "state holds non-finite values");
  return fallback_status(h);
}

int selbm_wall_stress(selbm_t *h, const double dir[3], double *tau) {
  if (!h || !dir || !tau) return SELBM_ERR_ARG;
  if (!h->initialized) return h->fail(SELBM_ERR_STATE, "state not initialised");
  const int dim = h->S.dim;
  double d[3] = {dir[0], dir[1], dim == 3 ? dir[2] : 0.0}, nrm = 0;
  for (int c = 0; c < dim; ++c) nrm += d[c] * d[c];
  if (!(nrm > 0)) return h->fail(SELBM_ERR_ARG, "wall_stress: zero direction");
  for (int c = 0; c < 3; ++c) d[c] /= std::sqrt(nrm);
  *tau = 0.0;
  if (h->n_wallpts == 0) return SELBM_OK;
  int rc = finalize(h);
  if (rc) return rc;
  const size_t nl = h->nloc();
  if ((rc = ensure_io(h, (nl * (1 + dim) + 2 * (size_t)h->n_wallpts) * 8))) return rc;
  double *rho_l = h->d_io, *u_l = h->d_io + nl, *part = h->d_io + nl * (1 + dim);
  const double mu = h->P.rho0 * h->P.nu;
  cudaError_t e = h->prec == SELBM_FP64
                      ? launch_moments<double>(h->lat, (const double *)h->BUF, h->d_l2g, h->Gs(), nl, h->P.rho0, rho_l, u_l, h->stream)
                      : launch_moments<float>(h->lat, (const float *)h->BUF, h->d_l2g, h->Gs(), nl, h->P.rho0, rho_l, u_l, h->stream);
  if (e == cudaSuccess)
    e = h->prec == SELBM_FP64
            ? launch_wall_stress<double>(u_l, dim, h->S.n1, h->S.Np, h->S.E, h->S.affine, (const double *)h->d_el_drdx,
                                         (const double *)h->d_drdx, (const double *)h->d_D, h->d_walls, h->d_wall_off, d,
                                         mu, part, h->stream)
            : launch_wall_stress<float>(u_l, dim, h->S.n1, h->S.Np, h->S.E, h->S.affine, (const float *)h->d_el_drdx,
                                        (const float *)h->d_drdx, (const float *)h->d_D, h->d_walls, h->d_wall_off, d,
                                        mu, part, h->stream);
  std::vector<double> hp(2 * (size_t)h->n_wallpts);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), part, hp.size() * 8, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "wall_stress");
  double num = 0, den = 0;
  for (int k = 0; k < h->n_wallpts; ++k) { num += hp[2 * k]; den += hp[2 * k + 1]; }
  *tau = den > 0 ? num / den : 0.0;
  return SELBM_OK;
}

int selbm_radial_profile(selbm_t *h, const double origin[3], const double axis[3], double radius, int nbins,
                         double *mean, double *mass) {
  if (!h || !origin || !axis || !mean || !mass) return SELBM_ERR_ARG;
  if (!h->initialized) return h->fail(SELBM_ERR_STATE, "state not initialised");
  if (nbins < 1 || nbins > SELBM_PROFILE_MAX_BINS) return h->fail(SELBM_ERR_ARG, "radial_profile: nbins out of range");
  if (!(radius > 0)) return h->fail(SELBM_ERR_ARG, "radial_profile: radius must be positive");
  const int dim = h->S.dim;
  double a[3] = {axis[0], axis[1], dim == 3 ? axis[2] : 0.0}, nrm = 0;
  for (int c = 0; c < dim; ++c) nrm += a[c] * a[c];
  if (!(nrm > 0)) return h->fail(SELBM_ERR_ARG, "radial_profile: zero axis");
  for (int c = 0; c < 3; ++c) a[c] /= std::sqrt(nrm);
  const double o[3] = {origin[0], origin[1], dim == 3 ? origin[2] : 0.0};
  int rc = finalize(h);
  if (rc) return rc;
  cudaError_t e = cudaSuccess;
  if (!h->d_xg) {
    std::vector<double> xg((size_t)h->S.G * dim);
    for (int g = 0; g < h->S.G; ++g)
      for (int c = 0; c < dim; ++c) xg[(size_t)g * dim + c] = h->S.X[(size_t)h->S.first_copy[g] * dim + c];
    e = upload(&h->d_xg, xg);
    if (e != cudaSuccess) return h->cuda_fail(e, "radial_profile");
  }
  const size_t nl = h->nloc();
  const int blocks = 256;
  if ((rc = ensure_io(h, (nl * (1 + dim) + (size_t)blocks * 2 * nbins) * 8))) return rc;
  double *rho_l = h->d_io, *u_l = h->d_io + nl, *part = h->d_io + nl * (1 + dim);
  e = h->prec == SELBM_FP64
          ? launch_moments<double>(h->lat, (const double *)h->BUF, h->d_l2g, h->Gs(), nl, h->P.rho0, rho_l, u_l, h->stream)
          : launch_moments<float>(h->lat, (const float *)h->BUF, h->d_l2g, h->Gs(), nl, h->P.rho0, rho_l, u_l, h->stream);
  if (e == cudaSuccess)
    e = launch_radial_profile(u_l, dim, h->d_first, h->d_xg, h->d_mass, h->S.G, o, a, radius, nbins, blocks, part,
                              h->stream);
  std::vector<double> hp((size_t)blocks * 2 * nbins);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), part, hp.size() * 8, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "radial_profile");
  for (int b = 0; b < nbins; ++b) {
    double su = 0, sm = 0;
    for (int k = 0; k < blocks; ++k) { su += hp[((size_t)k * nbins + b) * 2]; sm += hp[((size_t)k * nbins + b) * 2 + 1]; }
    mean[b] = sm > 0 ? su / sm : 0.0;
    mass[b] = sm;
  }
  return SELBM_OK;
}

int selbm_mesh_check(const selbm_mesh *mesh, int32_t lattice, int32_t order, int64_t out_i[6], double out_d[4]) {
  if (!mesh) { g_create_error = "NULL mesh"; return SELBM_ERR_ARG; }
  Setup S;
  std::string err;
  int rc = build_setup(*mesh, lattice, order, &S, &err);
  if (rc != SELBM_OK) { g_create_error = err; return rc; }
  return mesh_check_out(S, out_i, out_d);
}

int selbm_mesh_check_nodes(const selbm_mesh_nodes *mesh, int32_t lattice, int32_t order, int64_t out_i[6],
                           double out_d[4]) {
  if (!mesh) { g_create_error = "NULL mesh"; return SELBM_ERR_ARG; }
  Setup S;
  std::string err;
  int rc = build_setup_nodes(*mesh, lattice, order, &S, &err);
  if (rc != SELBM_OK) { g_create_error = err; return rc; }
  return mesh_check_out(S, out_i, out_d);
}


int selbm_timers(selbm_t *h, int enable) {
  if (!h) return SELBM_ERR_ARG;
  cudaStreamSynchronize(h->stream);
  for (auto &u : h->ev_used) { h->ev_pool.push_back(u.second.first); h->ev_pool.push_back(u.second.second); }
  h->ev_used.clear();
  h->timing = enable != 0;
  return SELBM_OK;
}

int selbm_timers_read(selbm_t *h, double ms[SELBM_TIMER_KINDS], int64_t n[SELBM_TIMER_KINDS]) {
  if (!h || !ms || !n) return SELBM_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "timers");
  for (int k = 0; k < SELBM_TIMER_KINDS; ++k) { ms[k] = 0.0; n[k] = 0; }
  for (auto &u : h->ev_used) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, u.second.first, u.second.second) == cudaSuccess) {
      ms[u.first] += t;
      n[u.first] += 1;
    }
    h->ev_pool.push_back(u.second.first);
    h->ev_pool.push_back(u.second.second);
  }
  h->ev_used.clear();
  return SELBM_OK;
}

// ---------------------------------------------------------------------------
// learned per-element filter control
// ---------------------------------------------------------------------------
static uint16_t float_to_bf16_bits(float x) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  if ((b & 0x7F800000u) == 0x7F800000u) return (uint16_t)(b >> 16);   // inf / nan unchanged
  b += 0x7FFFu + ((b >> 16) & 1u);                                    // round to nearest, ties to even
  return (uint16_t)(b >> 16);
}

int selbm_set_learned_filter(selbm_t *h, const float *params, const float *lo, const float *hi, double mass_bound,
                             double ke_bound) {
  if (!h || !params || !lo || !hi) return SELBM_ERR_ARG;
  const int nin = 2 * h->S.n1, P = mlp_nparams(nin);
  if (control_smem_bytes(h->lat, h->S.Np, h->S.n1, h->rsz) > 227 * 1024)
    return h->fail(SELBM_ERR_ARG, "learned filter: element tile does not fit in shared memory (use FP32 or a lower order)");
  for (int i = 0; i < nin; ++i)
    if (!(hi[i] > lo[i])) return h->fail(SELBM_ERR_ARG, "learned filter: hi must exceed lo for every feature");
  if (h->filter_pending && (h->filter_on || h->learned)) {
    // apply the pending filter with the old settings first
    int rc = finalize(h);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(h->FA, h->BUF, (size_t)h->Q * h->Gs() * h->rsz, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "set_learned_filter");
    h->filter_pending = false;
  }
  std::vector<uint16_t> wb(P);
  for (int i = 0; i < P; ++i) wb[i] = float_to_bf16_bits(params[i]);
  cudaError_t e = cudaMemcpyAsync(h->d_W, wb.data(), P * 2, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) {
    if (h->prec == SELBM_FP64) {
      std::vector<double> l(lo, lo + nin), u(hi, hi + nin);
      e = cudaMemcpyAsync(h->d_lo, l.data(), nin * 8, cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_hi, u.data(), nin * 8, cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    } else {
      e = cudaMemcpyAsync(h->d_lo, lo, nin * 4, cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_hi, hi, nin * 4, cudaMemcpyHostToDevice, h->stream);
    }
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_acc, 0, 8 * sizeof(double), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_flag, 0, 2 * sizeof(int), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_nfb, 0, 2 * sizeof(int), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "set_learned_filter");
  h->invalidate_graph();
  h->nin = nin;
  h->mass_bound = mass_bound;
  h->ke_bound = ke_bound;
  h->learned = true;
  return SELBM_OK;
}

int selbm_clear_learned_filter(selbm_t *h) {
  if (!h) return SELBM_ERR_ARG;
  if (h->learned && h->filter_pending) {
    int rc = finalize(h);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(h->FA, h->BUF, (size_t)h->Q * h->Gs() * h->rsz, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "clear_learned_filter");
    h->filter_pending = false;
  }
  h->learned = false;
  h->invalidate_graph();
  return SELBM_OK;
}

int selbm_learned_status(selbm_t *h, int64_t out[4]) {
  if (!h || !out) return SELBM_ERR_ARG;
  int flag[2] = {0, 0}, nfb[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(flag, h->d_flag, sizeof(flag), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(nfb, h->d_nfb, sizeof(nfb), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_nfb, 0, sizeof(nfb), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "learned_status");
  out[0] = flag[0]; out[1] = nfb[0]; out[2] = h->learned ? 1 : 0; out[3] = 0;
  return SELBM_OK;
}

int selbm_element_sigma(selbm_t *h, double *sigma) {
  if (!h || !sigma) return SELBM_ERR_ARG;
  const size_t cnt = (size_t)h->S.E * h->S.n1;
  cudaError_t e;
  if (h->prec == SELBM_FP64) {
    e = cudaMemcpyAsync(sigma, h->d_sigma_e, cnt * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  } else {
    std::vector<float> tmp(cnt);
    e = cudaMemcpyAsync(tmp.data(), h->d_sigma_e, cnt * 4, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    for (size_t i = 0; i < cnt; ++i) sigma[i] = tmp[i];
  }
  if (e != cudaSuccess) return h->cuda_fail(e, "element_sigma");
  return SELBM_OK;
}

int selbm_features(selbm_t *h, float *feat) {
  if (!h || !feat) return SELBM_ERR_ARG;
  if (!h->initialized) return h->fail(SELBM_ERR_STATE, "state not initialised");
  cudaError_t e;
  auto run = [&](auto tag) {
    using Real = decltype(tag);
    const Setup &S = h->S;
    ControlArgs<Real> c{};
    c.E = S.E; c.Np = S.Np; c.n = S.n1; c.N = S.N; c.G = S.G; c.Gs = h->Gs(); c.Nb = S.Nb;
    c.l2g = h->d_l2g; c.bslot = h->d_bslot; c.f = (const Real *)h->FA; c.rho0 = h->P.rho0; c.affine = S.affine ? 1 : 0;
    c.el_J = (const Real *)h->d_el_J; c.wJ = (const Real *)h->d_wJ; c.gllw = (const Real *)h->d_gllw;
    c.Vm = (const Real *)h->d_Vm; c.Vinv = (const Real *)h->d_Vinv; c.W = nullptr; c.sigma_out = nullptr; c.feat_out = feat;
    return launch_control<Real>(h->lat, c, h->stream);
  };
  e = h->prec == SELBM_FP64 ? run(double()) : run(float());
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "features");
  return SELBM_OK;
}

int selbm_element_errors(selbm_t *h, selbm_t *ref, double *err) {
  if (!h || !ref || !err) return SELBM_ERR_ARG;
  if (h->S.E != ref->S.E || h->S.dim != ref->S.dim) return h->fail(SELBM_ERR_ARG, "element_errors: meshes differ");
  const int dim = h->S.dim;
  const size_t nl = h->nloc(), nlr = ref->nloc();
  double *buf = nullptr, *I = nullptr, *wq = nullptr;
  cudaError_t e = cudaMalloc((void **)&buf, (nl + nlr) * (1 + dim) * sizeof(double));
  std::vector<double> Ih;
  build_interp(ref->S.N, h->S.N, &Ih);
  if (e == cudaSuccess) e = cudaMalloc((void **)&I, Ih.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void **)&wq, nl * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(I, Ih.data(), Ih.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(wq, h->S.wJ.data(), nl * sizeof(double), cudaMemcpyHostToDevice);
  int rc = SELBM_OK;
  if (e == cudaSuccess) {
    double *rho = buf, *u = buf + nl, *rhoR = buf + nl * (1 + dim), *uR = rhoR + nlr;
    rc = selbm_moments(h, rho, u, 1);
    if (!rc) rc = selbm_moments(ref, rhoR, uR, 1);
    if (!rc) {
      e = launch_element_errors(h->S.E, dim, h->S.n1, ref->S.n1, rho, u, rhoR, uR, I, wq, err, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
  }
  cudaFree(buf); cudaFree(I); cudaFree(wq);
  if (rc) return rc;
  if (e != cudaSuccess) return h->cuda_fail(e, "element_errors");
  return SELBM_OK;
}

int selbm_mlp_nparams(int32_t nin) { return nin > 0 ? mlp_nparams(nin) : SELBM_ERR_ARG; }

int selbm_mlp_grad(const float *params, int32_t nin, int32_t order, const float *x, const float *y, int64_t M,
                   float *grad, float *loss, void *stream) {
  if (!params || !x || !y || !grad || !loss || nin <= 0 || M <= 0 || order < 4) return SELBM_ERR_ARG;
  return mlp_grad(params, nin, order, x, y, M, grad, loss, (cudaStream_t)stream) == cudaSuccess ? SELBM_OK : SELBM_ERR_CUDA;
}

int selbm_mlp_forward(const float *params, int32_t nin, int32_t order, const float *x, int64_t M, int32_t bf16,
                      float *out, void *stream) {
  if (!params || !x || !out || nin <= 0 || M <= 0 || order < 4) return SELBM_ERR_ARG;
  return mlp_forward(params, nin, order, x, M, bf16, out, (cudaStream_t)stream) == cudaSuccess ? SELBM_OK : SELBM_ERR_CUDA;
}

int selbm_mlp_train(float *params, float *m, float *v, int32_t nin, int32_t order, const float *x, const float *y,
                    int64_t M, int32_t batch, int32_t epochs, float lr, uint64_t seed, int64_t *adam_t,
                    float *loss_hist, void *stream) {
  if (!params || !m || !v || !x || !y || !adam_t || nin <= 0 || M <= 0 || batch <= 0 || epochs < 0 || order < 4)
    return SELBM_ERR_ARG;
  return mlp_train(params, m, v, nin, order, x, y, M, batch, epochs, lr, seed, adam_t, loss_hist, (cudaStream_t)stream) ==
                 cudaSuccess
             ? SELBM_OK
             : SELBM_ERR_CUDA;
}

int selbm_sync(selbm_t *h) {
  if (!h) return SELBM_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "sync");
  return fallback_status(h);
}

}  // extern "C"

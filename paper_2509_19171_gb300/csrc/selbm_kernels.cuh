// Device-side data structures and launch helpers of the filtered SELBM hot path.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdlib>

#include "../../include/selbm.h"

namespace slb {

// One element-local wall node: up to three wall faces meet at a node of a hex.
template <typename Real>
struct WallPt {
  int32_t i, b, nf, wid[3];
  Real n[3][3];
  Real wsJs[3];
};

// Everything a stage / assembly / utility kernel reads.  Passed by value.
template <typename Real>
struct KParams {
  int E, Np, Nb, N, n, G, Gb;
  int Gs;                    // population stride of the state arrays (G rounded up to a multiple of 8)
  int stage;                 // 1, 2, 3
  Real A, B;                 // f^s = A f^0 + B (f^{s-1} + dt L(f^{s-1}))
  Real dt, omega, rho0, half_dt;
  Real g[3];
  int has_force, apply_filter;
  int wall_max;              // most wall nodes on one element (sizes a shared-memory buffer)
  const int32_t *l2g;        // [E][Np]
  const uint8_t *owner;      // [E][Np]
  const int32_t *bslot;      // [Np] boundary slot of each local node, -1 inside
  const Real *el_drdx;       // [E][dim][dim] affine metrics
  const Real *el_J;          // [E]
  const Real *drdx;          // [E][Np][dim][dim] general metrics
  const Real *wJ;            // [E][Np]
  const Real *gllw;          // [n]
  const Real *Dm, *Fm;       // [n][n]
  const WallPt<Real> *walls; // element-grouped wall nodes
  const int32_t *wall_off;   // [E+1]
  const Real *wall_u;        // [nwalls][3]
  const int32_t *bnode_g, *bnode_off, *bnode_slot;
  const Real *bnode_minv;    // [Gb] 1 / assembled mass
  const Real *fin;           // f^{s-1} on unique nodes [Q][G]
  const Real *f0;            // f^0 [Q][G]
  Real *fout;                // f^s [Q][G]
  Real *f0out;               // stage 1: f^0 written by owners
  Real *T;                   // assembly trace [Q][E*Nb]
  Real *rho;                 // [G] density of the step (forcing)
  const Real *fS;            // [3][G] extra acceleration field S on unique nodes, or NULL
  const Real *famp;          // [1] its time factor A(t) for the current step (device)
};

// body acceleration at unique node g: g + A(t) S_g (Sec. 4, pipe perturbation force)
template <typename Real>
__device__ __forceinline__ void node_accel(const KParams<Real> &p, size_t g, Real (&acc)[3]) {
  acc[0] = p.g[0];
  acc[1] = p.g[1];
  acc[2] = p.g[2];
  if (p.fS) {
    const Real A = *p.famp;
    const size_t G = (size_t)p.G;
    acc[0] += A * p.fS[g];
    acc[1] += A * p.fS[G + g];
    acc[2] += A * p.fS[2 * G + g];
  }
}

// Launchers (defined in selbm_kernels.cu).  lat = SELBM_D2Q9 / D3Q19 / D3Q27.
template <typename Real>
cudaError_t launch_stage(int lat, bool affine, const KParams<Real> &p, cudaStream_t s);
template <typename Real>
cudaError_t launch_dss(int lat, const KParams<Real> &p, cudaStream_t s);
// filtered copy of fin into fout on unique nodes (owners write)
template <typename Real>
cudaError_t launch_finalize(int lat, const KParams<Real> &p, cudaStream_t s);

template <typename Real>
cudaError_t launch_init(int lat, const double *rho, const double *u, const int32_t *first, int G, int Gs, double rho0,
                        double half_dt, const double g[3], int has_force, const Real *fS, double amp, Real *out,
                        cudaStream_t s);
// g = sum_{i < m} c_i f_i and b = base - cb g over n values (m <= 4): the argument of a stage
// of the printed four-stage scheme and the base that makes A b + B (g + dt L g) with A = 1,
// B = cb equal to base + cb dt L g
template <typename Real>
cudaError_t launch_combine(size_t n, const Real *f0, const Real *f1, const Real *f2, const Real *f3, int m,
                           const double c[4], const Real *base, double cb, Real *g, Real *b, cudaStream_t s);
// per-node acceleration field: fS[k][g] = S[first[g]][k] (k < dim), 0 for k >= dim
template <typename Real>
cudaError_t launch_force_field(const double *S, const int32_t *first, int G, int dim, Real *fS, cudaStream_t s);
// non-equilibrium second moment at every local node, out [nloc][dim][dim]
template <typename Real>
cudaError_t launch_stress(int lat, const Real *buf, const int32_t *l2g, int G, int Gs, size_t nloc, double rho0, double half_dt,
                          double factor, const double g[3], int has_force, const Real *fS, double amp, double *out,
                          cudaStream_t s);
// time factor of the field for the step starting at ft[0]; advances ft[0] by dt
template <typename Real>
cudaError_t launch_force_amp(double *ft, Real *amp, double dt, double period, double t_end, cudaStream_t s);
template <typename Real>
cudaError_t launch_set_state(int lat, const double *f, const int32_t *first, int G, int Gs, size_t nloc, double rho0, Real *out, cudaStream_t s);
template <typename Real>
cudaError_t launch_get_state(int lat, const Real *buf, const int32_t *l2g, int Gs, size_t nloc, double rho0, double *f, cudaStream_t s);
template <typename Real>
cudaError_t launch_moments(int lat, const Real *buf, const int32_t *l2g, int Gs, size_t nloc, double rho0, double *rho, double *u, cudaStream_t s);
int diag_blocks();
template <typename Real>
cudaError_t launch_diag(int lat, const Real *buf, const double *mass, int G, int Gs, double rho0, double *partial, double *out, cudaStream_t s);

// host copies of the matrices of the register-blocked stage kernel
struct FastHost {
  const double *D, *U, *W, *w;   // D_hat [n][n]; filter F = I + U W (U n x r, W r x n, stride n); GLL weights
  int r;
};
template <typename Real>
bool launch_fast_d2q9(int N, bool affine, const KParams<Real> &p, const FastHost &f, cudaStream_t s, cudaError_t *err);
template <typename Real>
bool launch_fast_d3q19(int N, bool affine, const KParams<Real> &p, const FastHost &f, cudaStream_t s, cudaError_t *err);
template <typename Real>
bool launch_fast_d3q27(int N, bool affine, const KParams<Real> &p, const FastHost &f, cudaStream_t s, cudaError_t *err);

// population-split step (3D; orders compiled for D3Q19: 4, 7 and D3Q27: 5, 7)
struct SplitHost {
  const double *D, *U, *W, *w;   // D_hat; fixed filter F = I + U W; GLL weights
  int r;
  const double *Vm, *Vinv, *fixed_sigma;   // modal <-> nodal; transfer function of the fixed filter
};
template <typename Real>
struct LearnedPtrs {
  const __nv_bfloat16 *W;        // network parameters; NULL = features only
  const Real *lo, *hi;           // [2n] training range of the features
  const int *flag;               // sticky drift fallback flag or NULL
  double *acc;                   // drift accumulators or NULL
  Real *sigma_out;               // [E][n] or NULL
  float *feat_out;               // [E][2n] or NULL
  int *n_fallback;               // elements that kept the fixed filter, or NULL
  int outputs;                   // 0: features / transfer functions only
};
enum { PRO_FIXED = 1, PRO_LEARNED = 2 };
template <typename Real>
bool split_stage_d3q19(int N, bool affine, const KParams<Real> &p, const SplitHost &h, cudaStream_t s, cudaError_t *err);
template <typename Real>
bool split_stage_d3q27(int N, bool affine, const KParams<Real> &p, const SplitHost &h, cudaStream_t s, cudaError_t *err);
template <typename Real>
bool split_prologue_d3q19(int N, bool affine, int mode, const KParams<Real> &p, const SplitHost &h,
                          const LearnedPtrs<Real> &lp, cudaStream_t s, cudaError_t *err);
template <typename Real>
bool split_prologue_d3q27(int N, bool affine, int mode, const KParams<Real> &p, const SplitHost &h,
                          const LearnedPtrs<Real> &lp, cudaStream_t s, cudaError_t *err);
// learned control of the split form: rho - rho0 and |u| on unique nodes into q [2][Gs] (+ the
// drift integrals into lp.acc), element features X [E][2n], then the network -> lp.sigma_out [E][n]
template <typename Real>
bool split_control_d3q19(int N, const KParams<Real> &p, const SplitHost &h, const LearnedPtrs<Real> &lp, Real *q,
                         Real *X, const double *mass, cudaStream_t s, cudaError_t *err);
template <typename Real>
bool split_control_d3q27(int N, const KParams<Real> &p, const SplitHost &h, const LearnedPtrs<Real> &lp, Real *q,
                         Real *X, const double *mass, cudaStream_t s, cudaError_t *err);
// which: 0 collision on unique nodes (writes fout -> f0out), 1 assembly of the learned
// filter's weighted shares at shared nodes + collision
template <typename Real>
cudaError_t split_collide_d3q19(int which, const KParams<Real> &p, cudaStream_t s);
template <typename Real>
cudaError_t split_collide_d3q27(int which, const KParams<Real> &p, cudaStream_t s);
inline bool split_compiled(int lat, int N) {
  return (lat == SELBM_D3Q19 && (N == 4 || N == 7)) || (lat == SELBM_D3Q27 && (N == 5 || N == 7));
}

// pipe statistics (selbm_stats.cu)
template <typename Real>
cudaError_t launch_wall_stress(const double *u, int dim, int n, int Np, int E, int affine, const Real *el_drdx,
                               const Real *drdx, const Real *Dm, const void *walls, const int32_t *wall_off,
                               const double dir[3], double mu, double *out, cudaStream_t s);
cudaError_t launch_radial_profile(const double *u, int dim, const int32_t *first, const double *xg, const double *mass,
                                  int G, const double origin[3], const double axis[3], double radius, int nbins,
                                  int blocks, double *partial, cudaStream_t s);

template <typename Real>
cudaError_t launch_eps(const double *u, int dim, int n, int Np, int E, int affine, const Real *el_drdx, const Real *drdx,
                       const Real *el_J, const Real *wJ, const Real *gllw, const Real *Dm, double mu, double *partial,
                       double *out, cudaStream_t s);

void upload_lattice_constants();
size_t stage_smem_bytes(int lat, int Np, int n, int real_size);

}  // namespace slb

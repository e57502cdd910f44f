// Learned per-element filter control and MLP training (declarations).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace slb {

// arguments of the control kernel (one CTA per element)
template <typename Real>
struct ControlArgs {
  int E, Np, n, N, G, Nb;
  int Gs;                      // population stride of the state arrays
  const int32_t *l2g;          // [E][Np]
  const int32_t *bslot;        // [Np] boundary slot of each local node, -1 inside
  const Real *f;               // state on unique nodes [Q][G] (deviation form)
  double rho0;
  int affine;
  const Real *el_J, *wJ, *gllw;
  const Real *Vm;              // [n][n] modal -> nodal
  const Real *Vinv;            // [n][n] nodal -> modal
  const __nv_bfloat16 *W;      // network parameters; NULL = features only
  const Real *lo, *hi;         // [2n] training range of the features
  const Real *fixed_sigma;     // [n] transfer function of the fixed filter (fallback)
  const int *flag;             // global fallback flag (device) or NULL
  double *acc;                 // drift accumulators (device) or NULL
  Real *sigma_out;             // [E][n]
  float *feat_out;             // [E][2n] or NULL
  int *n_fallback;             // elements that kept the fixed filter (device counter) or NULL
  Real *fout;                  // filtered element-interior nodes [Q][G], or NULL (no filtering)
  Real *T;                     // [Q][E*Nb] weighted shares of element-boundary nodes
};
size_t control_smem_bytes(int lat, int Np, int n, int real_size);

template <typename Real>
cudaError_t launch_control(int lat, const ControlArgs<Real> &c, cudaStream_t s);
cudaError_t launch_drift_check(double *acc, int *flag, double mass_bound, double ke_bound, int check_ke, cudaStream_t s);
cudaError_t launch_element_errors(int E, int dim, int n, int nR, const double *rho, const double *u, const double *rhoR,
                                  const double *uR, const double *I, const double *wq, double *err, cudaStream_t s);

int mlp_nparams(int nin);
cudaError_t mlp_grad(const float *params, int nin, int N, const float *X, const float *Y, int64_t M, float *grad,
                     float *loss, cudaStream_t s);
cudaError_t mlp_forward(const float *params, int nin, int N, const float *X, int64_t M, int bf16, float *out,
                        cudaStream_t s);
cudaError_t mlp_train(float *params, float *m, float *v, int nin, int N, const float *X, const float *Y, int64_t M,
                      int batch, int epochs, float lr, uint64_t seed, int64_t *adam_t, float *loss_hist,
                      cudaStream_t s);

}  // namespace slb

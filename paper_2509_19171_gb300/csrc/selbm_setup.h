// Host-side setup of the filtered SELBM (FP64): lattice tables, GLL operators,
// element map and metrics, global numbering, assembly map, wall tables.
// Everything here runs once per handle; the hot path only reads its output.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/selbm.h"

namespace slb {

constexpr double kCs2 = 1.0 / 3.0;
constexpr int kMaxQ = 27;
constexpr int kMaxN = 14;

struct Lattice {
  int dim = 0, Q = 0;
  std::vector<int> e;     // [Q][3] (zero-padded)
  std::vector<double> t;  // [Q]
  std::vector<int> opp;   // [Q]
};

// Velocity set ordered by speed class then ternary code (see selbm.h).
bool build_lattice(int which, Lattice *L);

struct GLL {
  int N = 0;
  std::vector<double> xi, w, D;  // D row-major [N+1][N+1], D[i][j] = l_j'(xi_i)
};
void build_gll(int N, GLL *g);

// Filter matrix F = V diag(sigma) V^{-1} in the basis 1, xi, L_k - L_{k-2}
// (row-major [N+1][N+1]); boundary rows are set to exact identity rows.
void build_filter(const GLL &g, const selbm_filter &f, std::vector<double> *F, std::vector<double> *sigma);
// Modal basis at the GLL nodes, V[i][k] = phi_k(xi_i) (1, xi, L_k - L_{k-2}), and its inverse.
void build_modal(const GLL &g, std::vector<double> *V, std::vector<double> *Vinv);
// Lagrange interpolation matrix I[i][j] = l_j(x_to[i]) from GLL(N_from) to GLL(N_to) nodes.
void build_interp(int N_from, int N_to, std::vector<double> *I);
// Low-rank form of the same filter: F = I + U W over the r damped modes (sigma_k != 1),
// U[j][q] = phi_{k_q}(xi_j), W[q][i] = (sigma_{k_q} - 1) (V^{-1})[k_q][i]; both stored with row stride N+1.
void build_filter_lowrank(const GLL &g, const selbm_filter &f, std::vector<double> *U, std::vector<double> *W, int *r);

// One wall-face node: element, local node, boundary slot, outward normal,
// surface quadrature weight w_s J_s, wall id (1-based).
struct WallNode {
  int e, i, b, wid;
  double n[3];
  double wsJs;
};

struct Setup {
  int dim = 0, E = 0, N = 0, n1 = 0, Np = 0, Nb = 0, G = 0, Gb = 0;
  Lattice lat;
  GLL gll;
  std::vector<double> X;        // [E][Np][dim] node coordinates
  std::vector<double> drdx;     // [E][Np][dim][dim]  dr_l/dx_k  (l row)
  std::vector<double> J;        // [E][Np]
  std::vector<double> wJ;       // [E][Np]
  bool affine = true;           // every element has constant metrics
  std::vector<double> el_drdx;  // [E][dim][dim] (affine case)
  std::vector<double> el_J;     // [E]
  std::vector<int32_t> l2g;     // [E][Np]
  std::vector<uint8_t> owner;   // [E][Np] 1 = first copy of its global node
  std::vector<int32_t> bslot;   // [Np] boundary slot b or -1 for element-interior nodes
  std::vector<int32_t> bnode_g;     // [Gb] global id of each boundary global node
  std::vector<int32_t> bnode_off;   // [Gb+1]
  std::vector<int32_t> bnode_slot;  // copies: e*Nb + b, ascending (e, i)
  std::vector<double> mass;         // [G] assembled lumped mass
  std::vector<int32_t> first_copy;  // [G] local index e*Np+i of the first copy
  std::vector<WallNode> walls;      // sorted by element
  std::vector<int32_t> wall_off;    // [E+1]
  std::vector<double> wall_u;       // [nwalls][3]
  double min_spacing = 0.0;
};

// Returns SELBM_OK or an error code with a message in *err.
int build_setup(const selbm_mesh &mesh, int lattice, int N, Setup *S, std::string *err);
// The same from GLL node coordinates and face connectivity.
int build_setup_nodes(const selbm_mesh_nodes &mesh, int lattice, int N, Setup *S, std::string *err);

}  // namespace slb

// Host-side FP64 setup of the filtered SELBM.  See selbm_setup.h.
#include "selbm_setup.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <unordered_map>

namespace slb {

// ---------------------------------------------------------------------------
// lattice (paper Sec. 2.1; weights are the standard ones the paper cites)
// ---------------------------------------------------------------------------
bool build_lattice(int which, Lattice *L) {
  int dim;
  double wc[4];
  if (which == SELBM_D2Q9) {
    dim = 2; wc[0] = 4.0 / 9.0; wc[1] = 1.0 / 9.0; wc[2] = 1.0 / 36.0; wc[3] = 0.0;
  } else if (which == SELBM_D3Q19) {
    dim = 3; wc[0] = 1.0 / 3.0; wc[1] = 1.0 / 18.0; wc[2] = 1.0 / 36.0; wc[3] = 0.0;
  } else if (which == SELBM_D3Q27) {
    dim = 3; wc[0] = 8.0 / 27.0; wc[1] = 2.0 / 27.0; wc[2] = 1.0 / 54.0; wc[3] = 1.0 / 216.0;
  } else {
    return false;
  }
  L->dim = dim;
  L->e.clear(); L->t.clear(); L->opp.clear();
  const int ncode = dim == 2 ? 9 : 27;
  for (int cls = 0; cls <= dim; ++cls) {
    if (wc[cls] == 0.0) continue;
    for (int code = 0; code < ncode; ++code) {      // ternary code ascending
      int c[3] = {code % 3 - 1, (code / 3) % 3 - 1, dim == 3 ? code / 9 - 1 : 0};
      if (c[0] * c[0] + c[1] * c[1] + c[2] * c[2] != cls) continue;
      L->e.insert(L->e.end(), c, c + 3);
      L->t.push_back(wc[cls]);
    }
  }
  L->Q = (int)L->t.size();
  for (int a = 0; a < L->Q; ++a) {
    for (int b = 0; b < L->Q; ++b) {
      if (L->e[3 * b] == -L->e[3 * a] && L->e[3 * b + 1] == -L->e[3 * a + 1] && L->e[3 * b + 2] == -L->e[3 * a + 2]) {
        L->opp.push_back(b);
        break;
      }
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// GLL (Sec. 2.2)
// ---------------------------------------------------------------------------
// Legendre L_n(x) and L_n'(x) by the three-term recurrences.
static void legendre_pair(int n, double x, double *L, double *dL) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) { *L = 1.0; *dL = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    double d2 = d0 + (2 * k + 1) * p1;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *L = p1; *dL = d1;
}

void build_gll(int N, GLL *g) {
  g->N = N;
  const int n = N + 1;
  g->xi.assign(n, 0.0);
  g->w.assign(n, 0.0);
  g->D.assign(n * n, 0.0);
  // GLL nodes are the roots of q(x) = L_{N-1}(x) - x L_N(x) = (1-x^2) L_N'(x) / N.
  // Newton from the Chebyshev-Lobatto points.
  for (int j = 0; j < n; ++j) {
    double x = -std::cos(M_PI * j / N);
    if (j == 0 || j == N) { g->xi[j] = x; continue; }
    for (int it = 0; it < 100; ++it) {
      double La, dLa, Lb, dLb;
      legendre_pair(N - 1, x, &La, &dLa);
      legendre_pair(N, x, &Lb, &dLb);
      double q = La - x * Lb, dq = dLa - Lb - x * dLb;
      double dx = q / dq;
      x -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    g->xi[j] = x;
  }
  for (int j = 0; j < n / 2; ++j) {          // exact symmetry
    double s = 0.5 * (g->xi[N - j] - g->xi[j]);
    g->xi[j] = -s; g->xi[N - j] = s;
  }
  if (n % 2) g->xi[N / 2] = 0.0;
  g->xi[0] = -1.0; g->xi[N] = 1.0;
  std::vector<double> LN(n);
  for (int i = 0; i < n; ++i) {
    double L, dL;
    legendre_pair(N, g->xi[i], &L, &dL);
    LN[i] = L;
    g->w[i] = 2.0 / (N * (N + 1) * L * L);
  }
  // closed form of the GLL collocation derivative: D_ij = L_N(x_i) / (L_N(x_j) (x_i - x_j)),
  // D_00 = -N(N+1)/4, D_NN = N(N+1)/4, other diagonal entries 0.
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      g->D[i * n + j] = (i == j) ? 0.0 : LN[i] / (LN[j] * (g->xi[i] - g->xi[j]));
  g->D[0] = -0.25 * N * (N + 1);
  g->D[n * n - 1] = 0.25 * N * (N + 1);
}

// ---------------------------------------------------------------------------
// filter (Sec. 2.4)
// ---------------------------------------------------------------------------
static bool invert(std::vector<double> A, int n, std::vector<double> *out) {
  std::vector<double> I(n * n, 0.0);
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[p * n + c])) p = r;
    if (std::fabs(A[p * n + c]) < 1e-300) return false;
    for (int k = 0; k < n; ++k) { std::swap(A[c * n + k], A[p * n + k]); std::swap(I[c * n + k], I[p * n + k]); }
    double d = 1.0 / A[c * n + c];
    for (int k = 0; k < n; ++k) { A[c * n + k] *= d; I[c * n + k] *= d; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double m = A[r * n + c];
      if (m == 0.0) continue;
      for (int k = 0; k < n; ++k) { A[r * n + k] -= m * A[c * n + k]; I[r * n + k] -= m * I[c * n + k]; }
    }
  }
  *out = I;
  return true;
}

void build_filter(const GLL &g, const selbm_filter &f, std::vector<double> *F, std::vector<double> *sigma) {
  const int N = g.N, n = N + 1;
  sigma->assign(n, 1.0);
  for (int k = 0; k < n; ++k) {
    if (f.gamma != 0.0 && k > f.kc) {
      double r = (k - f.kc) / (N - f.kc);
      (*sigma)[k] = f.shape == 0 ? 1.0 - f.gamma * r * r : std::pow(1.0 - f.gamma, std::pow(r, f.p));
    }
  }
  std::vector<double> V(n * n), Vi;
  for (int i = 0; i < n; ++i) {
    double x = g.xi[i];
    std::vector<double> Lk(n);
    for (int k = 0; k < n; ++k) { double L, dL; legendre_pair(k, x, &L, &dL); Lk[k] = L; }
    for (int k = 0; k < n; ++k) V[i * n + k] = (k == 0) ? 1.0 : (k == 1 ? x : Lk[k] - Lk[k - 2]);
  }
  invert(V, n, &Vi);
  F->assign(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += V[i * n + k] * (*sigma)[k] * Vi[k * n + j];
      (*F)[i * n + j] = s;
    }
  for (int j = 0; j < n; ++j) {            // end rows are exact identity rows (phi_k(+-1) = 0, k >= 2)
    (*F)[j] = (j == 0) ? 1.0 : 0.0;
    (*F)[N * n + j] = (j == N) ? 1.0 : 0.0;
  }
}

void build_modal(const GLL &g, std::vector<double> *V, std::vector<double> *Vinv) {
  const int N = g.N, n = N + 1;
  V->assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    const double x = g.xi[i];
    std::vector<double> Lk(n);
    for (int k = 0; k < n; ++k) { double L, dL; legendre_pair(k, x, &L, &dL); Lk[k] = L; }
    for (int k = 0; k < n; ++k) (*V)[i * n + k] = (k == 0) ? 1.0 : (k == 1 ? x : Lk[k] - Lk[k - 2]);
  }
  invert(*V, n, Vinv);
}

void build_interp(int N_from, int N_to, std::vector<double> *I) {
  GLL a, b;
  build_gll(N_from, &a);
  build_gll(N_to, &b);
  const int nf = N_from + 1, nt = N_to + 1;
  I->assign(nt * nf, 1.0);
  for (int i = 0; i < nt; ++i)
    for (int j = 0; j < nf; ++j)
      for (int m = 0; m < nf; ++m)
        if (m != j) (*I)[i * nf + j] *= (b.xi[i] - a.xi[m]) / (a.xi[j] - a.xi[m]);
}

void build_filter_lowrank(const GLL &g, const selbm_filter &f, std::vector<double> *U, std::vector<double> *W, int *r) {
  const int N = g.N, n = N + 1;
  std::vector<double> F, sigma;
  build_filter(g, f, &F, &sigma);
  std::vector<double> V(n * n), Vi;
  for (int i = 0; i < n; ++i) {
    const double x = g.xi[i];
    std::vector<double> Lk(n);
    for (int k = 0; k < n; ++k) { double L, dL; legendre_pair(k, x, &L, &dL); Lk[k] = L; }
    for (int k = 0; k < n; ++k) V[i * n + k] = (k == 0) ? 1.0 : (k == 1 ? x : Lk[k] - Lk[k - 2]);
  }
  invert(V, n, &Vi);
  U->assign(n * n, 0.0);
  W->assign(n * n, 0.0);
  int q = 0;
  for (int k = 0; k < n; ++k) {
    if (sigma[k] == 1.0) continue;
    for (int j = 0; j < n; ++j) (*U)[j * n + q] = V[j * n + k];
    for (int i = 0; i < n; ++i) (*W)[q * n + i] = (sigma[k] - 1.0) * Vi[k * n + i];
    ++q;
  }
  *r = q;
}

// ---------------------------------------------------------------------------
// element map (Gordon-Hall blend with circular arcs)
// ---------------------------------------------------------------------------
static void edge_point(const double *Pa, const double *Pb, double x, bool arc, double R, int dim, double *out) {
  const double la = 0.5 * (1.0 - x), lb = 0.5 * (1.0 + x);
  for (int k = 0; k < dim; ++k) out[k] = la * Pa[k] + lb * Pb[k];
  if (arc) {
    double ta = std::atan2(Pa[1], Pa[0]), tb = std::atan2(Pb[1], Pb[0]);
    if (tb - ta > M_PI) tb -= 2 * M_PI;
    if (ta - tb > M_PI) tb += 2 * M_PI;
    double th = la * ta + lb * tb;
    out[0] = R * std::cos(th);
    out[1] = R * std::sin(th);
  }
}

static void quad_point(const double *C /*[4][dim]*/, const int *cv, double r, double s, double R, int dim, double *out) {
  double e0[3], e1[3], e2[3], e3[3];
  edge_point(C + 0 * dim, C + 2 * dim, s, cv[0], R, dim, e0);
  edge_point(C + 1 * dim, C + 3 * dim, s, cv[1], R, dim, e1);
  edge_point(C + 0 * dim, C + 1 * dim, r, cv[2], R, dim, e2);
  edge_point(C + 2 * dim, C + 3 * dim, r, cv[3], R, dim, e3);
  const double rm = 0.5 * (1 - r), rp = 0.5 * (1 + r), sm = 0.5 * (1 - s), sp = 0.5 * (1 + s);
  for (int k = 0; k < dim; ++k) {
    double bil = rm * sm * C[0 * dim + k] + rp * sm * C[1 * dim + k] + rm * sp * C[2 * dim + k] + rp * sp * C[3 * dim + k];
    out[k] = rm * e0[k] + rp * e1[k] + sm * e2[k] + sp * e3[k] - bil;
  }
}

// ---------------------------------------------------------------------------
// global numbering by coordinate matching
// ---------------------------------------------------------------------------
struct Key {
  int64_t k[3];
  bool operator==(const Key &o) const { return k[0] == o.k[0] && k[1] == o.k[1] && k[2] == o.k[2]; }
};
struct KeyHash {
  size_t operator()(const Key &a) const {
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < 3; ++i) { h ^= (uint64_t)a.k[i]; h *= 1099511628211ull; h ^= h >> 29; }
    return (size_t)h;
  }
};

// ---------------------------------------------------------------------------
// node-coordinate mesh form (Sec. 2.2 isoparametric elements): the element map through the
// given GLL nodes, interpolated to the solver's nodes; nodes identified by face connectivity
// ---------------------------------------------------------------------------
// local index of node (a, b) of face f (face coordinates: tangential indices in increasing
// axis order), order N
static int face_node(int dim, int N, int f, int a, int b) {
  const int n = N + 1, axis = f / 2, fixed = (f % 2) ? N : 0;
  int idx[3] = {0, 0, 0};
  idx[axis] = fixed;
  if (dim == 2) {
    idx[1 - axis] = a;
    return idx[0] + n * idx[1];
  }
  const int t0 = axis == 0 ? 1 : 0, t1 = axis == 2 ? 1 : 2;
  idx[t0] = a;
  idx[t1] = b;
  return idx[0] + n * idx[1] + n * n * idx[2];
}

// face coordinates on the neighbour's face for orientation code `code`
static void orient_map(int code, int N, int a, int b, int *a2, int *b2) {
  int u = (code & 1) ? b : a, v = (code & 1) ? a : b;
  *a2 = (code & 2) ? N - u : u;
  *b2 = (code & 4) ? N - v : v;
}

// x at the solver's GLL nodes (order N) from the coordinates at the GLL nodes of order N_g:
// X[e][p][k] = sum over the given nodes of the tensor-product Lagrange basis at node p
static int nodes_to_gll(const selbm_mesh_nodes &m, int N, const GLL &g, std::vector<double> *X, std::string *err) {
  (void)g;
  const int dim = m.dim, E = m.nelem, Ng = m.order;
  if (!m.xyz) { *err = "mesh xyz is NULL"; return SELBM_ERR_ARG; }
  if (Ng < 1 || Ng > kMaxN) { *err = "mesh order out of range [1, 14]"; return SELBM_ERR_ARG; }
  const int ng = Ng + 1, n = N + 1;
  int Npg = 1, Np = 1;
  for (int k = 0; k < dim; ++k) { Npg *= ng; Np *= n; }
  std::vector<double> I;
  build_interp(Ng, N, &I);                                   // [n][ng]
  X->assign((size_t)E * Np * dim, 0.0);
  std::vector<double> a, b;
  for (int e = 0; e < E; ++e)
    for (int c = 0; c < dim; ++c) {
      const double *in = m.xyz + ((size_t)e * dim + c) * Npg;
      for (int v = 0; v < Npg; ++v)
        if (!std::isfinite(in[v])) { *err = "mesh xyz holds a non-finite value"; return SELBM_ERR_MESH; }
      // axis by axis: sizes (ng, ng, ng) -> (n, ng, ng) -> (n, n, ng) -> (n, n, n)
      a.assign(in, in + Npg);
      int s0 = ng, s1 = ng, s2 = dim == 3 ? ng : 1;
      for (int axis = 0; axis < dim; ++axis) {
        int d[3] = {s0, s1, s2};
        int o[3] = {s0, s1, s2};
        o[axis] = n;
        b.assign((size_t)o[0] * o[1] * o[2], 0.0);
        for (int k = 0; k < o[2]; ++k)
          for (int j = 0; j < o[1]; ++j)
            for (int i = 0; i < o[0]; ++i) {
              const int out_i[3] = {i, j, k};
              double acc = 0.0;
              for (int m2 = 0; m2 < ng; ++m2) {
                int src[3] = {i, j, k};
                src[axis] = m2;
                acc += I[out_i[axis] * ng + m2] * a[src[0] + d[0] * (src[1] + d[1] * src[2])];
              }
              b[i + o[0] * (j + o[1] * k)] = acc;
            }
        a.swap(b);
        s0 = o[0]; s1 = o[1]; s2 = o[2];
      }
      for (int p = 0; p < Np; ++p) (*X)[((size_t)e * Np + p) * dim + c] = a[p];
    }
  return SELBM_OK;
}

static int uf_find(std::vector<int64_t> &par, int64_t x) {
  while (par[x] != x) {
    par[x] = par[par[x]];
    x = par[x];
  }
  return (int)x;
}

// global numbering from face connectivity: the nodes of matched faces are joined (union-find),
// each class numbered in order of its first local copy; checks mutual pairs and that matched
// nodes differ by one translation per face
static int number_by_connectivity(const selbm_mesh_nodes &m, int N, Setup *S, int32_t *G, std::string *err) {
  const int dim = m.dim, E = m.nelem, nf = 2 * dim, n = N + 1;
  int Np = 1;
  for (int k = 0; k < dim; ++k) Np *= n;
  if (!m.face_nbr || !m.face_nbr_face || !m.face_orient) { *err = "face connectivity arrays are NULL"; return SELBM_ERR_ARG; }
  double scale = 0.0;
  {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (size_t q = 0; q < (size_t)E * Np; ++q)
      for (int k = 0; k < dim; ++k) {
        lo[k] = std::min(lo[k], S->X[q * dim + k]);
        hi[k] = std::max(hi[k], S->X[q * dim + k]);
      }
    for (int k = 0; k < dim; ++k) scale = std::max(scale, hi[k] - lo[k]);
  }
  const double tol = 1e-9 * scale;
  std::vector<int64_t> par((size_t)E * Np);
  for (size_t q = 0; q < par.size(); ++q) par[q] = (int64_t)q;
  const int nb = dim == 3 ? n : 1;                   // second face coordinate range
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < nf; ++f) {
      const int e2 = m.face_nbr[(size_t)e * nf + f];
      if (e2 < 0) continue;
      if (e2 >= E) { *err = "face_nbr names an element beyond nelem"; return SELBM_ERR_MESH; }
      const int f2 = m.face_nbr_face[(size_t)e * nf + f], code = m.face_orient[(size_t)e * nf + f];
      if (f2 < 0 || f2 >= nf) { *err = "face_nbr_face out of range"; return SELBM_ERR_MESH; }
      if (code < 0 || code > 7 || (dim == 2 && (code & 5))) { *err = "face_orient out of range"; return SELBM_ERR_MESH; }
      if (e2 == e && f2 == f) { *err = "a face is its own neighbour"; return SELBM_ERR_MESH; }
      if (m.face_nbr[(size_t)e2 * nf + f2] != e || m.face_nbr_face[(size_t)e2 * nf + f2] != f) {
        *err = "face connectivity is not mutual";
        return SELBM_ERR_MESH;
      }
      if (m.face_bc && m.face_bc[(size_t)e * nf + f] > 0) { *err = "a wall face has a neighbour"; return SELBM_ERR_MESH; }
      const int code2 = m.face_orient[(size_t)e2 * nf + f2];
      double shift[3] = {0, 0, 0};
      for (int b = 0; b < nb; ++b)
        for (int a = 0; a < n; ++a) {
          int a2, b2, a3, b3;
          orient_map(code, N, a, b, &a2, &b2);
          if (dim == 2) b2 = 0;
          orient_map(code2, N, a2, b2, &a3, &b3);   // back from the neighbour's side
          if (dim == 2) b3 = 0;
          if (a3 != a || b3 != b) { *err = "face orientations of a face pair are not inverse"; return SELBM_ERR_MESH; }
          const size_t q = (size_t)e * Np + face_node(dim, N, f, a, b);
          const size_t q2 = (size_t)e2 * Np + face_node(dim, N, f2, a2, b2);
          for (int k = 0; k < dim; ++k) {
            const double dk = S->X[q2 * dim + k] - S->X[q * dim + k];
            if (a == 0 && b == 0) shift[k] = dk;
            else if (std::fabs(dk - shift[k]) > tol) {
              *err = "matched face nodes do not coincide up to one translation (orientation?)";
              return SELBM_ERR_MESH;
            }
          }
          const int r1 = uf_find(par, (int64_t)q), r2 = uf_find(par, (int64_t)q2);
          if (r1 != r2) par[std::max(r1, r2)] = std::min(r1, r2);
        }
    }
  S->l2g.assign((size_t)E * Np, -1);
  S->owner.assign((size_t)E * Np, 0);
  std::vector<int32_t> id((size_t)E * Np, -1);
  int32_t g = 0;
  for (size_t q = 0; q < (size_t)E * Np; ++q) {
    const int r = uf_find(par, (int64_t)q);
    if (id[r] < 0) {
      id[r] = g++;
      S->owner[q] = 1;
    }
    S->l2g[q] = id[r];
  }
  *G = g;
  return SELBM_OK;
}

// The two mesh forms of the ABI: element corners (+ arcs, periods) or GLL node coordinates with
// face connectivity.  Everything after the coordinates and the global numbering is shared.
struct MeshInput {
  int dim = 0, nelem = 0;
  const selbm_mesh *corners = nullptr;
  const selbm_mesh_nodes *nodes = nullptr;
  const int32_t *face_bc = nullptr;
  int nwalls = 0;
  const double *wall_velocity = nullptr;
};

static int build_setup_impl(const MeshInput &mi, int lattice, int N, Setup *S, std::string *err) {
  const int dim = mi.dim;
  if (dim != 2 && dim != 3) { *err = "mesh.dim must be 2 or 3"; return SELBM_ERR_ARG; }
  if (mi.nelem <= 0) { *err = "mesh has no elements"; return SELBM_ERR_ARG; }
  if (N < 2 || N > kMaxN) { *err = "order N out of range [2, 14]"; return SELBM_ERR_ARG; }
  if (!build_lattice(lattice, &S->lat)) { *err = "unknown lattice"; return SELBM_ERR_ARG; }
  if (S->lat.dim != dim) { *err = "lattice dimension does not match the mesh"; return SELBM_ERR_ARG; }
  S->dim = dim; S->E = mi.nelem; S->N = N; S->n1 = N + 1;
  const int n = N + 1, E = mi.nelem;
  int Np = 1, Nint = 1;
  for (int k = 0; k < dim; ++k) { Np *= n; Nint *= (N - 1); }
  S->Np = Np; S->Nb = Np - Nint;
  build_gll(N, &S->gll);
  const std::vector<double> &xi = S->gll.xi, &w = S->gll.w, &D = S->gll.D;

  // reference index table
  std::vector<int> ijk(Np * 3, 0);
  for (int p = 0; p < Np; ++p) {
    ijk[3 * p] = p % n; ijk[3 * p + 1] = (p / n) % n; ijk[3 * p + 2] = dim == 3 ? p / (n * n) : 0;
  }
  S->bslot.assign(Np, -1);
  {
    int b = 0;
    for (int p = 0; p < Np; ++p) {
      bool bd = false;
      for (int k = 0; k < dim; ++k) bd |= (ijk[3 * p + k] == 0 || ijk[3 * p + k] == N);
      if (bd) S->bslot[p] = b++;
    }
  }

  // node coordinates
  S->X.assign((size_t)E * Np * dim, 0.0);
  if (mi.corners) {
    const selbm_mesh &mesh = *mi.corners;
    for (int e = 0; e < E; ++e) {
      const double *C = mesh.verts + (size_t)e * (1 << dim) * dim;
      int cv[4] = {0, 0, 0, 0};
      if (mesh.curved)
        for (int f = 0; f < 4; ++f) cv[f] = mesh.curved[(size_t)e * 2 * dim + f] != 0;
      for (int p = 0; p < Np; ++p) {
        double r = xi[ijk[3 * p]], s = xi[ijk[3 * p + 1]];
        double *out = &S->X[((size_t)e * Np + p) * dim];
        if (dim == 2) {
          quad_point(C, cv, r, s, mesh.radius, 2, out);
        } else {
          double t = xi[ijk[3 * p + 2]], lo[3], hi[3];
          quad_point(C, cv, r, s, mesh.radius, 3, lo);
          quad_point(C + 4 * 3, cv, r, s, mesh.radius, 3, hi);
          for (int k = 0; k < 3; ++k) out[k] = 0.5 * (1 - t) * lo[k] + 0.5 * (1 + t) * hi[k];
        }
      }
    }
  } else {
    int rc = nodes_to_gll(*mi.nodes, N, S->gll, &S->X, err);
    if (rc != SELBM_OK) return rc;
  }

  // metrics: dx_k/dr_l = D along axis l applied to x_k; inverse; J; wJ
  S->drdx.assign((size_t)E * Np * dim * dim, 0.0);
  S->J.assign((size_t)E * Np, 0.0);
  S->wJ.assign((size_t)E * Np, 0.0);
  const int stride[3] = {1, n, n * n};
  double minJ = 1e300;
  for (int e = 0; e < E; ++e) {
    const double *Xe = &S->X[(size_t)e * Np * dim];
    for (int p = 0; p < Np; ++p) {
      double a[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};  // a[k][l] = dx_k/dr_l
      for (int l = 0; l < dim; ++l) {
        int il = ijk[3 * p + l];
        int base = p - il * stride[l];
        for (int k = 0; k < dim; ++k) {
          double s = 0.0;
          for (int m = 0; m < n; ++m) s += D[il * n + m] * Xe[(size_t)(base + m * stride[l]) * dim + k];
          a[k][l] = s;
        }
      }
      double det, inv[3][3];
      if (dim == 2) {
        det = a[0][0] * a[1][1] - a[0][1] * a[1][0];
        inv[0][0] = a[1][1] / det; inv[0][1] = -a[0][1] / det;
        inv[1][0] = -a[1][0] / det; inv[1][1] = a[0][0] / det;
      } else {
        det = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
              a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            int i1 = (j + 1) % 3, i2 = (j + 2) % 3, j1 = (i + 1) % 3, j2 = (i + 2) % 3;
            inv[i][j] = (a[i1][j1] * a[i2][j2] - a[i1][j2] * a[i2][j1]) / det;   // cofactor transpose
          }
      }
      minJ = std::min(minJ, det);
      size_t q = (size_t)e * Np + p;
      S->J[q] = det;
      double wq = 1.0;
      for (int l = 0; l < dim; ++l) wq *= w[ijk[3 * p + l]];
      S->wJ[q] = wq * det;
      for (int l = 0; l < dim; ++l)
        for (int k = 0; k < dim; ++k) S->drdx[(q * dim + l) * dim + k] = inv[l][k];   // inv(dx/dr)[l][k] = dr_l/dx_k
    }
  }
  if (!(minJ > 0.0)) { *err = "non-positive Jacobian in the element map"; return SELBM_ERR_MESH; }

  // affine detection: constant metrics inside every element
  S->affine = true;
  S->el_drdx.assign((size_t)E * dim * dim, 0.0);
  S->el_J.assign(E, 0.0);
  for (int e = 0; e < E && S->affine; ++e) {
    const double *g0 = &S->drdx[(size_t)e * Np * dim * dim];
    double J0 = S->J[(size_t)e * Np], gmax = 0.0;
    for (int c = 0; c < dim * dim; ++c) gmax = std::max(gmax, std::fabs(g0[c]));
    for (int p = 1; p < Np && S->affine; ++p) {
      const double *gp = &S->drdx[((size_t)e * Np + p) * dim * dim];
      for (int c = 0; c < dim * dim; ++c)
        if (std::fabs(gp[c] - g0[c]) > 1e-11 * gmax) S->affine = false;
      if (std::fabs(S->J[(size_t)e * Np + p] - J0) > 1e-11 * J0) S->affine = false;
    }
    for (int c = 0; c < dim * dim; ++c) S->el_drdx[(size_t)e * dim * dim + c] = g0[c];
    S->el_J[e] = J0;
  }

  // global numbering: coordinates (corner form) or face connectivity (node form)
  int32_t G = 0;
  if (mi.nodes) {
    int rc = number_by_connectivity(*mi.nodes, N, S, &G, err);
    if (rc != SELBM_OK) return rc;
  } else {
    const selbm_mesh &mesh = *mi.corners;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (size_t q = 0; q < (size_t)E * Np; ++q)
      for (int k = 0; k < dim; ++k) { lo[k] = std::min(lo[k], S->X[q * dim + k]); hi[k] = std::max(hi[k], S->X[q * dim + k]); }
    double scale = 0.0;
    for (int k = 0; k < dim; ++k) scale = std::max(scale, hi[k] - lo[k]);
    const double quantum = 1e-7 * scale;
    std::unordered_map<Key, int32_t, KeyHash> map;
    map.reserve((size_t)E * Np);
    S->l2g.assign((size_t)E * Np, -1);
    S->owner.assign((size_t)E * Np, 0);
    for (size_t q = 0; q < (size_t)E * Np; ++q) {
      double y[3] = {0, 0, 0};
      for (int k = 0; k < dim; ++k) {
        y[k] = S->X[q * dim + k];
        double L = mesh.period ? mesh.period[k] : 0.0;
        if (L > 0.0) {
          double o = mesh.origin ? mesh.origin[k] : 0.0;
          double v = std::fmod(y[k] - o, L);
          if (v < 0) v += L;
          if (L - v < 1e-7 * scale) v -= L;
          y[k] = v;
        }
      }
      // candidate keys: nearest cell, plus the other side for coordinates close to a cell edge
      int64_t base[3], alt[3];
      bool amb[3] = {false, false, false};
      for (int k = 0; k < 3; ++k) {
        double u = y[k] / quantum;
        base[k] = (int64_t)std::llround(u);
        double fr = u - std::floor(u);
        alt[k] = fr < 0.5 ? base[k] + 1 : base[k] - 1;
        amb[k] = std::fabs(fr - 0.5) < 1e-3;
      }
      int32_t found = -1;
      for (int m = 0; m < 8 && found < 0; ++m) {
        Key key;
        bool ok = true;
        for (int k = 0; k < 3; ++k) {
          bool use_alt = (m >> k) & 1;
          if (use_alt && !amb[k]) { ok = false; break; }
          key.k[k] = use_alt ? alt[k] : base[k];
        }
        if (!ok) continue;
        auto it = map.find(key);
        if (it != map.end()) found = it->second;
      }
      if (found < 0) {
        Key key{{base[0], base[1], base[2]}};
        map.emplace(key, G);
        S->l2g[q] = G++;
        S->owner[q] = 1;
      } else {
        S->l2g[q] = found;
      }
    }
  }
  S->G = G;

  // renumber: element-interior nodes first, element by element in local order (each
  // element's interior is one contiguous block, written whole by the element kernels),
  // then element-boundary nodes in order of first appearance (one contiguous range,
  // written by the assembly)
  {
    std::vector<int32_t> nid(G, -1);
    int32_t next = 0;
    for (size_t q = 0; q < (size_t)E * Np; ++q)
      if (S->bslot[q % Np] < 0 && nid[S->l2g[q]] < 0) nid[S->l2g[q]] = next++;
    for (size_t q = 0; q < (size_t)E * Np; ++q)
      if (nid[S->l2g[q]] < 0) nid[S->l2g[q]] = next++;
    for (size_t q = 0; q < (size_t)E * Np; ++q) S->l2g[q] = nid[S->l2g[q]];
  }

  // consistency: interior nodes are unique; boundary nodes only match boundary nodes
  std::vector<int32_t> count(G, 0), nbd(G, 0);
  for (size_t q = 0; q < (size_t)E * Np; ++q) {
    count[S->l2g[q]]++;
    if (S->bslot[q % Np] >= 0) nbd[S->l2g[q]]++;
  }
  for (size_t q = 0; q < (size_t)E * Np; ++q) {
    int g = S->l2g[q];
    if (S->bslot[q % Np] < 0 && count[g] != 1) { *err = "element-interior node matched another node"; return SELBM_ERR_MESH; }
    if (S->bslot[q % Np] >= 0 && nbd[g] != count[g]) { *err = "boundary node matched an interior node"; return SELBM_ERR_MESH; }
  }

  // mass and first copies
  S->mass.assign(G, 0.0);
  S->first_copy.assign(G, -1);
  for (size_t q = 0; q < (size_t)E * Np; ++q) {
    int g = S->l2g[q];
    S->mass[g] += S->wJ[q];
    if (S->first_copy[g] < 0) S->first_copy[g] = (int32_t)q;
  }

  // assembly map over boundary global nodes (ascending global id; copies ascending (e, i))
  std::vector<int32_t> bidx(G, -1);
  S->bnode_g.clear();
  for (int g = 0; g < G; ++g)
    if (nbd[g] > 0) { bidx[g] = (int32_t)S->bnode_g.size(); S->bnode_g.push_back(g); }
  S->Gb = (int)S->bnode_g.size();
  S->bnode_off.assign(S->Gb + 1, 0);
  for (int u = 0; u < S->Gb; ++u) S->bnode_off[u + 1] = S->bnode_off[u] + nbd[S->bnode_g[u]];
  S->bnode_slot.assign(S->bnode_off[S->Gb], 0);
  std::vector<int32_t> fill(S->Gb, 0);
  for (int e = 0; e < E; ++e)
    for (int p = 0; p < Np; ++p) {
      int b = S->bslot[p];
      if (b < 0) continue;
      int u = bidx[S->l2g[(size_t)e * Np + p]];
      S->bnode_slot[S->bnode_off[u] + fill[u]++] = e * S->Nb + b;
    }

  // wall faces: outward normal +-grad r_l/|grad r_l|, w_s J_s = prod(tangential w) J |grad r_l|
  S->wall_u.assign((size_t)std::max(mi.nwalls, 0) * 3, 0.0);
  for (int k = 0; k < mi.nwalls; ++k)
    for (int c = 0; c < dim; ++c) S->wall_u[k * 3 + c] = mi.wall_velocity ? mi.wall_velocity[k * dim + c] : 0.0;
  S->walls.clear();
  S->wall_off.assign(E + 1, 0);
  for (int e = 0; e < E; ++e) {
    for (int f = 0; f < 2 * dim; ++f) {
      int wid = mi.face_bc ? mi.face_bc[(size_t)e * 2 * dim + f] : 0;
      if (wid <= 0) continue;
      if (wid > mi.nwalls) { *err = "face_bc refers to a wall id beyond nwalls"; return SELBM_ERR_MESH; }
      int axis = f / 2, side = f % 2;
      for (int p = 0; p < Np; ++p) {
        if (ijk[3 * p + axis] != (side ? N : 0)) continue;
        size_t q = (size_t)e * Np + p;
        const double *g = &S->drdx[(q * dim + axis) * dim];
        double gn = 0.0;
        for (int k = 0; k < dim; ++k) gn += g[k] * g[k];
        gn = std::sqrt(gn);
        WallNode wn;
        wn.e = e; wn.i = p; wn.b = S->bslot[p]; wn.wid = wid;
        for (int k = 0; k < 3; ++k) wn.n[k] = k < dim ? (side ? 1.0 : -1.0) * g[k] / gn : 0.0;
        double ws = 1.0;
        for (int l = 0; l < dim; ++l)
          if (l != axis) ws *= w[ijk[3 * p + l]];
        wn.wsJs = ws * S->J[q] * gn;
        S->walls.push_back(wn);
      }
    }
    S->wall_off[e + 1] = (int32_t)S->walls.size();
  }

  // smallest GLL node spacing
  double hmin = 1e300;
  for (int e = 0; e < E; ++e)
    for (int p = 0; p < Np; ++p)
      for (int l = 0; l < dim; ++l) {
        if (ijk[3 * p + l] == N) continue;
        const double *a = &S->X[((size_t)e * Np + p) * dim];
        const double *b = &S->X[((size_t)e * Np + p + stride[l]) * dim];
        double d2 = 0.0;
        for (int k = 0; k < dim; ++k) d2 += (a[k] - b[k]) * (a[k] - b[k]);
        hmin = std::min(hmin, std::sqrt(d2));
      }
  S->min_spacing = hmin;
  return SELBM_OK;
}

int build_setup(const selbm_mesh &mesh, int lattice, int N, Setup *S, std::string *err) {
  MeshInput mi;
  mi.dim = mesh.dim;
  mi.nelem = mesh.nelem;
  mi.corners = &mesh;
  mi.face_bc = mesh.face_bc;
  mi.nwalls = mesh.nwalls;
  mi.wall_velocity = mesh.wall_velocity;
  if (!mesh.verts) { *err = "mesh has no elements"; return SELBM_ERR_ARG; }
  return build_setup_impl(mi, lattice, N, S, err);
}

int build_setup_nodes(const selbm_mesh_nodes &mesh, int lattice, int N, Setup *S, std::string *err) {
  MeshInput mi;
  mi.dim = mesh.dim;
  mi.nelem = mesh.nelem;
  mi.nodes = &mesh;
  mi.face_bc = mesh.face_bc;
  mi.nwalls = mesh.nwalls;
  mi.wall_velocity = mesh.wall_velocity;
  return build_setup_impl(mi, lattice, N, S, err);
}

}  // namespace slb

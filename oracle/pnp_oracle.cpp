// pnp_oracle.cpp -- plain FP64 CPU oracle for the VMS-stabilised PNP block.
//
// TEST INFRASTRUCTURE.  This file is the independent reference that the CUDA path is
// checked against.  Only the tests, the smoke check and the CPU-baseline and reference
// legs of the benchmark load it; the library's product path never calls, links or includes it,
// and it shares no code, header or table with the CUDA sources.
//
// What it computes (Kim et al., "Direct numerical simulation of electrokinetic
// transport phenomena in fluids: variational multi-scale stabilization and
// octree-based mesh refinement", arXiv 2301.05985):
//   * the non-dimensional Poisson and Nernst-Planck equations of Sec. 2.2
//     (Eqs. nondim_poisson, nondim_np): -2 Lambda^2 lap(phi) = sum_s z_s c_s and
//     dc/dt + v.grad c = div(grad c + z c grad phi);
//   * BDF time discretisation with coefficients beta0..beta2 (Def. 1 of Sec. 3);
//   * the fully discrete VMS form of Def. 3 (Poisson and Nernst-Planck rows), with
//     the fine-scale closure c^f = -tau_c R_c and tau_c of Sec. 3.1 (C_I = 6,
//     G_ij = (2/h)^2 delta_ij on cubes);
//   * the analytic Jacobian of that residual (Sec. 4.1, Eq. newton_linear_system);
//   * Q1 elements on a 2:1-balanced octree (Sec. 4.2) with conforming hanging-node
//     constraints (the paper does not describe them; face-centre = mean of 4 face
//     corners, edge-midpoint = mean of 2 edge ends);
//   * the semi-implicit VMS Navier-Stokes block of Def. 3 (momentum and solenoidality
//     rows, linear in (v, p)) with its closure v^f = -tau_m R_m, p^f = -tau_sol R_sol of
//     Sec. 3.1, and the manufactured (u, v, p) of Eq. manufac_sol;
//   * optional periodic side walls (the electroconvection setup of Sec. 5.2): on a
//     periodic axis every coordinate is taken modulo the domain length, so the faces
//     x = 0 and x = 1 are one set of nodes and carry no boundary condition.
//
// Everything is written out plainly: std::map on integer coordinates for the mesh,
// direct evaluation of the tensor-product shape functions at each Gauss point,
// element-by-element assembly.  No sum factorisation, no blocking, no reordering.

#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <utility>
#include <vector>

namespace {

typedef std::array<int64_t, 3> IPt;

struct Mesh {
  int dim = 0;
  int L = 0;                                   // max level: coordinates in units of 2^-L
  int periodic = 0;                            // bit k: faces x_k = 0 and x_k = 1 are one
  std::vector<IPt> el_anchor;
  std::vector<int> el_level;
  std::vector<std::vector<int64_t>> el_nodes;  // 2^dim corner node ids (lexicographic corner order)
  std::vector<IPt> node_xyz;
  std::map<IPt, int64_t> node_of;
  // constraint rows: node -> list of (independent node, weight).  Identity for free nodes.
  std::vector<std::vector<std::pair<int64_t, double>>> cons;
  std::vector<char> hanging;
};

// Parameters of one residual evaluation.  Must match the ctypes mirror in oracle.py.
struct Params {
  double eps;      // Lambda, the non-dimensional Debye length
  double dt;       // time step
  double beta0, beta1, beta2;  // BDF coefficients
  double C_I;      // tau_c constant (6 in the paper)
  double t;        // time level of the unknown (manufactured-solution forcing only)
  int32_t steady;  // 1: drop the time-derivative terms (and 4/dt^2 in tau_c)
  int32_t vms;     // 0: tau_c := 0 (plain Galerkin; used by the exact-integration checks)
  int32_t mms;     // 1: add manufactured-solution forcing and use its Dirichlet values
  int32_t pad;
  int32_t bc_type[6][3];  // per face, per field: 0 natural, 1 Dirichlet
  double bc_val[6][3];
};

const double kZ[2] = {+1.0, -1.0};  // valences of c+ and c-

// ------------------------------------------------------------------ manufactured solution
// Sec. 5.1, Eq. manufac_sol (2D); in 3D every field is multiplied by cos(pi z) and the
// third velocity component is zero (still divergence-free).  Returns, for fields
// [c+, c-, phi, u, v, w], the value, gradient and Laplacian at (x, t); "steady"
// freezes the time factor at 1.
struct MmsField { double val; double grad[3]; double lap; double dval_dt; };

void mms_fields(int dim, const double* x, double t, int steady, MmsField out[6]) {
  const double k = 2.0 * M_PI;
  const double T = steady ? 1.0 : std::cos(2.0 * t);
  const double Tp = steady ? 0.0 : -2.0 * std::sin(2.0 * t);
  const double sx = std::sin(k * x[0]), cx = std::cos(k * x[0]);
  const double sy = std::sin(k * x[1]), cy = std::cos(k * x[1]);
  // A = cos(kx) sin(ky), B = sin(kx) cos(ky)
  const double A = cx * sy, B = sx * cy;
  const double Ag[2] = {-k * sx * sy, k * cx * cy};
  const double Bg[2] = {k * cx * cy, -k * sx * sy};
  const double Alap = -2.0 * k * k * A, Blap = -2.0 * k * k * B;
  double Z = 1.0, Zp = 0.0, Zpp = 0.0;
  if (dim == 3) {
    Z = std::cos(M_PI * x[2]);
    Zp = -M_PI * std::sin(M_PI * x[2]);
    Zpp = -M_PI * M_PI * Z;
  }
  // sign * T * {A or B} * Z
  const int which[5] = {0, 1, 0, 1, 0};   // A, B, A, B, A  for c+, c-, phi, u, v
  const double sgn[5] = {+1, +1, -1, +1, -1};
  for (int f = 0; f < 5; ++f) {
    const double g = which[f] ? B : A;
    const double* gg = which[f] ? Bg : Ag;
    const double gl = which[f] ? Blap : Alap;
    const double s = sgn[f];
    out[f].val = s * T * g * Z;
    out[f].dval_dt = s * Tp * g * Z;
    out[f].grad[0] = s * T * gg[0] * Z;
    out[f].grad[1] = s * T * gg[1] * Z;
    out[f].grad[2] = s * T * g * Zp;
    out[f].lap = s * T * (gl * Z + g * Zpp);
  }
  out[5] = MmsField{0.0, {0.0, 0.0, 0.0}, 0.0, 0.0};
}

// Forcing that makes the manufactured fields an exact solution of
//   dc_s/dt + v.grad c_s - div(grad c_s + z_s c_s grad phi) = f_s,
//   -2 Lambda^2 lap(phi) - sum_s z_s c_s = f_phi.
void mms_forcing(int dim, const double* x, double t, double eps, int steady, double f[3]) {
  MmsField m[6];
  mms_fields(dim, x, t, steady, m);
  const MmsField& ph = m[2];
  for (int s = 0; s < 2; ++s) {
    const MmsField& c = m[s];
    double adv = 0.0, gcgp = 0.0;
    for (int a = 0; a < dim; ++a) {
      adv += m[3 + a].val * c.grad[a];
      gcgp += c.grad[a] * ph.grad[a];
    }
    // div(z c grad phi) = z (grad c . grad phi + c lap phi)
    f[s] = c.dval_dt + adv - c.lap - kZ[s] * (gcgp + c.val * ph.lap);
  }
  f[2] = -2.0 * eps * eps * ph.lap - (m[0].val - m[1].val);
}

// ------------------------------------------------------------------ mesh construction
int corner_count(int dim) { return 1 << dim; }

// On a periodic axis a point is taken modulo the domain length (x = 1 is x = 0).
void wrap_point(const Mesh& m, IPt& p) {
  const int64_t size = int64_t(1) << m.L;
  for (int k = 0; k < m.dim; ++k)
    if ((m.periodic >> k) & 1) p[k] = ((p[k] % size) + size) % size;
}

IPt corner_point(const Mesh& m, const IPt& a, int64_t s, int c) {
  IPt p = a;
  for (int k = 0; k < m.dim; ++k)
    if ((c >> k) & 1) p[k] += s;
  wrap_point(m, p);
  return p;
}

// Error codes (same meaning as the library's public codes where they overlap).
enum { ORA_OK = 0, ORA_ERR_ARG = 1, ORA_ERR_UNBALANCED = 3 };

int build_mesh(Mesh& m, int dim, int L, int64_t n, const int32_t* anchors, const uint8_t* levels, int periodic) {
  if (dim != 2 && dim != 3) return ORA_ERR_ARG;
  if (L < 0 || L > 20 || n <= 0) return ORA_ERR_ARG;
  if (periodic < 0 || periodic >= (1 << dim)) return ORA_ERR_ARG;
  m.dim = dim;
  m.L = L;
  m.periodic = periodic;
  const int64_t size = int64_t(1) << L;
  std::map<IPt, int> leaf;  // anchor -> level
  for (int64_t e = 0; e < n; ++e) {
    IPt a = {0, 0, 0};
    for (int k = 0; k < dim; ++k) a[k] = anchors[e * dim + k];
    const int l = levels[e];
    if (l > L) return ORA_ERR_ARG;
    if (periodic && l == 0) return ORA_ERR_ARG;  // an element would meet itself across the wrap
    const int64_t s = int64_t(1) << (L - l);
    for (int k = 0; k < dim; ++k)
      if (a[k] < 0 || a[k] % s != 0 || a[k] + s > size) return ORA_ERR_ARG;
    if (leaf.count(a)) return ORA_ERR_ARG;  // duplicate anchor (same or different level)
    leaf[a] = l;
  }
  // Two octants overlap only if one is an ancestor of the other.
  long double vol = 0;
  for (auto& kv : leaf) {
    const IPt& a = kv.first;
    const int l = kv.second;
    for (int lc = 0; lc < l; ++lc) {
      const int64_t sc = int64_t(1) << (L - lc);
      IPt b = {0, 0, 0};
      for (int k = 0; k < dim; ++k) b[k] = (a[k] / sc) * sc;
      auto it = leaf.find(b);
      if (it != leaf.end() && it->second == lc) return ORA_ERR_ARG;
    }
    vol += std::pow((long double)2.0, -(long double)(dim * l));
  }
  if (std::fabs((double)(vol - 1.0L)) > 1e-12) return ORA_ERR_ARG;  // not a complete cover

  // 2:1 balance across faces, edges and corners: the leaf containing the same-size
  // neighbour region of every leaf must be at most one level coarser.
  for (auto& kv : leaf) {
    const IPt& a = kv.first;
    const int l = kv.second;
    const int64_t s = int64_t(1) << (L - l);
    const int nd = dim == 3 ? 27 : 9;
    for (int d = 0; d < nd; ++d) {
      int off[3] = {d % 3 - 1, (d / 3) % 3 - 1, (d / 9) % 3 - 1};
      if (dim == 2) off[2] = 0;
      if (off[0] == 0 && off[1] == 0 && off[2] == 0) continue;
      IPt r = a;
      bool inside = true;
      for (int k = 0; k < dim; ++k) {
        r[k] = a[k] + off[k] * s;
        if ((periodic >> k) & 1) continue;  // wrapped below
        if (r[k] < 0 || r[k] >= size) inside = false;
      }
      if (!inside) continue;
      wrap_point(m, r);
      for (int lc = l; lc >= 0; --lc) {
        const int64_t sc = int64_t(1) << (L - lc);
        IPt b = {0, 0, 0};
        for (int k = 0; k < dim; ++k) b[k] = (r[k] / sc) * sc;
        auto it = leaf.find(b);
        if (it != leaf.end() && it->second == lc) {
          if (lc < l - 1) return ORA_ERR_UNBALANCED;
          break;
        }
      }
    }
  }

  // Elements in the given input order; nodes numbered in order of first appearance.
  const int nc = corner_count(dim);
  m.el_anchor.resize(n);
  m.el_level.resize(n);
  m.el_nodes.assign(n, std::vector<int64_t>(nc));
  for (int64_t e = 0; e < n; ++e) {
    IPt a = {0, 0, 0};
    for (int k = 0; k < dim; ++k) a[k] = anchors[e * dim + k];
    m.el_anchor[e] = a;
    m.el_level[e] = levels[e];
    const int64_t s = int64_t(1) << (L - levels[e]);
    for (int c = 0; c < nc; ++c) {
      IPt p = corner_point(m, a, s, c);
      auto it = m.node_of.find(p);
      int64_t id;
      if (it == m.node_of.end()) {
        id = (int64_t)m.node_xyz.size();
        m.node_of[p] = id;
        m.node_xyz.push_back(p);
      } else {
        id = it->second;
      }
      m.el_nodes[e][c] = id;
    }
  }
  const int64_t nn = (int64_t)m.node_xyz.size();
  m.hanging.assign(nn, 0);
  m.cons.assign(nn, {});
  // A node that sits at the midpoint of an edge, or the centre of a face, of some
  // element is hanging; its value is the mean of that edge's ends / face's corners.
  for (int64_t e = 0; e < n; ++e) {
    const int64_t s = int64_t(1) << (L - m.el_level[e]);
    if (s < 2) continue;
    const IPt& a = m.el_anchor[e];
    // enumerate points of {0, s/2, s}^dim with 1 (edge midpoint) or 2 (face centre, 3D) mid coords
    const int np = dim == 3 ? 27 : 9;
    for (int q = 0; q < np; ++q) {
      int t3[3] = {q % 3, (q / 3) % 3, (q / 9) % 3};
      if (dim == 2) t3[2] = 0;
      int nmid = 0;
      for (int k = 0; k < dim; ++k) nmid += (t3[k] == 1);
      if (nmid == 0 || nmid == dim) continue;  // a corner, or the element centre
      IPt p = a;
      for (int k = 0; k < dim; ++k) p[k] = a[k] + t3[k] * (s / 2);
      wrap_point(m, p);
      auto it = m.node_of.find(p);
      if (it == m.node_of.end()) continue;
      const int64_t h = it->second;
      // parents: replace each mid coordinate by 0 or s
      std::vector<std::pair<int64_t, double>> par;
      const int npar = 1 << nmid;
      for (int pc = 0; pc < npar; ++pc) {
        IPt pp = a;
        int bit = 0;
        for (int k = 0; k < dim; ++k) {
          if (t3[k] == 1) {
            pp[k] = a[k] + (((pc >> bit) & 1) ? s : 0);
            ++bit;
          } else {
            pp[k] = a[k] + t3[k] * (s / 2);
          }
        }
        wrap_point(m, pp);
        auto pit = m.node_of.find(pp);
        if (pit == m.node_of.end()) return ORA_ERR_UNBALANCED;
        par.push_back({pit->second, 1.0 / npar});
      }
      if (m.hanging[h]) {
        // found again from another coarse element: must agree on the parent set
        std::set<int64_t> s1, s2;
        for (auto& pw : m.cons[h]) s1.insert(pw.first);
        for (auto& pw : par) s2.insert(pw.first);
        if (s1 != s2) return ORA_ERR_UNBALANCED;
        continue;
      }
      m.hanging[h] = 1;
      m.cons[h] = par;
    }
  }
  for (int64_t i = 0; i < nn; ++i) {
    if (!m.hanging[i]) {
      m.cons[i] = {{i, 1.0}};
    } else {
      for (auto& pw : m.cons[i])
        if (m.hanging[pw.first]) return ORA_ERR_UNBALANCED;  // chained constraints
    }
  }
  return ORA_OK;
}

// ------------------------------------------------------------------ boundary rows
// Dirichlet value of (node, field), if any: faces are scanned in increasing index and
// the last Dirichlet face that contains the node wins.  Hanging nodes are never
// Dirichlet rows (they stay constrained).
bool dirichlet(const Mesh& m, const Params& p, int64_t i, int f, double* g) {
  if (m.hanging[i]) return false;
  const int64_t size = int64_t(1) << m.L;
  bool is = false;
  for (int face = 0; face < 2 * m.dim; ++face) {
    const int ax = face / 2;
    if ((m.periodic >> ax) & 1) continue;  // identified faces carry no condition
    const int64_t want = (face & 1) ? size : 0;
    if (m.node_xyz[i][ax] != want) continue;
    if (p.bc_type[face][f] != 1) continue;
    is = true;
    if (p.mms) {
      double x[3] = {0, 0, 0};
      for (int k = 0; k < m.dim; ++k) x[k] = (double)m.node_xyz[i][k] / (double)size;
      MmsField mf[6];
      mms_fields(m.dim, x, p.t, p.steady, mf);
      *g = mf[f].val;
    } else {
      *g = p.bc_val[face][f];
    }
  }
  return is;
}

// ------------------------------------------------------------------ quadrature-point state
struct Qp {
  double N[8];        // shape functions
  double dN[8][3];    // physical gradients
  double w;           // quadrature weight (h/2)^dim
  double x[3];        // physical coordinates
};

// Tensor-product Q1 shape functions at the Gauss point with sign pattern q, in the
// element of anchor a and edge h (coordinates in [0,1]).
void eval_qp(const Mesh& m, int64_t e, int q, Qp& Q) {
  const int dim = m.dim;
  const double size = (double)(int64_t(1) << m.L);
  const double h = std::ldexp(1.0, -m.el_level[e]);
  const double g = 1.0 / std::sqrt(3.0);
  double xi[3] = {0, 0, 0};
  for (int k = 0; k < dim; ++k) {
    xi[k] = ((q >> k) & 1) ? g : -g;
    Q.x[k] = (double)m.el_anchor[e][k] / size + 0.5 * h * (xi[k] + 1.0);
  }
  if (dim == 2) Q.x[2] = 0.0;
  Q.w = std::pow(0.5 * h, dim);
  const int nc = corner_count(dim);
  for (int c = 0; c < nc; ++c) {
    double f1[3], d1[3];
    for (int k = 0; k < dim; ++k) {
      const double sk = ((c >> k) & 1) ? 1.0 : -1.0;
      f1[k] = 0.5 * (1.0 + sk * xi[k]);
      d1[k] = 0.5 * sk;
    }
    double N = 1.0;
    for (int k = 0; k < dim; ++k) N *= f1[k];
    Q.N[c] = N;
    for (int a = 0; a < 3; ++a) Q.dN[c][a] = 0.0;
    for (int a = 0; a < dim; ++a) {
      double d = d1[a] * (2.0 / h);
      for (int k = 0; k < dim; ++k)
        if (k != a) d *= f1[k];
      Q.dN[c][a] = d;
    }
  }
}

// Element nodal values of a node-major 3-field vector through the constraints.
void gather3(const Mesh& m, int64_t e, const double* U, double out[8][3]) {
  const int nc = corner_count(m.dim);
  for (int c = 0; c < nc; ++c) {
    const int64_t i = m.el_nodes[e][c];
    for (int f = 0; f < 3; ++f) out[c][f] = 0.0;
    for (auto& pw : m.cons[i])
      for (int f = 0; f < 3; ++f) out[c][f] += pw.second * U[3 * pw.first + f];
  }
}

void gatherd(const Mesh& m, int64_t e, const double* V, double out[8][3]) {
  // velocity: node-major with 3 slots per node (the last is ignored in 2D)
  gather3(m, e, V, out);
}

struct QpPhys {
  double c[2], gc[2][3], gp[3], va[3], hs[2], f[3];
  double tau, R[2], P[2][3];
  double kappa;
};

// State at one Gauss point: interpolated fields, tau_c, strong residual R_s and the
// transport vector P_s = v - z_s grad(phi).
void qp_state(const Mesh& m, const Params& p, int64_t e, const Qp& Q, const double Ue[8][3],
              const double Uke[8][3], const double Ukm1e[8][3], const double Ve[8][3], QpPhys& S) {
  const int dim = m.dim, nc = corner_count(dim);
  const double h = std::ldexp(1.0, -m.el_level[e]);
  for (int s = 0; s < 2; ++s) {
    S.c[s] = 0; S.hs[s] = 0;
    for (int a = 0; a < 3; ++a) S.gc[s][a] = 0;
  }
  for (int a = 0; a < 3; ++a) { S.gp[a] = 0; S.va[a] = 0; }
  for (int c = 0; c < nc; ++c) {
    for (int s = 0; s < 2; ++s) {
      S.c[s] += Q.N[c] * Ue[c][s];
      for (int a = 0; a < dim; ++a) S.gc[s][a] += Q.dN[c][a] * Ue[c][s];
      if (!p.steady) S.hs[s] += Q.N[c] * (p.beta1 * Uke[c][s] + p.beta2 * Ukm1e[c][s]) / p.dt;
    }
    for (int a = 0; a < dim; ++a) {
      S.gp[a] += Q.dN[c][a] * Ue[c][2];
      S.va[a] += Q.N[c] * Ve[c][a];
    }
  }
  S.kappa = p.steady ? 0.0 : p.beta0 / p.dt;
  if (p.mms) {
    mms_forcing(dim, Q.x, p.t, p.eps, p.steady, S.f);
  } else {
    S.f[0] = S.f[1] = S.f[2] = 0.0;
  }
  // tau_c = (4/dt^2 + v.G.v + C_I G:G)^(-1/2), G = (2/h)^2 I  (Sec. 3.1)
  double vv = 0;
  for (int a = 0; a < dim; ++a) vv += S.va[a] * S.va[a];
  const double G = (2.0 / h) * (2.0 / h);
  const double arg = (p.steady ? 0.0 : 4.0 / (p.dt * p.dt)) + G * vv + p.C_I * dim * G * G;
  S.tau = p.vms ? 1.0 / std::sqrt(arg) : 0.0;
  for (int s = 0; s < 2; ++s) {
    // R_s = (beta0 c + beta1 c^k + beta2 c^{k-1})/dt + v.grad c - div(grad c + z c grad phi) - f.
    // On an axis-aligned Q1 cube lap(c) = lap(phi) = 0, so the divergence reduces to
    // z grad c . grad phi.
    double adv = 0, mig = 0;
    for (int a = 0; a < dim; ++a) {
      adv += S.va[a] * S.gc[s][a];
      mig += S.gc[s][a] * S.gp[a];
    }
    S.R[s] = S.kappa * S.c[s] + S.hs[s] + adv - kZ[s] * mig - S.f[s];
    for (int a = 0; a < 3; ++a) S.P[s][a] = (a < dim) ? S.va[a] - kZ[s] * S.gp[a] : 0.0;
  }
}

// ------------------------------------------------------------------ residual
void element_residual(const Mesh& m, const Params& p, int64_t e, const double* U, const double* Uk,
                      const double* Ukm1, const double* adv, double Fe[8][3]) {
  const int dim = m.dim, nc = corner_count(dim);
  double Ue[8][3], Uke[8][3], Ukm1e[8][3], Ve[8][3];
  gather3(m, e, U, Ue);
  gather3(m, e, Uk, Uke);
  gather3(m, e, Ukm1, Ukm1e);
  gatherd(m, e, adv, Ve);
  for (int c = 0; c < nc; ++c)
    for (int f = 0; f < 3; ++f) Fe[c][f] = 0.0;
  const double lam2 = 2.0 * p.eps * p.eps;
  for (int q = 0; q < nc; ++q) {
    Qp Q;
    eval_qp(m, e, q, Q);
    QpPhys S;
    qp_state(m, p, e, Q, Ue, Uke, Ukm1e, Ve, S);
    for (int i = 0; i < nc; ++i) {
      // Nernst-Planck rows (Def. 3):
      // (q, (b0 c + b1 c^k + b2 c^{k-1})/dt) + (q, v.grad c) - (q, f)
      //   + (grad q, grad c + z c grad phi + tau R (v - z grad phi))
      for (int s = 0; s < 2; ++s) {
        double adv_s = 0, flux = 0;
        for (int a = 0; a < dim; ++a) adv_s += S.va[a] * S.gc[s][a];
        for (int a = 0; a < dim; ++a)
          flux += Q.dN[i][a] * (S.gc[s][a] + kZ[s] * S.c[s] * S.gp[a] + S.tau * S.R[s] * S.P[s][a]);
        Fe[i][s] += Q.w * (Q.N[i] * (S.kappa * S.c[s] + S.hs[s] + adv_s - S.f[s]) + flux);
      }
      // Poisson row (Def. 3): 2 Lambda^2 (grad q, grad phi) - (q, sum z c) + (q, sum z tau R) - (q, f_phi)
      double gg = 0;
      for (int a = 0; a < dim; ++a) gg += Q.dN[i][a] * S.gp[a];
      double charge = 0, fine = 0;
      for (int s = 0; s < 2; ++s) {
        charge += kZ[s] * S.c[s];
        fine += kZ[s] * S.tau * S.R[s];
      }
      Fe[i][2] += Q.w * (lam2 * gg - Q.N[i] * charge + Q.N[i] * fine - Q.N[i] * S.f[2]);
    }
  }
}

// Element contributions of elements e0 <= e < e1, assembled with the transpose of the
// constraints and added into F (no other rows touched).
void residual_elements(const Mesh& m, const Params& p, const double* U, const double* Uk, const double* Ukm1,
                       const double* adv, int64_t e0, int64_t e1, double* F) {
  const int nc = corner_count(m.dim);
  for (int64_t e = e0; e < e1; ++e) {
    double Fe[8][3];
    element_residual(m, p, e, U, Uk, Ukm1, adv, Fe);
    // assemble with the transpose of the constraints
    for (int c = 0; c < nc; ++c)
      for (auto& pw : m.cons[m.el_nodes[e][c]])
        for (int f = 0; f < 3; ++f) F[3 * pw.first + f] += pw.second * Fe[c][f];
  }
}

void residual(const Mesh& m, const Params& p, const double* U, const double* Uk, const double* Ukm1,
              const double* adv, double* F) {
  const int64_t nn = (int64_t)m.node_xyz.size();
  for (int64_t i = 0; i < 3 * nn; ++i) F[i] = 0.0;
  residual_elements(m, p, U, Uk, Ukm1, adv, 0, (int64_t)m.el_nodes.size(), F);
  for (int64_t i = 0; i < nn; ++i) {
    if (m.hanging[i]) {
      // constraint row: U_h - sum_p w_p U_p
      for (int f = 0; f < 3; ++f) {
        double v = U[3 * i + f];
        for (auto& pw : m.cons[i]) v -= pw.second * U[3 * pw.first + f];
        F[3 * i + f] = v;
      }
      continue;
    }
    for (int f = 0; f < 3; ++f) {
      double g;
      if (dirichlet(m, p, i, f, &g)) F[3 * i + f] = U[3 * i + f] - g;
    }
  }
}

// ------------------------------------------------------------------ analytic Jacobian
// Element Jacobian J[(i,fi),(j,fj)] = d Fe[i][fi] / d Ue[j][fj] (before constraints).
void element_jacobian(const Mesh& m, const Params& p, int64_t e, const double* U, const double* Uk,
                      const double* Ukm1, const double* adv, double Je[24][24]) {
  const int dim = m.dim, nc = corner_count(dim);
  double Ue[8][3], Uke[8][3], Ukm1e[8][3], Ve[8][3];
  gather3(m, e, U, Ue);
  gather3(m, e, Uk, Uke);
  gather3(m, e, Ukm1, Ukm1e);
  gatherd(m, e, adv, Ve);
  std::memset(Je, 0, sizeof(double) * 24 * 24);
  const double lam2 = 2.0 * p.eps * p.eps;
  for (int q = 0; q < nc; ++q) {
    Qp Q;
    eval_qp(m, e, q, Q);
    QpPhys S;
    qp_state(m, p, e, Q, Ue, Uke, Ukm1e, Ve, S);
    for (int j = 0; j < nc; ++j) {
      // derivatives of R_s with respect to the trial functions of node j
      double dRdc[2], dRdp[2];
      for (int s = 0; s < 2; ++s) {
        double pg = 0, gcg = 0;
        for (int a = 0; a < dim; ++a) {
          pg += S.P[s][a] * Q.dN[j][a];
          gcg += S.gc[s][a] * Q.dN[j][a];
        }
        dRdc[s] = S.kappa * Q.N[j] + pg;
        dRdp[s] = -kZ[s] * gcg;
      }
      for (int i = 0; i < nc; ++i) {
        double gij = 0, gip = 0, vgj = 0;
        for (int a = 0; a < dim; ++a) {
          gij += Q.dN[i][a] * Q.dN[j][a];
          gip += Q.dN[i][a] * S.gp[a];
          vgj += S.va[a] * Q.dN[j][a];
        }
        for (int s = 0; s < 2; ++s) {
          double giP = 0;
          for (int a = 0; a < dim; ++a) giP += Q.dN[i][a] * S.P[s][a];
          // d F_s,i / d c_s,j
          Je[3 * i + s][3 * j + s] +=
              Q.w * (Q.N[i] * (S.kappa * Q.N[j] + vgj) + gij + kZ[s] * Q.N[j] * gip + S.tau * dRdc[s] * giP);
          // d F_s,i / d phi_j
          Je[3 * i + s][3 * j + 2] +=
              Q.w * (kZ[s] * S.c[s] * gij + S.tau * dRdp[s] * giP - S.tau * S.R[s] * kZ[s] * gij);
          // d F_phi,i / d c_s,j
          Je[3 * i + 2][3 * j + s] += Q.w * (-Q.N[i] * kZ[s] * Q.N[j] + Q.N[i] * kZ[s] * S.tau * dRdc[s]);
        }
        Je[3 * i + 2][3 * j + 2] +=
            Q.w * (lam2 * gij + Q.N[i] * (kZ[0] * S.tau * dRdp[0] + kZ[1] * S.tau * dRdp[1]));
      }
    }
  }
}

// Triplets of the global Jacobian (duplicates to be summed by the caller).
int64_t jacobian_triplets(const Mesh& m, const Params& p, const double* U, const double* Uk,
                          const double* Ukm1, const double* adv, int64_t* I, int64_t* J, double* X) {
  const int64_t nn = (int64_t)m.node_xyz.size();
  const int nc = corner_count(m.dim);
  // row kind: 0 = PDE row, 1 = Dirichlet, 2 = hanging
  std::vector<char> kind(3 * nn, 0);
  for (int64_t i = 0; i < nn; ++i)
    for (int f = 0; f < 3; ++f) {
      double g;
      if (m.hanging[i]) kind[3 * i + f] = 2;
      else if (dirichlet(m, p, i, f, &g)) kind[3 * i + f] = 1;
    }
  int64_t k = 0;
  auto put = [&](int64_t r, int64_t c, double v) {
    if (I) { I[k] = r; J[k] = c; X[k] = v; }
    ++k;
  };
  for (int64_t e = 0; e < (int64_t)m.el_nodes.size(); ++e) {
    double Je[24][24];
    if (I) element_jacobian(m, p, e, U, Uk, Ukm1, adv, Je);
    for (int ci = 0; ci < nc; ++ci)
      for (auto& pi : m.cons[m.el_nodes[e][ci]])
        for (int fi = 0; fi < 3; ++fi) {
          const int64_t r = 3 * pi.first + fi;
          if (kind[r] != 0) continue;
          for (int cj = 0; cj < nc; ++cj)
            for (auto& pj : m.cons[m.el_nodes[e][cj]])
              for (int fj = 0; fj < 3; ++fj)
                put(r, 3 * pj.first + fj, I ? pi.second * pj.second * Je[3 * ci + fi][3 * cj + fj] : 0.0);
        }
  }
  for (int64_t i = 0; i < nn; ++i)
    for (int f = 0; f < 3; ++f) {
      const int64_t r = 3 * i + f;
      if (kind[r] == 1) put(r, r, 1.0);
      if (kind[r] == 2) {
        put(r, r, 1.0);
        for (auto& pw : m.cons[i]) put(r, 3 * pw.first + f, -pw.second);
      }
    }
  return k;
}

// ------------------------------------------------------------------ matrix-free Jv
// Directional derivative of the residual written from the linearised Gauss-point
// expressions (an independent derivation from element_jacobian).
// Element contributions of elements e0 <= e < e1 added into JV (no other rows touched).
void jv_elements(const Mesh& m, const Params& p, const double* U, const double* Uk, const double* Ukm1,
                 const double* adv, const double* V, int64_t e0, int64_t e1, double* JV) {
  const int dim = m.dim, nc = corner_count(dim);
  const double lam2 = 2.0 * p.eps * p.eps;
  for (int64_t e = e0; e < e1; ++e) {
    double Ue[8][3], Uke[8][3], Ukm1e[8][3], Ve[8][3], De[8][3], Fe[8][3];
    gather3(m, e, U, Ue);
    gather3(m, e, Uk, Uke);
    gather3(m, e, Ukm1, Ukm1e);
    gatherd(m, e, adv, Ve);
    gather3(m, e, V, De);
    for (int c = 0; c < nc; ++c)
      for (int f = 0; f < 3; ++f) Fe[c][f] = 0.0;
    for (int q = 0; q < nc; ++q) {
      Qp Q;
      eval_qp(m, e, q, Q);
      QpPhys S;
      qp_state(m, p, e, Q, Ue, Uke, Ukm1e, Ve, S);
      double dc[2] = {0, 0}, dgc[2][3] = {{0, 0, 0}, {0, 0, 0}}, dgp[3] = {0, 0, 0};
      for (int c = 0; c < nc; ++c) {
        for (int s = 0; s < 2; ++s) {
          dc[s] += Q.N[c] * De[c][s];
          for (int a = 0; a < dim; ++a) dgc[s][a] += Q.dN[c][a] * De[c][s];
        }
        for (int a = 0; a < dim; ++a) dgp[a] += Q.dN[c][a] * De[c][2];
      }
      double dR[2], mass[2];
      for (int s = 0; s < 2; ++s) {
        double vdg = 0, a1 = 0, a2 = 0;
        for (int a = 0; a < dim; ++a) {
          vdg += S.va[a] * dgc[s][a];
          a1 += dgc[s][a] * S.gp[a];
          a2 += S.gc[s][a] * dgp[a];
        }
        mass[s] = S.kappa * dc[s] + vdg;
        dR[s] = mass[s] - kZ[s] * (a1 + a2);
      }
      for (int i = 0; i < nc; ++i) {
        for (int s = 0; s < 2; ++s) {
          double flux = 0;
          for (int a = 0; a < dim; ++a)
            flux += Q.dN[i][a] * (dgc[s][a] + kZ[s] * (dc[s] * S.gp[a] + S.c[s] * dgp[a]) +
                                  S.tau * dR[s] * S.P[s][a] - S.tau * S.R[s] * kZ[s] * dgp[a]);
          Fe[i][s] += Q.w * (Q.N[i] * mass[s] + flux);
        }
        double gg = 0;
        for (int a = 0; a < dim; ++a) gg += Q.dN[i][a] * dgp[a];
        const double charge = kZ[0] * dc[0] + kZ[1] * dc[1];
        const double fine = S.tau * (kZ[0] * dR[0] + kZ[1] * dR[1]);
        Fe[i][2] += Q.w * (lam2 * gg - Q.N[i] * charge + Q.N[i] * fine);
      }
    }
    for (int c = 0; c < nc; ++c)
      for (auto& pw : m.cons[m.el_nodes[e][c]])
        for (int f = 0; f < 3; ++f) JV[3 * pw.first + f] += pw.second * Fe[c][f];
  }
}

void jv(const Mesh& m, const Params& p, const double* U, const double* Uk, const double* Ukm1,
        const double* adv, const double* V, double* JV) {
  const int64_t nn = (int64_t)m.node_xyz.size();
  for (int64_t i = 0; i < 3 * nn; ++i) JV[i] = 0.0;
  jv_elements(m, p, U, Uk, Ukm1, adv, V, 0, (int64_t)m.el_nodes.size(), JV);
  for (int64_t i = 0; i < nn; ++i) {
    if (m.hanging[i]) {
      for (int f = 0; f < 3; ++f) {
        double v = V[3 * i + f];
        for (auto& pw : m.cons[i]) v -= pw.second * V[3 * pw.first + f];
        JV[3 * i + f] = v;
      }
      continue;
    }
    for (int f = 0; f < 3; ++f) {
      double g;
      if (dirichlet(m, p, i, f, &g)) JV[3 * i + f] = V[3 * i + f];
    }
  }
}

// ------------------------------------------------------------------ Navier-Stokes block
// The semi-implicit VMS momentum and solenoidality rows of Def. 3 (Sec. 3.1), linear in
// the unknown (v, p) at t^{k+1}:
//   momentum, test w_i:
//     (1/Sc)(w_i, (b0 v_i + b1 v_i^k + b2 v_i^{k-1})/dt) + (1/Sc)(w_i, v~_j d_j v_i)
//     + (1/Sc)(d_j w_i, v~_j tau_m R_m,i) + (w_i, d_i p) + (d_i w_i, tau_sol R_sol)
//     + (d_j w_i, d_j v_i) + kappa/(2 Lambda^2) (w_i, (sum_s z_s c_s) d_i phi) - (w_i, f_i)
//   solenoidality, test q:
//     (q, d_i v_i) + (d_i q, tau_m R_m,i)
// with the strong residuals
//     R_m,i = (1/Sc)((b0 v_i + b1 v_i^k + b2 v_i^{k-1})/dt + v~_j d_j v_i) + d_i p
//             + kappa/(2 Lambda^2)(sum_s z_s c_s) d_i phi - f_i     (lap v = 0 on a Q1 cube)
//     R_sol = d_i v_i,
//     tau_m = (4/dt^2 + v~.G.v~ + C_I Sc^2 G:G)^(-1/2),   tau_sol = 1 / (tr(G) tau_m),
// G = (2/h)^2 I, and 1/Re = Sc (the velocity scale D/L of Sec. 2.2 makes Re = 1/Sc).  The
// fine-scale velocity is v^f = -tau_m R_m (Sec. 3.1), so the solenoidality row carries
// +(d_i q, tau_m R_m,i): the printed minus sign in front of that term (next to the
// misprinted test function) contradicts v^f = -tau_m R_m and would destabilise the
// pressure.  v~ = 2 v^k - v^{k-1} (Eq. averaging1) is an input.  (c_s, phi) is the PNP
// state the body force is taken from (the latest block iterate).  f is the forcing of
// the manufactured solution (zero otherwise).
//
// Unknowns: node-major [nn][4] = (v_x, v_y, v_z, p); in 2D slot 2 is inactive (its row
// is X_2 = 0).  Row kinds: hanging-node constraint rows, Dirichlet rows X - g (per face
// and component, the last Dirichlet face containing the node wins) and, with `pin`, the
// pressure row of the node at the origin, X_3 - pin_val.
struct NsParams {
  double Sc;     // Schmidt number (inertia coefficient 1/Sc)
  double kappa;  // electrohydrodynamic coupling constant
  double eps;    // Lambda: body-force coefficient kappa / (2 Lambda^2)
  double dt;
  double beta0, beta1, beta2;
  double C_I;
  double t;      // time level of the unknown (manufactured solution only)
  double pin_val;
  int32_t steady;  // 1: drop the time-derivative terms and 4/dt^2 in tau_m
  int32_t vms;     // 0: tau_m = tau_sol = 0
  int32_t mms;     // 1: manufactured forcing and Dirichlet values
  int32_t pin;     // 1: pressure of the origin node fixed to pin_val
  int32_t bc_type[6][4];
  double bc_val[6][4];
  double Sc_inv() const { return 1.0 / Sc; }
};

// Manufactured (u, v, w, p) of Eq. manufac_sol (3D: times cos(pi z), w = 0): value,
// gradient, Laplacian, time derivative; the momentum forcing that makes them (with the
// manufactured c+-, phi) an exact solution of the non-dimensional NS equation of Sec. 2.2,
//   (1/Sc)(dv/dt + v.grad v) + grad p - lap v + kappa/(2 Lambda^2)(c+ - c-) grad phi = f.
void ns_mms(const NsParams& p, int dim, const double* x, double t, MmsField out[4], double f[3]) {
  MmsField m[6];
  mms_fields(dim, x, t, p.steady, m);
  out[0] = m[3];
  out[1] = m[4];
  out[2] = m[5];
  // p = cos(2t) sin(2 pi x) cos(2 pi y) (3D: cos(pi z)): the same function as u
  out[3] = m[3];
  const double body = p.kappa / (2.0 * p.eps * p.eps) * (m[0].val - m[1].val);
  for (int i = 0; i < 3; ++i) {
    f[i] = 0.0;
    if (i >= dim) continue;
    double adv = 0.0;
    for (int j = 0; j < dim; ++j) adv += out[j].val * out[i].grad[j];
    f[i] = p.Sc_inv() * (out[i].dval_dt + adv) + out[3].grad[i] - out[i].lap + body * m[2].grad[i];
  }
}

// Dirichlet value of (node, slot), if any.
bool ns_dirichlet(const Mesh& m, const NsParams& p, int64_t i, int f, double* g) {
  if (m.hanging[i]) return false;
  if (m.dim == 2 && f == 2) {
    *g = 0.0;
    return true;
  }
  const int64_t size = int64_t(1) << m.L;
  bool is = false;
  for (int face = 0; face < 2 * m.dim; ++face) {
    const int ax = face / 2;
    if ((m.periodic >> ax) & 1) continue;
    const int64_t want = (face & 1) ? size : 0;
    if (m.node_xyz[i][ax] != want) continue;
    if (p.bc_type[face][f] != 1) continue;
    is = true;
    if (p.mms) {
      double x[3] = {0, 0, 0};
      for (int k = 0; k < m.dim; ++k) x[k] = (double)m.node_xyz[i][k] / (double)size;
      MmsField mf[4];
      double fr[3];
      ns_mms(p, m.dim, x, p.t, mf, fr);
      *g = mf[f].val;
    } else {
      *g = p.bc_val[face][f];
    }
  }
  if (!is && f == 3 && p.pin) {
    bool origin = true;
    for (int k = 0; k < m.dim; ++k) origin = origin && m.node_xyz[i][k] == 0;
    if (origin) {
      *g = p.pin_val;
      return true;
    }
  }
  return is;
}

// Element nodal values of a node-major 4-slot vector through the constraints.
void gather4(const Mesh& m, int64_t e, const double* X, double out[8][4]) {
  const int nc = corner_count(m.dim);
  for (int c = 0; c < nc; ++c) {
    for (int f = 0; f < 4; ++f) out[c][f] = 0.0;
    for (auto& pw : m.cons[m.el_nodes[e][c]])
      for (int f = 0; f < 4; ++f) out[c][f] += pw.second * X[4 * pw.first + f];
  }
}

// Element rows of the NS system from element-local nodal values (X through the
// constraints).  `with_data` = 0 drops every term that does not depend on X (history,
// body force, forcing): then Fe is the element matrix times Xe.
void ns_element_core(const Mesh& m, const NsParams& p, int64_t e, const double Xe[8][4], const double Ae[8][3],
                     const double Vke[8][3], const double Vkm1e[8][3], const double Ue[8][3], int with_data,
                     double Fe[8][4]) {
  const int dim = m.dim, nc = corner_count(dim);
  for (int c = 0; c < nc; ++c)
    for (int f = 0; f < 4; ++f) Fe[c][f] = 0.0;
  const double h = std::ldexp(1.0, -m.el_level[e]);
  const double G = (2.0 / h) * (2.0 / h);
  const double kap = p.steady ? 0.0 : p.beta0 / p.dt;
  const double isc = p.Sc_inv();
  const double fb = p.kappa / (2.0 * p.eps * p.eps);
  for (int q = 0; q < nc; ++q) {
    Qp Q;
    eval_qp(m, e, q, Q);
    double v[3] = {0, 0, 0}, gv[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, gp[3] = {0, 0, 0};
    double va[3] = {0, 0, 0}, hv[3] = {0, 0, 0}, cp = 0, cm = 0, gphi[3] = {0, 0, 0};
    for (int c = 0; c < nc; ++c) {
      for (int i = 0; i < dim; ++i) {
        v[i] += Q.N[c] * Xe[c][i];
        va[i] += Q.N[c] * Ae[c][i];
        if (!p.steady) hv[i] += Q.N[c] * (p.beta1 * Vke[c][i] + p.beta2 * Vkm1e[c][i]) / p.dt;
        for (int j = 0; j < dim; ++j) gv[i][j] += Q.dN[c][j] * Xe[c][i];  // d v_i / d x_j
        gp[i] += Q.dN[c][i] * Xe[c][3];
        gphi[i] += Q.dN[c][i] * Ue[c][2];
      }
      cp += Q.N[c] * Ue[c][0];
      cm += Q.N[c] * Ue[c][1];
    }
    double f[3] = {0, 0, 0};
    if (p.mms && with_data) {
      MmsField mf[4];
      ns_mms(p, dim, Q.x, p.t, mf, f);
    }
    double vv = 0, div = 0;
    for (int i = 0; i < dim; ++i) {
      vv += va[i] * va[i];
      div += gv[i][i];
    }
    // tau_m = (4/dt^2 + v~.G.v~ + C_I (1/Re)^2 G:G)^(-1/2), G:G = d (2/h)^4, 1/Re = Sc
    const double arg = (p.steady ? 0.0 : 4.0 / (p.dt * p.dt)) + G * vv + p.C_I * p.Sc * p.Sc * dim * G * G;
    const double tau_m = p.vms ? 1.0 / std::sqrt(arg) : 0.0;
    const double tau_s = p.vms ? 1.0 / (dim * G * tau_m) : 0.0;  // 1 / (tr(G) tau_m)
    double Rm[3] = {0, 0, 0};
    for (int i = 0; i < dim; ++i) {
      double adv_i = 0;
      for (int j = 0; j < dim; ++j) adv_i += va[j] * gv[i][j];
      Rm[i] = isc * (kap * v[i] + adv_i) + gp[i];
      if (with_data) Rm[i] += isc * hv[i] + fb * (cp - cm) * gphi[i] - f[i];
    }
    for (int a = 0; a < nc; ++a) {
      double vgN = 0;  // v~ . grad N_a
      for (int j = 0; j < dim; ++j) vgN += va[j] * Q.dN[a][j];
      for (int i = 0; i < dim; ++i) {
        double visc = 0;
        for (int j = 0; j < dim; ++j) visc += Q.dN[a][j] * gv[i][j];
        // the Galerkin terms other than the viscous one are N_a R_m,i (lap v = 0)
        Fe[a][i] += Q.w * (Q.N[a] * Rm[i] + visc + isc * vgN * tau_m * Rm[i] + Q.dN[a][i] * tau_s * div);
      }
      double pspg = 0;
      for (int i = 0; i < dim; ++i) pspg += Q.dN[a][i] * tau_m * Rm[i];
      Fe[a][3] += Q.w * (Q.N[a] * div + pspg);
    }
  }
}

void ns_element(const Mesh& m, const NsParams& p, int64_t e, const double* X, const double* adv,
                const double* Vk, const double* Vkm1, const double* U, int with_data, double Fe[8][4]) {
  double Xe[8][4], Ae[8][3], Vke[8][3], Vkm1e[8][3], Ue[8][3];
  gather4(m, e, X, Xe);
  gather3(m, e, adv, Ae);
  gather3(m, e, Vk, Vke);
  gather3(m, e, Vkm1, Vkm1e);
  gather3(m, e, U, Ue);
  ns_element_core(m, p, e, Xe, Ae, Vke, Vkm1e, Ue, with_data, Fe);
}

// Row fix-ups of the NS system: constraint rows of hanging nodes and Dirichlet rows.
// affine = 1: the rows of the residual (X - g); 0: the rows of the matrix (X).
void ns_rows(const Mesh& m, const NsParams& p, const double* X, int affine, double* F) {
  const int64_t nn = (int64_t)m.node_xyz.size();
  for (int64_t i = 0; i < nn; ++i) {
    if (m.hanging[i]) {
      for (int f = 0; f < 4; ++f) {
        double v = X[4 * i + f];
        for (auto& pw : m.cons[i]) v -= pw.second * X[4 * pw.first + f];
        F[4 * i + f] = v;
      }
      continue;
    }
    for (int f = 0; f < 4; ++f) {
      double g;
      if (ns_dirichlet(m, p, i, f, &g)) F[4 * i + f] = X[4 * i + f] - (affine ? g : 0.0);
    }
  }
}

// Element contributions of elements e0 <= e < e1, assembled with the transpose of the
// constraints and added into F (no other rows touched).
void ns_apply_elements(const Mesh& m, const NsParams& p, const double* X, const double* adv, const double* Vk,
                       const double* Vkm1, const double* U, int with_data, int64_t e0, int64_t e1, double* F) {
  const int nc = corner_count(m.dim);
  for (int64_t e = e0; e < e1; ++e) {
    double Fe[8][4];
    ns_element(m, p, e, X, adv, Vk, Vkm1, U, with_data, Fe);
    for (int c = 0; c < nc; ++c)
      for (auto& pw : m.cons[m.el_nodes[e][c]])
        for (int f = 0; f < 4; ++f) F[4 * pw.first + f] += pw.second * Fe[c][f];
  }
}

void ns_apply(const Mesh& m, const NsParams& p, const double* X, const double* adv, const double* Vk,
              const double* Vkm1, const double* U, int with_data, double* F) {
  const int64_t nn = (int64_t)m.node_xyz.size();
  for (int64_t i = 0; i < 4 * nn; ++i) F[i] = 0.0;
  ns_apply_elements(m, p, X, adv, Vk, Vkm1, U, with_data, 0, (int64_t)m.el_nodes.size(), F);
  ns_rows(m, p, X, with_data, F);
}

// Triplets of the NS matrix: each element matrix column is the element operator (without
// data) applied to a unit vector of the element's nodal values; assembled with the
// constraints, then the Dirichlet / constraint rows.
int64_t ns_matrix_triplets(const Mesh& m, const NsParams& p, const double* adv, int64_t* I, int64_t* J,
                           double* Xv) {
  const int64_t nn = (int64_t)m.node_xyz.size();
  const int nc = corner_count(m.dim);
  std::vector<char> kind(4 * nn, 0);
  for (int64_t i = 0; i < nn; ++i)
    for (int f = 0; f < 4; ++f) {
      double g;
      if (m.hanging[i]) kind[4 * i + f] = 2;
      else if (ns_dirichlet(m, p, i, f, &g)) kind[4 * i + f] = 1;
    }
  int64_t k = 0;
  auto put = [&](int64_t r, int64_t c, double v) {
    if (I) { I[k] = r; J[k] = c; Xv[k] = v; }
    ++k;
  };
  for (int64_t e = 0; e < (int64_t)m.el_nodes.size(); ++e) {
    double Ke[32][32];
    if (I) {
      // column (cj, fj): the element rows (no data) of the element-local unit vector
      double Ae[8][3], Z3[8][3] = {};
      gather3(m, e, adv, Ae);
      for (int cj = 0; cj < nc; ++cj)
        for (int fj = 0; fj < 4; ++fj) {
          double Xe[8][4] = {}, Fe[8][4];
          Xe[cj][fj] = 1.0;
          ns_element_core(m, p, e, Xe, Ae, Z3, Z3, Z3, 0, Fe);
          for (int ci = 0; ci < nc; ++ci)
            for (int fi = 0; fi < 4; ++fi) Ke[4 * ci + fi][4 * cj + fj] = Fe[ci][fi];
        }
    }
    for (int ci = 0; ci < nc; ++ci)
      for (auto& pi : m.cons[m.el_nodes[e][ci]])
        for (int fi = 0; fi < 4; ++fi) {
          const int64_t r = 4 * pi.first + fi;
          if (kind[r] != 0) continue;
          for (int cj = 0; cj < nc; ++cj)
            for (auto& pj : m.cons[m.el_nodes[e][cj]])
              for (int fj = 0; fj < 4; ++fj)
                put(r, 4 * pj.first + fj, I ? pi.second * pj.second * Ke[4 * ci + fi][4 * cj + fj] : 0.0);
        }
  }
  for (int64_t i = 0; i < nn; ++i)
    for (int f = 0; f < 4; ++f) {
      const int64_t r = 4 * i + f;
      if (kind[r] == 1) put(r, r, 1.0);
      if (kind[r] == 2) {
        put(r, r, 1.0);
        for (auto& pw : m.cons[i]) put(r, 4 * pw.first + f, -pw.second);
      }
    }
  return k;
}

}  // namespace

// ------------------------------------------------------------------ boundary flux
// Integral over boundary face `face` (axis face/2, the high side when face is odd) of
// n . (grad c_s + z_s c_s grad phi) for s = +, -, n the outward unit normal: the per
// species terms of the boundary current of Sec. 5.2 (the net species flux through the
// top boundary).  Each element with a side on that face contributes the tensor Gauss
// rule with 2^(d-1) points on its side, the Q1 fields through the constraints.
void boundary_flux(const Mesh& m, int face, const double* U, double out[2]) {
  const int dim = m.dim;
  const int ax = face / 2;
  const bool high = face & 1;
  const int64_t size = int64_t(1) << m.L;
  const double g = 1.0 / std::sqrt(3.0);
  const double nrm = high ? 1.0 : -1.0;
  out[0] = out[1] = 0.0;
  if ((m.periodic >> ax) & 1) return;  // an identified face is not a boundary
  const int nc = corner_count(dim);
  for (size_t e = 0; e < m.el_anchor.size(); ++e) {
    const int64_t s = int64_t(1) << (m.L - m.el_level[e]);
    const int64_t side = m.el_anchor[e][ax] + (high ? s : 0);
    if (side != (high ? size : 0)) continue;
    const double h = std::ldexp(1.0, -m.el_level[e]);
    double u[8][3];
    gather3(m, (int64_t)e, U, u);
    // 2^(dim-1) Gauss points of the side, weight (h/2)^(dim-1) each
    const int nq = 1 << (dim - 1);
    for (int q = 0; q < nq; ++q) {
      double xi[3] = {0, 0, 0};
      int bit = 0;
      for (int k = 0; k < dim; ++k) {
        if (k == ax) {
          xi[k] = high ? 1.0 : -1.0;
        } else {
          xi[k] = ((q >> bit) & 1) ? g : -g;
          ++bit;
        }
      }
      double val[3] = {0, 0, 0}, grad[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      for (int c = 0; c < nc; ++c) {
        double f1[3], d1[3];
        for (int k = 0; k < dim; ++k) {
          const double sk = ((c >> k) & 1) ? 1.0 : -1.0;
          f1[k] = 0.5 * (1.0 + sk * xi[k]);
          d1[k] = 0.5 * sk * (2.0 / h);
        }
        double N = 1.0;
        for (int k = 0; k < dim; ++k) N *= f1[k];
        for (int f = 0; f < 3; ++f) val[f] += N * u[c][f];
        for (int a = 0; a < dim; ++a) {
          double d = d1[a];
          for (int k = 0; k < dim; ++k)
            if (k != a) d *= f1[k];
          for (int f = 0; f < 3; ++f) grad[f][a] += d * u[c][f];
        }
      }
      const double w = std::pow(0.5 * h, dim - 1);
      for (int sp = 0; sp < 2; ++sp) {
        const double z = sp == 0 ? 1.0 : -1.0;
        out[sp] += w * nrm * (grad[sp][ax] + z * val[sp] * grad[2][ax]);
      }
    }
  }
}

// ------------------------------------------------------------------ plane integral
// Integral of each field over the plane x_ax = coord (integer units): every point of the
// plane lies in the elements whose closed range [a, a + s] along ax holds coord; an
// element whose side lies in the plane shares it with its neighbour across, so the
// element above the plane takes it (below only at the top face).  Cross-section at
// xi_ax = 2 (coord - a) / s - 1, tensor Gauss rule with 2^(d-1) points.
void plane_integral(const Mesh& m, int ax, int64_t coord, const double* U, double out[3]) {
  const int dim = m.dim;
  const int64_t size = int64_t(1) << m.L;
  const double g = 1.0 / std::sqrt(3.0);
  out[0] = out[1] = out[2] = 0.0;
  const int nc = corner_count(dim);
  for (size_t e = 0; e < m.el_anchor.size(); ++e) {
    const int64_t s = int64_t(1) << (m.L - m.el_level[e]);
    const int64_t a = m.el_anchor[e][ax];
    if (coord < a || coord > a + s) continue;          // the plane misses the element
    if (coord == a + s && coord != size) continue;     // the element above takes the side
    const double h = std::ldexp(1.0, -m.el_level[e]);
    double u[8][3];
    gather3(m, (int64_t)e, U, u);
    const int nq = 1 << (dim - 1);
    for (int q = 0; q < nq; ++q) {
      double xi[3] = {0, 0, 0};
      int bit = 0;
      for (int k = 0; k < dim; ++k) {
        if (k == ax) {
          xi[k] = 2.0 * (double)(coord - a) / (double)s - 1.0;
        } else {
          xi[k] = ((q >> bit) & 1) ? g : -g;
          ++bit;
        }
      }
      const double w = std::pow(0.5 * h, dim - 1);
      for (int c = 0; c < nc; ++c) {
        double N = 1.0;
        for (int k = 0; k < dim; ++k) N *= 0.5 * (1.0 + (((c >> k) & 1) ? 1.0 : -1.0) * xi[k]);
        for (int f = 0; f < 3; ++f) out[f] += w * N * u[c][f];
      }
    }
  }
}

// ================================================================== C interface
extern "C" {

void ora_plane_integral(void* h, int ax, int64_t coord, const double* U, double* out) {
  plane_integral(*static_cast<Mesh*>(h), ax, coord, U, out);
}

void ora_boundary_flux(void* h, int face, const double* U, double* out) {
  boundary_flux(*static_cast<Mesh*>(h), face, U, out);
}

void* ora_mesh_build(int dim, int max_level, int64_t n, const int32_t* anchors, const uint8_t* levels,
                     int periodic, int32_t* err) {
  Mesh* m = new Mesh();
  const int rc = build_mesh(*m, dim, max_level, n, anchors, levels, periodic);
  *err = rc;
  if (rc != ORA_OK) {
    delete m;
    return nullptr;
  }
  return m;
}

void ora_mesh_free(void* h) { delete static_cast<Mesh*>(h); }

void ora_mesh_sizes(void* h, int64_t* ne, int64_t* nn, int64_t* nh) {
  const Mesh& m = *static_cast<Mesh*>(h);
  *ne = (int64_t)m.el_nodes.size();
  *nn = (int64_t)m.node_xyz.size();
  int64_t c = 0;
  for (char x : m.hanging) c += x;
  *nh = c;
}

// Integer node coordinates [nn][dim], hanging flags [nn], element corner ids [ne][2^dim].
void ora_mesh_nodes(void* h, int64_t* xyz, int32_t* hanging, int64_t* el_nodes) {
  const Mesh& m = *static_cast<Mesh*>(h);
  for (size_t i = 0; i < m.node_xyz.size(); ++i) {
    for (int k = 0; k < m.dim; ++k) xyz[i * m.dim + k] = m.node_xyz[i][k];
    hanging[i] = m.hanging[i];
  }
  const int nc = corner_count(m.dim);
  for (size_t e = 0; e < m.el_nodes.size(); ++e)
    for (int c = 0; c < nc; ++c) el_nodes[e * nc + c] = m.el_nodes[e][c];
}

// Constraint triplets (row node, parent node, weight) of the hanging nodes.
int64_t ora_mesh_constraints(void* h, int64_t* rows, int64_t* cols, double* w) {
  const Mesh& m = *static_cast<Mesh*>(h);
  int64_t k = 0;
  for (size_t i = 0; i < m.node_xyz.size(); ++i) {
    if (!m.hanging[i]) continue;
    for (auto& pw : m.cons[i]) {
      if (rows) { rows[k] = (int64_t)i; cols[k] = pw.first; w[k] = pw.second; }
      ++k;
    }
  }
  return k;
}

void ora_residual(void* h, const Params* p, const double* U, const double* Uk, const double* Ukm1,
                  const double* adv, double* F) {
  residual(*static_cast<Mesh*>(h), *p, U, Uk, Ukm1, adv, F);
}

int64_t ora_jacobian(void* h, const Params* p, const double* U, const double* Uk, const double* Ukm1,
                     const double* adv, int64_t* I, int64_t* J, double* X) {
  return jacobian_triplets(*static_cast<Mesh*>(h), *p, U, Uk, Ukm1, adv, I, J, X);
}

void ora_jv(void* h, const Params* p, const double* U, const double* Uk, const double* Ukm1,
            const double* adv, const double* V, double* JV) {
  jv(*static_cast<Mesh*>(h), *p, U, Uk, Ukm1, adv, V, JV);
}

// The element contributions of elements e0 <= e < e1 (oracle element order), added into
// F / JV: no zeroing, no Dirichlet or constraint rows.  Summed over a partition of the
// elements and followed by those rows they give ora_residual / ora_jv (up to summation
// order); used to time the oracle on a sample of elements and across host threads.
void ora_residual_elements(void* h, const Params* p, const double* U, const double* Uk, const double* Ukm1,
                           const double* adv, int64_t e0, int64_t e1, double* F) {
  residual_elements(*static_cast<Mesh*>(h), *p, U, Uk, Ukm1, adv, e0, e1, F);
}

void ora_jv_elements(void* h, const Params* p, const double* U, const double* Uk, const double* Ukm1,
                     const double* adv, const double* V, int64_t e0, int64_t e1, double* JV) {
  jv_elements(*static_cast<Mesh*>(h), *p, U, Uk, Ukm1, adv, V, e0, e1, JV);
}

// Strong residuals R_+, R_- and tau_c at one Gauss point of element e (for the
// strong-form check): out = [R+, R-, tau].
void ora_qp_eval(void* h, const Params* p, int64_t e, int q, const double* U, const double* Uk,
                 const double* Ukm1, const double* adv, double* out) {
  const Mesh& m = *static_cast<Mesh*>(h);
  double Ue[8][3], Uke[8][3], Ukm1e[8][3], Ve[8][3];
  gather3(m, e, U, Ue);
  gather3(m, e, Uk, Uke);
  gather3(m, e, Ukm1, Ukm1e);
  gatherd(m, e, adv, Ve);
  Qp Q;
  eval_qp(m, e, q, Q);
  QpPhys S;
  qp_state(m, *p, e, Q, Ue, Uke, Ukm1e, Ve, S);
  out[0] = S.R[0];
  out[1] = S.R[1];
  out[2] = S.tau;
}

// Values of the Q1 field U (node-major [nn][3]) at integer points pts [npts][dim]
// (units of 2^-max_level, inside the closed domain): the point is located in a leaf by
// trying every level from the root down, then the element's trilinear interpolant (with
// hanging corners expressed through their constraints) is evaluated.
void ora_eval_points(void* h, const double* U, int64_t npts, const int64_t* pts, double* out) {
  const Mesh& m = *static_cast<Mesh*>(h);
  std::map<std::pair<IPt, int>, int64_t> leaf;
  for (size_t e = 0; e < m.el_anchor.size(); ++e) leaf[{m.el_anchor[e], m.el_level[e]}] = (int64_t)e;
  const int64_t size = int64_t(1) << m.L;
  const int nc = corner_count(m.dim);
  for (int64_t i = 0; i < npts; ++i) {
    IPt p = {0, 0, 0};
    for (int k = 0; k < m.dim; ++k) p[k] = pts[i * m.dim + k];
    int64_t e = -1;
    for (int l = 0; l <= m.L && e < 0; ++l) {
      const int64_t s = int64_t(1) << (m.L - l);
      IPt a = {0, 0, 0};
      for (int k = 0; k < m.dim; ++k) a[k] = std::min((p[k] / s) * s, size - s);
      auto it = leaf.find({a, l});
      if (it != leaf.end()) e = it->second;
    }
    for (int f = 0; f < 3; ++f) out[3 * i + f] = std::nan("");
    if (e < 0) continue;
    const int64_t s = int64_t(1) << (m.L - m.el_level[e]);
    double val[3] = {0, 0, 0};
    for (int c = 0; c < nc; ++c) {
      double N = 1.0;
      for (int k = 0; k < m.dim; ++k) {
        const double t = (double)(p[k] - m.el_anchor[e][k]) / (double)s;  // in [0, 1]
        N *= ((c >> k) & 1) ? t : 1.0 - t;
      }
      for (auto& pw : m.cons[m.el_nodes[e][c]])
        for (int f = 0; f < 3; ++f) val[f] += N * pw.second * U[3 * pw.first + f];
    }
    for (int f = 0; f < 3; ++f) out[3 * i + f] = val[f];
  }
}

// Row kinds [nn][3] (0 = PDE row, 1 = Dirichlet, 2 = hanging) and Dirichlet values.
void ora_bc_rows(void* h, const Params* p, int32_t* kind, double* g) {
  const Mesh& m = *static_cast<Mesh*>(h);
  for (size_t i = 0; i < m.node_xyz.size(); ++i)
    for (int f = 0; f < 3; ++f) {
      double v = 0.0;
      int k = 0;
      if (m.hanging[i]) k = 2;
      else if (dirichlet(m, *p, (int64_t)i, f, &v)) k = 1;
      kind[3 * i + f] = k;
      g[3 * i + f] = v;
    }
}

// Manufactured solution at points x [n][3]: out [n][6] = (c+, c-, phi, u, v, w) and
// forcing [n][3] = (f+, f-, f_phi).
void ora_mms(int dim, double eps, double t, int steady, int64_t n, const double* x, double* vals,
             double* forcing) {
  for (int64_t i = 0; i < n; ++i) {
    MmsField mf[6];
    mms_fields(dim, x + 3 * i, t, steady, mf);
    for (int f = 0; f < 6; ++f) vals[6 * i + f] = mf[f].val;
    mms_forcing(dim, x + 3 * i, t, eps, steady, forcing + 3 * i);
  }
}

// ------------------------------------------------------------------ Navier-Stokes block
// F = the NS rows of the unknown X [nn][4] (with_data = 1: the residual of the linear
// system, affine in X; 0: the matrix times X), given v~ (adv), the velocity history
// (Vk, Vkm1) and the PNP state U the body force is taken from, all [nn][3].
void ora_ns_apply(void* h, const NsParams* p, const double* X, const double* adv, const double* Vk,
                  const double* Vkm1, const double* U, int with_data, double* F) {
  ns_apply(*static_cast<Mesh*>(h), *p, X, adv, Vk, Vkm1, U, with_data, F);
}

// The element contributions of elements e0 <= e < e1 added into F (no zeroing, no
// Dirichlet or constraint rows); for timing the oracle on a sample across host threads.
void ora_ns_apply_elements(void* h, const NsParams* p, const double* X, const double* adv, const double* Vk,
                           const double* Vkm1, const double* U, int with_data, int64_t e0, int64_t e1, double* F) {
  ns_apply_elements(*static_cast<Mesh*>(h), *p, X, adv, Vk, Vkm1, U, with_data, e0, e1, F);
}

// Triplets of the NS matrix (duplicates to be summed by the caller); pass null arrays to
// count them.
int64_t ora_ns_matrix(void* h, const NsParams* p, const double* adv, int64_t* I, int64_t* J, double* X) {
  return ns_matrix_triplets(*static_cast<Mesh*>(h), *p, adv, I, J, X);
}

// Row kinds [nn][4] (0 = PDE row, 1 = Dirichlet or pressure pin, 2 = hanging) and values.
void ora_ns_bc_rows(void* h, const NsParams* p, int32_t* kind, double* g) {
  const Mesh& m = *static_cast<Mesh*>(h);
  for (size_t i = 0; i < m.node_xyz.size(); ++i)
    for (int f = 0; f < 4; ++f) {
      double v = 0.0;
      int k = 0;
      if (m.hanging[i]) k = 2;
      else if (ns_dirichlet(m, *p, (int64_t)i, f, &v)) k = 1;
      kind[4 * i + f] = k;
      g[4 * i + f] = v;
    }
}

// Manufactured (u, v, w, p) [n][4] and momentum forcing [n][3] at points x [n][3].
void ora_ns_mms(const NsParams* p, int dim, double t, int64_t n, const double* x, double* vals, double* forcing) {
  for (int64_t i = 0; i < n; ++i) {
    MmsField mf[4];
    ns_mms(*p, dim, x + 3 * i, t, mf, forcing + 3 * i);
    for (int f = 0; f < 4; ++f) vals[4 * i + f] = mf[f].val;
  }
}

}  // extern "C"


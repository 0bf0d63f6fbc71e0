// FastVPINNs CPU oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, FP64 restatement of what the FastVPINNs loss path computes,
// used to check the CUDA library.  Only the tests, the smoke check and the
// benchmark's CPU-baseline leg may load it.  It shares no code, header,
// table or constant with the CUDA path.
//
// Written from arXiv 2404.12063 ("FastVPINNs"):
//   * model problem  -eps Lap u + b.grad u = f, u = g on the boundary (Sec. 2.1, Eq. CD2D_strong)
//   * MLP u_NN = l o T^(h) o ... o T^(1), tanh hidden layers, linear output (Sec. 2.2, Eq. NN)
//   * cell residual W_k = int_K (grad u . grad v_k - f v_k) by quadrature (Sec. 2.3,
//     Eq. VPINNs_Bound_Loss and the quadrature sum below it), per-element loops
//     in the hp-VPINN style of Algorithm 1 (with the subtraction of F taken out
//     of the quadrature loop, as App. A.2 assembles F)
//   * loss: Algorithm 3 (mean over test functions, sum over elements) by
//     default, or Eq. (loss) (1/N_elem) sum_k |W_k|^2; plus tau L_b (Eq.
//     PINNs_Loss_components) and gamma L_s (Sec. 4.7)
//   * bilinear map, its Jacobian and inverse (App. A.1)
//   * Gauss-Lobatto-Legendre quadrature and test functions v_n = P_{n+1} - P_{n-1} (Sec. 4.5)
//   * space-dependent diffusion (Sec. 4.7.2): a network with two outputs (u, eps);
//     eps(x, y) replaces the scalar eps in the diffusion term at every node
//
// Readings taken where the paper is silent or garbled:
//   - the printed inverse Jacobian (App. A.1) swaps xi and eta in its second
//     row; the true inverse (1/D)[[y_eta, -y_xi], [-x_eta, x_xi]] is used.
//   - the convection term b.grad u tested against v, with eps multiplying only
//     the diffusion term (Alg. 3 prints only the diffusion terms).
//   - test index j = (m-1) T + (n-1), m along xi; quadrature index q = a Q + b, a along xi.
//   - with two outputs, the second output is eps(x, y) itself (linear output, no
//     activation): the paper states that the network outputs both fields and
//     names no transform.  Boundary and sensor terms use the first output only.
//
// Gradients: a hand-written reverse sweep (FP64).  The same loss is also
// instantiated on std::complex<double> so that complex-step derivatives
// (Squire & Trapp 1998) can pin that sweep.

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

using cplx = std::complex<double>;

inline double re(double v) { return v; }
inline double re(const cplx& v) { return v.real(); }

// ---------------------------------------------------------------- Legendre
// Three-term recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}, and the
// derivative recurrence P'_{k+1} = P'_{k-1} + (2k+1) P_k.
void legendre(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    double d2 = d0 + (2.0 * k + 1.0) * p1;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *P = p1; *dP = d1;
}

// GLL rule with Q points: the endpoints +-1 and the Q-2 roots of P'_{Q-1},
// found by Newton's method from Chebyshev-Lobatto starting points; weights
// w_i = 2 / (Q (Q-1) P_{Q-1}(x_i)^2).
bool gll(int Q, std::vector<double>& x, std::vector<double>& w) {
  if (Q < 2 || Q > 128) return false;
  const int N = Q - 1;
  x.assign(Q, 0.0); w.assign(Q, 0.0);
  x[0] = -1.0; x[N] = 1.0;
  for (int i = 1; i < N; ++i) {
    double t = -std::cos(M_PI * i / N);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(N, t, &P, &dP);
      // Legendre ODE: (1 - t^2) P'' = 2 t P' - N (N+1) P
      double d2P = (2.0 * t * dP - N * (N + 1.0) * P) / (1.0 - t * t);
      double dt = dP / d2P;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[i] = t;
  }
  for (int i = 0; i < Q; ++i) {
    double P, dP;
    legendre(N, x[i], &P, &dP);
    w[i] = 2.0 / (Q * (Q - 1.0) * P * P);
  }
  return true;
}

// Test function v_n(s) = P_{n+1}(s) - P_{n-1}(s), n >= 1, and its derivative.
void test_fn(int n, double s, double* v, double* dv) {
  double Pa, dPa, Pb, dPb;
  legendre(n + 1, s, &Pa, &dPa);
  legendre(n - 1, s, &Pb, &dPb);
  *v = Pa - Pb;
  *dv = dPa - dPb;
}

// ---------------------------------------------------------------- geometry
struct Geo {           // bilinear map at one reference point (App. A.1)
  double x, y;         // mapped point
  double x_xi, x_eta, y_xi, y_eta, D;
};

Geo bilinear(const double* vx, const double* vy, double xi, double eta) {
  const double xc0 = (vx[0] + vx[1] + vx[2] + vx[3]) / 4.0;
  const double xc1 = (-vx[0] + vx[1] + vx[2] - vx[3]) / 4.0;
  const double xc2 = (-vx[0] - vx[1] + vx[2] + vx[3]) / 4.0;
  const double xc3 = (vx[0] - vx[1] + vx[2] - vx[3]) / 4.0;
  const double yc0 = (vy[0] + vy[1] + vy[2] + vy[3]) / 4.0;
  const double yc1 = (-vy[0] + vy[1] + vy[2] - vy[3]) / 4.0;
  const double yc2 = (-vy[0] - vy[1] + vy[2] + vy[3]) / 4.0;
  const double yc3 = (vy[0] - vy[1] + vy[2] - vy[3]) / 4.0;
  Geo g;
  g.x = xc0 + xc1 * xi + xc2 * eta + xc3 * xi * eta;
  g.y = yc0 + yc1 * xi + yc2 * eta + yc3 * xi * eta;
  g.x_xi = xc1 + xc3 * eta;
  g.x_eta = xc2 + xc3 * xi;
  g.y_xi = yc1 + yc3 * eta;
  g.y_eta = yc2 + yc3 * xi;
  g.D = g.x_xi * g.y_eta - g.x_eta * g.y_xi;
  return g;
}

void cell_vertices(const double* verts, const int* cells, int e, double* vx, double* vy) {
  for (int k = 0; k < 4; ++k) {
    int n = cells[4 * e + k];
    vx[k] = verts[2 * n];
    vy[k] = verts[2 * n + 1];
  }
}

// ---------------------------------------------------------------- MLP
// widths[0..L]: widths[0] = 2 inputs, widths[L] = 1 output, L affine maps.
// Flat parameter layout per layer: W (row-major [out][in]) then b.
struct Net {
  int L;
  std::vector<int> w;
  std::vector<size_t> off;  // offset of layer i's W; its b follows at off + out*in
  size_t n_params;
  Net(int L_, const int* widths) : L(L_), w(widths, widths + L_ + 1) {
    size_t o = 0;
    for (int i = 0; i < L; ++i) { off.push_back(o); o += (size_t)w[i + 1] * w[i] + w[i + 1]; }
    n_params = o;
  }
  int max_width() const { int m = 0; for (int v : w) m = v > m ? v : m; return m; }
};

// Forward pass with forward-mode tangents d/dx, d/dy (chain rule through each
// layer: z = W h + b, z' = W h', t = tanh z, t' = (1 - t^2) z').
// If `tape` is given, records per hidden layer t, z'_x, z'_y for the reverse sweep.
// With two outputs, *e_out receives the second output's value (eps(x, y)).
template <class T>
void mlp_forward(const Net& net, const T* p, T x, T y, T* u, T* ux, T* uy,
                 std::vector<T>* tape = nullptr, T* e_out = nullptr) {
  const int mw = net.max_width();
  std::vector<T> h(mw), hx(mw), hy(mw), nh(mw), nhx(mw), nhy(mw);
  h[0] = x; h[1] = y;
  hx[0] = 1.0; hx[1] = 0.0;
  hy[0] = 0.0; hy[1] = 1.0;
  if (tape) tape->clear();
  for (int i = 0; i < net.L; ++i) {
    const int nin = net.w[i], nout = net.w[i + 1];
    const T* W = p + net.off[i];
    const T* b = W + (size_t)nout * nin;
    for (int o = 0; o < nout; ++o) {
      T z = b[o], zx = 0.0, zy = 0.0;
      for (int k = 0; k < nin; ++k) {
        z += W[o * nin + k] * h[k];
        zx += W[o * nin + k] * hx[k];
        zy += W[o * nin + k] * hy[k];
      }
      if (i + 1 < net.L) {
        T t = std::tanh(z);
        T s = 1.0 - t * t;
        nh[o] = t; nhx[o] = s * zx; nhy[o] = s * zy;
        if (tape) { tape->push_back(t); tape->push_back(zx); tape->push_back(zy); }
      } else {
        nh[o] = z; nhx[o] = zx; nhy[o] = zy;
      }
    }
    std::swap(h, nh); std::swap(hx, nhx); std::swap(hy, nhy);
  }
  *u = h[0]; *ux = hx[0]; *uy = hy[0];
  if (e_out) *e_out = net.w[net.L] > 1 ? h[1] : T(0.0);
}

// Reverse sweep through mlp_forward for seeds (ub, uxb, uyb) on (u, u_x, u_y)
// and, with two outputs, eb on the second output's value; adds d/dtheta into g.
// Uses the tape written by mlp_forward at the same point.
void mlp_reverse(const Net& net, const double* p, double x, double y, const std::vector<double>& tape,
                 double ub, double uxb, double uyb, double* g, double eb = 0.0) {
  const int L = net.L;
  // rebuild layer inputs from the tape: input of layer i is the output of layer i-1
  std::vector<size_t> toff(L, 0);
  { size_t o = 0; for (int i = 0; i + 1 < L; ++i) { toff[i] = o; o += 3 * (size_t)net.w[i + 1]; } }
  auto h_in = [&](int i, int k, int which) -> double {   // which: 0 value, 1 d/dx, 2 d/dy
    if (i == 0) {
      if (which == 0) return k == 0 ? x : y;
      if (which == 1) return k == 0 ? 1.0 : 0.0;
      return k == 0 ? 0.0 : 1.0;
    }
    const double* r = &tape[toff[i - 1] + 3 * (size_t)k];
    const double t = r[0], s = 1.0 - t * t;
    return which == 0 ? t : (which == 1 ? s * r[1] : s * r[2]);
  };
  const int mw = net.max_width();
  std::vector<double> zb(mw), zxb(mw), zyb(mw), hb(mw), hxb(mw), hyb(mw);
  // output layer (linear): seeds are the adjoints of z, z'_x, z'_y directly
  zb[0] = ub; zxb[0] = uxb; zyb[0] = uyb;
  if (net.w[L] > 1) { zb[1] = eb; zxb[1] = 0.0; zyb[1] = 0.0; }
  for (int i = L - 1; i >= 0; --i) {
    const int nin = net.w[i], nout = net.w[i + 1];
    const double* W = p + net.off[i];
    double* gW = g + net.off[i];
    double* gb = gW + (size_t)nout * nin;
    for (int o = 0; o < nout; ++o) {
      gb[o] += zb[o];
      for (int k = 0; k < nin; ++k)
        gW[o * nin + k] += zb[o] * h_in(i, k, 0) + zxb[o] * h_in(i, k, 1) + zyb[o] * h_in(i, k, 2);
    }
    if (i == 0) break;
    for (int k = 0; k < nin; ++k) {
      double a = 0, ax = 0, ay = 0;
      for (int o = 0; o < nout; ++o) {
        a += W[o * nin + k] * zb[o];
        ax += W[o * nin + k] * zxb[o];
        ay += W[o * nin + k] * zyb[o];
      }
      hb[k] = a; hxb[k] = ax; hyb[k] = ay;
    }
    // through layer i-1's tanh and tangent rule:
    //   t = tanh z, t'_s = (1-t^2) z'_s
    //   zbar = (1-t^2) (tbar - 2 t sum_s z'_s t'bar_s),  z'bar_s = (1-t^2) t'bar_s
    for (int k = 0; k < nin; ++k) {
      const double* r = &tape[toff[i - 1] + 3 * (size_t)k];
      const double t = r[0], s = 1.0 - t * t;
      zxb[k] = s * hxb[k];
      zyb[k] = s * hyb[k];
      zb[k] = s * (hb[k] - 2.0 * t * (r[1] * hxb[k] + r[2] * hyb[k]));
    }
  }
}

}  // namespace

// =====================================================================
// C interface (ctypes).  All arrays are host arrays, row-major.
// =====================================================================
extern "C" {

struct OracleProblem {
  int n_vertices;
  const double* vertices;   // [n_vertices][2]
  int n_elements;
  const int* cells;         // [n_elements][4], counter-clockwise b0..b3
  int Q, T;                 // GLL points / test functions per direction
  const double* f_quad;     // [n_elements][Q*Q] source f at the mapped quadrature points
  int n_layers;             // number of affine maps
  const int* widths;        // [n_layers + 1]
  int n_bd;
  const double* bd_xy;      // [n_bd][2]
  const double* bd_g;       // [n_bd]
  double tau;
  int n_s;
  const double* s_xy;       // [n_s][2]
  const double* s_u;        // [n_s]
  double gamma;
  double bx, by;
  int norm;                 // 0: Algorithm 3 (1/N_test) sum R^2; 1: Eq. (loss) (1/N_elem) sum R^2
};

int oracle_gll(int Q, double* x, double* w) {
  std::vector<double> xs, ws;
  if (!gll(Q, xs, ws)) return 1;
  std::memcpy(x, xs.data(), Q * sizeof(double));
  std::memcpy(w, ws.data(), Q * sizeof(double));
  return 0;
}

void oracle_legendre(int n, int m, const double* s, double* P, double* dP) {
  for (int i = 0; i < m; ++i) legendre(n, s[i], &P[i], &dP[i]);
}

void oracle_test_fn(int n, int m, const double* s, double* v, double* dv) {
  for (int i = 0; i < m; ++i) test_fn(n, s[i], &v[i], &dv[i]);
}

// Bilinear-map data at every quadrature node: out [n_e][Q*Q][7] =
// (x, y, x_xi, x_eta, y_xi, y_eta, D).
int oracle_geometry(int n_v, const double* verts, int n_e, const int* cells, int Q, double* out) {
  (void)n_v;
  std::vector<double> xs, ws;
  if (!gll(Q, xs, ws)) return 1;
  for (int e = 0; e < n_e; ++e) {
    double vx[4], vy[4];
    cell_vertices(verts, cells, e, vx, vy);
    for (int a = 0; a < Q; ++a)
      for (int b = 0; b < Q; ++b) {
        Geo g = bilinear(vx, vy, xs[a], xs[b]);
        double* o = out + ((size_t)e * Q * Q + a * Q + b) * 7;
        o[0] = g.x; o[1] = g.y; o[2] = g.x_xi; o[3] = g.x_eta; o[4] = g.y_xi; o[5] = g.y_eta; o[6] = g.D;
      }
  }
  return 0;
}

// Geometry at arbitrary reference points (for finite-difference pins of the map).
void oracle_map_points(const double* vx, const double* vy, int m, const double* xi, const double* eta, double* out) {
  for (int i = 0; i < m; ++i) {
    Geo g = bilinear(vx, vy, xi[i], eta[i]);
    double* o = out + 7 * (size_t)i;
    o[0] = g.x; o[1] = g.y; o[2] = g.x_xi; o[3] = g.x_eta; o[4] = g.y_xi; o[5] = g.y_eta; o[6] = g.D;
  }
}

// MLP value and gradient at points: out u[n], ux[n], uy[n].
void oracle_mlp(int n_layers, const int* widths, const double* p, int n, const double* xy,
                double* u, double* ux, double* uy) {
  Net net(n_layers, widths);
  for (int i = 0; i < n; ++i) mlp_forward<double>(net, p, xy[2 * i], xy[2 * i + 1], &u[i], &ux[i], &uy[i]);
}

// Second output (eps(x, y)) of a two-output network at n points.
void oracle_mlp_eps(int n_layers, const int* widths, const double* p, int n, const double* xy, double* eps) {
  Net net(n_layers, widths);
  for (int i = 0; i < n; ++i) {
    double u, ux, uy;
    mlp_forward<double>(net, p, xy[2 * i], xy[2 * i + 1], &u, &ux, &uy, nullptr, &eps[i]);
  }
}

// Complex-step d u/dx and d u/dy of the MLP value (independent of the tangent code path).
void oracle_mlp_cstep_x(int n_layers, const int* widths, const double* p, int n, const double* xy, double h,
                        double* dudx, double* dudy) {
  Net net(n_layers, widths);
  std::vector<cplx> pc(p, p + net.n_params);
  for (int i = 0; i < n; ++i) {
    cplx u, ux, uy;
    mlp_forward<cplx>(net, pc.data(), cplx(xy[2 * i], h), cplx(xy[2 * i + 1], 0.0), &u, &ux, &uy);
    dudx[i] = u.imag() / h;
    mlp_forward<cplx>(net, pc.data(), cplx(xy[2 * i], 0.0), cplx(xy[2 * i + 1], h), &u, &ux, &uy);
    dudy[i] = u.imag() / h;
  }
}

// Per-element weak residuals for a GIVEN gradient field (ux, uy at the
// quadrature nodes, [n_e][Q*Q]), loop form:
//   R[e][j] = sum_q w_q D_q ( eps (ux dv_j/dx + uy dv_j/dy) + (b . grad u) v_j - f_q v_j ).
int oracle_residuals_given_grad(const OracleProblem* pb, const double* ux, const double* uy, double eps,
                                double* R) {
  const int Q = pb->Q, T = pb->T, Nq = Q * Q, Nt = T * T;
  std::vector<double> xs, ws;
  if (!gll(Q, xs, ws) || T < 1) return 1;
  for (int e = 0; e < pb->n_elements; ++e) {
    double vx[4], vy[4];
    cell_vertices(pb->vertices, pb->cells, e, vx, vy);
    double* Re = R + (size_t)e * Nt;
    for (int j = 0; j < Nt; ++j) Re[j] = 0.0;
    for (int a = 0; a < Q; ++a)
      for (int b = 0; b < Q; ++b) {
        const int q = a * Q + b;
        Geo g = bilinear(vx, vy, xs[a], xs[b]);
        const double wq = ws[a] * ws[b];
        const double gx = ux[(size_t)e * Nq + q], gy = uy[(size_t)e * Nq + q];
        const double fq = pb->f_quad[(size_t)e * Nq + q];
        for (int m = 1; m <= T; ++m)
          for (int n = 1; n <= T; ++n) {
            double vm, dvm, vn, dvn;
            test_fn(m, xs[a], &vm, &dvm);
            test_fn(n, xs[b], &vn, &dvn);
            const double v = vm * vn, v_xi = dvm * vn, v_eta = vm * dvn;
            const double v_x = (g.y_eta * v_xi - g.y_xi * v_eta) / g.D;
            const double v_y = (-g.x_eta * v_xi + g.x_xi * v_eta) / g.D;
            const int j = (m - 1) * T + (n - 1);
            Re[j] += wq * g.D * (eps * (gx * v_x + gy * v_y) + (pb->bx * gx + pb->by * gy) * v - fq * v);
          }
      }
  }
  return 0;
}

// Tensor variant (Algorithm 3 / App. A.2): stacked premultipliers
//   Gx[e][j][q] = w_q D_q dv_j/dx,  Gy = w_q D_q dv_j/dy,  Gv = w_q D_q v_j,
//   F[e][j] = sum_q Gv[e][j][q] f_q.
int oracle_build_tensors(const OracleProblem* pb, double* Gx, double* Gy, double* Gv, double* F) {
  const int Q = pb->Q, T = pb->T, Nq = Q * Q, Nt = T * T;
  std::vector<double> xs, ws;
  if (!gll(Q, xs, ws) || T < 1) return 1;
  for (int e = 0; e < pb->n_elements; ++e) {
    double vx[4], vy[4];
    cell_vertices(pb->vertices, pb->cells, e, vx, vy);
    for (int j = 0; j < Nt; ++j) F[(size_t)e * Nt + j] = 0.0;
    for (int a = 0; a < Q; ++a)
      for (int b = 0; b < Q; ++b) {
        const int q = a * Q + b;
        Geo g = bilinear(vx, vy, xs[a], xs[b]);
        const double wq = ws[a] * ws[b];
        for (int m = 1; m <= T; ++m)
          for (int n = 1; n <= T; ++n) {
            double vm, dvm, vn, dvn;
            test_fn(m, xs[a], &vm, &dvm);
            test_fn(n, xs[b], &vn, &dvn);
            const double v = vm * vn, v_xi = dvm * vn, v_eta = vm * dvn;
            const int j = (m - 1) * T + (n - 1);
            const size_t idx = ((size_t)e * Nt + j) * Nq + q;
            Gx[idx] = wq * g.D * ((g.y_eta * v_xi - g.y_xi * v_eta) / g.D);
            Gy[idx] = wq * g.D * ((-g.x_eta * v_xi + g.x_xi * v_eta) / g.D);
            Gv[idx] = wq * g.D * v;
            F[(size_t)e * Nt + j] += Gv[idx] * pb->f_quad[(size_t)e * Nq + q];
          }
      }
  }
  return 0;
}

// Tensor-variant contraction: R = eps (Gx ux + Gy uy) + Gv (bx ux + by uy) - F,
// one matrix-vector product per element (Algorithm 3's matvec over the stack).
void oracle_contract(int n_e, int Nt, int Nq, const double* Gx, const double* Gy, const double* Gv,
                     const double* F, const double* ux, const double* uy, double eps, double bx, double by,
                     double* R) {
  for (int e = 0; e < n_e; ++e)
    for (int j = 0; j < Nt; ++j) {
      double ax = 0, ay = 0, av = 0;
      for (int q = 0; q < Nq; ++q) {
        const size_t idx = ((size_t)e * Nt + j) * Nq + q;
        const double gx = ux[(size_t)e * Nq + q], gy = uy[(size_t)e * Nq + q];
        ax += Gx[idx] * gx;
        ay += Gy[idx] * gy;
        av += Gv[idx] * (bx * gx + by * gy);
      }
      R[(size_t)e * Nt + j] = eps * (ax + ay) + av - F[(size_t)e * Nt + j];
    }
}

// Mapped quadrature points [n_e][Q*Q][2] (for evaluating f there).
int oracle_quad_points(int n_v, const double* verts, int n_e, const int* cells, int Q, double* xy) {
  (void)n_v;
  std::vector<double> xs, ws;
  if (!gll(Q, xs, ws)) return 1;
  for (int e = 0; e < n_e; ++e) {
    double vx[4], vy[4];
    cell_vertices(verts, cells, e, vx, vy);
    for (int a = 0; a < Q; ++a)
      for (int b = 0; b < Q; ++b) {
        Geo g = bilinear(vx, vy, xs[a], xs[b]);
        xy[((size_t)e * Q * Q + a * Q + b) * 2] = g.x;
        xy[((size_t)e * Q * Q + a * Q + b) * 2 + 1] = g.y;
      }
  }
  return 0;
}

}  // extern "C"

namespace {

// The whole loss for scalar type S (double, or complex for complex-step).
// Returns L and its parts (Lv, Lb, Ls); element residuals optionally.
template <class S>
void loss_generic(const OracleProblem* pb, const Net& net, const S* p, S eps, S* parts, double* R_out) {
  const int Q = pb->Q, T = pb->T, Nq = Q * Q, Nt = T * T;
  std::vector<double> xs, ws;
  gll(Q, xs, ws);
  S Lv = 0.0;
  std::vector<S> R(Nt);
  for (int e = 0; e < pb->n_elements; ++e) {
    double vx[4], vy[4];
    cell_vertices(pb->vertices, pb->cells, e, vx, vy);
    for (int j = 0; j < Nt; ++j) R[j] = 0.0;
    for (int a = 0; a < Q; ++a)
      for (int b = 0; b < Q; ++b) {
        const int q = a * Q + b;
        Geo g = bilinear(vx, vy, xs[a], xs[b]);
        S u, ux, uy, ep;
        mlp_forward<S>(net, p, S(g.x), S(g.y), &u, &ux, &uy, nullptr, &ep);
        const S epq = net.w[net.L] > 1 ? ep : eps;     // eps(x, y) or the scalar
        const double wq = ws[a] * ws[b];
        const double fq = pb->f_quad[(size_t)e * Nq + q];
        for (int m = 1; m <= T; ++m)
          for (int n = 1; n <= T; ++n) {
            double vm, dvm, vn, dvn;
            test_fn(m, xs[a], &vm, &dvm);
            test_fn(n, xs[b], &vn, &dvn);
            const double v = vm * vn, v_xi = dvm * vn, v_eta = vm * dvn;
            const double v_x = (g.y_eta * v_xi - g.y_xi * v_eta) / g.D;
            const double v_y = (-g.x_eta * v_xi + g.x_xi * v_eta) / g.D;
            R[(m - 1) * T + (n - 1)] +=
                wq * g.D * (epq * (ux * v_x + uy * v_y) + (pb->bx * ux + pb->by * uy) * v - fq * v);
          }
      }
    for (int j = 0; j < Nt; ++j) {
      Lv += R[j] * R[j];
      if (R_out) R_out[(size_t)e * Nt + j] = re(R[j]);
    }
  }
  Lv = Lv / double(pb->norm == 0 ? Nt : pb->n_elements);
  S Lb = 0.0, Ls = 0.0;
  for (int d = 0; d < pb->n_bd; ++d) {
    S u, ux, uy;
    mlp_forward<S>(net, p, S(pb->bd_xy[2 * d]), S(pb->bd_xy[2 * d + 1]), &u, &ux, &uy);
    Lb += (u - pb->bd_g[d]) * (u - pb->bd_g[d]);
  }
  if (pb->n_bd > 0) Lb = Lb / double(pb->n_bd);
  for (int s = 0; s < pb->n_s; ++s) {
    S u, ux, uy;
    mlp_forward<S>(net, p, S(pb->s_xy[2 * s]), S(pb->s_xy[2 * s + 1]), &u, &ux, &uy);
    Ls += (u - pb->s_u[s]) * (u - pb->s_u[s]);
  }
  if (pb->n_s > 0) Ls = Ls / double(pb->n_s);
  parts[0] = Lv + pb->tau * Lb + pb->gamma * Ls;
  parts[1] = Lv; parts[2] = Lb; parts[3] = Ls;
}

}  // namespace

extern "C" {

// Loss value and (optionally) its gradient by the hand-written reverse sweep.
//   loss4: (L, Lv, Lb, Ls);  grad: [n_params] or null;  dL_deps: scalar or null;
//   R: [n_e][N_t] element residuals or null;
//   ubar: [n_e][Q*Q][2] adjoint seeds dL/du_x, dL/du_y at the quadrature nodes, or null;
//   upts: [n_e][Q*Q][3] (u, u_x, u_y) at the quadrature nodes, or null.
// Elements are split over n_threads OpenMP threads (each with its own gradient
// buffer; the buffers are summed in thread order).
//   ebar: [n_e][Q*Q] adjoint seed dL/deps(x_q) of a two-output network, or null;
//   epts: [n_e][Q*Q] eps(x_q) of a two-output network, or null.
// With two outputs dL_deps is 0 (eps is part of theta).
int oracle_loss_grad(const OracleProblem* pb, const double* p, double eps, double* loss4, double* grad,
                     double* dL_deps, double* R_out, double* ubar_out, double* upts_out, int n_threads,
                     double* ebar_out, double* epts_out) {
  const int Q = pb->Q, T = pb->T, Nq = Q * Q, Nt = T * T;
  std::vector<double> xs, ws;
  if (!gll(Q, xs, ws) || T < 1 || pb->n_layers < 1) return 1;
  Net net(pb->n_layers, pb->widths);
  const double rscale = 2.0 / double(pb->norm == 0 ? Nt : pb->n_elements);   // d(Lv)/dR = rscale * R
  if (n_threads < 1) n_threads = 1;
  std::vector<std::vector<double>> gbuf(n_threads, std::vector<double>(net.n_params, 0.0));
  std::vector<double> lv_e(pb->n_elements, 0.0), de_e(pb->n_elements, 0.0);

#pragma omp parallel for num_threads(n_threads) schedule(static)
  for (int e = 0; e < pb->n_elements; ++e) {
#ifdef _OPENMP
    const int tid = omp_get_thread_num();
#else
    const int tid = 0;
#endif
    double vx[4], vy[4];
    cell_vertices(pb->vertices, pb->cells, e, vx, vy);
    std::vector<double> R(Nt, 0.0), A(Nt, 0.0);
    std::vector<double> U(Nq), UX(Nq), UY(Nq), EP(Nq, eps);
    std::vector<Geo> geo(Nq);
    std::vector<std::vector<double>> tapes(Nq);
    const bool two = net.w[net.L] > 1;
    // value + gradient of the network at every node, then the residual sums
    for (int a = 0; a < Q; ++a)
      for (int b = 0; b < Q; ++b) {
        const int q = a * Q + b;
        geo[q] = bilinear(vx, vy, xs[a], xs[b]);
        double ep = 0.0;
        mlp_forward<double>(net, p, geo[q].x, geo[q].y, &U[q], &UX[q], &UY[q], grad ? &tapes[q] : nullptr, &ep);
        if (two) EP[q] = ep;
      }
    for (int a = 0; a < Q; ++a)
      for (int b = 0; b < Q; ++b) {
        const int q = a * Q + b;
        const Geo& g = geo[q];
        const double wq = ws[a] * ws[b];
        const double fq = pb->f_quad[(size_t)e * Nq + q];
        for (int m = 1; m <= T; ++m)
          for (int n = 1; n <= T; ++n) {
            double vm, dvm, vn, dvn;
            test_fn(m, xs[a], &vm, &dvm);
            test_fn(n, xs[b], &vn, &dvn);
            const double v = vm * vn, v_xi = dvm * vn, v_eta = vm * dvn;
            const double v_x = (g.y_eta * v_xi - g.y_xi * v_eta) / g.D;
            const double v_y = (-g.x_eta * v_xi + g.x_xi * v_eta) / g.D;
            const int j = (m - 1) * T + (n - 1);
            const double diff = wq * g.D * (UX[q] * v_x + UY[q] * v_y);
            A[j] += diff;
            R[j] += EP[q] * diff + wq * g.D * ((pb->bx * UX[q] + pb->by * UY[q]) * v - fq * v);
          }
      }
    double lv = 0.0, de = 0.0;
    for (int j = 0; j < Nt; ++j) {
      lv += R[j] * R[j];
      de += rscale * R[j] * A[j];          // dLv/deps = sum_j dLv/dR_j * A_j
      if (R_out) R_out[(size_t)e * Nt + j] = R[j];
    }
    lv_e[e] = lv;
    de_e[e] = two ? 0.0 : de;
    if (epts_out)
      for (int q = 0; q < Nq; ++q) epts_out[(size_t)e * Nq + q] = two ? EP[q] : 0.0;
    if (upts_out)
      for (int q = 0; q < Nq; ++q) {
        double* o = upts_out + ((size_t)e * Nq + q) * 3;
        o[0] = U[q]; o[1] = UX[q]; o[2] = UY[q];
      }
    if (grad || ubar_out || ebar_out) {
      // adjoint seeds at each node: dL/du_x = sum_j Rbar_j w D (eps dv_j/dx + bx v_j), likewise y
      for (int a = 0; a < Q; ++a)
        for (int b = 0; b < Q; ++b) {
          const int q = a * Q + b;
          const Geo& g = geo[q];
          const double wq = ws[a] * ws[b];
          double sx = 0.0, sy = 0.0, eb = 0.0;
          for (int m = 1; m <= T; ++m)
            for (int n = 1; n <= T; ++n) {
              double vm, dvm, vn, dvn;
              test_fn(m, xs[a], &vm, &dvm);
              test_fn(n, xs[b], &vn, &dvn);
              const double v = vm * vn, v_xi = dvm * vn, v_eta = vm * dvn;
              const double v_x = (g.y_eta * v_xi - g.y_xi * v_eta) / g.D;
              const double v_y = (-g.x_eta * v_xi + g.x_xi * v_eta) / g.D;
              const double Rb = rscale * R[(m - 1) * T + (n - 1)];
              sx += Rb * wq * g.D * (EP[q] * v_x + pb->bx * v);
              sy += Rb * wq * g.D * (EP[q] * v_y + pb->by * v);
              eb += Rb * wq * g.D * (UX[q] * v_x + UY[q] * v_y);   // d R_j / d eps(x_q)
            }
          if (ubar_out) {
            ubar_out[((size_t)e * Nq + q) * 2] = sx;
            ubar_out[((size_t)e * Nq + q) * 2 + 1] = sy;
          }
          if (ebar_out) ebar_out[(size_t)e * Nq + q] = two ? eb : 0.0;
          if (grad) mlp_reverse(net, p, g.x, g.y, tapes[q], 0.0, sx, sy, gbuf[tid].data(), two ? eb : 0.0);
        }
    }
  }

  double Lv = 0.0, dLde = 0.0;
  for (int e = 0; e < pb->n_elements; ++e) { Lv += lv_e[e]; dLde += de_e[e]; }
  Lv /= double(pb->norm == 0 ? Nt : pb->n_elements);
  std::vector<double> g(net.n_params, 0.0);
  for (int t = 0; t < n_threads; ++t)
    for (size_t i = 0; i < net.n_params; ++i) g[i] += gbuf[t][i];

  double Lb = 0.0, Ls = 0.0;
  std::vector<double> tape;
  for (int d = 0; d < pb->n_bd; ++d) {
    double u, ux, uy;
    const double x = pb->bd_xy[2 * d], y = pb->bd_xy[2 * d + 1];
    mlp_forward<double>(net, p, x, y, &u, &ux, &uy, grad ? &tape : nullptr);
    Lb += (u - pb->bd_g[d]) * (u - pb->bd_g[d]);
    if (grad) mlp_reverse(net, p, x, y, tape, 2.0 * pb->tau * (u - pb->bd_g[d]) / pb->n_bd, 0.0, 0.0, g.data());
  }
  if (pb->n_bd > 0) Lb /= pb->n_bd;
  for (int s = 0; s < pb->n_s; ++s) {
    double u, ux, uy;
    const double x = pb->s_xy[2 * s], y = pb->s_xy[2 * s + 1];
    mlp_forward<double>(net, p, x, y, &u, &ux, &uy, grad ? &tape : nullptr);
    Ls += (u - pb->s_u[s]) * (u - pb->s_u[s]);
    if (grad) mlp_reverse(net, p, x, y, tape, 2.0 * pb->gamma * (u - pb->s_u[s]) / pb->n_s, 0.0, 0.0, g.data());
  }
  if (pb->n_s > 0) Ls /= pb->n_s;
  loss4[0] = Lv + pb->tau * Lb + pb->gamma * Ls;
  loss4[1] = Lv; loss4[2] = Lb; loss4[3] = Ls;
  if (grad) std::memcpy(grad, g.data(), net.n_params * sizeof(double));
  if (dL_deps) *dL_deps = dLde;
  return 0;
}

// Complex-step derivatives dL/dtheta_i (idx[k] >= 0) or dL/deps (idx[k] == -1):
// L(theta + i h e_k) evaluated in complex arithmetic, derivative = Im(L)/h.
int oracle_loss_cstep(const OracleProblem* pb, const double* p, double eps, int n_idx, const int* idx, double h,
                      double* out, int n_threads) {
  Net net(pb->n_layers, pb->widths);
  if (n_threads < 1) n_threads = 1;
#pragma omp parallel for num_threads(n_threads) schedule(dynamic, 1)
  for (int k = 0; k < n_idx; ++k) {
    std::vector<cplx> pc(p, p + net.n_params);
    cplx ec(eps, 0.0);
    if (idx[k] >= 0) pc[idx[k]] += cplx(0.0, h);
    else ec += cplx(0.0, h);
    cplx parts[4];
    loss_generic<cplx>(pb, net, pc.data(), ec, parts, nullptr);
    out[k] = parts[0].imag() / h;
  }
  return 0;
}

// Loss value only, by the same generic code instantiated on double.
int oracle_loss_value(const OracleProblem* pb, const double* p, double eps, double* loss4, double* R_out) {
  Net net(pb->n_layers, pb->widths);
  loss_generic<double>(pb, net, p, eps, loss4, R_out);
  return 0;
}

}  // extern "C"

/*
 * FP64 CPU oracle for the image-plane chi^2 path of LENSTOOL-style parametric
 * lens modelling (Rexroth, Schaefer, Fourestey & Kneib 2019, "High Performance
 * Computing for gravitational lens modeling: single vs double precision on
 * GPUs and CPUs").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA library: it is a plain, slow, single-pass restatement of the
 * method, written to be checked against the paper by eye.  Every
 * floating-point operation is IEEE double with no contraction
 * (-ffp-contract=off), evaluated in the order written.
 *
 * What it computes, step by step (Sect. 2.2.2 and Fig. 1):
 *   1. alpha(theta) = sum over potentials of the per-potential scaled
 *      deflection, in potential index order (superposition of gradients,
 *      Sect. 2.2.2; Algorithm 1 for the SIE).
 *   2. beta = theta - (D_ls/D_s) alpha(theta)   (lens equation, Eq. 13).
 *   3. barycentre of each system: mean over its observed images of beta.
 *   4. every grid cell split into two triangles; every mapped triangle
 *      tested for containing each system's barycentre (Fig. 1).
 *   5. predicted image = barycentric interpolation inside a containing
 *      triangle.
 *   6. chi^2 = sum_i sum_j |x_obs,ij - x_ij|^2 / sigma_ij^2  (Eq. 11), each
 *      observed image matched to the nearest predicted image of its system.
 *   7. d chi^2 / d(params) with the triangle assignment and matching frozen,
 *      by forward-mode dual numbers through the same templated code.
 *   8. magnifications and the source-plane chi^2 (extensions the relensing
 *      pipeline of Fig. 1 motivates): the deflection Jacobian d alpha/d theta
 *      by dual numbers (alpha depends on theta only through theta - c, so it
 *      is minus the derivative w.r.t. the potential centre), the point
 *      magnification 1/det(I - r d alpha/d theta), and the triangle
 *      magnification (image-plane area over lensed source-plane area).
 *
 * Readings where the paper is silent (the PIEMD profile, grid placement,
 * cell diagonal, tie rule, matching, penalty) are the ones listed in the
 * design notes of this repository; each function below states the one it
 * uses.
 *
 * Parity pins: deflections (SIS closed form, PIEMD quadrature/Poisson/curl/
 * circular and SIS limits, SIE reduction to SIS), triangle search (exact
 * rational brute force, lens-equation residual convergence, SIS image count),
 * chi^2 (noiseless convergence) and gradient (central differences, SIS
 * analytic) are all exercised by the CPU test suite.
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace lto {

const double kC = 299792.458;          // speed of light, km/s
const double kArcsec = 206264.80625;   // arcsec per radian
const double kPi = 3.14159265358979323846;
const double kU64 = 1.1102230246251565e-16;  // 2^-53

enum { SIS = 0, PIEMD = 1, SIE = 2 };
enum { R_KIND = 0, R_X, R_Y, R_E, R_PHI, R_RC, R_RCUT, R_SV, N_ROWS };

// ---------------------------------------------------------------- dual numbers
struct Dual {
  double v, d;
  Dual(double v_ = 0.0, double d_ = 0.0) : v(v_), d(d_) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
inline Dual operator+(double a, Dual b) { return Dual(a + b.v, b.d); }
inline Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
inline Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
inline Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
inline Dual operator/(double a, Dual b) {
  double q = a / b.v;
  return Dual(q, -q * b.d / b.v);
}
inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}
inline Dual atan(Dual a) { return Dual(std::atan(a.v), a.d / (1.0 + a.v * a.v)); }
inline Dual atanh(Dual a) { return Dual(std::atanh(a.v), a.d / (1.0 - a.v * a.v)); }
inline Dual sin(Dual a) { return Dual(std::sin(a.v), a.d * std::cos(a.v)); }
inline Dual cos(Dual a) { return Dual(std::cos(a.v), -a.d * std::sin(a.v)); }
inline double val(double a) { return a; }
inline double val(Dual a) { return a.v; }
using std::atan;
using std::atanh;
using std::cos;
using std::sin;
using std::sqrt;

// ------------------------------------------------------------ per-potential
// b0 = 4 pi (sigma_v / c)^2, the SIS/SIE normalisation of Sect. 2.2.2
// (the scaled deflection with D_ls/D_s factored out, Eq. 12), in arcsec.
template <class T>
T b0_of(T sv) {
  T t = sv / kC;
  return 4.0 * kPi * t * t * kArcsec;
}

// atan(t)/t as a function of t2 = t*t >= 0; the Taylor branch keeps the
// q -> 1 (k -> 0) limit exact and differentiable.
template <class T>
T atanc_sq(T t2) {
  if (val(t2) < 1e-6) return 1.0 - t2 * (1.0 / 3.0 - t2 * (1.0 / 5.0 - t2 * (1.0 / 7.0)));
  T t = sqrt(t2);
  return atan(t) / t;
}
// atanh(t)/t as a function of t2 = t*t, 0 <= t2 < 1.
template <class T>
T atanhc_sq(T t2) {
  if (val(t2) < 1e-6) return 1.0 + t2 * (1.0 / 3.0 + t2 * (1.0 / 5.0 + t2 * (1.0 / 7.0)));
  T t = sqrt(t2);
  return atanh(t) / t;
}

/*
 * Scaled deflection of one potential at (x, y).  p[] holds the 8 parameter
 * rows of this potential (kind, x, y, e, phi, r_core, r_cut, sigma_v).
 *
 * SIS (Sect. 2.1): alpha = b0 (theta - c)/|theta - c|; alpha = 0 at the
 *   centre, where it is undefined.
 * SIE (Algorithm 1): translate, rotate by phi, R = sqrt(x'^2 (1-eps) +
 *   y'^2 (1+eps)), g = ((1-eps) b0 x'/R, (1+eps) b0 y'/R), rotate by -phi.
 * PIEMD (dPIE; the paper only names it, Sect. 5): convergence
 *   kappa = (b0/2) s/(s-a) [1/psi_a - 1/psi_s],
 *   psi_w = sqrt(q^2 (w^2 + x'^2) + y'^2), q = 1 - e, a = r_core, s = r_cut,
 *   whose deflection in the rotated frame is, per cored term w,
 *   F_x = atan(k x'/(psi_w + w))/k, F_y = atanh(k y'/(psi_w + q^2 w))/k,
 *   k^2 = 1 - q^2, and alpha' = b0 s/(s-a) [F(a) - F(s)], rotated by -phi.
 *   (Checked by quadrature of the homoeoidal integrals, by Poisson's
 *   equation and by its circular and SIS limits in the test suite.)
 */
template <class T>
void alpha_one(const T* p, double x, double y, T& ax, T& ay) {
  int kind = (int)val(p[R_KIND]);
  T dx = x - p[R_X];
  T dy = y - p[R_Y];
  T b0 = b0_of(p[R_SV]);
  if (kind == SIS) {
    T R = sqrt(dx * dx + dy * dy);
    if (val(R) == 0.0) { ax = T(0.0); ay = T(0.0); return; }
    ax = b0 * dx / R;
    ay = b0 * dy / R;
    return;
  }
  T c = cos(p[R_PHI]);
  T s = sin(p[R_PHI]);
  T xp = dx * c + dy * s;
  T yp = dy * c - dx * s;
  T gx, gy;
  if (kind == SIE) {
    T eps = p[R_E];
    T R = sqrt(xp * xp * (1.0 - eps) + yp * yp * (1.0 + eps));
    if (val(R) == 0.0) { ax = T(0.0); ay = T(0.0); return; }
    gx = (1.0 - eps) * b0 * xp / R;
    gy = (1.0 + eps) * b0 * yp / R;
  } else {
    T q = 1.0 - p[R_E];
    T k2 = (1.0 - q) * (1.0 + q);
    T q2 = q * q;
    T a = p[R_RC];
    T sc = p[R_RCUT];
    T scale = b0 * (sc / (sc - a));
    T fx[2], fy[2];
    for (int t = 0; t < 2; ++t) {
      T w = (t == 0) ? a : sc;
      T psi = sqrt(q2 * (w * w + xp * xp) + yp * yp);
      T zx = xp / (psi + w);
      T zy = yp / (psi + q2 * w);
      fx[t] = zx * atanc_sq(k2 * zx * zx);
      fy[t] = zy * atanhc_sq(k2 * zy * zy);
    }
    gx = scale * (fx[0] - fx[1]);
    gy = scale * (fy[0] - fy[1]);
  }
  // rotation by -phi (Algorithm 1: cos(-phi), sin(-phi))
  ax = gx * c - gy * s;
  ay = gy * c + gx * s;
}

// Total deflection: superposition in potential index order (Sect. 2.2.2).
// params is [8][n_pot]; *asum (optional) receives sum_k |a_kx| + |a_ky|.
template <class T>
void alpha_total(const T* params, int n_pot, double x, double y, T& ax, T& ay,
                 double* asum) {
  ax = T(0.0);
  ay = T(0.0);
  double sa = 0.0;
  T p[N_ROWS];
  for (int k = 0; k < n_pot; ++k) {
    for (int r = 0; r < N_ROWS; ++r) p[r] = params[r * n_pot + k];
    T kx, ky;
    alpha_one(p, x, y, kx, ky);
    ax = ax + kx;
    ay = ay + ky;
    sa += std::fabs(val(kx)) + std::fabs(val(ky));
  }
  if (asum) *asum = sa;
}

// ------------------------------------------------------------------- grids
struct Grid {
  double x0, y0, dx, dy;
  int nx, ny;
  double X(int i) const { return x0 + i * dx; }
  double Y(int j) const { return y0 + j * dy; }
};

void deflect_grid(const double* params, int n_pot, const Grid& g, int n_threads,
                  double* alpha, double* asum) {
#pragma omp parallel for schedule(dynamic, 4) num_threads(n_threads > 0 ? n_threads : 1)
  for (int j = 0; j < g.ny; ++j) {
    for (int i = 0; i < g.nx; ++i) {
      size_t n = (size_t)j * g.nx + i;
      double ax, ay, sa;
      alpha_total(params, n_pot, g.X(i), g.Y(j), ax, ay, &sa);
      alpha[2 * n] = ax;
      alpha[2 * n + 1] = ay;
      if (asum) asum[n] = sa;
    }
  }
}

// --------------------------------------------------------- triangle search
// Edge function e(a, b, p) = (b - a) x (p - a), each operation rounded.
inline double edge_fn(double ax, double ay, double bx, double by, double px, double py) {
  double t1 = (bx - ax) * (py - ay);
  double t2 = (by - ay) * (px - ax);
  return t1 - t2;
}
// Tie rule: an edge traversed counter-clockwise with direction (dx, dy)
// owns the points on it iff dy > 0, or dy == 0 and dx < 0.
inline bool owned(double dx, double dy) { return dy > 0.0 || (dy == 0.0 && dx < 0.0); }

struct Vtx { double x, y; };

/*
 * Point-in-mapped-triangle predicate (Fig. 1: "every time the source plane
 * triangle includes the barycenter").  Lensing may flip a triangle's parity,
 * so the test follows the sign s of its mapped determinant; a triangle whose
 * FP64 determinant is exactly 0 is degenerate and skipped.  The point is
 * inside iff every s*e_k > 0, or e_k == 0 and edge k, taken counter-clockwise,
 * owns it.  On a hit, w[] receives the barycentric weights of A, B, C.
 */
bool point_in_tri(Vtx A, Vtx B, Vtx C, Vtx P, double w[3]) {
  double det = edge_fn(A.x, A.y, B.x, B.y, C.x, C.y);
  if (det == 0.0) return false;
  double e0 = edge_fn(A.x, A.y, B.x, B.y, P.x, P.y);  // edge A->B
  double e1 = edge_fn(B.x, B.y, C.x, C.y, P.x, P.y);  // edge B->C
  double e2 = edge_fn(C.x, C.y, A.x, A.y, P.x, P.y);  // edge C->A
  double s = det > 0.0 ? 1.0 : -1.0;
  const Vtx* from[3] = {&A, &B, &C};
  const Vtx* to[3] = {&B, &C, &A};
  double e[3] = {e0, e1, e2};
  for (int k = 0; k < 3; ++k) {
    double se = s * e[k];
    if (se > 0.0) continue;
    if (se < 0.0) return false;
    // on the edge: direction of the edge in counter-clockwise traversal
    double dx = s > 0.0 ? to[k]->x - from[k]->x : from[k]->x - to[k]->x;
    double dy = s > 0.0 ? to[k]->y - from[k]->y : from[k]->y - to[k]->y;
    if (!owned(dx, dy)) return false;
  }
  w[0] = e1 / det;  // weight of A: edge opposite A is B->C
  w[1] = e2 / det;
  w[2] = e0 / det;
  return true;
}

/*
 * Whether two FP64 evaluations that may differ by up to d per coordinate
 * (different libm transcendentals) could decide this pair differently.
 * Used only to classify pairs for comparisons; it does not change a result.
 */
bool undecidable(Vtx A, Vtx B, Vtx C, Vtx P, double d) {
  double xmin = std::min(A.x, std::min(B.x, C.x)), xmax = std::max(A.x, std::max(B.x, C.x));
  double ymin = std::min(A.y, std::min(B.y, C.y)), ymax = std::max(A.y, std::max(B.y, C.y));
  if (P.x < xmin - 2 * d || P.x > xmax + 2 * d || P.y < ymin - 2 * d || P.y > ymax + 2 * d)
    return false;
  auto bound = [d](Vtx a, Vtx b, Vtx p) {
    double bx = std::fabs(b.x - a.x), by = std::fabs(b.y - a.y);
    double px = std::fabs(p.x - a.x), py = std::fabs(p.y - a.y);
    return 2 * d * (bx + by + px + py) + 8 * d * d + 4 * kU64 * (bx * py + by * px);
  };
  double det = edge_fn(A.x, A.y, B.x, B.y, C.x, C.y);
  if (std::fabs(det) <= bound(A, B, C)) return true;
  if (std::fabs(edge_fn(A.x, A.y, B.x, B.y, P.x, P.y)) <= bound(A, B, P)) return true;
  if (std::fabs(edge_fn(B.x, B.y, C.x, C.y, P.x, P.y)) <= bound(B, C, P)) return true;
  if (std::fabs(edge_fn(C.x, C.y, A.x, A.y, P.x, P.y)) <= bound(C, A, P)) return true;
  return false;
}

// Cell (i, j) has corners v00=(i,j), v10=(i+1,j), v01=(i,j+1), v11=(i+1,j+1);
// T0 = (v00, v10, v11), T1 = (v00, v11, v01); tri = 2 (j (nx-1) + i) + t.
inline void tri_nodes(const Grid& g, int64_t tri, int64_t node[3]) {
  int64_t cell = tri / 2;
  int t = (int)(tri % 2);
  int64_t i = cell % (g.nx - 1), j = cell / (g.nx - 1);
  int64_t v00 = j * g.nx + i, v10 = v00 + 1, v01 = v00 + g.nx, v11 = v01 + 1;
  node[0] = v00;
  node[1] = t == 0 ? v10 : v11;
  node[2] = t == 0 ? v11 : v01;
}

}  // namespace lto

using namespace lto;

extern "C" {

struct lto_hit {
  int32_t src;
  int32_t undecidable;
  int64_t tri;
  double x, y;
  double w[3];
};

struct lto_pair {
  int32_t src;
  int32_t inside;
  int64_t tri;
};

// alpha at n arbitrary points; params is [8][n_pot] for one sample.
int lto_alpha_points(const double* params, int n_pot, int n, const double* x,
                     const double* y, double* ax, double* ay, double* asum) {
  for (int m = 0; m < n; ++m) {
    double sa;
    alpha_total(params, n_pot, x[m], y[m], ax[m], ay[m], &sa);
    if (asum) asum[m] = sa;
  }
  return 0;
}

int lto_deflect_grid(const double* params, int n_pot, double x0, double y0, double dx,
                     double dy, int nx, int ny, int n_threads, double* alpha, double* asum) {
  Grid g{x0, y0, dx, dy, nx, ny};
  deflect_grid(params, n_pot, g, n_threads, alpha, asum);
  return 0;
}

/*
 * Triangle search (Fig. 1): for every source s (position src_xy[s], ratio
 * r[s]) and every mapped triangle, in (s, tri) order, record the hits with
 * their barycentric image positions.  Returns the number of hits (which may
 * exceed capacity; only the first `capacity` are written).  d_src[s] is the
 * uncertainty of the source position used to classify undecidable pairs
 * (0 for exact inputs); those pairs are written to und[] (und_cap entries)
 * and counted in *n_und.
 */
int64_t lto_find_images(const double* params, int n_pot, double x0, double y0, double dx,
                        double dy, int nx, int ny, int n_src, const double* src_xy,
                        const double* r, const double* d_src, int n_threads,
                        int64_t capacity, lto_hit* hits, int64_t und_cap, lto_pair* und,
                        int64_t* n_und) {
  Grid g{x0, y0, dx, dy, nx, ny};
  size_t nn = (size_t)nx * ny;
  const int nt = n_threads > 0 ? n_threads : 1;
  std::vector<double> alpha(2 * nn), asum(nn);
  deflect_grid(params, n_pot, g, nt, alpha.data(), asum.data());
  std::vector<Vtx> beta(nn);
  std::vector<double> dv(nn);
  // hits and undecidable pairs of each cell row, concatenated in row order
  // afterwards: the lists are in (source, triangle) order whatever the
  // number of threads
  const int rows = ny > 1 ? ny - 1 : 0;
  std::vector<std::vector<lto_hit>> row_hits(rows);
  std::vector<std::vector<lto_pair>> row_und(rows);
  int64_t count = 0, ucount = 0;
  for (int s = 0; s < n_src; ++s) {
    double rs = r[s];
#pragma omp parallel for schedule(static) num_threads(nt)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t n = (size_t)j * nx + i;
        double tx = g.X(i), ty = g.Y(j);
        beta[n].x = tx - rs * alpha[2 * n];
        beta[n].y = ty - rs * alpha[2 * n + 1];
        dv[n] = 64.0 * kU64 * (std::fabs(tx) + std::fabs(ty) + rs * asum[n]);
      }
    Vtx P{src_xy[2 * s], src_xy[2 * s + 1]};
    double dp = d_src ? d_src[s] : 0.0;
    int64_t tri_per_row = 2 * (int64_t)(nx - 1);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int jr = 0; jr < rows; ++jr) {
      row_hits[jr].clear();
      row_und[jr].clear();
      for (int64_t tri = jr * tri_per_row; tri < (jr + 1) * tri_per_row; ++tri) {
        int64_t v[3];
        tri_nodes(g, tri, v);
        Vtx A = beta[v[0]], B = beta[v[1]], C = beta[v[2]];
        double w[3];
        bool in = point_in_tri(A, B, C, P, w);
        double d = std::max(std::max(dv[v[0]], dv[v[1]]), std::max(dv[v[2]], dp));
        bool und_pair = undecidable(A, B, C, P, d);
        if (und_pair) row_und[jr].push_back(lto_pair{s, in ? 1 : 0, tri});
        if (in) {
          lto_hit h;
          h.src = s;
          h.undecidable = und_pair ? 1 : 0;
          h.tri = tri;
          h.w[0] = w[0];
          h.w[1] = w[1];
          h.w[2] = w[2];
          int64_t ia = v[0] % nx, ja = v[0] / nx, ib = v[1] % nx, jb = v[1] / nx;
          int64_t ic = v[2] % nx, jc = v[2] / nx;
          h.x = w[0] * g.X((int)ia) + w[1] * g.X((int)ib) + w[2] * g.X((int)ic);
          h.y = w[0] * g.Y((int)ja) + w[1] * g.Y((int)jb) + w[2] * g.Y((int)jc);
          row_hits[jr].push_back(h);
        }
      }
    }
    for (int jr = 0; jr < rows; ++jr) {
      for (const lto_pair& u : row_und[jr]) {
        if (ucount < und_cap) und[ucount] = u;
        ++ucount;
      }
      for (const lto_hit& h : row_hits[jr]) {
        if (count < capacity) hits[count] = h;
        ++count;
      }
    }
  }
  if (n_und) *n_und = ucount;
  return count;
}

/*
 * Barycentres (Sect. 2.2.2): beta_ij = theta_obs,ij - r_i alpha(theta_obs,ij)
 * for every observed image, and for every system the unweighted mean over its
 * images, summed in observation order.  d_bary[i] receives the uncertainty
 * used to classify undecidable pairs.
 */
int lto_barycentres(const double* params, int n_pot, int n_obs, const double* ox,
                    const double* oy, const int32_t* osys, int n_sys, const double* sys_r,
                    double* bary, double* d_bary) {
  std::vector<double> sx(n_sys, 0.0), sy(n_sys, 0.0), dmax(n_sys, 0.0);
  std::vector<int> cnt(n_sys, 0);
  for (int m = 0; m < n_obs; ++m) {
    int i = osys[m];
    double ax, ay, sa;
    alpha_total(params, n_pot, ox[m], oy[m], ax, ay, &sa);
    double bx = ox[m] - sys_r[i] * ax;
    double by = oy[m] - sys_r[i] * ay;
    sx[i] = sx[i] + bx;
    sy[i] = sy[i] + by;
    cnt[i] += 1;
    dmax[i] = std::max(dmax[i], 64.0 * kU64 * (std::fabs(ox[m]) + std::fabs(oy[m]) + sys_r[i] * sa));
  }
  for (int i = 0; i < n_sys; ++i) {
    bary[2 * i] = cnt[i] ? sx[i] / cnt[i] : 0.0;
    bary[2 * i + 1] = cnt[i] ? sy[i] / cnt[i] : 0.0;
    if (d_bary) d_bary[i] = 2.0 * dmax[i];
  }
  return 0;
}

/*
 * chi^2 of Eq. 11 for one sample.  For each observed image (in observation
 * order) the predicted image of its system nearest to it is taken (ties to
 * the lower triangle id); a system with no predicted image contributes
 * (L_diag / sigma)^2 per observed image, L_diag the grid diagonal.
 * Outputs: *chi2; match_tri[n_obs] (-1 if none), match_xy[n_obs][2];
 * bary[n_sys][2]; *n_hits, *n_und.  Hits go to hits[capacity].
 */
int lto_chi2(const double* params, int n_pot, double x0, double y0, double dx, double dy,
             int nx, int ny, int n_obs, const double* ox, const double* oy, const double* osig,
             const int32_t* osys, int n_sys, const double* sys_r, int n_threads,
             int64_t capacity, lto_hit* hits, double* chi2, int64_t* match_tri,
             double* match_xy, double* bary, int64_t* n_hits, int64_t* n_und) {
  std::vector<double> d_bary(n_sys);
  lto_barycentres(params, n_pot, n_obs, ox, oy, osys, n_sys, sys_r, bary, d_bary.data());
  std::vector<lto_pair> und(1);
  int64_t nh = lto_find_images(params, n_pot, x0, y0, dx, dy, nx, ny, n_sys, bary, sys_r,
                               d_bary.data(), n_threads, capacity, hits, 0, und.data(), n_und);
  if (n_hits) *n_hits = nh;
  if (nh > capacity) return 1;
  double Lx = (nx - 1) * dx, Ly = (ny - 1) * dy;
  double diag = std::sqrt(Lx * Lx + Ly * Ly);
  double total = 0.0;
  for (int m = 0; m < n_obs; ++m) {
    int i = osys[m];
    int64_t best = -1;
    double bd = 0.0;
    for (int64_t h = 0; h < nh; ++h) {
      if (hits[h].src != i) continue;
      double ex = ox[m] - hits[h].x, ey = oy[m] - hits[h].y;
      double d2 = ex * ex + ey * ey;
      if (best < 0 || d2 < bd || (d2 == bd && hits[h].tri < hits[best].tri)) {
        best = h;
        bd = d2;
      }
    }
    double term;
    if (best < 0) {
      double t = diag / osig[m];
      term = t * t;
      match_tri[m] = -1;
      match_xy[2 * m] = match_xy[2 * m + 1] = 0.0;
    } else {
      term = bd / (osig[m] * osig[m]);
      match_tri[m] = hits[best].tri;
      match_xy[2 * m] = hits[best].x;
      match_xy[2 * m + 1] = hits[best].y;
    }
    total = total + term;
  }
  *chi2 = total;
  return 0;
}

}  // extern "C"

namespace lto {

/*
 * chi^2 with the assignment frozen: observed image m is predicted by the
 * barycentric interpolation inside triangle match_tri[m] (or contributes the
 * constant penalty when match_tri[m] < 0).  Templated so the same code gives
 * the value (T = double) and forward-mode derivatives (T = Dual).
 */
template <class T>
T chi2_frozen(const T* params, int n_pot, const Grid& g, int n_obs, const double* ox,
              const double* oy, const double* osig, const int32_t* osys, int n_sys,
              const double* sys_r, const int64_t* match_tri) {
  std::vector<T> bx(n_sys, T(0.0)), by(n_sys, T(0.0));
  std::vector<int> cnt(n_sys, 0);
  for (int m = 0; m < n_obs; ++m) {
    int i = osys[m];
    T ax, ay;
    alpha_total(params, n_pot, ox[m], oy[m], ax, ay, nullptr);
    bx[i] = bx[i] + (ox[m] - sys_r[i] * ax);
    by[i] = by[i] + (oy[m] - sys_r[i] * ay);
    cnt[i] += 1;
  }
  for (int i = 0; i < n_sys; ++i)
    if (cnt[i]) {
      bx[i] = bx[i] / (double)cnt[i];
      by[i] = by[i] / (double)cnt[i];
    }
  double Lx = (g.nx - 1) * g.dx, Ly = (g.ny - 1) * g.dy;
  double diag = std::sqrt(Lx * Lx + Ly * Ly);
  T total(0.0);
  for (int m = 0; m < n_obs; ++m) {
    int i = osys[m];
    if (match_tri[m] < 0) {
      double t = diag / osig[m];
      total = total + t * t;
      continue;
    }
    int64_t v[3];
    tri_nodes(g, match_tri[m], v);
    T vx[3], vy[3];
    double tx[3], ty[3];
    for (int c = 0; c < 3; ++c) {
      tx[c] = g.X((int)(v[c] % g.nx));
      ty[c] = g.Y((int)(v[c] / g.nx));
      T ax, ay;
      alpha_total(params, n_pot, tx[c], ty[c], ax, ay, nullptr);
      vx[c] = tx[c] - sys_r[i] * ax;
      vy[c] = ty[c] - sys_r[i] * ay;
    }
    // barycentric weights from the edge functions, as in point_in_tri
    auto ef = [](T ax, T ay, T bx_, T by_, T px, T py) {
      return (bx_ - ax) * (py - ay) - (by_ - ay) * (px - ax);
    };
    T det = ef(vx[0], vy[0], vx[1], vy[1], vx[2], vy[2]);
    T wA = ef(vx[1], vy[1], vx[2], vy[2], bx[i], by[i]) / det;
    T wB = ef(vx[2], vy[2], vx[0], vy[0], bx[i], by[i]) / det;
    T wC = ef(vx[0], vy[0], vx[1], vy[1], bx[i], by[i]) / det;
    T px = wA * tx[0] + wB * tx[1] + wC * tx[2];
    T py = wA * ty[0] + wB * ty[1] + wC * ty[2];
    T ex = ox[m] - px, ey = oy[m] - py;
    total = total + (ex * ex + ey * ey) / (osig[m] * osig[m]);
  }
  return total;
}

}  // namespace lto

extern "C" {

int lto_chi2_frozen(const double* params, int n_pot, double x0, double y0, double dx,
                    double dy, int nx, int ny, int n_obs, const double* ox, const double* oy,
                    const double* osig, const int32_t* osys, int n_sys, const double* sys_r,
                    const int64_t* match_tri, double* chi2) {
  Grid g{x0, y0, dx, dy, nx, ny};
  *chi2 = chi2_frozen<double>(params, n_pot, g, n_obs, ox, oy, osig, osys, n_sys, sys_r,
                              match_tri);
  return 0;
}

/*
 * Deflection Jacobian J = d alpha / d theta at n points, jac[m] = (J_xx, J_xy,
 * J_yx, J_yy).  Forward-mode duals: seeding the centre row (x, then y) of
 * every potential at once gives sum_k d alpha_k / d c_k = -J, because each
 * alpha_k depends on theta and c_k only through theta - c_k.
 */
int lto_jacobian_points(const double* params, int n_pot, int n, const double* x,
                        const double* y, double* jac) {
  std::vector<Dual> p(N_ROWS * (size_t)n_pot);
  for (int m = 0; m < n; ++m) {
    for (int col = 0; col < 2; ++col) {  // derivative w.r.t. theta_x, then theta_y
      for (size_t t = 0; t < p.size(); ++t) p[t] = Dual(params[t], 0.0);
      const int row = col == 0 ? R_X : R_Y;
      for (int k = 0; k < n_pot; ++k) p[(size_t)row * n_pot + k].d = 1.0;
      Dual ax, ay;
      alpha_total(p.data(), n_pot, x[m], y[m], ax, ay, nullptr);
      jac[4 * m + col] = -ax.d;      // J_xx, J_xy
      jac[4 * m + 2 + col] = -ay.d;  // J_yx, J_yy
    }
  }
  return 0;
}

/*
 * Source-plane chi^2 of one sample (the LENSTOOL source-plane fit of Jullo et
 * al. 2007, which the paper cites for the chi^2): for every observed image m
 * of system i, beta_m = theta_m - r_i alpha(theta_m) (Eq. 13), the system's
 * barycentre as in step 3, and
 *   chi^2_S = sum_m |beta_m - beta_bar_i|^2 mu_m^2 / sigma_m^2,
 *   mu_m = 1 / det(I - r_i J(theta_m)),
 * i.e. the image-plane error budget carried to the source plane by the local
 * magnification.  mu[n_obs] receives mu_m.
 */
int lto_chi2_source(const double* params, int n_pot, int n_obs, const double* ox,
                    const double* oy, const double* osig, const int32_t* osys, int n_sys,
                    const double* sys_r, double* chi2, double* mu) {
  std::vector<double> bary(2 * (size_t)n_sys), jac(4 * (size_t)n_obs);
  lto_barycentres(params, n_pot, n_obs, ox, oy, osys, n_sys, sys_r, bary.data(), nullptr);
  lto_jacobian_points(params, n_pot, n_obs, ox, oy, jac.data());
  double c2 = 0.0;
  for (int m = 0; m < n_obs; ++m) {
    const int i = osys[m];
    const double r = sys_r[i];
    double ax, ay;
    alpha_total(params, n_pot, ox[m], oy[m], ax, ay, nullptr);
    const double bx = ox[m] - r * ax, by = oy[m] - r * ay;
    const double* J = &jac[4 * (size_t)m];
    const double det = (1.0 - r * J[0]) * (1.0 - r * J[3]) - (r * J[1]) * (r * J[2]);
    const double u = 1.0 / det;
    mu[m] = u;
    const double ex = bx - bary[2 * i], ey = by - bary[2 * i + 1];
    c2 = c2 + (ex * ex + ey * ey) * u * u / (osig[m] * osig[m]);
  }
  *chi2 = c2;
  return 0;
}

/*
 * Triangle magnification of the triangles tri[n] of a grid (numbering as in
 * step 4): the signed image-plane area divided by the signed area of the
 * triangle lensed with ratio r[n] (Eq. 13).  Negative for images of odd
 * parity; +-inf where the lensed triangle is degenerate.
 */
int lto_tri_magnification(const double* params, int n_pot, double x0, double y0, double dx,
                          double dy, int nx, int ny, int n, const int64_t* tri, const double* r,
                          double* mu) {
  Grid g{x0, y0, dx, dy, nx, ny};
  for (int m = 0; m < n; ++m) {
    int64_t node[3];
    tri_nodes(g, tri[m], node);
    double tx[3], ty[3], bx[3], by[3];
    for (int v = 0; v < 3; ++v) {
      tx[v] = g.X((int)(node[v] % nx));
      ty[v] = g.Y((int)(node[v] / nx));
      double ax, ay;
      alpha_total(params, n_pot, tx[v], ty[v], ax, ay, nullptr);
      bx[v] = tx[v] - r[m] * ax;
      by[v] = ty[v] - r[m] * ay;
    }
    const double area_img = (tx[1] - tx[0]) * (ty[2] - ty[0]) - (ty[1] - ty[0]) * (tx[2] - tx[0]);
    const double area_src = (bx[1] - bx[0]) * (by[2] - by[0]) - (by[1] - by[0]) * (bx[2] - bx[0]);
    mu[m] = area_img / area_src;
  }
  return 0;
}

/*
 * d chi^2 / d(x, y, e, phi, r_core, sigma_v) of every potential, with the
 * assignment match_tri[] frozen: one forward-mode dual pass per parameter.
 * grad is [n_pot][6].
 */
int lto_chi2_grad(const double* params, int n_pot, double x0, double y0, double dx,
                  double dy, int nx, int ny, int n_obs, const double* ox, const double* oy,
                  const double* osig, const int32_t* osys, int n_sys, const double* sys_r,
                  const int64_t* match_tri, double* chi2, double* grad) {
  Grid g{x0, y0, dx, dy, nx, ny};
  static const int rows[6] = {R_X, R_Y, R_E, R_PHI, R_RC, R_SV};
  std::vector<Dual> p(N_ROWS * (size_t)n_pot);
  for (size_t n = 0; n < p.size(); ++n) p[n] = Dual(params[n], 0.0);
  for (int k = 0; k < n_pot; ++k)
    for (int m = 0; m < 6; ++m) {
      size_t idx = (size_t)rows[m] * n_pot + k;
      p[idx].d = 1.0;
      Dual c = chi2_frozen<Dual>(p.data(), n_pot, g, n_obs, ox, oy, osig, osys, n_sys,
                                 sys_r, match_tri);
      p[idx].d = 0.0;
      grad[k * 6 + m] = c.d;
      if (chi2) *chi2 = c.v;
    }
  return 0;
}

}  // extern "C"

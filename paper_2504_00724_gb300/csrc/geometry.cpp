// Cut cells, Green-formula moments and Alg. 1 merging (Sec. 2.4, Sec. 3.1).
//
// A level's box is cut by closed parametric curves.  Crossings of each curve with the grid
// lines split it into arcs that each lie in one cell; in every cell that holds arcs, the
// loops "arc, then counter-clockwise along the cell edges to the next arc entry" bound the
// connected pieces of C_i cap Omega.  Moments int X^p Y^q dA (X, Y in the cell frame,
// units of h) follow from Green's formula int_C f dA = int_dC F dY with F = X^{p+1}/(p+1)
// (eq. volumeIntegral with xi0 at the cell centre): exact on straight pieces, Gauss-Legendre
// on arcs.  Alg. 1 then folds every component but the largest of a multi-piece cell into
// its largest neighbour, and merges each interface cell with volume <= theta h^2, smallest
// first, into the non-empty 4-neighbour with the longest common cut face (ties: larger
// volume, then +x, -x, +y, -y).
#include <algorithm>
#include <atomic>
#include <thread>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>

#include "host.h"

namespace ccm {

static const double TWO_PI = 6.283185307179586476925286766559;

// ------------------------------------------------------------------ curves

// edge of a polygon at parameter t: vertices a -> b and the position s in [0, 1) along it
static void polygon_edge(const Curve& c, double t, int& a, int& b, double& s) {
  const int n = (int)(c.V.size() / 2);
  const double u = t * (n / (2 * M_PI));
  const double k = std::floor(u);
  s = u - k;
  a = (int)(((long)k % n + n) % n);
  b = (a + 1) % n;
}

bool Curve::prepare() {
  if (kind != CCM_SPLINE) return true;
  const int n = (int)(V.size() / 2);
  knots.assign(n + 1, 0.0);
  for (int k = 0; k < n; ++k) {
    const int l = (k + 1) % n;
    const double ch = std::hypot(V[2 * l] - V[2 * k], V[2 * l + 1] - V[2 * k + 1]);
    if (!(ch > 0)) return false;
    knots[k + 1] = knots[k] + ch;
  }
  const double L = knots[n];
  for (int k = 0; k <= n; ++k) knots[k] = 2 * M_PI * knots[k] / L;
  knots[n] = 2 * M_PI;
  // periodic cubic spline: h_{k-1} M_{k-1} + 2 (h_{k-1} + h_k) M_k + h_k M_{k+1} = 6 (d_k - d_{k-1}),
  // d_k = (v_{k+1} - v_k) / h_k, indices mod n; dense elimination with partial pivoting
  for (int c = 0; c < 2; ++c) {
    std::vector<double> A((size_t)n * n, 0.0), r(n);
    for (int k = 0; k < n; ++k) {
      const int km = (k + n - 1) % n, kp = (k + 1) % n;
      const double hm = knots[km + 1] - knots[km], hk = knots[k + 1] - knots[k];
      A[(size_t)k * n + km] += hm;
      A[(size_t)k * n + k] += 2 * (hm + hk);
      A[(size_t)k * n + kp] += hk;
      const double dk = (V[2 * kp + c] - V[2 * k + c]) / hk, dm = (V[2 * k + c] - V[2 * km + c]) / hm;
      r[k] = 6 * (dk - dm);
    }
    for (int col = 0; col < n; ++col) {
      int piv = col;
      for (int row = col + 1; row < n; ++row)
        if (std::fabs(A[(size_t)row * n + col]) > std::fabs(A[(size_t)piv * n + col])) piv = row;
      if (piv != col) {
        for (int m = 0; m < n; ++m) std::swap(A[(size_t)piv * n + m], A[(size_t)col * n + m]);
        std::swap(r[piv], r[col]);
      }
      const double d = A[(size_t)col * n + col];
      if (!(std::fabs(d) > 0)) return false;
      for (int row = col + 1; row < n; ++row) {
        const double f = A[(size_t)row * n + col] / d;
        if (f == 0.0) continue;
        for (int m = col; m < n; ++m) A[(size_t)row * n + m] -= f * A[(size_t)col * n + m];
        r[row] -= f * r[col];
      }
    }
    M[c].assign(n, 0.0);
    for (int row = n - 1; row >= 0; --row) {
      double s = r[row];
      for (int m = row + 1; m < n; ++m) s -= A[(size_t)row * n + m] * M[c][m];
      M[c][row] = s / A[(size_t)row * n + row];
    }
  }
  poly.clear();
  for (int k = 0; k < n; ++k)
    for (int s = 0; s < 64; ++s) {
      double x, y;
      xy(knots[k] + (knots[k + 1] - knots[k]) * s / 64.0, x, y);
      poly.push_back(x);
      poly.push_back(y);
    }
  return true;
}

// even-odd rule against a closed polyline (x0, y0, x1, y1, ...)
static bool inside_polyline(const std::vector<double>& P, double x, double y) {
  const int n = (int)(P.size() / 2);
  bool in = false;
  for (int k = 0; k < n; ++k) {
    const double xa = P[2 * k], ya = P[2 * k + 1];
    const double xb = P[2 * ((k + 1) % n)], yb = P[2 * ((k + 1) % n) + 1];
    if (ya == yb) continue;
    if ((ya > y) != (yb > y) && x < xa + (y - ya) * (xb - xa) / (yb - ya)) in = !in;
  }
  return in;
}

// spline segment of t (mod 2 pi) and its local coordinates
static void spline_seg(const Curve& c, double t, int& k, double& hk, double& a, double& b) {
  const int n = (int)(c.V.size() / 2);
  double tt = std::fmod(t, 2 * M_PI);
  if (tt < 0) tt += 2 * M_PI;
  k = (int)(std::upper_bound(c.knots.begin(), c.knots.end(), tt) - c.knots.begin()) - 1;
  k = std::min(std::max(k, 0), n - 1);
  hk = c.knots[k + 1] - c.knots[k];
  a = (c.knots[k + 1] - tt) / hk;
  b = (tt - c.knots[k]) / hk;
}

void Curve::subintervals(double t0, double t1, std::vector<std::pair<double, double>>& out) const {
  out.clear();
  if (kind != CCM_POLYGON && kind != CCM_SPLINE) {
    out.push_back({t0, t1});
    return;
  }
  const int n = (int)(V.size() / 2);
  const double lo = std::min(t0, t1), hi = std::max(t0, t1);
  std::vector<double> cuts;
  for (int k = 0; k < n; ++k) {
    const double b = kind == CCM_SPLINE ? knots[k] : 2 * M_PI * k / n;
    double v = b + 2 * M_PI * std::ceil((lo - b) / (2 * M_PI));
    for (; v < hi; v += 2 * M_PI)
      if (v > lo) cuts.push_back(v);
  }
  std::sort(cuts.begin(), cuts.end());
  if (t1 < t0) std::reverse(cuts.begin(), cuts.end());
  double a = t0;
  for (double v : cuts) {
    out.push_back({a, v});
    a = v;
  }
  out.push_back({a, t1});
}

void Curve::xy(double t, double& x, double& y) const {
  if (kind == CCM_SPLINE) {
    int k;
    double hk, a, b;
    spline_seg(*this, t, k, hk, a, b);
    const int n = (int)(V.size() / 2), k1 = (k + 1) % n;
    double* o[2] = {&x, &y};
    for (int c = 0; c < 2; ++c)
      *o[c] = a * V[2 * k + c] + b * V[2 * k1 + c] + ((a * a * a - a) * M[c][k] + (b * b * b - b) * M[c][k1]) * hk * hk / 6;
    return;
  }
  if (kind == CCM_POLYGON) {
    int a, b;
    double s;
    polygon_edge(*this, t, a, b, s);
    x = V[2 * a] + (V[2 * b] - V[2 * a]) * s;
    y = V[2 * a + 1] + (V[2 * b + 1] - V[2 * a + 1]) * s;
    return;
  }
  switch (kind) {
    case CCM_CIRCLE:
      x = p[0] + p[2] * std::cos(t);
      y = p[1] + p[2] * std::sin(t);
      return;
    case CCM_ELLIPSE: {
      double X = p[2] * std::cos(t), Y = p[3] * std::sin(t);
      double c = std::cos(p[4]), s = std::sin(p[4]);
      x = p[0] + X * c - Y * s;
      y = p[1] + X * s + Y * c;
      return;
    }
    default: {
      double r = p[2] + p[3] * std::cos(p[4] * t);
      x = p[0] + r * std::cos(t);
      y = p[1] + r * std::sin(t);
    }
  }
}

void Curve::dxy(double t, double& x, double& y) const {
  if (kind == CCM_SPLINE) {
    int k;
    double hk, a, b;
    spline_seg(*this, t, k, hk, a, b);
    const int n = (int)(V.size() / 2), k1 = (k + 1) % n;
    double* o[2] = {&x, &y};
    for (int c = 0; c < 2; ++c)
      *o[c] = (V[2 * k1 + c] - V[2 * k + c]) / hk + ((1 - 3 * a * a) * M[c][k] + (3 * b * b - 1) * M[c][k1]) * hk / 6;
    return;
  }
  if (kind == CCM_POLYGON) {
    int a, b;
    double s;
    polygon_edge(*this, t, a, b, s);
    const double sc = (double)(V.size() / 2) / (2 * M_PI);
    x = (V[2 * b] - V[2 * a]) * sc;
    y = (V[2 * b + 1] - V[2 * a + 1]) * sc;
    return;
  }
  switch (kind) {
    case CCM_CIRCLE:
      x = -p[2] * std::sin(t);
      y = p[2] * std::cos(t);
      return;
    case CCM_ELLIPSE: {
      double X = -p[2] * std::sin(t), Y = p[3] * std::cos(t);
      double c = std::cos(p[4]), s = std::sin(p[4]);
      x = X * c - Y * s;
      y = X * s + Y * c;
      return;
    }
    default: {
      double r = p[2] + p[3] * std::cos(p[4] * t);
      double dr = -p[3] * p[4] * std::sin(p[4] * t);
      x = dr * std::cos(t) - r * std::sin(t);
      y = dr * std::sin(t) + r * std::cos(t);
    }
  }
}

bool Curve::inside(double x, double y) const {
  // even-odd rule: a ray towards +x crosses the boundary an odd number of times; a spline is
  // tested against its 64-per-cubic polyline (the test only classifies centres of cells the
  // curve does not enter, h/2 or more from it)
  if (kind == CCM_POLYGON) return inside_polyline(V, x, y);
  if (kind == CCM_SPLINE) return inside_polyline(poly, x, y);
  switch (kind) {
    case CCM_CIRCLE: {
      double dx = x - p[0], dy = y - p[1];
      return dx * dx + dy * dy < p[2] * p[2];
    }
    case CCM_ELLIPSE: {
      double dx = x - p[0], dy = y - p[1];
      double c = std::cos(p[4]), s = std::sin(p[4]);
      double X = (dx * c + dy * s) / p[2], Y = (-dx * s + dy * c) / p[3];
      return X * X + Y * Y < 1.0;
    }
    default: {
      double dx = x - p[0], dy = y - p[1];
      double th = std::atan2(dy, dx);
      return std::hypot(dx, dy) < p[2] + p[3] * std::cos(p[4] * th);
    }
  }
}

// ------------------------------------------------------------------ moment helpers

const Mom& pure_moments() {
  static Mom m = [] {
    Mom r{};
    for (int k = 0; k < NMOM; ++k) {
      int p = mono_p(k), q = mono_q(k);
      double ip = (p % 2) ? 0.0 : 2.0 * std::pow(0.5, p + 1) / (p + 1);
      double iq = (q % 2) ? 0.0 : 2.0 * std::pow(0.5, q + 1) / (q + 1);
      r[k] = ip * iq;
    }
    return r;
  }();
  return m;
}

static double binom(int n, int k) {
  static const double B[5][5] = {{1, 0, 0, 0, 0}, {1, 1, 0, 0, 0}, {1, 2, 1, 0, 0}, {1, 3, 3, 1, 0}, {1, 4, 6, 4, 1}};
  return B[n][k];
}

// moments about the frame X' = X + dx, Y' = Y + dy
Mom shift_moments(const Mom& m, double dx, double dy) {
  double px[5] = {1, dx, dx * dx, dx * dx * dx, dx * dx * dx * dx};
  double py[5] = {1, dy, dy * dy, dy * dy * dy, dy * dy * dy * dy};
  Mom out{};
  for (int k = 0; k < NMOM; ++k) {
    int p = mono_p(k), q = mono_q(k);
    double s = 0;
    for (int a = 0; a <= p; ++a)
      for (int b = 0; b <= q; ++b) s += binom(p, a) * binom(q, b) * px[p - a] * py[q - b] * m[mono_index(a, b)];
    out[k] = s;
  }
  return out;
}

const Mom& CutLevel::moments(int lin) const {
  auto it = mom.find(lin);
  return it == mom.end() ? pure_moments() : it->second;
}

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        // final derivative for the weight
        p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
          double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        break;
      }
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = -z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

static const int GL_ARC = 12;

struct GL {
  std::vector<double> x, w;
  explicit GL(int n) { gauss_legendre(n, x, w); }
};
static const GL& gl_arc() {
  static GL g(GL_ARC);
  return g;
}

// int over the piece of X^{p+1}/(p+1) Y^q dY, frame centred at (xc, yc), units of h
static void piece_moments(const Piece& pc, const std::vector<Curve>& curves, double xc, double yc,
                          double h, Mom& acc) {
  if (!pc.arc) {
    double X0 = (pc.ax - xc) / h, Y0 = (pc.ay - yc) / h;
    double X1 = (pc.bx - xc) / h, Y1 = (pc.by - yc) / h;
    if (Y0 == Y1) return;
    // pieces on cell edges are axis-parallel: vertical here, X constant
    double X = 0.5 * (X0 + X1);
    for (int k = 0; k < NMOM; ++k) {
      int p = mono_p(k), q = mono_q(k);
      acc[k] += std::pow(X, p + 1) / (p + 1) * (std::pow(Y1, q + 1) - std::pow(Y0, q + 1)) / (q + 1);
    }
    return;
  }
  const Curve& c = curves[pc.curve];
  const GL& g = gl_arc();
  std::vector<std::pair<double, double>> parts;
  c.subintervals(pc.t0, pc.t1, parts);
  for (const auto& ab : parts) {
    double tm = 0.5 * (ab.first + ab.second), tr = 0.5 * (ab.second - ab.first);
    for (int n = 0; n < GL_ARC; ++n) {
      double t = tm + tr * g.x[n], x, y, dx, dy;
      c.xy(t, x, y);
      c.dxy(t, dx, dy);
      double X = (x - xc) / h, Y = (y - yc) / h, wY = dy / h * tr * g.w[n];
      double Xp[6] = {1, X, X * X, X * X * X, X * X * X * X, X * X * X * X * X};
      double Yq[5] = {1, Y, Y * Y, Y * Y * Y, Y * Y * Y * Y};
      for (int k = 0; k < NMOM; ++k) {
        int p = mono_p(k), q = mono_q(k);
        acc[k] += Xp[p + 1] / (p + 1) * Yq[q] * wY;
      }
    }
  }
}

// int_S X^p Y^q ds and the same with n_x, n_y (outward normal = right-hand normal)
static void piece_bmoments(const Piece& pc, const std::vector<Curve>& curves, double xc, double yc,
                           double h, Mom& b0, Mom& bx, Mom& by) {
  const GL& g = gl_arc();
  auto add = [&](double X, double Y, double ds, double nx, double ny) {
    double Xp[5] = {1, X, X * X, X * X * X, X * X * X * X};
    double Yq[5] = {1, Y, Y * Y, Y * Y * Y, Y * Y * Y * Y};
    for (int k = 0; k < NMOM; ++k) {
      double v = Xp[mono_p(k)] * Yq[mono_q(k)] * ds;
      b0[k] += v;
      bx[k] += v * nx;
      by[k] += v * ny;
    }
  };
  if (!pc.arc) {
    for (int n = 0; n < GL_ARC; ++n) {
      double s = 0.5 * (g.x[n] + 1.0);
      double X0 = (pc.ax - xc) / h, Y0 = (pc.ay - yc) / h, X1 = (pc.bx - xc) / h, Y1 = (pc.by - yc) / h;
      double L = std::hypot(X1 - X0, Y1 - Y0);
      add(X0 + (X1 - X0) * s, Y0 + (Y1 - Y0) * s, L * 0.5 * g.w[n], (Y1 - Y0) / L, -(X1 - X0) / L);
    }
    return;
  }
  const Curve& c = curves[pc.curve];
  std::vector<std::pair<double, double>> parts;
  c.subintervals(pc.t0, pc.t1, parts);
  for (const auto& ab : parts) {
    double tm = 0.5 * (ab.first + ab.second), tr = 0.5 * (ab.second - ab.first);
    for (int n = 0; n < GL_ARC; ++n) {
      double t = tm + tr * g.x[n], x, y, dx, dy;
      c.xy(t, x, y);
      c.dxy(t, dx, dy);
      double sp = std::hypot(dx, dy), sg = tr > 0 ? 1.0 : -1.0;
      add((x - xc) / h, (y - yc) / h, sp / h * std::fabs(tr) * g.w[n], sg * dy / sp, -sg * dx / sp);
    }
  }
}

// ------------------------------------------------------------------ crossings

struct Crossing {
  double t;
  int axis;   // 0: vertical line x = x0 + k h, 1: horizontal line y = y0 + k h
  long k;
  bool operator<(const Crossing& o) const {
    if (t != o.t) return t < o.t;
    if (axis != o.axis) return axis < o.axis;
    return k < o.k;
  }
};

// root of f on [a, b] with f(a) f(b) < 0: bisection-secant (Illinois) to full precision
static double find_root(const std::function<double(double)>& f, double a, double b, double fa, double fb) {
  int side = 0;
  for (int it = 0; it < 300; ++it) {
    double c = (fa * b - fb * a) / (fa - fb);
    if (!(c > std::min(a, b) && c < std::max(a, b))) c = 0.5 * (a + b);
    double fc = f(c);
    if (fc == 0.0) return c;
    if ((fc > 0) == (fb > 0)) {
      b = c;
      fb = fc;
      if (side == -1) fa *= 0.5;
      side = -1;
    } else {
      a = c;
      fa = fc;
      if (side == 1) fb *= 0.5;
      side = 1;
    }
    if (std::fabs(b - a) <= 4e-16 * std::max(1.0, std::fabs(a))) break;
  }
  return std::fabs(fa) < std::fabs(fb) ? a : b;
}

static std::vector<Crossing> curve_crossings(const Curve& c, double x0, double y0, double h) {
  double tot = 0, px, py, qx, qy;
  c.xy(0.0, px, py);
  for (int s = 1; s <= 4096; ++s) {
    c.xy(TWO_PI * s / 4096, qx, qy);
    tot += std::hypot(qx - px, qy - py);
    px = qx;
    py = qy;
  }
  long ns = std::max<long>(4096, (long)std::ceil(64.0 * tot / h));
  std::vector<double> t(ns + 1), xs(ns + 1), ys(ns + 1);
  for (long s = 0; s <= ns; ++s) {
    t[s] = TWO_PI * (double)s / (double)ns;
    c.xy(t[s], xs[s], ys[s]);
  }
  xs[ns] = xs[0];
  ys[ns] = ys[0];
  std::vector<Crossing> out;
  for (int axis = 0; axis < 2; ++axis) {
    const std::vector<double>& v = axis == 0 ? xs : ys;
    double org = axis == 0 ? x0 : y0;
    long prev = (long)std::floor((v[0] - org) / h);
    for (long s = 0; s < ns; ++s) {
      long cur = (long)std::floor((v[s + 1] - org) / h);
      if (cur != prev) {
        long lo = std::min(prev, cur), hi = std::max(prev, cur);
        for (long k = lo + 1; k <= hi; ++k) {
          double L = org + k * h;
          double fa = v[s] - L, fb = v[s + 1] - L, tr;
          if (fa == 0.0) {
            tr = t[s];
          } else if (fb == 0.0) {
            tr = t[s + 1];
          } else if (fa * fb > 0.0) {
            continue;   // the cell index changed only by the rounding of (v - org) / h
          } else {
            auto f = [&](double tt) {
              double x, y;
              c.xy(tt, x, y);
              return (axis == 0 ? x : y) - L;
            };
            double fbe = f(t[s + 1]);
            if (fbe * fa > 0) tr = t[s + 1];       // the periodic seam t = 2 pi
            else tr = find_root(f, t[s], t[s + 1], fa, fbe);
          }
          out.push_back({std::fmod(tr, TWO_PI), axis, k});
        }
      }
      prev = cur;
    }
  }
  std::sort(out.begin(), out.end());
  // a curve that only touches a line crosses it twice at the same parameter: drop both
  bool changed = true;
  while (changed && out.size() > 1) {
    changed = false;
    size_t n = out.size();
    for (size_t a = 0; a < n; ++a) {
      size_t b = (a + 1) % n;
      double dt = std::fmod(out[b].t - out[a].t + TWO_PI, TWO_PI);
      if (out[a].axis == out[b].axis && out[a].k == out[b].k && dt < 1e-12) {
        std::vector<Crossing> keep;
        for (size_t m = 0; m < n; ++m)
          if (m != a && m != b) keep.push_back(out[m]);
        out.swap(keep);
        changed = true;
        break;
      }
    }
  }
  return out;
}

// ------------------------------------------------------------------ loops

struct Arc {
  int curve;
  double ts, te;          // traversal from ts to te
  double s_in, s_out;     // perimeter coordinates of entry and exit
  double Xin, Yin, Xout, Yout;
};

static double sigma_of(double X, double Y, int edge) {
  switch (edge) {
    case 0: return X + 0.5;          // bottom
    case 1: return 1.5 + Y;          // right
    case 2: return 2.5 - X;          // top
    default: return 3.5 - Y;         // left
  }
}

static const double CORNER_X[4] = {-0.5, 0.5, 0.5, -0.5};
static const double CORNER_Y[4] = {-0.5, -0.5, 0.5, 0.5};

int check_problem(const ccm_problem& prob) {
  if (!(prob.h > 0) || prob.nx < 4 || prob.ny < 4 || prob.ncurves < 0 || (prob.ncurves > 0 && !prob.curves))
    return CCM_EINVAL;
  if (!(prob.b * prob.b - 4 * prob.a * prob.c < 0)) return CCM_EINVAL;   // elliptic (Sec. 2)
  if (prob.box_bc != CCM_NONE && prob.box_bc != CCM_DIRICHLET && prob.box_bc != CCM_NEUMANN) return CCM_EINVAL;
  for (int k = 0; k < prob.ncurves; ++k) {
    const ccm_curve& c = prob.curves[k];
    if (c.kind < CCM_CIRCLE || c.kind > CCM_SPLINE || (c.orient != 1 && c.orient != -1) ||
        (c.bc != CCM_DIRICHLET && c.bc != CCM_NEUMANN && c.bc != CCM_ROBIN))
      return CCM_EINVAL;
    if (c.kind == CCM_POLYGON || c.kind == CCM_SPLINE) {
      if (c.npts < 3 || !c.pts) return CCM_EINVAL;
      double area2 = 0;
      for (int v = 0; v < c.npts; ++v) {
        const int w = (v + 1) % c.npts;
        if (!std::isfinite(c.pts[2 * v]) || !std::isfinite(c.pts[2 * v + 1])) return CCM_EINVAL;
        area2 += c.pts[2 * v] * c.pts[2 * w + 1] - c.pts[2 * w] * c.pts[2 * v + 1];
      }
      if (!(area2 > 0)) return CCM_EINVAL;      // counter-clockwise
    }
    if (c.bc == CCM_ROBIN && (!std::isfinite(c.robin[0]) || !std::isfinite(c.robin[1]) ||
                              (c.robin[0] == 0.0 && c.robin[1] == 0.0)))
      return CCM_EINVAL;
  }
  return CCM_OK;
}

int build_cut_level(const ccm_problem& prob, int nx, int ny, double h, double theta, CutLevel& cg,
                    std::string& err, CentreClassifier* cc) {
  cg.nx = nx;
  cg.ny = ny;
  cg.h = h;
  cg.x0 = prob.x0;
  cg.y0 = prob.y0;
  cg.box_bc = prob.box_bc;
  cg.curves.clear();
  for (int k = 0; k < prob.ncurves; ++k) {
    Curve c;
    c.kind = prob.curves[k].kind;
    std::memcpy(c.p, prob.curves[k].p, sizeof(c.p));
    c.orient = prob.curves[k].orient;
    c.bc = prob.curves[k].bc;
    if (c.kind == CCM_POLYGON || c.kind == CCM_SPLINE) {
      c.V.assign(prob.curves[k].pts, prob.curves[k].pts + 2 * prob.curves[k].npts);
      if (!c.prepare()) {
        err = "degenerate spline";
        return CCM_EGEOM;
      }
    }
    if (c.bc == CCM_ROBIN) {
      c.robin[0] = prob.curves[k].robin[0];
      c.robin[1] = prob.curves[k].robin[1];
    } else {
      c.robin[0] = c.bc == CCM_NEUMANN ? 0.0 : 1.0;
      c.robin[1] = c.bc == CCM_NEUMANN ? 1.0 : 0.0;
    }
    cg.curves.push_back(c);
  }
  const bool walls = prob.box_bc != CCM_NONE;
  const double x0 = prob.x0, y0 = prob.y0;
  const long N = (long)nx * ny;

  // ---- arcs per cell
  std::map<int, std::vector<Arc>> arcs;   // ordered by linear index
  for (int ci = 0; ci < (int)cg.curves.size(); ++ci) {
    const Curve& c = cg.curves[ci];
    std::vector<Crossing> cr = curve_crossings(c, x0, y0, h);
    if (cr.size() < 2) {
      err = "a curve does not cross the grid";
      return CCM_EGEOM;
    }
    size_t m = cr.size();
    for (size_t a = 0; a < m; ++a) {
      Crossing A = cr[a], B = cr[(a + 1) % m];
      double ta = A.t, tb = B.t;
      if (a == m - 1) tb += TWO_PI;
      if (tb - ta < 1e-12) continue;           // zero-length piece through a grid vertex
      double xm, ym;
      c.xy(0.5 * (ta + tb), xm, ym);
      int i = (int)std::floor((xm - x0) / h), j = (int)std::floor((ym - y0) / h);
      if (i < 0 || i >= nx || j < 0 || j >= ny) {
        err = "a curve leaves the box";
        return CCM_EGEOM;
      }
      double xc = cg.cx(i), yc = cg.cy(j);
      auto endpoint = [&](double tt, const Crossing& C, double& X, double& Y, int& edge) -> bool {
        double px, py;
        c.xy(tt, px, py);
        X = std::min(std::max((px - xc) / h, -0.5), 0.5);
        Y = std::min(std::max((py - yc) / h, -0.5), 0.5);
        if (C.axis == 0) {
          if (C.k == i) { X = -0.5; edge = 3; return true; }
          if (C.k == i + 1) { X = 0.5; edge = 1; return true; }
        } else {
          if (C.k == j) { Y = -0.5; edge = 0; return true; }
          if (C.k == j + 1) { Y = 0.5; edge = 2; return true; }
        }
        return false;
      };
      double Xa, Ya, Xb, Yb;
      int ea, eb;
      if (!endpoint(ta, A, Xa, Ya, ea) || !endpoint(tb, B, Xb, Yb, eb)) {
        err = "inconsistent curve crossing";
        return CCM_EGEOM;
      }
      Arc arc;
      arc.curve = ci;
      if (c.orient > 0) {
        arc.ts = ta; arc.te = tb;
        arc.s_in = sigma_of(Xa, Ya, ea); arc.s_out = sigma_of(Xb, Yb, eb);
        arc.Xin = Xa; arc.Yin = Ya; arc.Xout = Xb; arc.Yout = Yb;
      } else {
        arc.ts = tb; arc.te = ta;
        arc.s_in = sigma_of(Xb, Yb, eb); arc.s_out = sigma_of(Xa, Ya, ea);
        arc.Xin = Xb; arc.Yin = Yb; arc.Xout = Xa; arc.Yout = Ya;
      }
      arcs[j * nx + i].push_back(arc);
    }
  }

  // ---- classification of the other cells by their centres (on the device when a classifier
  // is given, else rows over host threads; every cell's test is independent)
  cg.status.assign(N, ST_EMPTY);
  cg.iface.assign(N, 0);
  if (cc) {
    if (int rc = cc->classify(cg, cg.status)) {
      err = "device centre classification failed";
      return rc;
    }
  } else {
    std::atomic<int> next_row{0};
    auto work = [&]() {
      for (int j = next_row.fetch_add(1); j < ny; j = next_row.fetch_add(1))
        for (int i = 0; i < nx; ++i) {
          double x = cg.cx(i), y = cg.cy(j);
          bool in = true;
          for (const Curve& c : cg.curves) {
            bool ins = c.inside(x, y);
            if ((c.orient > 0) != ins) { in = false; break; }
          }
          cg.status[(long)j * nx + i] = in ? ST_PURE : ST_EMPTY;
        }
    };
    const int nt = (int)std::min<long>(std::max(1u, std::thread::hardware_concurrency()), std::max(1L, (long)ny / 64));
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back(work);
    work();
    for (auto& t : th) t.join();
  }
  for (auto& kv : arcs) {
    cg.status[kv.first] = ST_CUT;
    cg.iface[kv.first] = 1;
    cg.first_curve[kv.first] = kv.second[0].curve;
    cg.arc_param[kv.first] = 0.5 * (kv.second[0].ts + kv.second[0].te);
  }

  // ---- loops of every interface cell
  std::unordered_map<int, std::vector<Region>> members;
  for (auto& kv : arcs) {
    int lin = kv.first, j = lin / nx, i = lin % nx;
    double xc = cg.cx(i), yc = cg.cy(j);
    std::vector<Arc>& A = kv.second;
    std::vector<char> done(A.size(), 0);
    std::vector<Region> loops;
    for (size_t first = 0; first < A.size(); ++first) {
      if (done[first]) continue;
      Region reg;
      reg.hi = i;
      reg.hj = j;
      size_t cur = first;
      int guard = 0;
      while (true) {
        if (++guard > 4 * (int)A.size() + 4) {
          err = "cut-cell loop construction failed";
          return CCM_EGEOM;
        }
        done[cur] = 1;
        Piece pa;
        pa.arc = true;
        pa.curve = A[cur].curve;
        pa.t0 = A[cur].ts;
        pa.t1 = A[cur].te;
        reg.pieces.push_back(pa);
        size_t best = 0;
        double bd = 1e300;
        for (size_t k = 0; k < A.size(); ++k) {
          double d = std::fmod(A[k].s_in - A[cur].s_out + 8.0, 4.0);
          if (d < bd) { bd = d; best = k; }
        }
        // walk counter-clockwise from the exit to the next entry through the corners
        std::vector<std::pair<double, double>> pts;
        pts.push_back({A[cur].Xout, A[cur].Yout});
        double sa = A[cur].s_out, sb = sa + bd;
        for (long cidx = (long)std::floor(sa) + 1; cidx < sb; ++cidx) pts.push_back({CORNER_X[cidx % 4], CORNER_Y[cidx % 4]});
        pts.push_back({A[best].Xin, A[best].Yin});
        for (size_t q = 0; q + 1 < pts.size(); ++q) {
          double Xa = pts[q].first, Ya = pts[q].second, Xb = pts[q + 1].first, Yb = pts[q + 1].second;
          if (Xa == Xb && Ya == Yb) continue;
          Piece ps;
          ps.ax = xc + Xa * h;
          ps.ay = yc + Ya * h;
          ps.bx = xc + Xb * h;
          ps.by = yc + Yb * h;
          ps.wall = walls && ((Xa == -0.5 && Xb == -0.5 && i == 0) || (Xa == 0.5 && Xb == 0.5 && i == nx - 1) ||
                              (Ya == -0.5 && Yb == -0.5 && j == 0) || (Ya == 0.5 && Yb == 0.5 && j == ny - 1));
          reg.pieces.push_back(ps);
        }
        cur = best;
        if (cur == first) break;
        if (done[cur]) {
          err = "cut-cell loop construction failed";
          return CCM_EGEOM;
        }
      }
      reg.mom.fill(0.0);
      for (const Piece& pc : reg.pieces) piece_moments(pc, cg.curves, xc, yc, h, reg.mom);
      loops.push_back(reg);
    }
    members[lin] = loops;
  }

  cg.vol.assign(N, 0.0);
  for (long q = 0; q < N; ++q)
    if (cg.status[q] == ST_PURE) cg.vol[q] = 1.0;
  for (auto& kv : members) {
    double v = 0;
    for (auto& r : kv.second) v += r.mom[0];
    cg.vol[kv.first] = v;
  }
  cg.owner.assign(N, -1);
  for (long q = 0; q < N; ++q)
    if (cg.status[q] != ST_EMPTY) cg.owner[q] = (int32_t)q;

  auto pure_region = [&](int lin) {
    int j = lin / nx, i = lin % nx;
    double xc = cg.cx(i), yc = cg.cy(j), hh = 0.5 * h;
    double PX[4] = {xc - hh, xc + hh, xc + hh, xc - hh}, PY[4] = {yc - hh, yc - hh, yc + hh, yc + hh};
    Region r;
    r.hi = i;
    r.hj = j;
    for (int k = 0; k < 4; ++k) {
      Piece ps;
      ps.ax = PX[k];
      ps.ay = PY[k];
      ps.bx = PX[(k + 1) % 4];
      ps.by = PY[(k + 1) % 4];
      ps.wall = walls && ((k == 0 && j == 0) || (k == 1 && i == nx - 1) || (k == 2 && j == ny - 1) || (k == 3 && i == 0));
      r.pieces.push_back(ps);
    }
    r.mom = pure_moments();
    return r;
  };
  auto cell_members = [&](int lin) -> std::vector<Region>& {
    auto it = members.find(lin);
    if (it != members.end()) return it->second;
    members[lin] = {pure_region(lin)};
    return members[lin];
  };
  auto absorb = [&](int dst, const std::vector<Region>& src) {
    std::vector<Region>& L = cell_members(dst);
    for (const Region& r : src) L.push_back(r);
    cg.status[dst] = ST_CUT;
    double v = 0;
    for (const Region& r : L) v += r.mom[0];
    cg.vol[dst] = v;
  };
  // length (units of h) of a loop's straight pieces on edge d (0:+x, 1:-x, 2:+y, 3:-y)
  auto face_len = [&](const Region& r, int d) {
    double xc = cg.cx(r.hi), yc = cg.cy(r.hj), L = 0;
    for (const Piece& pc : r.pieces) {
      if (pc.arc) continue;
      double X0 = (pc.ax - xc) / h, Y0 = (pc.ay - yc) / h, X1 = (pc.bx - xc) / h, Y1 = (pc.by - yc) / h;
      if (d == 0 && std::fabs(X0 - 0.5) < 1e-12 && std::fabs(X1 - 0.5) < 1e-12) L += std::fabs(Y1 - Y0);
      else if (d == 1 && std::fabs(X0 + 0.5) < 1e-12 && std::fabs(X1 + 0.5) < 1e-12) L += std::fabs(Y1 - Y0);
      else if (d == 2 && std::fabs(Y0 - 0.5) < 1e-12 && std::fabs(Y1 - 0.5) < 1e-12) L += std::fabs(X1 - X0);
      else if (d == 3 && std::fabs(Y0 + 0.5) < 1e-12 && std::fabs(Y1 + 0.5) < 1e-12) L += std::fabs(X1 - X0);
    }
    return L;
  };
  static const int DI[4] = {1, -1, 0, 0}, DJ[4] = {0, 0, 1, -1};

  // ---- Alg. 1 preprocessing: multi-component cells keep their largest component
  std::vector<int> iface_cells;
  for (auto& kv : arcs) iface_cells.push_back(kv.first);   // ascending (std::map)
  for (int lin : iface_cells) {
    std::vector<Region> loops = members[lin];
    if (loops.size() < 2) continue;
    int j = lin / nx, i = lin % nx;
    std::vector<int> order(loops.size());
    for (size_t k = 0; k < loops.size(); ++k) order[k] = (int)k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return loops[a].mom[0] > loops[b].mom[0]; });
    for (size_t oi = 1; oi < order.size(); ++oi) {
      const Region& reg = loops[order[oi]];
      int best = -1, bd = -1;
      double bv = -1;
      for (int d = 0; d < 4; ++d) {
        if (face_len(reg, d) <= 0.0) continue;
        int ii = i + DI[d], jj = j + DJ[d];
        if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) continue;
        double v = cg.vol[(long)jj * nx + ii];
        if (v <= 0.0) continue;
        // larger volume wins; on equal volume the earlier direction (the larger -d) wins
        if (best < 0 || v > bv) { best = jj * nx + ii; bv = v; bd = d; }
      }
      (void)bd;
      if (best < 0) {
        err = "isolated cut-cell component";
        return CCM_EGEOM;
      }
      absorb(best, {reg});
    }
    members[lin] = {loops[order[0]]};
    cg.vol[lin] = loops[order[0]].mom[0];
  }

  // ---- Alg. 1 merging of small interface cells
  std::unordered_map<int, int> parent;
  std::vector<int> cand;
  for (int lin : iface_cells)
    if (cg.vol[lin] <= theta) cand.push_back(lin);
  std::stable_sort(cand.begin(), cand.end(), [&](int a, int b) {
    if (cg.vol[a] != cg.vol[b]) return cg.vol[a] < cg.vol[b];
    return a < b;
  });
  for (int lin : cand) {
    int j = lin / nx, i = lin % nx;
    if (cg.vol[lin] > theta || cg.vol[lin] <= 0.0 || parent.count(lin)) continue;
    const std::vector<Region>& own = members[lin];
    int best = -1;
    double bf = -1, bv = -1;
    for (int d = 0; d < 4; ++d) {
      int ii = i + DI[d], jj = j + DJ[d];
      if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) continue;
      double v = cg.vol[(long)jj * nx + ii];
      if (v <= 0.0) continue;
      double fl = 0;
      for (const Region& r : own)
        if (r.hi == i && r.hj == j) fl += face_len(r, d);
      if (best < 0 || fl > bf || (fl == bf && v > bv)) {
        best = jj * nx + ii;
        bf = fl;
        bv = v;
      }
    }
    if (best < 0 || bf <= 0.0) {
      err = "small cut cell without a face to merge through";
      return CCM_EGEOM;
    }
    std::vector<Region> moved = own;
    absorb(best, moved);
    members[lin].clear();
    cg.vol[lin] = 0.0;
    cg.status[lin] = ST_EMPTY;
    parent[lin] = best;
  }
  for (auto& kv : parent) {
    int s = kv.second;
    while (parent.count(s)) s = parent[s];
    cg.owner[kv.first] = s;
  }

  // ---- final moments of non-pure survivors
  for (auto& kv : members) {
    int lin = kv.first;
    if (kv.second.empty() || cg.status[lin] == ST_PURE) continue;
    int j = lin / nx, i = lin % nx;
    Mom m{};
    for (const Region& r : kv.second) {
      Mom s = shift_moments(r.mom, r.hi - i, r.hj - j);
      for (int k = 0; k < NMOM; ++k) m[k] += s[k];
    }
    cg.mom[lin] = m;
    cg.regions[lin] = kv.second;
  }

  // ---- boundary segments: cut survivors with arcs or wall pieces, and pure wall cells
  std::vector<int> bcells;
  for (auto& kv : cg.regions) bcells.push_back(kv.first);
  if (walls) {
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        if (i != 0 && j != 0 && i != nx - 1 && j != ny - 1) continue;
        long q = (long)j * nx + i;
        if (cg.status[q] == ST_PURE) bcells.push_back((int)q);
      }
  }
  std::sort(bcells.begin(), bcells.end());
  bcells.erase(std::unique(bcells.begin(), bcells.end()), bcells.end());
  for (int lin : bcells) {
    std::vector<Region> regs;
    if (cg.status[lin] == ST_PURE) regs = {pure_region(lin)};
    else regs = cg.regions[lin];
    std::vector<Piece> bp;
    for (const Region& r : regs)
      for (const Piece& pc : r.pieces)
        if (pc.arc || pc.wall) bp.push_back(pc);
    if (bp.empty()) continue;
    // one operator gamma1 u + gamma2 du/dn per cell: the same type and, for Robin, the same
    // coefficients on every piece
    int bc = -1;
    std::array<double, 2> gam{1.0, 0.0};
    for (const Piece& pc : bp) {
      const int b = pc.arc ? cg.curves[pc.curve].bc : prob.box_bc;
      std::array<double, 2> g{b == CCM_NEUMANN ? 0.0 : 1.0, b == CCM_NEUMANN ? 1.0 : 0.0};
      if (pc.arc) g = {cg.curves[pc.curve].robin[0], cg.curves[pc.curve].robin[1]};
      if (bc < 0) {
        bc = b;
        gam = g;
      } else if (bc != b || (b == CCM_ROBIN && gam != g)) {
        err = "a cell mixes boundary-condition types";
        return CCM_EGEOM;
      }
    }
    int j = lin / nx, i = lin % nx;
    Mom b0{}, bx{}, by{};
    for (const Piece& pc : bp) piece_bmoments(pc, cg.curves, cg.cx(i), cg.cy(j), h, b0, bx, by);
    cg.seg_of[lin] = (int)cg.segs.size();
    cg.segs.push_back(lin);
    cg.seg_bc.push_back(bc);
    cg.seg_gamma.push_back(gam);
    cg.bm0.push_back(b0);
    cg.bmx.push_back(bx);
    cg.bmy.push_back(by);
    cg.seg_pieces.push_back(bp);
  }
  return CCM_OK;
}

// ------------------------------------------------------------------ caller quadrature

void cell_quadrature(const CutLevel& cg, std::vector<int32_t>& cell, std::vector<double>& xy,
                     std::vector<double>& w) {
  // eq. iteratedIntegral: outer Gauss rule along every boundary piece with dy != 0,
  // inner Gauss rule in xi from xi0 (the survivor's centre) to x(t)
  static GL inner(8);
  const GL& g = gl_arc();
  cell.clear();
  xy.clear();
  w.clear();
  std::vector<int> keys;
  for (auto& kv : cg.regions) keys.push_back(kv.first);
  std::sort(keys.begin(), keys.end());
  for (int lin : keys) {
    if (cg.status[lin] != ST_CUT) continue;
    double xi0 = cg.cx(lin % cg.nx);
    for (const Region& r : cg.regions.at(lin)) {
      for (const Piece& pc : r.pieces) {
        auto add = [&](double x, double y, double wy) {
          double half = 0.5 * (x - xi0);
          for (size_t l = 0; l < inner.x.size(); ++l) {
            cell.push_back(lin);
            xy.push_back(xi0 + half * (inner.x[l] + 1.0));
            xy.push_back(y);
            w.push_back(inner.w[l] * half * wy);
          }
        };
        if (!pc.arc) {
          if (pc.ay == pc.by) continue;
          for (int n = 0; n < GL_ARC; ++n) {
            double s = 0.5 * (g.x[n] + 1.0);
            add(pc.ax + (pc.bx - pc.ax) * s, pc.ay + (pc.by - pc.ay) * s, (pc.by - pc.ay) * 0.5 * g.w[n]);
          }
          continue;
        }
        const Curve& c = cg.curves[pc.curve];
        std::vector<std::pair<double, double>> parts;
        c.subintervals(pc.t0, pc.t1, parts);
        for (const auto& ab : parts) {
          double tm = 0.5 * (ab.first + ab.second), tr = 0.5 * (ab.second - ab.first);
          for (int n = 0; n < GL_ARC; ++n) {
            double x, y, dx, dy;
            c.xy(tm + tr * g.x[n], x, y);
            c.dxy(tm + tr * g.x[n], dx, dy);
            add(x, y, dy * tr * g.w[n]);
          }
        }
      }
    }
  }
}

void boundary_quadrature(const CutLevel& cg, std::vector<int32_t>& seg, std::vector<double>& xy,
                         std::vector<double>& w, std::vector<double>& nrm) {
  const GL& g = gl_arc();
  seg.clear();
  xy.clear();
  w.clear();
  nrm.clear();
  for (size_t s = 0; s < cg.segs.size(); ++s) {
    for (const Piece& pc : cg.seg_pieces[s]) {
      auto add = [&](double x, double y, double ds, double nx, double ny) {
        seg.push_back((int32_t)s);
        xy.push_back(x);
        xy.push_back(y);
        w.push_back(ds);
        nrm.push_back(nx);
        nrm.push_back(ny);
      };
      if (!pc.arc) {
        for (int n = 0; n < GL_ARC; ++n) {
          double t = 0.5 * (g.x[n] + 1.0);
          double L = std::hypot(pc.bx - pc.ax, pc.by - pc.ay);
          add(pc.ax + (pc.bx - pc.ax) * t, pc.ay + (pc.by - pc.ay) * t, L * 0.5 * g.w[n], (pc.by - pc.ay) / L,
              -(pc.bx - pc.ax) / L);
        }
        continue;
      }
      const Curve& c = cg.curves[pc.curve];
      std::vector<std::pair<double, double>> parts;
      c.subintervals(pc.t0, pc.t1, parts);
      for (const auto& ab : parts) {
        double tm = 0.5 * (ab.first + ab.second), tr = 0.5 * (ab.second - ab.first);
        for (int n = 0; n < GL_ARC; ++n) {
          double x, y, dx, dy;
          c.xy(tm + tr * g.x[n], x, y);
          c.dxy(tm + tr * g.x[n], dx, dy);
          double sp = std::hypot(dx, dy), sg = tr > 0 ? 1.0 : -1.0;
          add(x, y, sp * std::fabs(tr) * g.w[n], sg * dy / sp, -sg * dx / sp);
        }
      }
    }
  }
}

void cell_averages(const CutLevel& cg, void (*f)(void*, int64_t, const double*, const double*, double*), void* ctx,
                   double* out) {
  const long N = (long)cg.nx * cg.ny;
  std::fill(out, out + N, 0.0);
  // pure cells: 5 x 5 tensor Gauss-Legendre rule on the square, exact for Q_9
  std::vector<double> gx, gw;
  gauss_legendre(5, gx, gw);
  const long batch_cells = 8192;
  std::vector<long> cells;
  std::vector<double> x, y, v;
  auto flush = [&]() {
    if (cells.empty()) return;
    v.resize(x.size());
    f(ctx, (int64_t)x.size(), x.data(), y.data(), v.data());
    for (size_t k = 0; k < cells.size(); ++k) {
      double acc = 0.0;
      for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b) acc += gw[a] * gw[b] * v[k * 25 + a * 5 + b];
      out[cells[k]] = 0.25 * acc;
    }
    cells.clear();
    x.clear();
    y.clear();
  };
  for (long q = 0; q < N; ++q) {
    if (cg.status[q] != ST_PURE) continue;
    const double xc = cg.cx((int)(q % cg.nx)), yc = cg.cy((int)(q / cg.nx));
    cells.push_back(q);
    for (int a = 0; a < 5; ++a)
      for (int b = 0; b < 5; ++b) {
        x.push_back(xc + 0.5 * cg.h * gx[a]);
        y.push_back(yc + 0.5 * cg.h * gx[b]);
      }
    if ((long)cells.size() == batch_cells) flush();
  }
  flush();
  // cut and merged cells: the cut-cell rule, divided by the cell's area
  std::vector<int32_t> cc;
  std::vector<double> xy, w;
  cell_quadrature(cg, cc, xy, w);
  if (cc.empty()) return;
  const size_t n = cc.size();
  x.resize(n);
  y.resize(n);
  v.resize(n);
  for (size_t k = 0; k < n; ++k) {
    x[k] = xy[2 * k];
    y[k] = xy[2 * k + 1];
  }
  f(ctx, (int64_t)n, x.data(), y.data(), v.data());
  std::vector<double> sum(N, 0.0);
  for (size_t k = 0; k < n; ++k) sum[cc[k]] += w[k] * v[k];
  for (long q = 0; q < N; ++q)
    if (cg.status[q] == ST_CUT) out[q] = sum[q] / (cg.vol[q] * cg.h * cg.h);
}

void boundary_averages(const CutLevel& cg,
                       void (*g)(void*, int64_t, const double*, const double*, double*, double*, double*),
                       void* ctx, double* out) {
  std::vector<int32_t> seg;
  std::vector<double> xy, w, nrm;
  boundary_quadrature(cg, seg, xy, w, nrm);
  const size_t ns = cg.segs.size(), n = seg.size();
  std::vector<double> x(n), y(n), u(n), ux(n), uy(n), num(ns, 0.0), den(ns, 0.0);
  for (size_t k = 0; k < n; ++k) {
    x[k] = xy[2 * k];
    y[k] = xy[2 * k + 1];
  }
  if (n) g(ctx, (int64_t)n, x.data(), y.data(), u.data(), ux.data(), uy.data());
  for (size_t k = 0; k < n; ++k) {
    const int s = seg[k];
    const double g1 = cg.seg_gamma[s][0], g2 = cg.seg_gamma[s][1];
    double val = 0.0;
    if (g1 != 0.0) val += g1 * u[k];
    if (g2 != 0.0) val += g2 * (ux[k] * nrm[2 * k] + uy[k] * nrm[2 * k + 1]);
    num[s] += val * w[k];
    den[s] += w[k];
  }
  for (size_t s = 0; s < ns; ++s) out[s] = den[s] > 0.0 ? num[s] / den[s] : 0.0;
}

}  // namespace ccm

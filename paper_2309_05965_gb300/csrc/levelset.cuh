// Analytic level-set functions H and grad H on the device (Sec. 5.1):
// Gamma = {H = 0}, Omega = {H < 0}.  Parameter layouts are those of
// kfbi_levelset_kind in kfbi.h.  The translation unit that uses these for
// geometric decisions is compiled with -fmad=false so that every product and
// sum is rounded separately.
#pragma once
#include "kfbi_internal.cuh"

namespace kfbi {

// Union of n equal discs (d = 2) or balls (d = 3): the first centre k with the
// smallest |X - c_k|^2 - r^2, and that value.
__device__ inline int ls_nearest_ball(const double* p, int d, const double* X, double* val) {
  const double r = p[0];
  const int n = static_cast<int>(p[1]);
  int best = 0;
  double bv = 0.0;
  for (int k = 0; k < n; ++k) {
    const double* c = p + 2 + d * k;
    const double dx = X[0] - c[0], dy = X[1] - c[1];
    double v = dx * dx + dy * dy;
    if (d == 3) {
      const double dz = X[2] - c[2];
      v = v + dz * dz;
    }
    v = v - r * r;
    if (k == 0 || v < bv) {
      bv = v;
      best = k;
    }
  }
  *val = bv;
  return best;
}

// Grid-sampled H: per axis the first of the four interpolation nodes and the
// local coordinate t in the cell [i0, i0 + 1] (i0 clamped to [1, N - 2]); a
// coordinate within 1e-10 h of a node is taken as that node.
__device__ inline void ls_cell(const LevelSet& L, double x, int* base, double* t) {
  double u = (x - L.glo) / L.gh;
  const double k = rint(u);
  if (fabs(u - k) <= 1e-10) u = k;
  const double i0 = fmin(fmax(floor(u), 1.0), (double)(L.gn - 2));
  *base = (int)i0 - 1;
  *t = u - i0;
}

// cubic Lagrange basis on t = -1, 0, 1, 2 and its derivative
__device__ inline void ls_lagrange(double t, double* w, double* dw) {
  const double tm1 = t - 1.0, tm2 = t - 2.0, tp1 = t + 1.0;
  w[0] = -(t * tm1 * tm2) / 6.0;
  w[1] = (tp1 * tm1 * tm2) / 2.0;
  w[2] = -(tp1 * t * tm2) / 2.0;
  w[3] = (tp1 * t * tm1) / 6.0;
  dw[0] = -(tm1 * tm2 + t * tm2 + t * tm1) / 6.0;
  dw[1] = (tm1 * tm2 + tp1 * tm2 + tp1 * tm1) / 2.0;
  dw[2] = -(t * tm2 + tp1 * tm2 + tp1 * t) / 2.0;
  dw[3] = (t * tm1 + tp1 * tm1 + tp1 * t) / 6.0;
}

// the interpolant's value (and gradient if g) at X, sums in a fixed order
__device__ inline double ls_sampled(const LevelSet& L, const double* X, double* g) {
  const int d = L.gd, n1 = L.gn + 1;
  int base[3] = {0, 0, 0};
  double w[3][4], dw[3][4];
  for (int k = 0; k < d; ++k) {
    double t;
    ls_cell(L, X[k], &base[k], &t);
    ls_lagrange(t, w[k], dw[k]);
  }
  const double* S = L.grid;
  double val = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
  if (d == 2) {
    for (int a = 0; a < 4; ++a) {
      double row = 0.0, drow = 0.0;
      const double* r = S + (long long)(base[0] + a) * n1 + base[1];
      for (int b = 0; b < 4; ++b) {
        row = row + w[1][b] * r[b];
        drow = drow + dw[1][b] * r[b];
      }
      val = val + w[0][a] * row;
      g0 = g0 + dw[0][a] * row;
      g1 = g1 + w[0][a] * drow;
    }
  } else {
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        double row = 0.0, drow = 0.0;
        const double* r = S + ((long long)(base[0] + a) * n1 + (base[1] + b)) * n1 + base[2];
        for (int c = 0; c < 4; ++c) {
          row = row + w[2][c] * r[c];
          drow = drow + dw[2][c] * r[c];
        }
        const double wab = w[0][a] * w[1][b];
        val = val + wab * row;
        g0 = g0 + (dw[0][a] * w[1][b]) * row;
        g1 = g1 + (w[0][a] * dw[1][b]) * row;
        g2 = g2 + wab * drow;
      }
  }
  if (g) {
    g[0] = g0 / L.gh;
    g[1] = g1 / L.gh;
    g[2] = d == 3 ? g2 / L.gh : 0.0;
  }
  return val;
}

// H of the analytic kinds (the components a union is made of, and the
// one-interface kinds)
__device__ inline double ls_H_kind(int kind, const double* p, const double* X) {
  switch (kind) {
    case KFBI_LS_ELLIPSE: {
      double x = X[0] - p[0], y = X[1] - p[1];
      double c = cos(p[4]), s = sin(p[4]);
      double u = (x * c + y * s) / p[2];
      double v = (y * c - x * s) / p[3];
      return u * u + v * v - 1.0;
    }
    case KFBI_LS_STAR: {
      double x = X[0] - p[0], y = X[1] - p[1];
      double r = sqrt(x * x + y * y);
      double th = atan2(y, x);
      return r - p[2] - p[3] * sin(p[4] * th);
    }
    case KFBI_LS_ELLIPSOID: {
      double u = (X[0] - p[0]) / p[3];
      double v = (X[1] - p[1]) / p[4];
      double w = (X[2] - p[2]) / p[5];
      return u * u + v * v + w * w - 1.0;
    }
    case KFBI_LS_TORUS: {
      double rho = sqrt(X[0] * X[0] + X[1] * X[1]);
      double t = rho - p[0];
      return t * t + X[2] * X[2] - p[1] * p[1];
    }
    case KFBI_LS_MOLECULE: {
      const double r = p[0], level = p[1];
      int na = static_cast<int>(p[2]);
      double acc = 0.0;
      for (int k = 0; k < na; ++k) {
        double dx = X[0] - p[3 + 3 * k], dy = X[1] - p[4 + 3 * k], dz = X[2] - p[5 + 3 * k];
        acc = acc + exp(-(dx * dx + dy * dy + dz * dz) / (r * r));
      }
      return level - acc;
    }
  }
  return 0.0;
}

__device__ inline void ls_grad_kind(int kind, const double* p, const double* X, double* g) {
  switch (kind) {
    case KFBI_LS_ELLIPSE: {
      double x = X[0] - p[0], y = X[1] - p[1];
      double c = cos(p[4]), s = sin(p[4]);
      double a = p[2], b = p[3];
      double u = (x * c + y * s) / a;
      double v = (y * c - x * s) / b;
      g[0] = 2.0 * u * (c / a) + 2.0 * v * (-s / b);
      g[1] = 2.0 * u * (s / a) + 2.0 * v * (c / b);
      g[2] = 0.0;
      return;
    }
    case KFBI_LS_STAR: {
      double x = X[0] - p[0], y = X[1] - p[1];
      double r2 = x * x + y * y;
      double r = sqrt(r2);
      double th = atan2(y, x);
      double dth = p[3] * p[4] * cos(p[4] * th);
      g[0] = x / r + dth * y / r2;
      g[1] = y / r - dth * x / r2;
      g[2] = 0.0;
      return;
    }
    case KFBI_LS_ELLIPSOID: {
      g[0] = 2.0 * (X[0] - p[0]) / (p[3] * p[3]);
      g[1] = 2.0 * (X[1] - p[1]) / (p[4] * p[4]);
      g[2] = 2.0 * (X[2] - p[2]) / (p[5] * p[5]);
      return;
    }
    case KFBI_LS_TORUS: {
      double rho = sqrt(X[0] * X[0] + X[1] * X[1]);
      double f = 2.0 * (rho - p[0]) / rho;
      g[0] = f * X[0];
      g[1] = f * X[1];
      g[2] = 2.0 * X[2];
      return;
    }
    case KFBI_LS_MOLECULE: {
      double r = p[0];
      int na = static_cast<int>(p[2]);
      g[0] = g[1] = g[2] = 0.0;
      for (int k = 0; k < na; ++k) {
        double dx = X[0] - p[3 + 3 * k], dy = X[1] - p[4 + 3 * k], dz = X[2] - p[5 + 3 * k];
        double e = exp(-(dx * dx + dy * dy + dz * dz) / (r * r));
        double c = (2.0 / (r * r)) * e;
        g[0] = g[0] + c * dx;
        g[1] = g[1] + c * dy;
        g[2] = g[2] + c * dz;
      }
      return;
    }
  }
  g[0] = g[1] = g[2] = 0.0;
}

// ---- several interfaces (the remark on arbitrarily close interfaces,
// Sec. 5.2): interface k has its own function H_k; Omega^(k) = {H_k < 0}.
__device__ inline int ls_union_count(int kind) {
  switch (kind) {
    case KFBI_LS_ELLIPSE:
    case KFBI_LS_STAR:
      return 5;
    case KFBI_LS_ELLIPSOID:
      return 6;
    case KFBI_LS_TORUS:
      return 2;
  }
  return 0;
}

// component k of a union: its kind and parameters
__device__ inline const double* ls_union_comp(const double* p, int k, int* kind) {
  int at = 1;
  for (int j = 0; j < k; ++j) at += 1 + ls_union_count(static_cast<int>(p[at]));
  *kind = static_cast<int>(p[at]);
  return p + at + 1;
}

// the first component with the smallest H_k, and that value
__device__ inline int ls_union_argmin(const double* p, const double* X, double* val) {
  const int m = static_cast<int>(p[0]);
  int best = 0, at = 1;
  double bv = 0.0;
  for (int k = 0; k < m; ++k) {
    const int kind = static_cast<int>(p[at]);
    const double v = ls_H_kind(kind, p + at + 1, X);
    if (k == 0 || v < bv) {
      bv = v;
      best = k;
    }
    at += 1 + ls_union_count(kind);
  }
  *val = bv;
  return best;
}

__device__ inline int ls_n_iface(const LevelSet& L) {
  if (L.kind == KFBI_LS_DISCS || L.kind == KFBI_LS_SPHERES) return static_cast<int>(L.p[1]);
  if (L.kind == KFBI_LS_UNION) return static_cast<int>(L.p[0]);
  return 1;
}

__device__ inline double ls_H(const LevelSet& L, const double* X) {
  switch (L.kind) {
    case KFBI_LS_GRID:
      return ls_sampled(L, X, nullptr);
    case KFBI_LS_DISCS:
    case KFBI_LS_SPHERES: {
      double v;
      ls_nearest_ball(L.p, L.kind == KFBI_LS_DISCS ? 2 : 3, X, &v);
      return v;
    }
    case KFBI_LS_UNION: {
      double v;
      ls_union_argmin(L.p, X, &v);
      return v;
    }
  }
  return ls_H_kind(L.kind, L.p, X);
}

__device__ inline void ls_grad(const LevelSet& L, const double* X, double* g) {
  const double* p = L.p;
  switch (L.kind) {
    case KFBI_LS_GRID:
      ls_sampled(L, X, g);
      return;
    case KFBI_LS_DISCS:
    case KFBI_LS_SPHERES: {
      const int d = L.kind == KFBI_LS_DISCS ? 2 : 3;
      double v;
      const double* c = p + 2 + d * ls_nearest_ball(p, d, X, &v);
      g[0] = 2.0 * (X[0] - c[0]);
      g[1] = 2.0 * (X[1] - c[1]);
      g[2] = d == 3 ? 2.0 * (X[2] - c[2]) : 0.0;
      return;
    }
    case KFBI_LS_UNION: {
      double v;
      int kind;
      const double* q = ls_union_comp(p, ls_union_argmin(p, X, &v), &kind);
      ls_grad_kind(kind, q, X, g);
      return;
    }
  }
  ls_grad_kind(L.kind, p, X, g);
}

// side label of a point: 0 outside Omega, 1 + k in Omega^(k) (for a point
// in two overlapping components, the first with the smallest H_k)
__device__ inline int ls_label(const LevelSet& L, const double* X) {
  double v;
  int k = 0;
  if (L.kind == KFBI_LS_DISCS || L.kind == KFBI_LS_SPHERES)
    k = ls_nearest_ball(L.p, L.kind == KFBI_LS_DISCS ? 2 : 3, X, &v);
  else if (L.kind == KFBI_LS_UNION)
    k = ls_union_argmin(L.p, X, &v);
  else
    v = ls_H(L, X);
  return v < 0.0 ? k + 1 : 0;
}

// H_k of interface k alone (the arithmetic of ls_nearest_ball for a ball)
__device__ inline double ls_H_iface(const LevelSet& L, int k, const double* X) {
  if (L.kind == KFBI_LS_DISCS || L.kind == KFBI_LS_SPHERES) {
    const int d = L.kind == KFBI_LS_DISCS ? 2 : 3;
    const double r = L.p[0];
    const double* c = L.p + 2 + d * k;
    const double dx = X[0] - c[0], dy = X[1] - c[1];
    double v = dx * dx + dy * dy;
    if (d == 3) {
      const double dz = X[2] - c[2];
      v = v + dz * dz;
    }
    return v - r * r;
  }
  if (L.kind == KFBI_LS_UNION) {
    int kind;
    const double* q = ls_union_comp(L.p, k, &kind);
    return ls_H_kind(kind, q, X);
  }
  return ls_H(L, X);
}

__device__ inline void ls_grad_iface(const LevelSet& L, int k, const double* X, double* g) {
  if (L.kind == KFBI_LS_DISCS || L.kind == KFBI_LS_SPHERES) {
    const int d = L.kind == KFBI_LS_DISCS ? 2 : 3;
    const double* c = L.p + 2 + d * k;
    g[0] = 2.0 * (X[0] - c[0]);
    g[1] = 2.0 * (X[1] - c[1]);
    g[2] = d == 3 ? 2.0 * (X[2] - c[2]) : 0.0;
    return;
  }
  if (L.kind == KFBI_LS_UNION) {
    int kind;
    const double* q = ls_union_comp(L.p, k, &kind);
    ls_grad_kind(kind, q, X, g);
    return;
  }
  ls_grad(L, X, g);
}

}  // namespace kfbi

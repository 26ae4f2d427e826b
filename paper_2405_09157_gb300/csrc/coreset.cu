// Core-set certificates for the certified SVM search (a reading beyond the
// paper, built on Eq. (PD) and the core-set view of PD it cites in Sec. 4.2).
//
// Restricting Eq. (PD) to subsets of the two classes can only raise its
// minimum, so the exact polytope distance of a core set is an upper bound on
// OPT; the direction of that solution, evaluated on every point (the margin f
// of Sec. 5), is a lower bound. The core set is read off the MWU: in each
// class the K points nearest the hyperplane of the FTP's best direction w
// (smallest y_i x_i^T w). This file holds
//   * the exact solver of the small problem (host, FP64): a primal
//     active-set method (exact affine least-distance solves on the support,
//     the most violating point added, points leaving the support on the way
//     to the affine optimum dropped), pd_active_set;
//   * the device kernels that project every point on a direction, pick the
//     core set by a threshold per class, and gather its rows;
//   * svm_coreset_check, which the certified search of svm_solve calls.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "coreset.cuh"
#include "dispatch.cuh"

namespace pdscp {

// ---------------------------------------------------------------------------
// Host solver: polytope distance min ||P^T mu - Q^T gamma|| over the two
// simplices (Eq. PD), P: nP x d, Q: nQ x d row-major (FP64).
// ---------------------------------------------------------------------------
namespace {

struct ActiveSet {
  const double* P;
  const double* Q;
  int nP, nQ, d;
  // candidate k: a_k = P[k] (class 0) for k < nP, a_k = -Q[k - nP] (class 1) otherwise
  double dot_a(int k, const double* v) const {
    const double* x = k < nP ? P + (size_t)k * d : Q + (size_t)(k - nP) * d;
    double s = 0.0;
    for (int j = 0; j < d; ++j) s += x[j] * v[j];
    return k < nP ? s : -s;
  }
  double dot_aa(int k, int l) const {
    const double* x = k < nP ? P + (size_t)k * d : Q + (size_t)(k - nP) * d;
    const double* u = l < nP ? P + (size_t)l * d : Q + (size_t)(l - nP) * d;
    double s = 0.0;
    for (int j = 0; j < d; ++j) s += x[j] * u[j];
    return ((k < nP) == (l < nP)) ? s : -s;
  }
  void axpy_a(int k, double c, double* z) const {
    const double* x = k < nP ? P + (size_t)k * d : Q + (size_t)(k - nP) * d;
    const double cc = k < nP ? c : -c;
    for (int j = 0; j < d; ++j) z[j] += cc * x[j];
  }
};

// A symmetric matrix of variable order k kept in a buffer of a larger
// stride (capacity), so that a row/column is appended in O(k) and removed in
// O(k^2) without reallocating.
struct SymBuf {
  std::vector<double> a;
  int k = 0, cap = 0;
  void reserve(int c) {
    if (c <= cap) return;
    int nc = cap > 0 ? cap : 16;
    while (nc < c) nc *= 2;
    std::vector<double> b((size_t)nc * nc, 0.0);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) b[(size_t)i * nc + j] = a[(size_t)i * cap + j];
    a.swap(b);
    cap = nc;
  }
  double& at(int i, int j) { return a[(size_t)i * cap + j]; }
  double at(int i, int j) const { return a[(size_t)i * cap + j]; }
  void drop(int p) {  // removes row and column p
    for (int i = 0; i < k; ++i) {
      if (i == p) continue;
      double* row = a.data() + (size_t)i * cap;
      for (int j = p; j + 1 < k; ++j) row[j] = row[j + 1];
    }
    for (int i = p; i + 1 < k; ++i)
      std::copy(a.begin() + (size_t)(i + 1) * cap, a.begin() + (size_t)(i + 1) * cap + k - 1, a.begin() + (size_t)i * cap);
    --k;
  }
};

// Inverse of the KKT matrix of the affine least-distance problem on the
// support, K = [[0, E^T], [E, G]] (rows 0, 1: the two classes' sums; then
// the support's Gram matrix G and class indicators E), kept up to date by
// bordering (a point added) and by the inverse's partition formula (a point
// removed), O(k^2) each; rebuilt by Gauss-Jordan elimination when a pivot or
// the check of a solve's residual says the updates have lost accuracy.
struct KktInverse {
  SymBuf inv;
  std::vector<double> u, M;
  bool rebuild(const SymBuf& G, const std::vector<int>& cls) {
    const int k = G.k, n = k + 2;
    inv.reserve(n);
    inv.k = n;
    M.assign((size_t)n * n, 0.0);
    for (int i = 0; i < k; ++i) {
      M[(size_t)cls[i] * n + 2 + i] = M[(size_t)(2 + i) * n + cls[i]] = 1.0;
      for (int j = 0; j < k; ++j) M[(size_t)(2 + i) * n + 2 + j] = G.at(i, j);
    }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) inv.at(i, j) = i == j ? 1.0 : 0.0;
    for (int c = 0; c < n; ++c) {
      int piv = c;
      double best = std::fabs(M[(size_t)c * n + c]);
      for (int i = c + 1; i < n; ++i) {
        const double v = std::fabs(M[(size_t)i * n + c]);
        if (v > best) best = v, piv = i;
      }
      if (!(best > 1e-300)) return false;
      if (piv != c)
        for (int j = 0; j < n; ++j) {
          std::swap(M[(size_t)c * n + j], M[(size_t)piv * n + j]);
          std::swap(inv.at(c, j), inv.at(piv, j));
        }
      const double dv = 1.0 / M[(size_t)c * n + c];
      for (int j = 0; j < n; ++j) {
        M[(size_t)c * n + j] *= dv;
        inv.at(c, j) *= dv;
      }
      for (int i = 0; i < n; ++i) {
        if (i == c) continue;
        const double f = M[(size_t)i * n + c];
        if (f == 0.0) continue;
        for (int j = 0; j < n; ++j) {
          M[(size_t)i * n + j] -= f * M[(size_t)c * n + j];
          inv.at(i, j) -= f * inv.at(c, j);
        }
      }
    }
    return true;
  }
  // bordering: a new last row/column b (length n) with diagonal dd
  bool append(const std::vector<double>& b, double dd) {
    const int n = inv.k;
    u.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int j = 0; j < n; ++j) s += inv.at(i, j) * b[j];
      u[i] = s;
    }
    double bu = 0.0;
    for (int i = 0; i < n; ++i) bu += b[i] * u[i];
    const double sc = dd - bu;
    if (!(std::fabs(sc) > 1e-12 * (std::fabs(dd) + std::fabs(bu)))) return false;
    inv.reserve(n + 1);
    const double is = 1.0 / sc;
    for (int i = 0; i < n; ++i) {
      const double ui = u[i] * is;
      for (int j = 0; j < n; ++j) inv.at(i, j) += ui * u[j];
      inv.at(i, n) = -ui;
      inv.at(n, i) = -ui;
    }
    inv.at(n, n) = is;
    inv.k = n + 1;
    return true;
  }
  // removal of row/column p
  bool remove(int p) {
    const int n = inv.k;
    const double pp = inv.at(p, p);
    if (!(std::fabs(pp) > 1e-300)) return false;
    const double ip = 1.0 / pp;
    for (int i = 0; i < n; ++i) {
      if (i == p) continue;
      const double f = inv.at(i, p) * ip;
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j)
        if (j != p) inv.at(i, j) -= f * inv.at(p, j);
    }
    inv.drop(p);
    return true;
  }
};

// out[k] = X[k] . v for the rows of a matrix given transposed (XT: d x rows),
// as one scaled-row sum per feature (vectorisable; each dot product summed
// over the features in order)
void transposed_dots(const double* __restrict__ XT, int rows, int d, const double* __restrict__ v,
                     double* __restrict__ out) {
  std::fill(out, out + rows, 0.0);
  for (int j = 0; j < d; ++j) {
    const double vj = v[j];
    const double* x = XT + (size_t)j * rows;
    for (int k = 0; k < rows; ++k) out[k] += x[k] * vj;
  }
}

// the same in FP32
void transposed_dots_f(const float* __restrict__ XT, int rows, int d, const float* __restrict__ v,
                       float* __restrict__ out) {
  std::fill(out, out + rows, 0.0f);
  for (int j = 0; j < d; ++j) {
    const float vj = v[j];
    const float* x = XT + (size_t)j * rows;
    for (int k = 0; k < rows; ++k) out[k] += x[k] * vj;
  }
}

}  // namespace

int pd_active_set(const double* P, int nP, const double* Q, int nQ, int d, double tol, int max_iter, double* mu,
                  double* ga, double* z, double* gap_out, const double* mu0, const double* ga0) {
  ActiveSet A{P, Q, nP, nQ, d};
  const int m = nP + nQ;
  std::vector<double> zc(d, 0.0), cen(d, 0.0);
  for (int i = 0; i < nP; ++i)
    for (int j = 0; j < d; ++j) cen[j] += P[(size_t)i * d + j] / nP;
  for (int i = 0; i < nQ; ++i)
    for (int j = 0; j < d; ++j) cen[j] -= Q[(size_t)i * d + j] / nQ;
  // the candidates transposed (features x candidates, Q negated) for the scans
  std::vector<double> AT((size_t)d * m);
  for (int k = 0; k < nP; ++k)
    for (int j = 0; j < d; ++j) AT[(size_t)j * m + k] = P[(size_t)k * d + j];
  for (int k = 0; k < nQ; ++k)
    for (int j = 0; j < d; ++j) AT[(size_t)j * m + nP + k] = -Q[(size_t)k * d + j];
  // start: the pair nearest along the difference of the centroids
  int s0 = 0, s1 = nP;
  double b0 = INFINITY, b1 = INFINITY;
  for (int k = 0; k < m; ++k) {
    const double v = A.dot_a(k, cen.data());
    if (k < nP && v < b0) b0 = v, s0 = k;
    if (k >= nP && v < b1) b1 = v, s1 = k;
  }
  std::vector<int> S = {s0, s1};       // support (candidate indices)
  std::vector<int> cls = {0, 1};       // their classes
  std::vector<double> c = {1.0, 1.0};  // weights on the support
  if (mu0 && ga0) {
    // warm start: the positive weights given (renormalised per class), if
    // each class has some
    std::vector<int> S2, cls2;
    std::vector<double> c2;
    double w[2] = {0.0, 0.0};
    for (int k = 0; k < m; ++k) {
      const double v = k < nP ? mu0[k] : ga0[k - nP];
      if (v > 0.0) {
        S2.push_back(k);
        cls2.push_back(k < nP ? 0 : 1);
        c2.push_back(v);
        w[k < nP ? 0 : 1] += v;
      }
    }
    if (w[0] > 0.0 && w[1] > 0.0) {
      for (size_t i = 0; i < S2.size(); ++i) c2[i] /= w[cls2[i]];
      S.swap(S2);
      cls.swap(cls2);
      c.swap(c2);
    }
  }
  SymBuf G;  // the support's Gram matrix
  G.reserve(std::max<int>(2 * d + 8, (int)S.size() + 8));
  G.k = (int)S.size();
  for (int i = 0; i < G.k; ++i)
    for (int j = 0; j < G.k; ++j) G.at(i, j) = A.dot_aa(S[i], S[j]);
  std::vector<char> in(m, 0);
  for (int k : S) in[k] = 1;
  KktInverse K;
  K.inv.reserve(G.cap + 2);
  bool have_inv = K.rebuild(G, cls);
  auto rebuild_z = [&]() {
    std::fill(zc.begin(), zc.end(), 0.0);
    for (size_t i = 0; i < S.size(); ++i) A.axpy_a(S[i], c[i], zc.data());
  };
  auto remove_at = [&](size_t pos) {
    G.drop((int)pos);
    in[S[pos]] = 0;
    S.erase(S.begin() + pos);
    cls.erase(cls.begin() + pos);
    c.erase(c.begin() + pos);
    if (have_inv) have_inv = K.remove(2 + (int)pos);
  };
  // the affine optimum on the support: x = K^-1 (1, 1, 0, ..., 0), checked
  // by its residual against G (rebuilt once if the updates drifted)
  std::vector<double> x;
  auto solve = [&]() -> bool {
    const int ks = (int)S.size(), n = ks + 2;
    for (int attempt = 0; attempt < 2; ++attempt) {
      if (!have_inv) have_inv = K.rebuild(G, cls);
      if (!have_inv) return false;
      x.assign(n, 0.0);
      for (int i = 0; i < n; ++i) x[i] = K.inv.at(i, 0) + K.inv.at(i, 1);
      double scale = 1.0, s0c = 0.0, s1c = 0.0;
      for (int i = 0; i < ks; ++i) (cls[i] ? s1c : s0c) += x[2 + i];
      double res = std::max(std::fabs(s0c - 1.0), std::fabs(s1c - 1.0));
      for (int i = 0; i < ks; ++i) {
        double gi = x[cls[i]], mag = std::fabs(gi);
        for (int j = 0; j < ks; ++j) {
          const double t = G.at(i, j) * x[2 + j];
          gi += t;
          mag += std::fabs(t);
        }
        res = std::max(res, std::fabs(gi));
        scale = std::max(scale, mag);
      }
      if (res <= 1e-10 * scale) return true;
      have_inv = false;  // drifted: rebuild and solve again
    }
    return false;
  };
  std::vector<double> av(m), bcol;
  // while far from the stopping gap the scans run in FP32 (on the transposed
  // candidates rounded once): they only pick the point to add; the stopping
  // test always rests on an FP64 scan (from the first FP32 estimate within
  // 4 tol of the gap on, every scan is FP64)
  const bool fast = tol >= 1e-7;
  bool exact = !fast;
  std::vector<float> ATf, zf(d), avf;
  if (fast) {
    ATf.resize(AT.size());
    for (size_t i = 0; i < AT.size(); ++i) ATf[i] = (float)AT[i];
    avf.resize(m);
  }
  rebuild_z();
  double gap = INFINITY;
  int it = 0;
  for (; it < max_iter; ++it) {
    double zz = 0.0;
    for (int j = 0; j < d; ++j) zz += zc[j] * zc[j];
    double lam[2], mn[2];
    int arg[2];
    for (int pass = 0; pass < 2; ++pass) {
      if (exact) {
        transposed_dots(AT.data(), m, d, zc.data(), av.data());  // a_k . z for every candidate
      } else {
        for (int j = 0; j < d; ++j) zf[j] = (float)zc[j];
        transposed_dots_f(ATf.data(), m, d, zf.data(), avf.data());
        for (int k = 0; k < m; ++k) av[k] = avf[k];
      }
      lam[0] = lam[1] = 0.0;
      for (size_t i = 0; i < S.size(); ++i) lam[cls[i]] += c[i] * av[S[i]];
      mn[0] = mn[1] = INFINITY;
      arg[0] = arg[1] = -1;
      for (int k = 0; k < m; ++k) {
        const double v = av[k];
        const int cl = k < nP ? 0 : 1;
        if (v < mn[cl]) mn[cl] = v, arg[cl] = k;
      }
      gap = zz - (mn[0] + mn[1]);
      if (exact || gap > 4.0 * tol * zz) break;
      exact = true;  // near the stopping gap: FP64 scans from here on
    }
    if (exact && gap <= tol * zz) break;
    const int cl = (lam[0] - mn[0] >= lam[1] - mn[1]) ? 0 : 1;
    const int add = arg[cl];
    if (add < 0 || in[add]) break;
    const int k = (int)S.size();
    bcol.assign(k + 2, 0.0);
    bcol[cl] = 1.0;
    G.reserve(k + 1);
    for (int i = 0; i < k; ++i) {
      const double g = A.dot_aa(S[i], add);
      G.at(i, k) = G.at(k, i) = g;
      bcol[2 + i] = g;
    }
    const double gaa = A.dot_aa(add, add);
    G.at(k, k) = gaa;
    G.k = k + 1;
    S.push_back(add);
    cls.push_back(cl);
    c.push_back(0.0);
    in[add] = 1;
    if (have_inv) have_inv = K.append(bcol, gaa);
    bool stalled = false;
    for (int minor = 0; minor < 4 * m + 8; ++minor) {
      const int ks = (int)S.size();
      if (!solve()) {
        stalled = true;
        break;
      }
      bool all_pos = true;
      for (int i = 0; i < ks; ++i)
        if (!(x[2 + i] > 0.0)) all_pos = false;
      if (all_pos) {
        for (int i = 0; i < ks; ++i) c[i] = x[2 + i];
        break;
      }
      double theta = 1.0;
      int hit = -1;
      for (int i = 0; i < ks; ++i)
        if (x[2 + i] <= 0.0 && c[i] - x[2 + i] > 0.0) {
          const double th = c[i] / (c[i] - x[2 + i]);
          if (th < theta) theta = th, hit = i;
        }
      for (int i = 0; i < ks; ++i) c[i] += theta * (x[2 + i] - c[i]);
      if (hit >= 0) c[hit] = 0.0;
      bool removed = false;
      for (int i = ks - 1; i >= 0; --i) {
        int others = 0;
        for (int j = 0; j < (int)S.size(); ++j)
          if (j != i && cls[j] == cls[i]) ++others;
        if (c[i] <= 0.0 && others > 0) {
          remove_at((size_t)i);
          removed = true;
        }
      }
      if (!removed) {
        stalled = true;
        break;
      }
    }
    rebuild_z();
    if (stalled || !in[add]) break;
  }
  double s0w = 0.0, s1w = 0.0;
  for (size_t i = 0; i < S.size(); ++i) {
    if (c[i] < 0.0) c[i] = 0.0;
    (S[i] < nP ? s0w : s1w) += c[i];
  }
  std::fill(mu, mu + nP, 0.0);
  std::fill(ga, ga + nQ, 0.0);
  for (size_t i = 0; i < S.size(); ++i) {
    if (S[i] < nP) mu[S[i]] = s0w > 0.0 ? c[i] / s0w : 0.0;
    else ga[S[i] - nP] = s1w > 0.0 ? c[i] / s1w : 0.0;
  }
  std::fill(z, z + d, 0.0);
  for (int i = 0; i < nP; ++i)
    if (mu[i] > 0.0)
      for (int j = 0; j < d; ++j) z[j] += mu[i] * P[(size_t)i * d + j];
  for (int i = 0; i < nQ; ++i)
    if (ga[i] > 0.0)
      for (int j = 0; j < d; ++j) z[j] -= ga[i] * Q[(size_t)i * d + j];
  if (gap_out) *gap_out = gap;
  return it;
}

// Minimum enclosing ball of the rows of P (m x d, FP64, translated near the
// origin by the caller) through its dual: weights mu on the simplex
// maximising phi(mu) = sum_i mu_i |p_i|^2 - |c_mu|^2, c_mu = sum_i mu_i p_i
// (phi(mu) <= OPT^2 for any mu: weak duality), by Frank-Wolfe steps toward
// the farthest row and away steps from the nearest row of the support, each
// with its exact line search (phi is a concave quadratic along both), until
// the farthest row lies within (1 + tol) sqrt(phi) of c_mu. Returns
// sqrt(phi); c (d): c_mu; *far: the farthest row's distance from it.
double meb_dual_fw(const double* P, int m, int d, double tol, int max_iter, std::vector<double>& mu,
                   std::vector<double>& c, double* far) {
  std::vector<double> PT((size_t)d * m), sq(m, 0.0), pc(m), d2(m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < d; ++j) {
      const double v = P[(size_t)i * d + j];
      PT[(size_t)j * m + i] = v;
      sq[i] += v * v;
    }
  mu.assign(m, 0.0);
  c.assign(d, 0.0);
  // start: the row farthest from the rows' mean, with all the weight
  std::vector<double> mean(d, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < d; ++j) mean[j] += P[(size_t)i * d + j] / m;
  int j0 = 0;
  double best = -1.0;
  for (int i = 0; i < m; ++i) {
    double t = 0.0;
    for (int j = 0; j < d; ++j) t += (P[(size_t)i * d + j] - mean[j]) * (P[(size_t)i * d + j] - mean[j]);
    if (t > best) best = t, j0 = i;
  }
  mu[j0] = 1.0;
  for (int j = 0; j < d; ++j) c[j] = P[(size_t)j0 * d + j];
  double phi = 0.0;
  for (int it = 0; it < max_iter; ++it) {
    double cc = 0.0, msq = 0.0;
    for (int j = 0; j < d; ++j) cc += c[j] * c[j];
    std::fill(pc.begin(), pc.end(), 0.0);
    for (int j = 0; j < d; ++j) {
      const double cj = c[j];
      const double* x = PT.data() + (size_t)j * m;
      for (int i = 0; i < m; ++i) pc[i] += x[i] * cj;
    }
    int jf = 0, ja = -1;
    for (int i = 0; i < m; ++i) {
      d2[i] = std::max(sq[i] - 2.0 * pc[i] + cc, 0.0);
      msq += mu[i] * sq[i];
      if (d2[i] > d2[jf]) jf = i;
      if (mu[i] > 0.0 && (ja < 0 || d2[i] < d2[ja])) ja = i;
    }
    phi = std::max(msq - cc, 0.0);
    if (d2[jf] <= (1.0 + tol) * (1.0 + tol) * phi) break;
    const double gfw = d2[jf] - phi, gaw = phi - d2[ja];
    if (gfw >= gaw || mu[ja] >= 1.0) {
      const double st = std::min(1.0, gfw / (2.0 * d2[jf]));
      for (int i = 0; i < m; ++i) mu[i] *= 1.0 - st;
      mu[jf] += st;
      for (int j = 0; j < d; ++j) c[j] = (1.0 - st) * c[j] + st * P[(size_t)jf * d + j];
    } else {
      const double smax = mu[ja] / (1.0 - mu[ja]);
      const double st = d2[ja] > 0.0 ? std::min(smax, gaw / (2.0 * d2[ja])) : smax;
      for (int i = 0; i < m; ++i) mu[i] *= 1.0 + st;
      mu[ja] -= st;
      if (st >= smax) mu[ja] = 0.0;
      for (int j = 0; j < d; ++j) c[j] = (1.0 + st) * c[j] - st * P[(size_t)ja * d + j];
    }
  }
  // the final weights renormalised onto the simplex, then c_mu, phi and the
  // farthest distance recomputed from them directly
  double wsum = 0.0;
  for (int i = 0; i < m; ++i) wsum += mu[i];
  for (int i = 0; i < m; ++i) mu[i] /= wsum;
  std::fill(c.begin(), c.end(), 0.0);
  for (int i = 0; i < m; ++i)
    if (mu[i] > 0.0)
      for (int j = 0; j < d; ++j) c[j] += mu[i] * P[(size_t)i * d + j];
  double msq = 0.0, cc = 0.0, fmax = 0.0;
  for (int j = 0; j < d; ++j) cc += c[j] * c[j];
  for (int i = 0; i < m; ++i) {
    msq += mu[i] * sq[i];
    double t = 0.0;
    for (int j = 0; j < d; ++j) t += (P[(size_t)i * d + j] - c[j]) * (P[(size_t)i * d + j] - c[j]);
    fmax = std::max(fmax, t);
  }
  if (far) *far = std::sqrt(fmax);
  return std::sqrt(std::max(msq - cc, 0.0));
}

}  // namespace pdscp

// ---------------------------------------------------------------------------
// Device side: projections, the per-class threshold pick, row gathering.
// ---------------------------------------------------------------------------
namespace pdscp {

namespace {

// order-preserving images of floats as unsigned ints (atomic min / max)
__device__ __forceinline__ unsigned int f2o(float v) {
  const unsigned int b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__host__ __device__ inline float o2f(unsigned int b) {
  b = (b & 0x80000000u) ? (b & 0x7fffffffu) : ~b;
  float f;
  memcpy(&f, &b, sizeof(f));
  return f;
}

// s_i = y_i x_i . w for every row, one warp per row (rows strided over the
// grid); mm[0..3] = images of min_P s, max_P s, min_Q s, max_Q s.
template <typename T>
__global__ void __launch_bounds__(256) svm_project_kernel(const T* X, const int8_t* y, int64_t n, int d,
                                                          const float* w, float* s, unsigned int* mm) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float lo[2] = {INFINITY, INFINITY}, hi[2] = {-INFINITY, -INFINITY};
  for (int64_t i = wid; i < n; i += nw) {
    const T* row = X + i * d;
    float acc = 0.f;
    for (int j = lane; j < d; j += 32) acc = fmaf(elem_to_float<T>(row + j), __ldg(w + j), acc);
    acc = warp_sum(acc);
    const bool pos = __ldg(y + i) > 0;
    const float v = pos ? acc : -acc;
    if (lane == 0) s[i] = v;
    const int c = pos ? 0 : 1;
    lo[c] = fminf(lo[c], v);
    hi[c] = fmaxf(hi[c], v);
  }
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (lo[c] <= hi[c]) {
        atomicMin(mm + 2 * c, f2o(lo[c]));
        atomicMax(mm + 2 * c + 1, f2o(hi[c]));
      }
    }
  }
}

// s_i = -|x_i - c|^2 for every row (SES core sets: the smallest s are the
// farthest points), one warp per row; mm[0], mm[1] = images of min s, max s
template <typename T>
__global__ void __launch_bounds__(256) ses_dist_kernel(const T* X, int64_t n, int d, const float* c, float* s,
                                                       unsigned int* mm) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float lo = INFINITY, hi = -INFINITY;
  for (int64_t i = wid; i < n; i += nw) {
    const T* row = X + i * d;
    float acc = 0.f;
    for (int j = lane; j < d; j += 32) {
      const float t = elem_to_float<T>(row + j) - __ldg(c + j);
      acc = fmaf(t, t, acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) s[i] = -acc;
    lo = fminf(lo, -acc);
    hi = fmaxf(hi, -acc);
  }
  if (lane == 0 && lo <= hi) {
    atomicMin(mm, f2o(lo));
    atomicMax(mm + 1, f2o(hi));
  }
}

// cnt[c] = number of rows of class c (0: P, 1: Q; every row is of class 0
// when y is null) with s <= th[c]
__global__ void __launch_bounds__(256) count_le_kernel(const float* s, const int8_t* y, int64_t n, float thP,
                                                       float thQ, unsigned long long* cnt) {
  unsigned int a = 0, b = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const bool pos = y ? __ldg(y + i) > 0 : true;
    const float v = s[i];
    if (pos) a += v <= thP ? 1u : 0u;
    else b += v <= thQ ? 1u : 0u;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (a) atomicAdd(cnt, (unsigned long long)a);
    if (b) atomicAdd(cnt + 1, (unsigned long long)b);
  }
}

// the indices of rows with s <= th[c], appended per class (at most cap each;
// pos[c] counts them all)
__global__ void __launch_bounds__(256) select_le_kernel(const float* s, const int8_t* y, int64_t n, float thP,
                                                        float thQ, int* idx, int cap, unsigned int* pos) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (y ? __ldg(y + i) > 0 : true) ? 0 : 1;
    if (s[i] <= (c == 0 ? thP : thQ)) {
      const unsigned int k = atomicAdd(pos + c, 1u);
      if (k < (unsigned int)cap) idx[(size_t)c * cap + k] = (int)i;
    }
  }
}

// rows idx[0..k) of X as float32 into out (k x d)
template <typename T>
__global__ void __launch_bounds__(256) gather_rows_kernel(const T* X, const int* idx, int k, int d, float* out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)k * d;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / d), j = (int)(e % d);
    out[e] = elem_to_float<T>(X + (int64_t)idx[r] * d + j);
  }
}

size_t r256c(size_t x) { return (x + 255) & ~(size_t)255; }

struct CsLayout {
  size_t s, mm, cnt, pos, sel, gidx, rows, w, total;
};
CsLayout cs_layout(int64_t n, int d) {
  CsLayout L;
  const size_t cap = (size_t)2 * kCoresetK;  // selection cap per class (threshold overshoot)
  const size_t kmax = (size_t)2 * kCoresetMaxPerClass;
  L.s = 0;
  L.mm = r256c((size_t)n * sizeof(float));
  L.cnt = L.mm + 256;
  L.pos = L.cnt + 256;
  L.sel = L.pos + 256;
  L.gidx = L.sel + r256c(2 * cap * sizeof(int));
  L.rows = L.gidx + r256c(kmax * sizeof(int));
  L.w = L.rows + r256c(kmax * (size_t)d * sizeof(float));
  L.total = L.w + r256c((size_t)d * sizeof(float));
  return L;
}

template <typename T>
cudaError_t launch_project(const void* X, const int8_t* y, int64_t n, int d, const float* w, float* s,
                           unsigned int* mm, cudaStream_t st) {
  const unsigned int init[4] = {0xffffffffu, 0u, 0xffffffffu, 0u};
  cudaError_t e = cudaMemcpyAsync(mm, init, sizeof(init), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  const int grid = device_sm_count() * 8;
  svm_project_kernel<T><<<grid, 256, 0, st>>>(reinterpret_cast<const T*>(X), y, n, d, w, s, mm);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ses_dist(const void* X, int64_t n, int d, const float* c, float* s, unsigned int* mm,
                            cudaStream_t st) {
  const unsigned int init[2] = {0xffffffffu, 0u};
  cudaError_t e = cudaMemcpyAsync(mm, init, sizeof(init), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  const int grid = device_sm_count() * 8;
  ses_dist_kernel<T><<<grid, 256, 0, st>>>(reinterpret_cast<const T*>(X), n, d, c, s, mm);
  return cudaGetLastError();
}

}  // namespace

size_t coreset_bytes(int64_t n, int d) { return cs_layout(n, d).total; }

pdscp_status svm_coreset_check(const void* X, int dtype, const int8_t* y, int64_t n, int d, const double* w0,
                               double eps, void* ws, cudaStream_t st, double* lb, double* ub,
                               std::vector<double>& w_lb) {
  const CsLayout L = cs_layout(n, d);
  char* base = reinterpret_cast<char*>(ws);
  float* s = reinterpret_cast<float*>(base + L.s);
  unsigned int* mm = reinterpret_cast<unsigned int*>(base + L.mm);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(base + L.cnt);
  unsigned int* pos = reinterpret_cast<unsigned int*>(base + L.pos);
  int* sel = reinterpret_cast<int*>(base + L.sel);
  int* gidx = reinterpret_cast<int*>(base + L.gidx);
  float* rows = reinterpret_cast<float*>(base + L.rows);
  float* wdev = reinterpret_cast<float*>(base + L.w);
  const int cap = 2 * kCoresetK;
  const int grid = device_sm_count() * 4;
  std::vector<float> wf(d);
  std::vector<double> w(w0, w0 + d);
  std::vector<int> core[2];  // the core set, sorted row indices per class
  *lb = 0.0;
  *ub = INFINITY;
  w_lb.assign(d, 0.0);
  auto fail_cuda = [](cudaError_t, const char* what) { return report_error(PDSCP_ERR_CUDA, what); };
  // projections of every point on w (unit norm taken by the caller's use of
  // the margin: here only their order matters, and min_P s + min_Q s)
  auto project = [&](const std::vector<double>& v, unsigned int* mm_host) -> cudaError_t {
    double nv = 0.0;
    for (int j = 0; j < d; ++j) nv += v[j] * v[j];
    nv = nv > 0.0 ? 1.0 / std::sqrt(nv) : 0.0;
    for (int j = 0; j < d; ++j) wf[j] = (float)(v[j] * nv);
    cudaError_t e = cudaMemcpyAsync(wdev, wf.data(), (size_t)d * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = dtype == PDSCP_F32 ? launch_project<float>(X, y, n, d, wdev, s, mm, st)
                             : launch_project<__nv_bfloat16>(X, y, n, d, wdev, s, mm, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mm_host, mm, 4 * sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
  };
  unsigned int mmh[4];
  cudaError_t e = project(w, mmh);
  if (e != cudaSuccess) return fail_cuda(e, "coreset: projection");
  std::vector<float> rowsh;
  std::vector<double> Pd, Qd, mu, ga, z(d), mu0, ga0;
  std::vector<std::pair<int, double>> prev[2];  // the last round's solution: (row, weight) per class
  for (int round = 0; round < kCoresetRounds; ++round) {
    // per class: a threshold taking between K and 2K points (bisection on
    // its float value over [min, max] of the class), or every point of a
    // class of at most K points
    auto count = [&](const float* th2, unsigned long long* got) -> cudaError_t {
      const unsigned long long z2[2] = {0ull, 0ull};
      cudaError_t e2 = cudaMemcpyAsync(cnt, z2, sizeof(z2), cudaMemcpyHostToDevice, st);
      if (e2 == cudaSuccess) count_le_kernel<<<grid, 256, 0, st>>>(s, y, n, th2[0], th2[1], cnt);
      if (e2 == cudaSuccess) e2 = cudaGetLastError();
      if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(got, cnt, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
      if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
      return e2;
    };
    float lo[2] = {o2f(mmh[0]), o2f(mmh[2])}, hi[2] = {o2f(mmh[1]), o2f(mmh[3])};
    unsigned long long got[2];
    if ((e = count(lo, got)) != cudaSuccess) return fail_cuda(e, "coreset: count");
    // lo takes fewer than K points (else it is the threshold); hi takes all of the class
    bool need[2];
    for (int c = 0; c < 2; ++c) {
      need[c] = got[c] < (unsigned long long)kCoresetK;
      if (!need[c]) hi[c] = lo[c];
    }
    for (int itb = 0; itb < 40 && (need[0] || need[1]); ++itb) {
      float mid[2];
      for (int c = 0; c < 2; ++c) mid[c] = need[c] ? lo[c] + 0.5f * (hi[c] - lo[c]) : hi[c];
      if ((e = count(mid, got)) != cudaSuccess) return fail_cuda(e, "coreset: count");
      for (int c = 0; c < 2; ++c) {
        if (!need[c]) continue;
        if (!(mid[c] > lo[c] && mid[c] < hi[c])) {  // no float left between lo and hi
          need[c] = false;
          continue;
        }
        if (got[c] < (unsigned long long)kCoresetK) {
          lo[c] = mid[c];
        } else {
          hi[c] = mid[c];
          if (got[c] <= (unsigned long long)cap) need[c] = false;
        }
      }
    }
    const float th[2] = {hi[0], hi[1]};
    unsigned int posh[2] = {0u, 0u};
    e = cudaMemcpyAsync(pos, posh, sizeof(posh), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) select_le_kernel<<<grid, 256, 0, st>>>(s, y, n, th[0], th[1], sel, cap, pos);
    if (e == cudaSuccess) e = cudaMemcpyAsync(posh, pos, sizeof(posh), cudaMemcpyDeviceToHost, st);
    std::vector<int> selh(2 * (size_t)cap);
    if (e == cudaSuccess) e = cudaMemcpyAsync(selh.data(), sel, selh.size() * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_cuda(e, "coreset: select");
    // merge the picked points into the core set (sorted: the set and so the
    // solve do not depend on the order of the device's atomic appends)
    for (int c = 0; c < 2; ++c) {
      std::vector<int> got(selh.begin() + (size_t)c * cap, selh.begin() + (size_t)c * cap + std::min<unsigned int>(posh[c], cap));
      std::sort(got.begin(), got.end());
      std::vector<int> merged;
      std::set_union(core[c].begin(), core[c].end(), got.begin(), got.end(), std::back_inserter(merged));
      if ((int)merged.size() > kCoresetMaxPerClass) merged.resize(kCoresetMaxPerClass);  // keeps the sorted head
      core[c].swap(merged);
    }
    const int nP = (int)core[0].size(), nQ = (int)core[1].size();
    if (nP == 0 || nQ == 0) break;
    std::vector<int> all(core[0]);
    all.insert(all.end(), core[1].begin(), core[1].end());
    const int k = nP + nQ;
    rowsh.resize((size_t)k * d);
    e = cudaMemcpyAsync(gidx, all.data(), (size_t)k * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
      if (dtype == PDSCP_F32)
        gather_rows_kernel<float><<<grid, 256, 0, st>>>(reinterpret_cast<const float*>(X), gidx, k, d, rows);
      else
        gather_rows_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(X), gidx, k,
                                                                d, rows);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(rowsh.data(), rows, rowsh.size() * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_cuda(e, "coreset: gather");
    Pd.assign(rowsh.begin(), rowsh.begin() + (size_t)nP * d);
    Qd.assign(rowsh.begin() + (size_t)nP * d, rowsh.end());
    mu.assign(nP, 0.0);
    ga.assign(nQ, 0.0);
    // warm start from the last round's solution (its rows are in the merged
    // core sets unless the size cap cut them)
    mu0.assign(nP, 0.0);
    ga0.assign(nQ, 0.0);
    for (int c = 0; c < 2; ++c)
      for (const auto& rw : prev[c]) {
        const auto pos = std::lower_bound(core[c].begin(), core[c].end(), rw.first);
        if (pos != core[c].end() && *pos == rw.first) (c ? ga0 : mu0)[pos - core[c].begin()] = rw.second;
      }
    double gap = 0.0;
    pd_active_set(Pd.data(), nP, Qd.data(), nQ, d, eps / 10.0, 4 * (nP + nQ) + 64, mu.data(), ga.data(), z.data(),
                  &gap, round > 0 ? mu0.data() : nullptr, round > 0 ? ga0.data() : nullptr);
    for (int c = 0; c < 2; ++c) {
      prev[c].clear();
      const std::vector<double>& wt = c ? ga : mu;
      for (size_t i = 0; i < wt.size(); ++i)
        if (wt[i] > 0.0) prev[c].emplace_back(core[c][i], wt[i]);
    }
    double zz = 0.0;
    for (int j = 0; j < d; ++j) zz += z[j] * z[j];
    if (!(zz > 0.0)) break;
    *ub = std::min(*ub, std::sqrt(zz));
    // the solution's direction over every point: its margin
    w.assign(z.begin(), z.end());
    e = project(w, mmh);
    if (e != cudaSuccess) return fail_cuda(e, "coreset: projection");
    const double m = (double)o2f(mmh[0]) + (double)o2f(mmh[2]);  // min_P x.w - max_Q x.w, |w| = 1
    if (m > *lb) {
      *lb = m;
      const double inv = 1.0 / std::sqrt(zz);
      for (int j = 0; j < d; ++j) w_lb[j] = z[j] * inv;
    }
    if (*ub <= (1.0 + eps) * *lb) break;
  }
  return PDSCP_OK;
}

pdscp_status ses_coreset_check(const void* X, int dtype, int64_t n, int d, const double* c0, double eps, void* ws,
                               cudaStream_t st, double* lb, double* ub, std::vector<double>& c_ub) {
  const CsLayout L = cs_layout(n, d);
  char* base = reinterpret_cast<char*>(ws);
  float* s = reinterpret_cast<float*>(base + L.s);
  unsigned int* mm = reinterpret_cast<unsigned int*>(base + L.mm);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(base + L.cnt);
  unsigned int* pos = reinterpret_cast<unsigned int*>(base + L.pos);
  int* sel = reinterpret_cast<int*>(base + L.sel);
  int* gidx = reinterpret_cast<int*>(base + L.gidx);
  float* rows = reinterpret_cast<float*>(base + L.rows);
  float* cdev = reinterpret_cast<float*>(base + L.w);
  const int cap = 2 * kCoresetK;
  const int kmax = 2 * kCoresetMaxPerClass;  // the rows region holds both classes' caps of the SVM checks
  const int grid = device_sm_count() * 4;
  std::vector<float> cf(d);
  *lb = 0.0;
  *ub = INFINITY;
  c_ub.assign(c0, c0 + d);
  auto fail_cuda = [](cudaError_t, const char* what) { return report_error(PDSCP_ERR_CUDA, what); };
  // s_i = -|x_i - c|^2 for every point; returns min s and max s
  auto dist_pass = [&](const std::vector<double>& c, float* smin, float* smax) -> cudaError_t {
    for (int j = 0; j < d; ++j) cf[j] = (float)c[j];
    cudaError_t e = cudaMemcpyAsync(cdev, cf.data(), (size_t)d * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = dtype == PDSCP_F32 ? launch_ses_dist<float>(X, n, d, cdev, s, mm, st)
                             : launch_ses_dist<__nv_bfloat16>(X, n, d, cdev, s, mm, st);
    unsigned int mmh[2];
    if (e == cudaSuccess) e = cudaMemcpyAsync(mmh, mm, sizeof(mmh), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
      *smin = o2f(mmh[0]);
      *smax = o2f(mmh[1]);
    }
    return e;
  };
  std::vector<double> c(c0, c0 + d);
  float smin = 0.f, smax = 0.f;
  cudaError_t e = dist_pass(c, &smin, &smax);
  if (e != cudaSuccess) return fail_cuda(e, "ses core set: distances");
  *ub = std::sqrt(std::max(-(double)smin, 0.0));  // the ball at c0 itself
  std::vector<int> core;  // the core set: sorted row indices
  std::vector<float> rowsh;
  std::vector<double> Pd, mu, cm;
  for (int round = 0; round < kCoresetRounds; ++round) {
    // a threshold on s taking between K and 2K points (the farthest from c),
    // by bisection over [min s, max s], or every point when n <= K
    auto count = [&](float th, unsigned long long* got) -> cudaError_t {
      const unsigned long long z2[2] = {0ull, 0ull};
      cudaError_t e2 = cudaMemcpyAsync(cnt, z2, sizeof(z2), cudaMemcpyHostToDevice, st);
      if (e2 == cudaSuccess) count_le_kernel<<<grid, 256, 0, st>>>(s, nullptr, n, th, th, cnt);
      if (e2 == cudaSuccess) e2 = cudaGetLastError();
      if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(got, cnt, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
      if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
      return e2;
    };
    float lo = smin, hi = smax;
    unsigned long long got[2];
    if ((e = count(lo, got)) != cudaSuccess) return fail_cuda(e, "ses core set: count");
    bool need = got[0] < (unsigned long long)kCoresetK;
    if (!need) hi = lo;
    for (int itb = 0; itb < 40 && need; ++itb) {
      const float mid = lo + 0.5f * (hi - lo);
      if (!(mid > lo && mid < hi)) break;  // no float left between lo and hi
      if ((e = count(mid, got)) != cudaSuccess) return fail_cuda(e, "ses core set: count");
      if (got[0] < (unsigned long long)kCoresetK) {
        lo = mid;
      } else {
        hi = mid;
        if (got[0] <= (unsigned long long)cap) need = false;
      }
    }
    unsigned int posh[2] = {0u, 0u};
    e = cudaMemcpyAsync(pos, posh, sizeof(posh), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) select_le_kernel<<<grid, 256, 0, st>>>(s, nullptr, n, hi, hi, sel, cap, pos);
    if (e == cudaSuccess) e = cudaMemcpyAsync(posh, pos, sizeof(posh), cudaMemcpyDeviceToHost, st);
    std::vector<int> selh(cap);
    if (e == cudaSuccess) e = cudaMemcpyAsync(selh.data(), sel, selh.size() * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_cuda(e, "ses core set: select");
    // merged into the core set, sorted (independent of the atomic appends' order)
    std::vector<int> picked(selh.begin(), selh.begin() + std::min<unsigned int>(posh[0], cap));
    std::sort(picked.begin(), picked.end());
    std::vector<int> merged;
    std::set_union(core.begin(), core.end(), picked.begin(), picked.end(), std::back_inserter(merged));
    if ((int)merged.size() > kmax) merged.resize(kmax);
    core.swap(merged);
    const int k = (int)core.size();
    if (k == 0) break;
    rowsh.resize((size_t)k * d);
    e = cudaMemcpyAsync(gidx, core.data(), (size_t)k * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
      if (dtype == PDSCP_F32)
        gather_rows_kernel<float><<<grid, 256, 0, st>>>(reinterpret_cast<const float*>(X), gidx, k, d, rows);
      else
        gather_rows_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(X), gidx, k,
                                                                d, rows);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(rowsh.data(), rows, rowsh.size() * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_cuda(e, "ses core set: gather");
    // the dual on the core set, translated by c0 (the ball problem is
    // translation invariant; near the origin phi loses no digits)
    Pd.resize((size_t)k * d);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < d; ++j) Pd[(size_t)i * d + j] = (double)rowsh[(size_t)i * d + j] - c0[j];
    double far = 0.0;
    const double lbr = meb_dual_fw(Pd.data(), k, d, eps / 10.0, 200000, mu, cm, &far);
    *lb = std::max(*lb, lbr);
    for (int j = 0; j < d; ++j) c[j] = cm[j] + c0[j];
    // the ball at c_mu over every point: an upper bound (and the distances
    // the next round picks from)
    if ((e = dist_pass(c, &smin, &smax)) != cudaSuccess) return fail_cuda(e, "ses core set: distances");
    const double r = std::sqrt(std::max(-(double)smin, 0.0));
    if (r < *ub) {
      *ub = r;
      c_ub = c;
    }
    if (*ub <= (1.0 + eps) * *lb) break;
  }
  return PDSCP_OK;
}

}  // namespace pdscp

using namespace pdscp;

extern "C" pdscp_status pdscp_meb_dual(const double* P, int32_t m, int32_t d, double tol, int32_t max_iter,
                                       double* mu, double* center, double* lb, double* far) {
  if (!P || !mu || !center || !lb || !far) return report_error(PDSCP_ERR_INVALID_ARG, "pdscp_meb_dual: null pointer");
  if (m < 1 || d < 1) return report_error(PDSCP_ERR_INVALID_ARG, "pdscp_meb_dual: m < 1 or d < 1");
  if (!(tol >= 0.0) || max_iter < 1) return report_error(PDSCP_ERR_INVALID_ARG, "pdscp_meb_dual: tol < 0 or max_iter < 1");
  std::vector<double> w, c;
  *lb = meb_dual_fw(P, m, d, tol, max_iter, w, c, far);
  std::copy(w.begin(), w.end(), mu);
  std::copy(c.begin(), c.end(), center);
  return PDSCP_OK;
}

extern "C" pdscp_status pdscp_polytope_distance(const double* P, int32_t nP, const double* Q, int32_t nQ, int32_t d,
                                                double tol, int32_t max_iter, double* mu, double* gamma,
                                                double* dist) {
  if (!P || !Q || !mu || !gamma || !dist) return report_error(PDSCP_ERR_INVALID_ARG, "pdscp_polytope_distance: null pointer");
  if (nP < 1 || nQ < 1 || d < 1) return report_error(PDSCP_ERR_INVALID_ARG, "pdscp_polytope_distance: empty set or d < 1");
  if (!(tol >= 0.0) || max_iter < 1) return report_error(PDSCP_ERR_INVALID_ARG, "pdscp_polytope_distance: tol < 0 or max_iter < 1");
  std::vector<double> z(d);
  pd_active_set(P, nP, Q, nQ, d, tol, max_iter, mu, gamma, z.data(), nullptr);
  double zz = 0.0;
  for (int j = 0; j < d; ++j) zz += z[j] * z[j];
  *dist = std::sqrt(zz);
  return PDSCP_OK;
}

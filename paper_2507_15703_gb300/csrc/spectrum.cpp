// Host FP64 spectrum helpers: P_inf(k) interpolation and the inversion of a
// target angular spectrum C_l into a non-negative 3-D spectrum P_inf(k).
//
// The relation used (paper Sec. II.A): with the convention
// xi(x) = int d^3k P(k) exp(i k.x) behind Eq. (2.4), the plane-wave expansion
// of exp(i k.x) on a sphere of radius r gives
//     C_l = 16 pi^2 int_0^inf k^2 P(k) j_l(k r)^2 dk,
// and summing (2l+1) C_l P_l(cos theta) / 4 pi (Eq. 2.1) returns xi_inf at the
// chord 2 r sin(theta/2) (Eq. 2.3).  The paper imposes the equivalent
// condition on xi with a linear program (Sec. II.B); here the C_l are matched
// directly in relative least squares under P >= 0 (Lawson-Hanson NNLS).
#include "spectrum.h"

#include <algorithm>
#include <cmath>
#include <limits>
#include <thread>

#include "cmb3d.h"

namespace cmb3d {

double pk_interp(const std::vector<double>& k, const std::vector<double>& p, double x) {
  if (k.empty()) return 0.0;
  if (x > k.back()) return 0.0;
  if (x <= k.front()) return p.front();
  const size_t i = static_cast<size_t>(std::upper_bound(k.begin(), k.end(), x) - k.begin());
  if (i >= k.size()) return p.back();
  const double t = (x - k[i - 1]) / (k[i] - k[i - 1]);
  return p[i - 1] + t * (p[i] - p[i - 1]);
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>* x, std::vector<double>* w) {
  x->assign(static_cast<size_t>(n), 0.0);
  w->assign(static_cast<size_t>(n), 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;                    // P_0, P_1
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);     // P_n'(z)
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    (*x)[static_cast<size_t>(i)] = -z;
    (*x)[static_cast<size_t>(n - 1 - i)] = z;
    const double wi = 2.0 / ((1.0 - z * z) * dp * dp);
    (*w)[static_cast<size_t>(i)] = wi;
    (*w)[static_cast<size_t>(n - 1 - i)] = wi;
  }
}

namespace {

// j_l(x)^2 for l = 0..lmax by Miller's downward recurrence
// j_{l-1} = (2l+1)/x j_l - j_{l+1}, started well above max(lmax, x) and
// normalised with the sum rule sum_l (2l+1) j_l(x)^2 = 1 (only squares are
// needed, so the overall sign does not matter).
void sph_bessel_sq(int lmax, double x, std::vector<double>* out) {
  out->assign(static_cast<size_t>(lmax) + 1, 0.0);
  if (x < 1e-300) {
    (*out)[0] = 1.0;
    return;
  }
  const int start = static_cast<int>(std::max<double>(lmax, x) + 30.0 + 6.0 * std::sqrt(std::max(x, 1.0)));
  double jp1 = 0.0, j = 1.0;       // j_{start+1}, j_{start} up to a common factor
  double sum = (2.0 * start + 1.0) * j * j;
  std::vector<double> vals(static_cast<size_t>(lmax) + 1, 0.0);
  if (start <= lmax) vals[static_cast<size_t>(start)] = j;
  for (int l = start; l >= 1; --l) {
    double jm1 = (2.0 * l + 1.0) / x * j - jp1;
    jp1 = j;
    j = jm1;
    if (std::fabs(j) > 1e100) {                     // rescale so that j^2 cannot overflow
      const double s = 1e-100;
      j *= s;
      jp1 *= s;
      sum *= s * s;
      for (int m = l; m <= lmax; ++m) vals[static_cast<size_t>(m)] *= s;
    }
    sum += (2.0 * (l - 1) + 1.0) * j * j;
    if (l - 1 <= lmax) vals[static_cast<size_t>(l - 1)] = j;
  }
  for (int l = 0; l <= lmax; ++l) (*out)[static_cast<size_t>(l)] = vals[static_cast<size_t>(l)] * vals[static_cast<size_t>(l)] / sum;
}

// Solve G[P,P] z = h[P] for the index set P by Cholesky; false if a pivot is
// not positive.  G is n x n row-major symmetric positive semi-definite.
bool chol_solve(const std::vector<double>& G, int n, const std::vector<int>& P, const std::vector<double>& h,
                std::vector<double>* z) {
  const int p = static_cast<int>(P.size());
  std::vector<double> Lm(static_cast<size_t>(p) * p, 0.0);
  for (int i = 0; i < p; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = G[static_cast<size_t>(P[static_cast<size_t>(i)]) * n + P[static_cast<size_t>(j)]];
      for (int k = 0; k < j; ++k) s -= Lm[static_cast<size_t>(i) * p + k] * Lm[static_cast<size_t>(j) * p + k];
      if (i == j) {
        if (!(s > 0.0)) return false;
        Lm[static_cast<size_t>(i) * p + i] = std::sqrt(s);
      } else {
        Lm[static_cast<size_t>(i) * p + j] = s / Lm[static_cast<size_t>(j) * p + j];
      }
    }
  }
  z->assign(static_cast<size_t>(p), 0.0);
  for (int i = 0; i < p; ++i) {                    // L y = h
    double s = h[static_cast<size_t>(P[static_cast<size_t>(i)])];
    for (int k = 0; k < i; ++k) s -= Lm[static_cast<size_t>(i) * p + k] * (*z)[static_cast<size_t>(k)];
    (*z)[static_cast<size_t>(i)] = s / Lm[static_cast<size_t>(i) * p + i];
  }
  for (int i = p - 1; i >= 0; --i) {               // L^T z = y
    double s = (*z)[static_cast<size_t>(i)];
    for (int k = i + 1; k < p; ++k) s -= Lm[static_cast<size_t>(k) * p + i] * (*z)[static_cast<size_t>(k)];
    (*z)[static_cast<size_t>(i)] = s / Lm[static_cast<size_t>(i) * p + i];
  }
  return true;
}

}  // namespace

std::vector<double> cl_design_matrix(const double* ell, int n, const std::vector<double>& knodes, double r,
                                     int nquad) {
  const int nk = static_cast<int>(knodes.size());
  std::vector<double> A(static_cast<size_t>(n) * nk, 0.0);
  std::vector<double> gx, gw;
  gauss_legendre(nquad, &gx, &gw);
  int lmax = 0;
  for (int i = 0; i < n; ++i) lmax = std::max(lmax, static_cast<int>(ell[i]));
  std::vector<double> jl2;
  const double c16 = 16.0 * M_PI * M_PI;
  for (int j = 0; j + 1 < nk; ++j) {
    const double a = knodes[static_cast<size_t>(j)], b = knodes[static_cast<size_t>(j) + 1];
    for (int g = 0; g < nquad; ++g) {
      const double k = 0.5 * (b - a) * gx[static_cast<size_t>(g)] + 0.5 * (b + a);
      const double w = 0.5 * (b - a) * gw[static_cast<size_t>(g)];
      const double s = (k - a) / (b - a);              // rising hat of node j+1
      sph_bessel_sq(lmax, k * r, &jl2);
      const double base = c16 * w * k * k;
      for (int i = 0; i < n; ++i) {
        const double v = base * jl2[static_cast<size_t>(ell[i])];
        A[static_cast<size_t>(i) * nk + j] += v * (1.0 - s);
        A[static_cast<size_t>(i) * nk + j + 1] += v * s;
      }
    }
  }
  return A;
}

int nnls(const std::vector<double>& A, int m, int n, const std::vector<double>& b, double ridge,
         std::vector<double>* xout) {
  // Normal equations G = A^T A + ridge * mean(diag) I, h = A^T b.
  std::vector<double> G(static_cast<size_t>(n) * n, 0.0), h(static_cast<size_t>(n), 0.0);
  for (int i = 0; i < m; ++i) {
    const double* a = &A[static_cast<size_t>(i) * n];
    for (int j = 0; j < n; ++j) {
      if (a[j] == 0.0) continue;
      h[static_cast<size_t>(j)] += a[j] * b[static_cast<size_t>(i)];
      double* g = &G[static_cast<size_t>(j) * n];
      for (int k = j; k < n; ++k) g[k] += a[j] * a[k];
    }
  }
  double dmean = 0.0;
  for (int j = 0; j < n; ++j) dmean += G[static_cast<size_t>(j) * n + j];
  dmean /= n;
  for (int j = 0; j < n; ++j) {
    G[static_cast<size_t>(j) * n + j] += ridge * dmean;
    for (int k = j + 1; k < n; ++k) G[static_cast<size_t>(k) * n + j] = G[static_cast<size_t>(j) * n + k];
  }
  double gmax = 0.0;
  for (double v : G) gmax = std::max(gmax, std::fabs(v));
  const double tol = 10.0 * std::numeric_limits<double>::epsilon() * gmax * n;

  std::vector<double> x(static_cast<size_t>(n), 0.0), w(h), z;
  std::vector<char> passive(static_cast<size_t>(n), 0);
  std::vector<int> P;
  auto gradient = [&]() {                           // w = h - G x
    for (int j = 0; j < n; ++j) {
      double s = h[static_cast<size_t>(j)];
      const double* g = &G[static_cast<size_t>(j) * n];
      for (int k = 0; k < n; ++k) s -= g[k] * x[static_cast<size_t>(k)];
      w[static_cast<size_t>(j)] = s;
    }
  };
  auto passive_set = [&]() {
    P.clear();
    for (int j = 0; j < n; ++j)
      if (passive[static_cast<size_t>(j)]) P.push_back(j);
  };
  const int max_steps = 30 * n + 100;
  int steps = 0;
  while (true) {
    int t = -1;
    double best = tol;
    for (int j = 0; j < n; ++j)
      if (!passive[static_cast<size_t>(j)] && w[static_cast<size_t>(j)] > best) {
        best = w[static_cast<size_t>(j)];
        t = j;
      }
    if (t < 0) break;
    if (++steps > max_steps) {
      *xout = x;
      return -1;
    }
    passive[static_cast<size_t>(t)] = 1;
    passive_set();
    if (!chol_solve(G, n, P, h, &z)) {
      // t is numerically dependent on the passive set: skip it until x moves
      passive[static_cast<size_t>(t)] = 0;
      w[static_cast<size_t>(t)] = 0.0;
      passive_set();
      continue;
    }
    for (int inner = 0; inner <= n; ++inner) {
      if (inner > 0 && !chol_solve(G, n, P, h, &z)) {
        *xout = x;
        return -1;
      }
      double zmin = std::numeric_limits<double>::infinity();
      for (double v : z) zmin = std::min(zmin, v);
      if (zmin > 0.0) {
        for (size_t c = 0; c < P.size(); ++c) x[static_cast<size_t>(P[c])] = z[c];
        break;
      }
      // move from x towards z until the first passive variable reaches zero
      double alpha = 1.0;
      for (size_t c = 0; c < P.size(); ++c)
        if (z[c] <= 0.0) {
          const double xj = x[static_cast<size_t>(P[c])];
          alpha = std::min(alpha, xj / (xj - z[c]));
        }
      for (size_t c = 0; c < P.size(); ++c) {
        double& xj = x[static_cast<size_t>(P[c])];
        const double x0 = xj;
        xj += alpha * (z[c] - xj);
        // the blocking variable(s) land on zero exactly
        if (xj <= 0.0 || (z[c] <= 0.0 && x0 / (x0 - z[c]) <= alpha * (1.0 + 1e-12))) {
          xj = 0.0;
          passive[static_cast<size_t>(P[c])] = 0;
        }
      }
      passive_set();
      if (P.empty()) break;
    }
    gradient();
  }
  *xout = x;
  return steps;
}

int fit_pk_from_cl(const double* ell, const double* cl, int n, int N, double L, double r, int nk,
                   std::vector<double>* knodes, std::vector<double>* pnodes, double* max_rel_err,
                   std::string* detail) {
  const double kmax = std::sqrt(3.0) * M_PI * N / L;
  knodes->resize(static_cast<size_t>(nk));
  for (int j = 0; j < nk; ++j) (*knodes)[static_cast<size_t>(j)] = kmax * j / (nk - 1);
  std::vector<double> A = cl_design_matrix(ell, n, *knodes, r, 16);
  std::vector<double> Aw(A.size()), b(static_cast<size_t>(n), 1.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < nk; ++j)
      Aw[static_cast<size_t>(i) * nk + j] = A[static_cast<size_t>(i) * nk + j] / cl[i];
  // Unit column norms: the non-negative solution is invariant under positive
  // column scaling, and the normal equations become far better conditioned.
  std::vector<double> cn(static_cast<size_t>(nk), 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < nk; ++j) cn[static_cast<size_t>(j)] += Aw[static_cast<size_t>(i) * nk + j] * Aw[static_cast<size_t>(i) * nk + j];
  for (int j = 0; j < nk; ++j) cn[static_cast<size_t>(j)] = cn[static_cast<size_t>(j)] > 0 ? std::sqrt(cn[static_cast<size_t>(j)]) : 1.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < nk; ++j) Aw[static_cast<size_t>(i) * nk + j] /= cn[static_cast<size_t>(j)];
  std::vector<double> x;
  const int it = nnls(Aw, n, nk, b, 0.0, &x);
  for (int j = 0; j < nk; ++j) x[static_cast<size_t>(j)] /= cn[static_cast<size_t>(j)];
  if (it < 0) {
    if (detail) *detail = "NNLS iteration limit reached";
    return CMB3D_EUNSUPPORTED;
  }
  double err = 0.0;
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < nk; ++j) s += A[static_cast<size_t>(i) * nk + j] * x[static_cast<size_t>(j)];
    err = std::max(err, std::fabs(s - cl[i]) / cl[i]);
  }
  *pnodes = x;
  *max_rel_err = err;
  return CMB3D_OK;
}

void sqrt_symmetric(const double* a, int n, double* s) {
  std::vector<double> A(a, a + static_cast<size_t>(n) * n), V(static_cast<size_t>(n) * n, 0.0);
  for (int i = 0; i < n; ++i) V[static_cast<size_t>(i) * n + i] = 1.0;
  auto at = [&](std::vector<double>& m, int i, int j) -> double& { return m[static_cast<size_t>(i) * n + j]; };
  double fro = 0.0;
  for (double x : A) fro += x * x;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += 2.0 * at(A, i, j) * at(A, i, j);
    if (off <= 1e-30 * fro) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = at(A, p, q);
        if (apq == 0.0) continue;
        // rotation angle zeroing A[p][q] (Golub & Van Loan, Alg. 8.4.1)
        const double tau = (at(A, q, q) - at(A, p, p)) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = t * c;
        for (int k = 0; k < n; ++k) {            // A <- A J (columns p, q)
          const double akp = at(A, k, p), akq = at(A, k, q);
          at(A, k, p) = c * akp - sn * akq;
          at(A, k, q) = sn * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {            // A <- J^T A (rows p, q)
          const double apk = at(A, p, k), aqk = at(A, q, k);
          at(A, p, k) = c * apk - sn * aqk;
          at(A, q, k) = sn * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {            // V <- V J
          const double vkp = at(V, k, p), vkq = at(V, k, q);
          at(V, k, p) = c * vkp - sn * vkq;
          at(V, k, q) = sn * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc += at(V, i, k) * std::sqrt(std::max(at(A, k, k), 0.0)) * at(V, j, k);
      s[static_cast<size_t>(i) * n + j] = acc;
    }
}

void sqrt_gamma_table(int N, int M, int h, double L, const std::vector<double>& knodes,
                      const std::vector<double>& pnodes, int threads, std::vector<float>* table) {
  const int H = N / 2;
  const int nq = 2 * H * H + 1;
  table->assign(static_cast<size_t>(nq) * h * h, 0.0f);
  std::vector<char> reach(static_cast<size_t>(nq), 0);
  for (int mx = 0; mx <= H; ++mx)
    for (int f = -H + 1; f <= H; ++f) reach[static_cast<size_t>(mx * mx + f * f)] = 1;
  const double dp = L / N;
  const double kxy = 2.0 * M_PI / (N * dp), kz = 2.0 * M_PI / (M * dp);
  const double vol = std::pow(2.0 * M_PI / dp, 3) / (static_cast<double>(M) * N * N);
  // cos(2 pi m d / M) for m < M, d < h
  std::vector<double> cs(static_cast<size_t>(M) * h);
  for (int m = 0; m < M; ++m)
    for (int d = 0; d < h; ++d)
      cs[static_cast<size_t>(m) * h + d] = std::cos(2.0 * M_PI * static_cast<double>((static_cast<long long>(m) * d) % M) / M);
  auto work = [&](int t) {
    std::vector<double> col(static_cast<size_t>(M)), xi(static_cast<size_t>(h)), g(static_cast<size_t>(h) * h),
        sq(static_cast<size_t>(h) * h);
    for (int q = t; q < nq; q += threads) {
      if (!reach[static_cast<size_t>(q)]) continue;
      for (int m = 0; m < M; ++m) {
        const int fz = m <= M / 2 ? m : m - M;
        const double k = std::sqrt(kxy * kxy * q + kz * kz * static_cast<double>(fz) * fz);
        col[static_cast<size_t>(m)] = (q == 0 && m == 0) ? 0.0 : pk_interp(knodes, pnodes, k) * vol;
      }
      for (int d = 0; d < h; ++d) {
        double acc = 0.0;
        for (int m = 0; m < M; ++m) acc += col[static_cast<size_t>(m)] * cs[static_cast<size_t>(m) * h + d];
        xi[static_cast<size_t>(d)] = acc;
      }
      for (int i = 0; i < h; ++i)
        for (int j = 0; j < h; ++j) g[static_cast<size_t>(i) * h + j] = xi[static_cast<size_t>(std::abs(i - j))];
      sqrt_symmetric(g.data(), h, sq.data());
      float* out = table->data() + static_cast<size_t>(q) * h * h;
      for (int i = 0; i < h * h; ++i) out[i] = static_cast<float>(sq[static_cast<size_t>(i)]);
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < threads; ++t) pool.emplace_back(work, t);
  work(0);
  for (auto& th : pool) th.join();
}

}  // namespace cmb3d

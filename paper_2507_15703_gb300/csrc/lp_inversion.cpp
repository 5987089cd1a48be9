// The paper's linear-programming inversion (Sec. II.B), host FP64.
//
// A flat-space spectrum P_inf >= 0 is sought whose correlation function
// xi_inf(r) = 4 pi int k P(k) sin(k r)/r dk (Eq. 2.4) equals the sphere's
// xi_sph(theta) (Eq. 2.1 with the beam-smoothed C_l of Eq. 2.2) at the chord
// r = 2 R sin(theta/2) (Eq. 2.3) for every separation up to the largest one
// the cap holds.  With P linear between uniform k nodes and the constraints
// taken at uniform separations this is the linear program
//     minimise c^T x,  c_j = sum_i A_ij  (Eq. 2.5),  A x >= b,  x >= 0,
// whose objective sum_i (A x)_i is smallest, sum_i b_i, exactly when A x = b.
//
// The program has many more constraints (m, one per separation) than
// unknowns (n, one per k node), so the simplex runs on its dual
//     maximise b^T y,  A^T y + t = c,  y, t >= 0,
// an n-row tableau.  The dual is always feasible (y = 1 gives A^T y = c), and
// the primal is feasible because the first node's column is positive: its hat
// covers k <= dk and k r <= dk rmax = 2 pi / 3 < pi for the default dk.
#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <functional>
#include <limits>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "cmb3d.h"
#include "spectrum.h"

namespace cmb3d {

int lp_grid(double R, double theta_max, double beam, double dr, double dk, double kmax, LpGrid* g,
            std::string* detail) {
  auto bad = [&](const char* why) {
    if (detail) *detail = why;
    return CMB3D_EINVAL;
  };
  if (!(std::isfinite(R) && R > 0)) return bad("R must be finite and > 0");
  if (!(std::isfinite(theta_max) && theta_max > 0 && theta_max <= M_PI)) return bad("theta_max must be in (0, pi]");
  if (!(std::isfinite(beam) && beam >= 0)) return bad("beam must be finite and >= 0");
  if (!(std::isfinite(dr) && dr >= 0) || !(std::isfinite(dk) && dk >= 0) || !(std::isfinite(kmax) && kmax > 0))
    return bad("dr, dk must be finite and >= 0, kmax finite and > 0");
  g->rmax = theta_max <= M_PI / 2 ? 2.0 * R * std::sin(theta_max) : 2.0 * R;
  g->dr = dr == 0.0 ? beam / 5.0 : dr;
  g->dk = dk == 0.0 ? 2.0 * M_PI / (3.0 * g->rmax) : dk;
  if (!(g->dr > 0)) return bad("dr = 0 needs a beam > 0 (dr = beam / 5)");
  if (!(kmax >= g->dk)) return bad("kmax must be at least dk");
  const double mm = std::floor(g->rmax / g->dr) + 1.0, nn = std::floor(kmax / g->dk);
  if (mm > 1e6 || nn > 1e5) {
    if (detail) *detail = "more than 1e6 separations or 1e5 k nodes";
    return CMB3D_EUNSUPPORTED;
  }
  g->m = static_cast<int>(mm);
  g->n = static_cast<int>(nn);
  return CMB3D_OK;
}

void lp_targets(const double* ell, const double* cl, int nl, double beam, double R, const LpGrid& g,
                std::vector<double>* b) {
  b->assign(static_cast<size_t>(g.m), 0.0);
  const int lmax = static_cast<int>(ell[nl - 1]);
  std::vector<double> weight(static_cast<size_t>(lmax) + 1, 0.0);     // (2l+1) C_l e^{-b^2 l^2} / 4 pi
  for (int i = 0; i < nl; ++i) {
    const double l = ell[i];
    weight[static_cast<size_t>(l)] += (2.0 * l + 1.0) * cl[i] * std::exp(-(beam * l) * (beam * l)) / (4.0 * M_PI);
  }
  for (int i = 0; i < g.m; ++i) {
    const double r = i * g.dr;
    const double x = 1.0 - r * r / (2.0 * R * R);                     // cos theta_i, Eq. 2.3 inverted
    double p0 = 1.0, p1 = x, acc = weight[0];
    if (lmax >= 1) acc += weight[1] * x;
    for (int l = 1; l < lmax; ++l) {                                   // (l+1) P_{l+1} = (2l+1) x P_l - l P_{l-1}
      const double p2 = ((2.0 * l + 1.0) * x * p1 - l * p0) / (l + 1.0);
      p0 = p1;
      p1 = p2;
      acc += weight[static_cast<size_t>(l) + 1] * p2;
    }
    (*b)[static_cast<size_t>(i)] = acc;
  }
}

void lp_matrix(const LpGrid& g, int threads, std::vector<double>* A) {
  const int m = g.m, n = g.n, nq = 16;
  A->assign(static_cast<size_t>(m) * n, 0.0);
  std::vector<double> gx, gw;
  gauss_legendre(nq, &gx, &gw);
  auto rows = [&](int i0, int i1) {
    for (int i = i0; i < i1; ++i) {
      const double r = i * g.dr;
      double* row = A->data() + static_cast<size_t>(i) * n;
      for (int a = 0; a < n; ++a) {                                    // node interval [k_a, k_a+1]
        const double ka = a * g.dk, kb = (a + 1) * g.dk;
        double left = 0.0, right = 0.0;
        for (int q = 0; q < nq; ++q) {
          const double k = 0.5 * (kb - ka) * gx[q] + 0.5 * (kb + ka);
          const double w = 0.5 * (kb - ka) * gw[q];
          const double kern = r == 0.0 ? k * k : k * std::sin(k * r) / r;
          left += w * kern * (kb - k) / (kb - ka);
          right += w * kern * (k - ka) / (kb - ka);
        }
        row[a] += 4.0 * M_PI * left;
        if (a + 1 < n) row[a + 1] += 4.0 * M_PI * right;               // node n carries P = 0
      }
    }
  };
  threads = std::max(1, std::min(threads, m));
  std::vector<std::thread> pool;
  const int per = (m + threads - 1) / threads;
  for (int t = 0; t < threads; ++t) {
    const int i0 = t * per, i1 = std::min(m, i0 + per);
    if (i0 < i1) pool.emplace_back(rows, i0, i1);
  }
  for (auto& th : pool) th.join();
}

namespace {

// Persistent host threads for the row updates of a pivot: run(f) calls
// f(part, parts) once for every part, the caller taking part 0, and returns
// when all parts are done.
class RowPool {
 public:
  explicit RowPool(int parts) : parts_(std::max(1, parts)) {
    for (int t = 1; t < parts_; ++t) workers_.emplace_back([this, t] { loop(t); });
  }
  ~RowPool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& w : workers_) w.join();
  }
  int parts() const { return parts_; }
  void run(const std::function<void(int, int)>& f) {
    if (parts_ == 1) {
      f(0, 1);
      return;
    }
    {
      std::lock_guard<std::mutex> lk(mu_);
      job_ = &f;
      pending_ = parts_ - 1;
      ++gen_;
    }
    cv_.notify_all();
    f(0, parts_);
    std::unique_lock<std::mutex> lk(mu_);
    done_.wait(lk, [this] { return pending_ == 0; });
    job_ = nullptr;
  }

 private:
  void loop(int t) {
    long seen = 0;
    while (true) {
      const std::function<void(int, int)>* job;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
        if (stop_) return;
        seen = gen_;
        job = job_;
      }
      (*job)(t, parts_);
      std::lock_guard<std::mutex> lk(mu_);
      if (--pending_ == 0) done_.notify_one();
    }
  }
  int parts_;
  std::vector<std::thread> workers_;
  std::mutex mu_;
  std::condition_variable cv_, done_;
  const std::function<void(int, int)>* job_ = nullptr;
  long gen_ = 0;
  int pending_ = 0;
  bool stop_ = false;
};

// Dense simplex tableau of the dual, rows = dual constraints (one per primal
// unknown), columns = y (m), t (n), artificial variables, then the
// right-hand side.  z holds c_B^T B^{-1} a_col - cost_col; a column with
// z < 0 improves the (maximised) objective.
struct Tableau {
  int rows = 0, width = 0;             // width excludes the rhs column
  std::vector<double> T, z;            // rows x (width + 1), width + 1
  std::vector<int> basis;
  double& at(int r, int c) { return T[static_cast<size_t>(r) * (width + 1) + c]; }
  double rhs(int r) const { return T[static_cast<size_t>(r) * (width + 1) + width]; }

  RowPool* pool = nullptr;

  void pivot(int r, int e) {
    const size_t w1 = static_cast<size_t>(width) + 1;
    double* pr = T.data() + static_cast<size_t>(r) * w1;
    const double inv = 1.0 / pr[e];
    for (size_t c = 0; c < w1; ++c) pr[c] *= inv;
    pr[e] = 1.0;
    auto update = [&](int part, int parts) {            // rows are independent: same result for any split
      const int per = (rows + parts - 1) / parts;
      for (int i = part * per, i1 = std::min(rows, i + per); i < i1; ++i) {
        if (i == r) continue;
        double* pi = T.data() + static_cast<size_t>(i) * w1;
        const double f = pi[e];
        if (f == 0.0) continue;
        for (size_t c = 0; c < w1; ++c) pi[c] -= f * pr[c];
        pi[e] = 0.0;
      }
    };
    if (pool) pool->run(update);
    else update(0, 1);
    const double f = z[static_cast<size_t>(e)];
    if (f != 0.0) {
      for (size_t c = 0; c < w1; ++c) z[c] -= f * pr[c];
      z[static_cast<size_t>(e)] = 0.0;
    }
    basis[static_cast<size_t>(r)] = e;
  }

  void price(const std::vector<double>& cost) {                        // z from scratch
    const size_t w1 = static_cast<size_t>(width) + 1;
    z.assign(w1, 0.0);
    for (int c = 0; c < width; ++c) z[static_cast<size_t>(c)] = -cost[static_cast<size_t>(c)];
    for (int r = 0; r < rows; ++r) {
      const double cb = cost[static_cast<size_t>(basis[static_cast<size_t>(r)])];
      if (cb == 0.0) continue;
      const double* pr = T.data() + static_cast<size_t>(r) * w1;
      for (size_t c = 0; c < w1; ++c) z[c] += cb * pr[c];
    }
  }
};

constexpr double kPivTol = 1e-9, kOptTol = 1e-10, kFeasTol = 1e-10;

// Maximise over columns [0, ncols) from a feasible basis (Dantzig pricing on
// the equilibrated columns).  Returns 0 at the optimum, 1 when unbounded, 2 at
// the pivot limit.
int run_simplex(Tableau* tb, int ncols, long max_pivots, long* pivots) {
  int stalled = 0;
  bool bland = false;
  double last = tb->z[static_cast<size_t>(tb->width)];
  while (true) {
    int e = -1;
    double best = -kOptTol;
    for (int c = 0; c < ncols; ++c) {
      const double zc = tb->z[static_cast<size_t>(c)];
      if (zc < best) {
        e = c;
        if (bland) break;                                              // smallest improving index
        best = zc;
      }
    }
    if (e < 0) return 0;
    if (*pivots >= max_pivots) return 2;
    // ratio test with a feasibility allowance (Harris): the bound first, then
    // the largest pivot element among the rows within it
    double bound = std::numeric_limits<double>::infinity();
    for (int r = 0; r < tb->rows; ++r) {
      const double a = tb->at(r, e);
      if (a > kPivTol) bound = std::min(bound, (std::max(tb->rhs(r), 0.0) + kFeasTol) / a);
    }
    if (!std::isfinite(bound)) return 1;
    int leave = -1;
    double big = 0.0;
    for (int r = 0; r < tb->rows; ++r) {
      const double a = tb->at(r, e);
      if (a <= kPivTol || std::max(tb->rhs(r), 0.0) / a > bound) continue;
      if (bland) {
        if (leave < 0 || tb->basis[static_cast<size_t>(r)] < tb->basis[static_cast<size_t>(leave)]) leave = r;
      } else if (a > big) {
        big = a;
        leave = r;
      }
    }
    tb->pivot(leave, e);
    for (int r = 0; r < tb->rows; ++r)                                 // rounding below the bound
      if (tb->rhs(r) < 0.0 && tb->rhs(r) > -kFeasTol) tb->at(r, tb->width) = 0.0;
    ++*pivots;
    const double obj = tb->z[static_cast<size_t>(tb->width)];
    if (obj > last + 1e-13 * std::max(1.0, std::fabs(last))) {
      stalled = 0;
      bland = false;
    } else if (++stalled > 50) {
      bland = true;                                                    // no cycling under Bland's rule
    }
    last = obj;
  }
}

// Dense Gaussian elimination with partial pivoting; false if singular.
bool solve_dense(std::vector<double> M, int n, std::vector<double>* x) {
  std::vector<double>& v = *x;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(M[static_cast<size_t>(r) * n + c]) > std::fabs(M[static_cast<size_t>(p) * n + c])) p = r;
    const double piv = M[static_cast<size_t>(p) * n + c];
    if (!(std::fabs(piv) > 1e-300)) return false;
    if (p != c) {
      for (int k = 0; k < n; ++k) std::swap(M[static_cast<size_t>(p) * n + k], M[static_cast<size_t>(c) * n + k]);
      std::swap(v[static_cast<size_t>(p)], v[static_cast<size_t>(c)]);
    }
    for (int r = c + 1; r < n; ++r) {
      const double f = M[static_cast<size_t>(r) * n + c] / piv;
      if (f == 0.0) continue;
      for (int k = c; k < n; ++k) M[static_cast<size_t>(r) * n + k] -= f * M[static_cast<size_t>(c) * n + k];
      v[static_cast<size_t>(r)] -= f * v[static_cast<size_t>(c)];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    double s = v[static_cast<size_t>(c)];
    for (int k = c + 1; k < n; ++k) s -= M[static_cast<size_t>(c) * n + k] * v[static_cast<size_t>(k)];
    v[static_cast<size_t>(c)] = s / M[static_cast<size_t>(c) * n + c];
  }
  return true;
}

}  // namespace

int lp_solve(const std::vector<double>& A, int m, int n, const std::vector<double>& b, long max_pivots,
             std::vector<double>* x_out, long* pivots, std::string* detail) {
  *pivots = 0;
  // Equilibrate: columns to unit max, then rows to unit max; targets and
  // costs to unit max (positive factors change neither the feasible set nor
  // the minimiser).
  std::vector<double> sig(static_cast<size_t>(n), 1.0), rho(static_cast<size_t>(m), 1.0);
  for (int j = 0; j < n; ++j) {
    double mx = 0.0;
    for (int i = 0; i < m; ++i) mx = std::max(mx, std::fabs(A[static_cast<size_t>(i) * n + j]));
    if (mx > 0) sig[static_cast<size_t>(j)] = 1.0 / mx;
  }
  for (int i = 0; i < m; ++i) {
    double mx = 0.0;
    for (int j = 0; j < n; ++j) mx = std::max(mx, std::fabs(A[static_cast<size_t>(i) * n + j] * sig[static_cast<size_t>(j)]));
    if (mx > 0) rho[static_cast<size_t>(i)] = 1.0 / mx;
  }
  auto ahat = [&](int i, int j) {
    return rho[static_cast<size_t>(i)] * A[static_cast<size_t>(i) * n + j] * sig[static_cast<size_t>(j)];
  };
  double beta = 0.0, gamma = 0.0;
  for (int i = 0; i < m; ++i) beta = std::max(beta, std::fabs(rho[static_cast<size_t>(i)] * b[static_cast<size_t>(i)]));
  if (!(beta > 0)) beta = 1.0;
  std::vector<double> bhat(static_cast<size_t>(m)), chat(static_cast<size_t>(n), 0.0);
  for (int i = 0; i < m; ++i) bhat[static_cast<size_t>(i)] = rho[static_cast<size_t>(i)] * b[static_cast<size_t>(i)] / beta;
  for (int j = 0; j < n; ++j) {
    double c = 0.0;                                                    // Eq. 2.5 on the original matrix
    for (int i = 0; i < m; ++i) c += A[static_cast<size_t>(i) * n + j];
    chat[static_cast<size_t>(j)] = c * sig[static_cast<size_t>(j)];
    gamma = std::max(gamma, std::fabs(chat[static_cast<size_t>(j)]));
  }
  if (!(gamma > 0)) gamma = 1.0;
  for (double& c : chat) c /= gamma;

  // Dual tableau: row j is sum_i Ahat_ij y_i + t_j = chat_j; a row with
  // chat_j < 0 is negated and gets an artificial variable.
  int nart = 0;
  for (int j = 0; j < n; ++j) nart += chat[static_cast<size_t>(j)] < 0;
  Tableau tb;
  tb.rows = n;
  tb.width = m + n + nart;
  tb.T.assign(static_cast<size_t>(n) * (tb.width + 1), 0.0);
  tb.basis.assign(static_cast<size_t>(n), 0);
  for (int j = 0, a = 0; j < n; ++j) {
    const double s = chat[static_cast<size_t>(j)] < 0 ? -1.0 : 1.0;
    for (int i = 0; i < m; ++i) tb.at(j, i) = s * ahat(i, j);
    tb.at(j, m + j) = s;
    tb.at(j, tb.width) = s * chat[static_cast<size_t>(j)];
    if (s < 0) {
      tb.at(j, m + n + a) = 1.0;
      tb.basis[static_cast<size_t>(j)] = m + n + a++;
    } else {
      tb.basis[static_cast<size_t>(j)] = m + j;
    }
  }
  const double entries = static_cast<double>(n) * (tb.width + 1);
  const unsigned hc = std::thread::hardware_concurrency();
  RowPool pool(entries < 2e5 ? 1 : static_cast<int>(std::max(1u, std::min({hc, 16u, static_cast<unsigned>(n)}))));
  tb.pool = &pool;
  std::vector<double> cost(static_cast<size_t>(tb.width), 0.0);
  if (nart > 0) {                                                      // phase 1: maximise -sum(artificial)
    for (int a = 0; a < nart; ++a) cost[static_cast<size_t>(m + n + a)] = -1.0;
    tb.price(cost);
    const int st = run_simplex(&tb, tb.width, max_pivots, pivots);
    if (st == 2) {
      if (detail) *detail = "simplex pivot limit reached (phase 1)";
      return CMB3D_EUNSUPPORTED;
    }
    if (tb.z[static_cast<size_t>(tb.width)] < -1e-8) {
      if (detail) *detail = "linear program infeasible";
      return CMB3D_EINVAL;
    }
    for (int r = 0; r < n; ++r) {                                      // drive artificials at zero out
      if (tb.basis[static_cast<size_t>(r)] < m + n) continue;
      for (int c = 0; c < m + n; ++c)
        if (std::fabs(tb.at(r, c)) > kPivTol) {
          tb.pivot(r, c);
          ++*pivots;
          break;
        }
    }
    std::fill(cost.begin(), cost.end(), 0.0);
  }
  for (int i = 0; i < m; ++i) cost[static_cast<size_t>(i)] = bhat[static_cast<size_t>(i)];
  tb.price(cost);
  const int st = run_simplex(&tb, m + n, max_pivots, pivots);          // phase 2 (no artificial enters)
  if (st == 2) {
    if (detail) *detail = "simplex pivot limit reached";
    return CMB3D_EUNSUPPORTED;
  }
  if (st == 1) {
    if (detail) *detail = "dual unbounded: linear program infeasible";
    return CMB3D_EINVAL;
  }

  // Primal solution: the prices of the slack columns ...
  std::vector<double> xs(static_cast<size_t>(n));
  for (int j = 0; j < n; ++j) xs[static_cast<size_t>(j)] = tb.z[static_cast<size_t>(m + j)];
  // ... re-solved on the equilibrated data: the constraints of basic y are
  // tight and the unknowns of basic t are zero.
  std::vector<int> rows_e, cols_u;
  std::vector<char> tbasic(static_cast<size_t>(n), 0);
  bool art_left = false;
  for (int r = 0; r < n; ++r) {
    const int v = tb.basis[static_cast<size_t>(r)];
    if (v < m) rows_e.push_back(v);
    else if (v < m + n) tbasic[static_cast<size_t>(v - m)] = 1;
    else art_left = true;
  }
  for (int j = 0; j < n; ++j)
    if (!tbasic[static_cast<size_t>(j)]) cols_u.push_back(j);
  auto violation = [&](const std::vector<double>& x) {
    double v = 0.0;
    for (int j = 0; j < n; ++j) v = std::max(v, -x[static_cast<size_t>(j)]);
    for (int i = 0; i < m; ++i) {
      double s = 0.0;
      for (int j = 0; j < n; ++j) s += ahat(i, j) * x[static_cast<size_t>(j)];
      v = std::max(v, bhat[static_cast<size_t>(i)] - s);
    }
    return v;
  };
  if (!art_left && rows_e.size() == cols_u.size() && !rows_e.empty()) {
    const int k = static_cast<int>(rows_e.size());
    std::vector<double> M(static_cast<size_t>(k) * k), v(static_cast<size_t>(k));
    for (int a = 0; a < k; ++a) {
      for (int c = 0; c < k; ++c) M[static_cast<size_t>(a) * k + c] = ahat(rows_e[static_cast<size_t>(a)], cols_u[static_cast<size_t>(c)]);
      v[static_cast<size_t>(a)] = bhat[static_cast<size_t>(rows_e[static_cast<size_t>(a)])];
    }
    if (solve_dense(M, k, &v)) {
      std::vector<double> xr(static_cast<size_t>(n), 0.0);
      for (int c = 0; c < k; ++c) xr[static_cast<size_t>(cols_u[static_cast<size_t>(c)])] = v[static_cast<size_t>(c)];
      if (violation(xr) <= std::max(violation(xs), 1e-12)) xs.swap(xr);
    }
  }
  x_out->assign(static_cast<size_t>(n), 0.0);
  for (int j = 0; j < n; ++j)
    (*x_out)[static_cast<size_t>(j)] = std::max(0.0, xs[static_cast<size_t>(j)]) * sig[static_cast<size_t>(j)] * beta;
  return CMB3D_OK;
}

}  // namespace cmb3d

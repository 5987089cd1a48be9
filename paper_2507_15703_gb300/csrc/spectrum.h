// Host FP64 helpers for the box spectrum: P_inf(k) interpolation and the
// C_l -> P_inf(k) inversion of cmb3d_set_spectrum(CMB3D_SPEC_CL).
#pragma once

#include <string>
#include <vector>

namespace cmb3d {

// P_inf(k): linear in k between nodes, nodes' first value below the first
// node, zero above the last node.
double pk_interp(const std::vector<double>& k, const std::vector<double>& p, double x);

// Gauss-Legendre nodes and weights of order n on [-1, 1].
void gauss_legendre(int n, std::vector<double>* x, std::vector<double>* w);

// Fit P_inf >= 0 on nk uniform nodes of [0, sqrt(3) pi N / L] to the target
// C_l (relative least squares, Lawson-Hanson NNLS) using
// C_l = 16 pi^2 int k^2 P(k) j_l(k r)^2 dk.  Returns a CMB3D_* status; on
// success fills knodes, pnodes and the maximum relative C_l error.
int fit_pk_from_cl(const double* ell, const double* cl, int n, int N, double L, double r, int nk,
                   std::vector<double>* knodes, std::vector<double>* pnodes, double* max_rel_err,
                   std::string* detail);

// A[l][j] = 16 pi^2 int k^2 hat_j(k) j_l(k r)^2 dk on the hat basis of knodes,
// Gauss-Legendre with `nquad` points per node interval.  Row-major, n x nk.
std::vector<double> cl_design_matrix(const double* ell, int n, const std::vector<double>& knodes, double r,
                                     int nquad);

// Non-negative least squares min ||A x - b||^2 + ridge * mean(diag(A^T A)) ||x||^2,
// x >= 0: the active-set method of Lawson & Hanson (1974, Ch. 23) run on the
// normal equations (Bro & de Jong 1997), each passive subsystem solved by
// Cholesky (a candidate whose subsystem is not positive definite is skipped
// until x moves).  A is m x n row-major.  Returns the number of outer steps,
// or -1 on failure.
int nnls(const std::vector<double>& A, int m, int n, const std::vector<double>& b, double ridge,
         std::vector<double>* x);

// Symmetric square root S = V diag(sqrt(max(lambda, 0))) V^T of a symmetric
// n x n matrix (row-major, FP64), by cyclic Jacobi rotations to convergence
// (off-diagonal norm below 1e-15 of the Frobenius norm, or 100 sweeps).
void sqrt_symmetric(const double* a, int n, double* s);

// The 2-D Fourier method (paper Sec. II.D.2): for every q_perp = m_x^2 + m_y^2
// in [0, 2 (N/2)^2] that the half plane m_x in [0, N/2], m_y signed in
// (-N/2, N/2] reaches, the symmetric square root of the h x h covariance
//   Gamma_ij = xi(|i - j| dp),  xi(d dp) = sum_{m_z} P_box(m) cos(2 pi m_z d / M),
//   P_box(m) = P_inf(|k|) (2 pi / dp)^3 / (M N^2),  dp = L / N,
//   k = (2 pi m_x/(N dp), 2 pi m_y/(N dp), 2 pi m_z/(M dp)),  P_box(0) = 0
// (Eq. 2.11 with M != N), rounded to FP32: table[q][z][i], (2 (N/2)^2 + 1) x h x h.
// Unreached q_perp are left zero.  Runs on `threads` host threads.
void sqrt_gamma_table(int N, int M, int h, double L, const std::vector<double>& knodes,
                      const std::vector<double>& pnodes, int threads, std::vector<float>* table);

// ---- The linear-programming inversion of the paper (Sec. II.B) ----------
//
// Find P_inf >= 0 on uniform k nodes whose xi_inf (Eq. 2.4) matches the
// sphere's xi_sph (Eq. 2.1, C_l smoothed by exp(-b^2 l^2), Eq. 2.2) at the
// chords r_i = i dr (Eq. 2.3) up to the largest separation of the cap:
// minimise c^T x, c_j = sum_i A_ij (Eq. 2.5), subject to A x >= b, x >= 0.

struct LpGrid {
  double rmax = 0, dr = 0, dk = 0;  // largest chord, separation step, node step
  int m = 0;                        // constraints: r_i = i dr, i < m = floor(rmax/dr) + 1
  int n = 0;                        // unknowns: P at k_j = j dk, j < n = floor(kmax/dk); P(n dk) = 0
};

// The grid of a cap of polar half-angle theta_max on a sphere of radius R:
// rmax = 2 R sin(theta_max) (2 R beyond pi/2); dr = 0 selects beam / 5 and
// dk = 0 selects 2 pi / (3 rmax).  Returns a CMB3D_* status.
int lp_grid(double R, double theta_max, double beam, double dr, double dk, double kmax, LpGrid* g,
            std::string* detail);

// b_i = sum_l (2l+1) C_l exp(-beam^2 l^2) P_l(cos theta_i) / (4 pi) with
// cos theta_i = 1 - r_i^2 / (2 R^2); Legendre polynomials by recurrence.
void lp_targets(const double* ell, const double* cl, int nl, double beam, double R, const LpGrid& g,
                std::vector<double>* b);

// A_ij = 4 pi int k phi_j(k) sin(k r_i)/r_i dk (k^2 at r = 0) for the hat
// functions phi_j of the nodes, Gauss-Legendre with 16 points per node
// interval.  Row-major m x n, rows split over `threads` host threads.
void lp_matrix(const LpGrid& g, int threads, std::vector<double>* A);

// Solve min c^T x, c_j = sum_i A_ij, A x >= b, x >= 0 (A m x n row-major):
// a dense two-phase simplex on the dual problem (max b^T y, A^T y <= c,
// y >= 0; n rows), with equilibrated rows and columns, Dantzig pricing and
// Bland's rule after a run of degenerate pivots; the primal solution is read
// from the optimal basis and re-solved on the original data.  Returns a
// CMB3D_* status (CMB3D_EUNSUPPORTED if `max_pivots` is reached).
int lp_solve(const std::vector<double>& A, int m, int n, const std::vector<double>& b, long max_pivots,
             std::vector<double>* x, long* pivots, std::string* detail);

}  // namespace cmb3d

// Host FP64 helpers for the box spectrum: P_inf(k) interpolation and the
// C_l -> P_inf(k) inversion of cmb3d_set_spectrum(CMB3D_SPEC_CL).
#pragma once

#include <string>
#include <vector>

namespace cmb3d {

// P_inf(k): linear in k between nodes, nodes' first value below the first
// node, zero above the last node.
double pk_interp(const std::vector<double>& k, const std::vector<double>& p, double x);

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

}  // namespace cmb3d

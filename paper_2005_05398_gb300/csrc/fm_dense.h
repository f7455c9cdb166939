// Small dense and banded linear algebra on the host (row-major, float64).
//
// Used by the set-up of the tensor-trick preconditioner (the 1D generalized
// eigenproblems D(A1, A2) of Section 3.2, Eq. WW-scale; the banded y systems)
// and by the Ritz problems of the restarted Arnoldi driver.
#pragma once
#include <vector>

namespace fmh {

// LU with partial pivoting of the n x n matrix A (in place).  Returns false if singular.
bool lu_factor(int n, double* A, int* piv);
void lu_solve(int n, const double* LU, const int* piv, double* b);           // one right-hand side
bool invert(int n, const double* A, double* Ainv);                            // Ainv = A^{-1}

// Eigen-decomposition of a real matrix whose spectrum is real: A V = V diag(lam).
// Householder reduction to Hessenberg form, shifted QR (Wilkinson shifts) for the
// eigenvalues, inverse iteration on the Hessenberg matrix for the eigenvectors.
// Returns 0, or -1 when a complex pair (or no convergence) is met.  V columns have
// unit 2-norm.  lam is in no particular order.
int eig_real(int n, const double* A, double* lam, double* V);

// All eigenvalues (re, im) of a general real matrix, and unit eigenvectors for the
// real ones (zero columns for complex ones).  Returns 0, 1 (a complex eigenvalue
// occurred) or -1 (no convergence).
int eig_general(int n, const double* A, double* re, double* im, double* V);

// Eigenvalues (complex, as re/im) of a real upper-Hessenberg matrix (Francis double-shift QR).
// Returns 0 or -1 (no convergence).
int hess_eigvals(int n, const double* H, double* re, double* im);

// (W-bar, W, lambda) with W-bar A1 W = diag(lambda) and W-bar A2 W = I (Eq. WW-scale),
// eigenvalues ordered ascending (descending when 'descending').  Returns 0, -1 (complex
// spectrum) or -2 (singular A2 / W).
int decompose(int n, const double* A1, const double* A2, bool descending,
              double* Wbar, double* W, double* lam);

// Like decompose(), descending, for pencils that may have complex-conjugate eigenvalue pairs:
// a pair contributes two real columns, the real and imaginary parts of the eigenvector of the
// member with positive imaginary part, phased so that its coefficient 'top' is real positive
// (kind = 1 and 2; real eigenvalues kind = 0; lam = real parts; top < 0: the largest coefficient
// is made real positive).  W-bar = (A2 W)^{-1}, so
// W-bar A2 W = I and W-bar A1 W is block diagonal with 2x2 blocks for the pairs.
int decompose_pairs(int n, const double* A1, const double* A2, int top, double* Wbar, double* W, double* lam,
                    int* kind);

// All eigenvalues and unit eigenvectors (real and imaginary parts) of a general real matrix.
int eig_general2(int n, const double* A, double* re, double* im, double* Vr, double* Vi);

// Banded LU with partial pivoting (the row-swap form of LAPACK's gbtrf).  The matrix is
// given as a row-major band: row i holds columns i-kl .. i+ku+kl in B[i*(2kl+ku+1) + (j-i+kl)]
// (the last kl columns receive fill-in).  On return U(i, i+d) = B[i*w + kl + d] (d = 0..kl+ku),
// the multipliers L(j+r, j) are in Lmul[j*kl + r - 1] (r = 1..kl) and piv[j] is the row
// swapped with j.  Returns false if a pivot is zero.
bool band_lu(int n, int kl, int ku, double* B, double* Lmul, int* piv);
void band_solve(int n, int kl, int ku, const double* B, const double* Lmul, const int* piv, double* x);

}  // namespace fmh

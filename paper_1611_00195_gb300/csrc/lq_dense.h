// Host dense complex linear algebra used by the deflation-space eigensolver (lq_dense.cu).
#pragma once
#include <complex>

namespace lq {
// eigenvalues w[n] and unit eigenvectors (columns of V, row-major n x n; V may be null)
int dense_eig(int n, const std::complex<double>* A, std::complex<double>* w, std::complex<double>* V);
// Hermitian positive definite G = L L^H, L returned in place (lower, row-major)
int dense_cholesky(int n, std::complex<double>* G);
// in-place inverse (row-major)
int dense_inverse(int n, std::complex<double>* A);
}  // namespace lq

// Host-side linear algebra of the codec's PCA initialisation (see aew_pca.cpp).
#pragma once

namespace aew {

// All eigenpairs of the symmetric n x n matrix A (row-major, FP64): eigenvalues w[n]
// in descending order, eigenvectors as the columns of V (row-major n x n: V[i][j] is
// component i of eigenvector j).  Returns false if the QL iteration does not converge.
bool sym_eig(int n, const double* A, double* w, double* V);

// Weights (row-major, layer y -> y W + b) of the GELU autoencoder that computes the
// rank-k code mu + (y - mu) V_k V_k^T exactly; V as from sym_eig with leading dimension
// n_in, n_hid >= 2k (hidden units beyond 2k get zero weights).
void pca_pair_weights(int n_in, int n_hid, int k, const double* mu, const double* V,
                      float* W1, float* b1, float* W2, float* b2, float* W3, float* b3,
                      float* W4, float* b4);

}  // namespace aew

// Host-side linear algebra of the codec's PCA initialisation (Sec. 1: a linear
// autoencoder learns the principal subspace of its data), in FP64:
//
//  * sym_eig: all eigenpairs of a dense symmetric matrix.  Householder reduction to
//    tridiagonal form T = Q^T A Q, then the implicit-shift QL iteration on T (Bowdler,
//    Martin, Reinsch and Wilkinson, "The QR and QL algorithms for symmetric matrices",
//    Numer. Math. 11, 1968), with each iteration's plane rotations recorded and then
//    applied to the rows of the eigenvector matrix in parallel (rows are independent).
//  * pca_pair_weights: the weights of a GELU autoencoder n_in -> n_hid -> k -> n_hid ->
//    n_in that computes the rank-k affine code y -> mu + (y - mu) V V^T exactly, from
//    GELU(a) - GELU(-a) = a: hidden units j and k + j carry +a_j and -a_j.
#include "aew_pca.h"

#include <algorithm>
#include <cmath>
#include <limits>
#include <numeric>
#include <thread>
#include <vector>

namespace aew {
namespace {

// body(lo, hi) over [0, n) split across the hardware threads (serial for small n)
template <class F>
void parallel_for(int n, F body) {
  const unsigned hw = std::thread::hardware_concurrency();
  int nth = (int)std::min<unsigned>(hw ? hw : 1, 32);
  if (n < 256 || nth <= 1) {
    body(0, n);
    return;
  }
  nth = std::min(nth, n / 64);
  std::vector<std::thread> th;
  th.reserve(nth);
  for (int t = 0; t < nth; ++t) {
    const int lo = (int)((long long)n * t / nth), hi = (int)((long long)n * (t + 1) / nth);
    th.emplace_back([=] { body(lo, hi); });
  }
  for (auto& x : th) x.join();
}

struct Rot {
  int i;
  double c, s;
};

}  // namespace

bool sym_eig(int n, const double* A, double* w, double* V) {
  if (n < 1) return false;
  const size_t N = (size_t)n;
  std::vector<double> a(A, A + N * N);
  std::vector<double> Q(N * N, 0.0);   // row-major: Q[i][j]
  for (int i = 0; i < n; ++i) Q[(size_t)i * N + i] = 1.0;
  std::vector<double> d(N, 0.0), e(N, 0.0), v(N), p(N);

  // ---- Householder reduction: step k zeroes column k below the subdiagonal
  for (int k = 0; k + 2 < n; ++k) {
    const int lo = k + 1, m = n - lo;
    double sig = 0.0;
    for (int i = lo; i < n; ++i) sig += a[(size_t)i * N + k] * a[(size_t)i * N + k];
    sig = std::sqrt(sig);
    if (sig == 0.0) {
      e[k] = 0.0;
      continue;
    }
    const double x0 = a[(size_t)lo * N + k];
    const double alpha = x0 > 0 ? -sig : sig;
    double vn = 0.0;
    for (int i = 0; i < m; ++i) {
      v[i] = a[(size_t)(lo + i) * N + k] - (i == 0 ? alpha : 0.0);
      vn += v[i] * v[i];
    }
    vn = std::sqrt(vn);
    for (int i = 0; i < m; ++i) v[i] /= vn;
    e[k] = alpha;
    // p = A22 v, then q = p - (v.p) v, A22 -= 2 (v q^T + q v^T)
    parallel_for(m, [&](int r0, int r1) {
      for (int i = r0; i < r1; ++i) {
        const double* row = &a[(size_t)(lo + i) * N + lo];
        double s = 0.0;
        for (int j = 0; j < m; ++j) s += row[j] * v[j];
        p[i] = s;
      }
    });
    double K = 0.0;
    for (int i = 0; i < m; ++i) K += v[i] * p[i];
    for (int i = 0; i < m; ++i) p[i] -= K * v[i];
    parallel_for(m, [&](int r0, int r1) {
      for (int i = r0; i < r1; ++i) {
        double* row = &a[(size_t)(lo + i) * N + lo];
        const double vi = v[i], pi = p[i];
        for (int j = 0; j < m; ++j) row[j] -= 2.0 * (vi * p[j] + pi * v[j]);
      }
    });
    // Q <- Q H_k = Q - 2 (Q v) v^T on columns lo..n-1
    parallel_for(n, [&](int r0, int r1) {
      for (int i = r0; i < r1; ++i) {
        double* row = &Q[(size_t)i * N + lo];
        double s = 0.0;
        for (int j = 0; j < m; ++j) s += row[j] * v[j];
        s *= 2.0;
        for (int j = 0; j < m; ++j) row[j] -= s * v[j];
      }
    });
  }
  for (int k = 0; k < n; ++k) d[k] = a[(size_t)k * N + k];
  if (n >= 2) e[n - 2] = a[(size_t)(n - 1) * N + (n - 2)];
  e[n - 1] = 0.0;

  // ---- implicit-shift QL on the tridiagonal (d, e), e[i] coupling d[i] and d[i+1]
  std::vector<Rot> rots;
  rots.reserve(N);
  const double eps = std::numeric_limits<double>::epsilon();
  for (int l = 0; l < n; ++l) {
    for (int iter = 0;; ++iter) {
      int m = l;
      for (; m < n - 1; ++m) {
        const double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
        if (std::fabs(e[m]) <= eps * dd) break;
      }
      if (m == l) break;
      if (iter >= 100) return false;
      // Wilkinson-type shift from the leading 2 x 2 block
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = std::hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
      double s = 1.0, c = 1.0, pp = 0.0;
      bool deflated = false;
      rots.clear();
      for (int i = m - 1; i >= l; --i) {
        const double f = s * e[i], b = c * e[i];
        r = std::hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {   // an underflowed coupling: split here and restart
          d[i + 1] -= pp;
          e[m] = 0.0;
          deflated = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - pp;
        r = (d[i] - g) * s + 2.0 * c * b;
        pp = s * r;
        d[i + 1] = g + pp;
        g = c * r - b;
        rots.push_back({i, c, s});
      }
      // eigenvectors: Z[:, i], Z[:, i+1] rotated, in the order the rotations were made
      if (!rots.empty()) {
        parallel_for(n, [&](int r0, int r1) {
          for (int row = r0; row < r1; ++row) {
            double* z = &Q[(size_t)row * N];
            for (const Rot& q : rots) {
              const double f = z[q.i + 1];
              z[q.i + 1] = q.s * z[q.i] + q.c * f;
              z[q.i] = q.c * z[q.i] - q.s * f;
            }
          }
        });
      }
      if (deflated) continue;
      d[l] -= pp;
      e[l] = g;
      e[m] = 0.0;
    }
  }

  // ---- sort descending
  std::vector<int> idx(N);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return d[x] > d[y]; });
  for (int j = 0; j < n; ++j) {
    w[j] = d[idx[j]];
    for (int i = 0; i < n; ++i) V[(size_t)i * N + j] = Q[(size_t)i * N + idx[j]];
  }
  return true;
}

void pca_pair_weights(int n_in, int n_hid, int k, const double* mu, const double* V,
                      float* W1, float* b1, float* W2, float* b2, float* W3, float* b3,
                      float* W4, float* b4) {
  const size_t NI = (size_t)n_in, NH = (size_t)n_hid, K = (size_t)k;
  std::fill(W1, W1 + NI * NH, 0.f);
  std::fill(b1, b1 + NH, 0.f);
  std::fill(W2, W2 + NH * K, 0.f);
  std::fill(b2, b2 + K, 0.f);
  std::fill(W3, W3 + K * NH, 0.f);
  std::fill(b3, b3 + NH, 0.f);
  std::fill(W4, W4 + NH * NI, 0.f);
  for (int j = 0; j < k; ++j) {
    double muv = 0.0;
    for (int i = 0; i < n_in; ++i) {
      const double vij = V[(size_t)i * NI + j];   // component i of eigenvector j
      muv += mu[i] * vij;
      W1[(size_t)i * NH + j] = (float)vij;
      W1[(size_t)i * NH + k + j] = (float)-vij;
      W4[(size_t)j * NI + i] = (float)vij;
      W4[(size_t)(k + j) * NI + i] = (float)-vij;
    }
    b1[j] = (float)-muv;
    b1[k + j] = (float)muv;
    W2[(size_t)j * K + j] = 1.f;
    W2[(size_t)(k + j) * K + j] = -1.f;
    W3[(size_t)j * NH + j] = 1.f;
    W3[(size_t)j * NH + k + j] = -1.f;
  }
  for (int i = 0; i < n_in; ++i) b4[i] = (float)mu[i];
}

}  // namespace aew

// Host-side lattice set-up: hopping matrix of Eq. 3 on the periodic square or honeycomb lattice and
// e^{cK} by a cyclic Jacobi eigensolver (no LAPACK in the build).
#include <cmath>
#include <vector>

namespace nmc_host {

// K_ij = -t for nearest neighbours, set once per pair (so a length-2 direction has one bond
// and a length-1 direction none).
// lattice 0: periodic Lx x Ly square lattice, i = x + Lx*y.
// lattice 1: periodic honeycomb of Lx x Ly cells with two sites each, i = 2 (x + Lx*y) + sub;
//            the A site (sub 0) of cell (x,y) bonds to the B sites (sub 1) of cells (x,y),
//            (x-1,y) and (x,y-1).
void hopping(int lattice, int Lx, int Ly, double t, std::vector<double>& K) {
  const int N = Lx * Ly * (lattice == 1 ? 2 : 1);
  K.assign((size_t)N * N, 0.0);
  if (lattice == 1) {
    for (int y = 0; y < Ly; ++y)
      for (int x = 0; x < Lx; ++x) {
        const int a = 2 * (x + Lx * y);
        const int bx[3] = {x, (x + Lx - 1) % Lx, x}, by[3] = {y, y, (y + Ly - 1) % Ly};
        for (int d = 0; d < 3; ++d) {
          const int b = 2 * (bx[d] + Lx * by[d]) + 1;
          K[(size_t)a * N + b] = -t;
          K[(size_t)b * N + a] = -t;
        }
      }
    return;
  }
  const int dx[4] = {1, -1, 0, 0}, dy[4] = {0, 0, 1, -1};
  for (int y = 0; y < Ly; ++y)
    for (int x = 0; x < Lx; ++x) {
      const int i = x + Lx * y;
      for (int d = 0; d < 4; ++d) {
        const int j = ((x + dx[d]) % Lx + Lx) % Lx + Lx * (((y + dy[d]) % Ly + Ly) % Ly);
        if (j != i) K[(size_t)i * N + j] = -t;
      }
    }
}

// Cyclic Jacobi for a symmetric matrix A (n x n, row-major; destroyed).
// On return w holds the eigenvalues and V (row-major) the eigenvectors as columns.
// Rotation per (p,q): tau = (a_qq - a_pp)/(2 a_pq), t = sign(tau)/(|tau| + sqrt(1+tau^2)),
// c = 1/sqrt(1+t^2), s = t c; A <- J^T A J zeroes a_pq (Golub & Van Loan, Sec. 8.5).
void jacobi_eigh(int n, std::vector<double>& A, std::vector<double>& w, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  auto a = [&](int r, int c) -> double& { return A[(size_t)r * n + c]; };
  double total = 0.0;
  for (double v : A) total += v * v;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += a(p, q) * a(p, q);
    if (off <= 1e-32 * total || off == 0.0) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a(p, q);
        if (apq == 0.0) continue;
        const double tau = (a(q, q) - a(p, p)) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double akp = a(k, p), akq = a(k, q);
          a(k, p) = c * akp - s * akq;
          a(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = a(p, k), aqk = a(q, k);
          a(p, k) = c * apk - s * aqk;
          a(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = a(i, i);
}

// out = V diag(e^{c w}) V^T
void expk_from_eig(int n, const std::vector<double>& w, const std::vector<double>& V, double c,
                   std::vector<double>& out) {
  out.assign((size_t)n * n, 0.0);
  std::vector<double> ew(n);
  for (int k = 0; k < n; ++k) ew[k] = std::exp(c * w[k]);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += V[(size_t)i * n + k] * ew[k] * V[(size_t)j * n + k];
      out[(size_t)i * n + j] = s;
    }
}

}  // namespace nmc_host

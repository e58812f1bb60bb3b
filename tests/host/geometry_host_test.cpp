// Host driver for the library's metric terms (the geometry precompute of
// Sec. 2: contravariant metrics Ja^i in the 2D cross-product and 3D
// invariant-curl forms, and the Jacobian J), as build_level computes them
// before they are uploaded.  Needs no GPU.
//
// Input (stdin): dim K M; the mapping nodes, K x (M+1)^dim x 3 doubles as
// hexadecimal floats; the orders, K x 3.  Output: per element and Gauss node
// the 9 values of Ja[i][c] and J, as hexadecimal floats.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_1806_11456_gb300/csrc/dg_internal.h"

int main() {
  int dim = 0, K = 0, M = 0;
  if (std::scanf("%d %d %d", &dim, &K, &M) != 3 || K < 1) return 2;
  const int npe = dim == 3 ? (M + 1) * (M + 1) * (M + 1) : (M + 1) * (M + 1);
  std::vector<double> X((size_t)K * npe * 3);
  char buf[64];
  for (auto& v : X) {
    if (std::scanf("%63s", buf) != 1) return 2;
    v = std::strtod(buf, nullptr);
  }
  std::vector<int> ord((size_t)K * 3);
  for (auto& v : ord)
    if (std::scanf("%d", &v) != 1) return 2;
  for (int e = 0; e < K; ++e) {
    int n[3] = {ord[e * 3] + 1, ord[e * 3 + 1] + 1, dim == 3 ? ord[e * 3 + 2] + 1 : 1};
    const int nn = n[0] * n[1] * n[2];
    std::vector<double> Ja((size_t)nn * 9), J(nn);
    dg::element_geometry_host(M, dim, X.data() + (size_t)e * npe * 3, n, Ja.data(), J.data());
    for (int nd = 0; nd < nn; ++nd) {
      for (int c = 0; c < 9; ++c) std::printf("%a ", Ja[nd * 9 + c]);
      std::printf("%a\n", J[nd]);
    }
  }
  return 0;
}

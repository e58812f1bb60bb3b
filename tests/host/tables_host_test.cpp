// Host driver for the library's 1-D tables (Gauss nodes and weights, the
// collocation and weak-form derivative matrices, the Lagrange basis at -1 and
// +1) and its transfer matrices between node counts (L2 projection down,
// interpolation up), as built once per process and uploaded to the GPU.
// Needs no GPU.  Output: one line per table, "name n [m] values..." with the
// values as hexadecimal floats.
#include <cstdio>
#include <vector>

#include "../../paper_1806_11456_gb300/csrc/dg_internal.h"

int main() {
  const dg::Tables1D& T = dg::tables();
  for (int n = 1; n < dg::kNP; ++n) {
    std::printf("x %d", n);
    for (int i = 0; i < n; ++i) std::printf(" %a", T.x[n][i]);
    std::printf("\nw %d", n);
    for (int i = 0; i < n; ++i) std::printf(" %a", T.w[n][i]);
    std::printf("\nD %d", n);
    for (int i = 0; i < n; ++i)
      for (int a = 0; a < n; ++a) std::printf(" %a", T.D[n][i][a]);
    std::printf("\nDhat %d", n);
    for (int i = 0; i < n; ++i)
      for (int a = 0; a < n; ++a) std::printf(" %a", T.Dhat[n][i][a]);
    std::printf("\nlm %d", n);
    for (int i = 0; i < n; ++i) std::printf(" %a", T.lm[n][i]);
    std::printf("\nlp %d", n);
    for (int i = 0; i < n; ++i) std::printf(" %a", T.lp[n][i]);
    std::printf("\n");
  }
  std::vector<double> M((size_t)dg::kNP * dg::kNP);
  for (int nf = 1; nf < dg::kNP; ++nf)
    for (int nt = 1; nt < dg::kNP; ++nt) {
      dg::transfer_matrix(nf, nt, M.data());
      std::printf("T %d %d", nf, nt);
      for (int k = 0; k < nt * nf; ++k) std::printf(" %a", M[k]);
      std::printf("\n");
    }
  return 0;
}

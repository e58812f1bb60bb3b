// Host driver for the library's order adaptation (dg_adapt: the per-element
// order selection of Sec. 3.3.2 and the order-jump fix-point of Secs. 4.1.2 /
// 4.2.1), which runs entirely on the host.  It builds a mesh handle holding
// only the host fields dg_adapt reads (dimension, element count, face table,
// reference orders), so no device memory and no GPU are needed.
//
// Input (stdin, whitespace separated): dim K; the face table, K x 6 x 4
// int32 (neighbour, neighbour face, orientation, boundary tag); the
// reference orders, K x 3; tau_max n_min n_max cap jump_rule conform_tag;
// the tau table, K x 3 x 16 doubles written as hexadecimal floats (exact).
// Output (stdout): the new orders, K x 3, or "error <message>".
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_1806_11456_gb300/csrc/dg_internal.h"

int main() {
  int dim = 0, K = 0;
  if (std::scanf("%d %d", &dim, &K) != 2 || K < 1) return 2;
  dg_mesh m;
  m.dim = dim;
  m.K = K;
  m.ftab.resize((size_t)K * 6 * 4);
  for (auto& v : m.ftab)
    if (std::scanf("%d", &v) != 1) return 2;
  m.orders.resize((size_t)K * 3);
  for (auto& v : m.orders)
    if (std::scanf("%d", &v) != 1) return 2;
  dg_adapt_params ap{};
  char buf[64];
  if (std::scanf("%63s %d %d %d %d %d", buf, &ap.n_min, &ap.n_max, &ap.cap, &ap.jump_rule, &ap.conform_tag) != 6)
    return 2;
  ap.tau_max = std::strtod(buf, nullptr);
  std::vector<double> tau((size_t)K * 3 * 16);
  for (auto& v : tau) {
    if (std::scanf("%63s", buf) != 1) return 2;
    v = std::strtod(buf, nullptr);
  }
  std::vector<int32_t> out((size_t)K * 3);
  if (dg_adapt(&m, tau.data(), &ap, out.data()) != DG_OK) {
    std::printf("error %s\n", dg_last_error());
    return 0;
  }
  for (int32_t v : out) std::printf("%d\n", v);
  return 0;
}

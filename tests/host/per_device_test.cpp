// Host unit test of the per-device bookkeeping (PerDevice in dg_internal.h):
// each device index has its own entry, state set for one device is not seen
// by another, and indexes outside [0, kMax) are refused.  Needs no GPU.
#include <cstdio>

#include "../../paper_1806_11456_gb300/csrc/dg_internal.h"

struct Entry {
  void* table = nullptr;
  bool ready = false;
};

int main() {
  dg::PerDevice<Entry> pd;
  int fails = 0;
  auto check = [&](bool c, const char* what) {
    if (!c) {
      std::printf("FAIL: %s\n", what);
      ++fails;
    }
  };
  for (int d = 0; d < dg::PerDevice<Entry>::kMax; ++d) check(pd.get(d) && !pd.get(d)->ready, "starts unset");
  static int t0 = 0, t1 = 0;
  pd.get(0)->table = &t0;
  pd.get(0)->ready = true;
  check(!pd.get(1)->ready && pd.get(1)->table == nullptr, "device 1 does not see device 0's entry");
  pd.get(1)->table = &t1;
  pd.get(1)->ready = true;
  check(pd.get(0)->table == &t0 && pd.get(1)->table == &t1, "entries stay distinct");
  check(pd.get(0) != pd.get(1), "distinct storage");
  check(pd.get(-1) == nullptr && pd.get(dg::PerDevice<Entry>::kMax) == nullptr, "out-of-range index refused");
  if (fails == 0) std::printf("per-device bookkeeping ok\n");
  return fails == 0 ? 0 : 1;
}

// Instantiates the fused solver for one column length L2 = BCCB_L2 and every row
// length L1 in {16, 32, 64, 128, 256}; the build compiles this file once per L2.
#include "solver.h"

#ifndef BCCB_L2
#error "compile with -DBCCB_L2=<16|32|64|128|256>"
#endif

#define BCCB_CAT2(a, b) a##b
#define BCCB_CAT(a, b) BCCB_CAT2(a, b)

namespace bccb {

const FusedEntry* BCCB_CAT(fused_lookup_L2_, BCCB_L2)(int L1, bool admm) {
  static const FusedEntry table[] = {
      fused_entry<16, BCCB_L2, false>(),  fused_entry<16, BCCB_L2, true>(),
      fused_entry<32, BCCB_L2, false>(),  fused_entry<32, BCCB_L2, true>(),
      fused_entry<64, BCCB_L2, false>(),  fused_entry<64, BCCB_L2, true>(),
      fused_entry<128, BCCB_L2, false>(), fused_entry<128, BCCB_L2, true>(),
      fused_entry<256, BCCB_L2, false>(), fused_entry<256, BCCB_L2, true>(),
  };
  for (const FusedEntry& e : table)
    if (e.L1 == L1 && e.admm == (admm ? 1 : 0)) return &e;
  return nullptr;
}

}  // namespace bccb

// Instantiates the fused solver for one column length L2 = BCCB_L2 and every row
// length L1 in {16, 32, 64, 128, 256}, with the 8192-element tile and, for grids of
// at least 8192 elements, the 4096-element tile (twice the CTAs per cluster); the
// build compiles this file once per L2.
#include "adjoint.cuh"
#include "solver.h"

#ifndef BCCB_L2
#error "compile with -DBCCB_L2=<16|32|64|128|256>"
#endif

#define BCCB_CAT2(a, b) a##b
#define BCCB_CAT(a, b) BCCB_CAT2(a, b)

namespace bccb {

#define BCCB_ENTRIES(L1)                                                            \
  fused_entry<L1, BCCB_L2, false>(), fused_entry<L1, BCCB_L2, true>()
#define BCCB_ENTRIES_HALF(L1)                                                       \
  fused_entry<L1, BCCB_L2, false, 4096>(), fused_entry<L1, BCCB_L2, true, 4096>()
// ISTA/FISTA on the circulant embedding of a Toeplitz Gram (both sides >= 32)
#define BCCB_BLOCK(L1) fused_entry<L1, BCCB_L2, false, kFusedTileElems, false, true>()
#define BCCB_BLOCK_HALF(L1) fused_entry<L1, BCCB_L2, false, 4096, false, true>()

// ISTA/FISTA with the state outside shared memory: rows of 256, 8192 elements per CTA, two CTAs
// per SM (needs at least 32 rows)
#define BCCB_SPARSE(L1) fused_entry<L1, BCCB_L2, false, kFusedTileElems, false, false, true>()

const FusedEntry* BCCB_CAT(fused_lookup_L2_, BCCB_L2)(int L1, bool admm, int tile, bool block, bool sparse) {
  static const FusedEntry table[] = {
      BCCB_ENTRIES(16), BCCB_ENTRIES(32), BCCB_ENTRIES(64), BCCB_ENTRIES(128), BCCB_ENTRIES(256),
#if BCCB_L2 >= 32
      BCCB_ENTRIES_HALF(256),
#endif
#if BCCB_L2 >= 64
      BCCB_ENTRIES_HALF(128),
#endif
#if BCCB_L2 >= 128
      BCCB_ENTRIES_HALF(64),
#endif
#if BCCB_L2 >= 256
      BCCB_ENTRIES_HALF(32),
#endif
#if BCCB_L2 >= 32
      BCCB_BLOCK(32), BCCB_BLOCK(64), BCCB_BLOCK(128), BCCB_BLOCK(256), BCCB_BLOCK_HALF(256),
#endif
#if BCCB_L2 >= 64
      BCCB_BLOCK_HALF(128),
#endif
#if BCCB_L2 >= 128
      BCCB_BLOCK_HALF(64),
#endif
#if BCCB_L2 >= 256
      BCCB_BLOCK_HALF(32),
#endif
#if BCCB_L2 >= 32
      BCCB_SPARSE(256),
#endif
  };
  for (const FusedEntry& e : table)
    if (e.L1 == L1 && e.admm == (admm ? 1 : 0) && e.tile == tile && e.block == (block ? 1 : 0) &&
        e.sparse == (sparse ? 1 : 0))
      return &e;
  return nullptr;
}

// forward pass of the unrolled network (per-layer multipliers, saved layer inputs): square grids
const FusedEntry* BCCB_CAT(learned_lookup_L2_, BCCB_L2)(int L1) {
  static const FusedEntry e = fused_entry<BCCB_L2, BCCB_L2, false, kFusedTileElems, true>();
  return L1 == BCCB_L2 ? &e : nullptr;
}

const AdjointEntry* BCCB_CAT(adjoint_lookup_L2_, BCCB_L2)(int L1) {
  static const AdjointEntry table[] = {adjoint_entry<16, BCCB_L2>(), adjoint_entry<32, BCCB_L2>(),
                                       adjoint_entry<64, BCCB_L2>(), adjoint_entry<128, BCCB_L2>(),
                                       adjoint_entry<256, BCCB_L2>()};
  for (const AdjointEntry& e : table)
    if (e.L1 == L1) return &e;
  return nullptr;
}

}  // namespace bccb

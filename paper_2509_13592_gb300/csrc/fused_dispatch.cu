// Maps a grid shape (L1, L2) and algorithm family to its fused-kernel launcher.
#include "solver.h"

namespace bccb {

const FusedEntry* fused_lookup_L2_16(int L1, bool admm, int tile, bool block, bool sparse);
const FusedEntry* fused_lookup_L2_32(int L1, bool admm, int tile, bool block, bool sparse);
const FusedEntry* fused_lookup_L2_64(int L1, bool admm, int tile, bool block, bool sparse);
const FusedEntry* fused_lookup_L2_128(int L1, bool admm, int tile, bool block, bool sparse);
const FusedEntry* fused_lookup_L2_256(int L1, bool admm, int tile, bool block, bool sparse);

const AdjointEntry* adjoint_lookup_L2_16(int L1);
const AdjointEntry* adjoint_lookup_L2_32(int L1);
const AdjointEntry* adjoint_lookup_L2_64(int L1);
const AdjointEntry* adjoint_lookup_L2_128(int L1);
const AdjointEntry* adjoint_lookup_L2_256(int L1);

const FusedEntry* learned_lookup_L2_16(int L1);
const FusedEntry* learned_lookup_L2_32(int L1);
const FusedEntry* learned_lookup_L2_64(int L1);
const FusedEntry* learned_lookup_L2_128(int L1);
const FusedEntry* learned_lookup_L2_256(int L1);

const FusedEntry* learned_lookup(int L1, int L2) {
  switch (L2) {
    case 16: return learned_lookup_L2_16(L1);
    case 32: return learned_lookup_L2_32(L1);
    case 64: return learned_lookup_L2_64(L1);
    case 128: return learned_lookup_L2_128(L1);
    case 256: return learned_lookup_L2_256(L1);
    default: return nullptr;
  }
}

const AdjointEntry* adjoint_lookup(int L1, int L2) {
  switch (L2) {
    case 16: return adjoint_lookup_L2_16(L1);
    case 32: return adjoint_lookup_L2_32(L1);
    case 64: return adjoint_lookup_L2_64(L1);
    case 128: return adjoint_lookup_L2_128(L1);
    case 256: return adjoint_lookup_L2_256(L1);
    default: return nullptr;
  }
}

const FusedEntry* fused_lookup(int L1, int L2, bool admm, int tile, bool block, bool sparse) {
  if (tile == 0) tile = kFusedTileElems;
  switch (L2) {
    case 16: return fused_lookup_L2_16(L1, admm, tile, block, sparse);
    case 32: return fused_lookup_L2_32(L1, admm, tile, block, sparse);
    case 64: return fused_lookup_L2_64(L1, admm, tile, block, sparse);
    case 128: return fused_lookup_L2_128(L1, admm, tile, block, sparse);
    case 256: return fused_lookup_L2_256(L1, admm, tile, block, sparse);
    default: return nullptr;
  }
}

}  // namespace bccb

// Shared-memory layout of a K-major bf16 operand tile of tcgen05.mma without swizzle, as the
// field kernels stage it (plain C++: the host tests check it). A tile is R rows by 16 k
// (8 features, k = 2 f + 0 for Re and 2 f + 1 for Im, one bf16 pair per (row, feature));
// core matrices of 8 rows by 8 k are 128 contiguous bytes (row r % 8 at byte 16 (r % 8)),
// the two core matrices of a row group lie 128 bytes apart along K (the descriptor's leading
// byte offset) and successive row groups 256 bytes apart (its stride byte offset).
#pragma once

namespace mlmc {
namespace umma {

constexpr int kLeadingBytes = 128;  // core matrices adjacent along K
constexpr int kStrideBytes = 256;   // core matrices adjacent along M / N (8-row groups)

// Byte offset of the bf16 pair of (row r, feature f) in a tile, 0 <= f < 8.
#if defined(__CUDACC__)
__host__ __device__
#endif
constexpr int pair_offset(int r, int f) {
  return (r >> 3) * kStrideBytes + (f >> 2) * kLeadingBytes + (r & 7) * 16 + (f & 3) * 4;
}

}  // namespace umma
}  // namespace mlmc

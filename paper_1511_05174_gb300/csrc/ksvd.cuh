// Internal declarations of the K-SVD sweep's launch configuration (not part of the ABI).
#pragma once

namespace csp {
// Ranks of the sweep's cluster for dimension M, T atoms and the update method
// (approx: the approximate update, whose M <= 192 configuration differs).
int ksvd_owner_split(int M, int T, bool approx);
}  // namespace csp

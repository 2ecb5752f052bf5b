// float instantiation of the block-parallel velocity sweep (ugks_blocked.cuh).
#include "ugks_blocked.cuh"

namespace ugks {
UGKS_INSTANTIATE_BLOCKED(float)
}  // namespace ugks

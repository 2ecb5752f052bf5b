// FP32 arithmetic with __half scaled storage of f (ugks_blocked.cuh, ugks_store.cuh).
#include "ugks_blocked.cuh"

namespace ugks {
UGKS_INSTANTIATE_SCALED(__half)
}  // namespace ugks

// Dslash instantiations for __nv_bfloat16 storage (one translation unit per precision
// so that the library compiles in parallel).
#include "dslash.cuh"

namespace tml {
TM_INSTANTIATE_DSLASH(__nv_bfloat16)
TM_INSTANTIATE_DSLASH_MMA(__nv_bfloat16)
}  // namespace tml

// Dslash instantiations for __half storage (one translation unit per precision
// so that the library compiles in parallel).
#include "dslash.cuh"

namespace tml {
TM_INSTANTIATE_DSLASH(__half)
TM_INSTANTIATE_DSLASH_MMA(__half)
}  // namespace tml

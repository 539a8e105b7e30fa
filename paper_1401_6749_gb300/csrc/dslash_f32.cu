// Dslash instantiations for float storage (one translation unit per precision
// so that the library compiles in parallel).
#include "dslash.cuh"

namespace tml {
TM_INSTANTIATE_DSLASH(float)
}  // namespace tml

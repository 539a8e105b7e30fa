// Dslash instantiation for float-float storage and arithmetic (18-real links:
// the operator in about 48-bit precision on the FP32 pipes).
#include "dslash.cuh"

namespace tml {
template tm_status_t dslash_launch<FFloat, 18>(const tm_op*, const DslashCall&, cudaStream_t);
}  // namespace tml

// Dslash instantiation for double storage (18-real links only: FP64 is
// arithmetic-bound on this GPU, so the link is not compressed).
#include "dslash.cuh"

namespace tml {
template tm_status_t dslash_launch<double, 18>(const tm_op*, const DslashCall&, cudaStream_t);
}  // namespace tml

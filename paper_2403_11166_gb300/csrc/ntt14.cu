// Instantiates the fused NTT / INTT kernels for N = 2^14 (Shoup / Harvey butterflies).
#include "ntt.cuh"
namespace pencil {
PENCIL_NTT_INSTANTIATE(, 14, false)
}  // namespace pencil

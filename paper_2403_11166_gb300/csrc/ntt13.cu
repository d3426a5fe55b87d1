// Instantiates the fused NTT / INTT kernels for N = 2^13 (Shoup / Harvey butterflies).
#include "ntt.cuh"
namespace pencil {
PENCIL_NTT_INSTANTIATE(, 13, false)
}  // namespace pencil

// Instantiates the fused NTT / INTT kernels for N = 2^13 (pseudo-Mersenne fold butterflies).
#include "ntt.cuh"
namespace pencil {
PENCIL_NTT_INSTANTIATE(, 13, true)
}  // namespace pencil

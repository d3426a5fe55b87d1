// Instantiates the fused NTT / INTT kernels for N = 2^12 (pseudo-Mersenne fold butterflies).
#include "ntt.cuh"
namespace pencil {
PENCIL_NTT_INSTANTIATE(, 12, true)
}  // namespace pencil

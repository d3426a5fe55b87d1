// Instantiates the fused NTT / INTT kernels for N = 2^14 (pseudo-Mersenne fold butterflies).
#include "ntt.cuh"
namespace pencil {
PENCIL_NTT_INSTANTIATE(, 14, true)
}  // namespace pencil

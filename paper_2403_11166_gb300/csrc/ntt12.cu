// Instantiates the fused NTT / INTT kernels for N = 2^12 (Shoup / Harvey butterflies).
#include "ntt.cuh"
namespace pencil {
PENCIL_NTT_INSTANTIATE(, 12, false)
}  // namespace pencil

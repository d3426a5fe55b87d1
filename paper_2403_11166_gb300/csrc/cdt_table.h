// Generated by gen_cdt.py: floor(2^63 * P(|E| <= j)) for the discrete Gaussian
// with sigma = 3.2 on [-19, 19].  Do not edit.
#pragma once
#include <stdint.h>
#define PENCIL_CDT_LEN 19
static const uint64_t kPencilCdt[PENCIL_CDT_LEN] = {
    0x0ff52b40a5917f1dull,
    0x2e5a25d4bf0e400eull,
    0x489ae26955b04bd6ull,
    0x5d2bc20f621bf185ull,
    0x6bc8694c3cc80ff4ull,
    0x7532d89ac6ba7dceull,
    0x7ab396cb74436798ull,
    0x7d9e4e916643eb07ull,
    0x7f05495819eb2051ull,
    0x7fa1ce9c0039a957ull,
    0x7fdfb3f212e8c4e8ull,
    0x7ff5e6f9d2314fccull,
    0x7ffd1f97bc4406a2ull,
    0x7fff40fa0088d11dull,
    0x7fffd2e835e1c57dull,
    0x7ffff6524386ff1eull,
    0x7ffffe1db4769da5ull,
    0x7fffffac0a1dcb08ull,
    0x7ffffff428673853ull,
};

// Table of the entropy filter with the cube's own grey-level probabilities
// (LNF_ENTROPY_LOCAL; the information entropy of the kernel, paper section
// "Related Work").  With c_g of the m cube voxels at grey level g, the cube's
// first order entropy is H = log2 m - (1/m) sum_g c_g log2 c_g, so
//   m 2^22 H = t[m] - sum_g t[c_g],   t[c] = round(2^22 c log2 c),
// and the filter keeps P0 iff that exceeds m theta.  The table depends only on
// the cube size; it is built here once per context, on the host, and read by
// the kernels from device memory.
//
// log2 is taken with 40 fractional bits by the classical repeated-squaring
// method (x = 2^k m, m in [1, 2) held with 62 fractional bits; each square,
// truncated to 62 fractional bits, that reaches 2 yields a 1 bit and is
// halved), the method the entropy filter's weights (Eq. 7) use; t[c] rounds
// c log2 c half up from 40 to 22 fractional bits.
#include "lnf_ctx.h"

#include <vector>

namespace {

unsigned long long log2_fixed40_host(unsigned long long x)
{
    int k = 63;
    while (!((x >> k) & 1ull))
        --k;
    unsigned long long m = k <= 62 ? (x << (62 - k)) : (x >> (k - 62));
    unsigned long long res = (unsigned long long)k << 40;
    for (int i = 1; i <= 40; ++i) {
        m = (unsigned long long)(((unsigned __int128)m * m) >> 62);
        if (m >= (1ull << 63)) {
            m >>= 1;
            res |= 1ull << (40 - i);
        }
    }
    return res;
}

}  // namespace

lnf_status lnf_lt_upload(lnf_ctx *ctx)
{
    std::vector<unsigned long long> t(LNF_LT_MAX + 1, 0ull);
    for (unsigned long long c = 2; c <= LNF_LT_MAX; ++c)
        t[c] = (c * log2_fixed40_host(c) + (1ull << 17)) >> 18;
    if (cudaMalloc(&ctx->d_lt, sizeof(unsigned long long) * t.size()) != cudaSuccess)
        return LNF_ENOMEM;
    if (cudaMemcpy(ctx->d_lt, t.data(), sizeof(unsigned long long) * t.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return LNF_ECUDA;
    return LNF_OK;
}

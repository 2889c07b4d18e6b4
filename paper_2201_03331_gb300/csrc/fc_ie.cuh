// Inclusion-exclusion helpers shared by the order-3 sweep and the order-3
// tensor-core kernel: full 3^k tables (k = 2, 3) from the cells whose
// genotypes are all in {0, 1} and lower-order tables.  Counts are packed as
// cases | controls << 16; every intermediate is a count, so the packed
// subtractions never borrow across the fields.
#pragma once
#include "fc_internal.cuh"

namespace fc {
namespace {

// Per-SNP genotype counts, packed per genotype as cases | controls << 16.
// m = marg row of the SNP: x = c0g0|c0g1<<16, y = c0g2|c1g0<<16, z = c1g1|c1g2<<16.
__device__ __forceinline__ void unpack_marg(const uint4 m, uint32_t t[3])
{
    t[0] = (m.x & 0xffffu) | (m.y & 0xffff0000u);
    t[1] = (m.x >> 16) | (m.z << 16);
    t[2] = (m.y & 0xffffu) | (m.z & 0xffff0000u);
}

// Full 3x3 table T[3a + b] of a SNP pair from its restricted cells
// R[2a + b] (a, b in {0,1}) and the per-SNP tables Ta, Tb.
__device__ __forceinline__ void full2(const uint32_t R[4], const uint32_t Ta[3], const uint32_t Tb[3],
                                      uint32_t T[9])
{
    T[0] = R[0]; T[1] = R[1]; T[3] = R[2]; T[4] = R[3];
    T[2] = Ta[0] - R[0] - R[1];
    T[5] = Ta[1] - R[2] - R[3];
    T[6] = Tb[0] - R[0] - R[2];
    T[7] = Tb[1] - R[1] - R[3];
    T[8] = Ta[2] - T[6] - T[7];
}

// Full 3x3x3 table T[9a + 3b + c] from the restricted cells Rr[4a + 2b + c]
// and the three full pair tables over positions (a,b), (a,c), (b,c).
__device__ __forceinline__ void full3(const uint32_t Rr[8], const uint32_t T01[9], const uint32_t T02[9],
                                      const uint32_t T12[9], uint32_t T[27])
{
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c) T[9 * a + 3 * b + c] = Rr[4 * a + 2 * b + c];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
#pragma unroll
        for (int b = 0; b < 2; ++b) T[18 + 3 * b + c] = T12[3 * b + c] - T[3 * b + c] - T[9 + 3 * b + c];
#pragma unroll
        for (int a = 0; a < 2; ++a) T[9 * a + 6 + c] = T02[3 * a + c] - T[9 * a + c] - T[9 * a + 3 + c];
        T[24 + c] = T12[6 + c] - T[6 + c] - T[15 + c];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) T[9 * a + 3 * b + 2] = T01[3 * a + b] - T[9 * a + 3 * b] - T[9 * a + 3 * b + 1];
}

}  // namespace
}  // namespace fc

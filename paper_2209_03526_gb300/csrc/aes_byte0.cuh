// aes_byte0.cuh -- byte 0 of an AES-128 output block from the shared-memory T-tables,
// for the Z_2 outputs of the one-hot mode: the control bit, Convert into Z_2 of a seed
// and of a value block, and the binary re-share PRF all read bits 0 and 1 of byte 0 only.
//
// Byte 0 of the final round is S[byte 0 of column 0 of round 9's state] xor byte 0 of the
// last round key (ShiftRows leaves row 0 in place), so round 9 needs column 0 alone (4
// lookups) and the final round one S-box lookup: 133 lookups per block instead of 160
// (148 for the column-0 variant).  Rounds 1..8 are the full rounds of device_fss.cuh.
#pragma once
#include <cstdint>

#include "device_fss.cuh"

namespace ogm {

// bits 0..7 of AES-128_rk(in), the rest zero
template <class Tab>
__device__ __forceinline__ uint32_t aes_one_b0(const Tab& T, const uint32_t* rk, const uint32_t in[4]) {
    uint32_t c[4];
#pragma unroll
    for (int j = 0; j < 4; j++) c[j] = in[j] ^ rk[j];
#pragma unroll
    for (int r = 1; r < 9; r++) aes_round(T, c, rk[4 * r], rk[4 * r + 1], rk[4 * r + 2], rk[4 * r + 3]);
    const uint32_t c0 = T.template lu<0, 0>(c[0]) ^ T.template lu<1, 1>(c[1]) ^ T.template lu<2, 2>(c[2]) ^
                        T.template lu<3, 3>(c[3]) ^ rk[36];
    return (T.template lu<0, 3>(c0) ^ rk[40]) & 0xFFu;   // table 3 holds S[x] in byte 0
}

// the same under round keys rk ^ (m & d): m = 0 selects key A, m = ~0 key B
template <class Tab>
__device__ __forceinline__ uint32_t aes_sel_b0(const Tab& T, const uint32_t* rk, const uint32_t* d, uint32_t m,
                                               const uint32_t in[4]) {
    uint32_t c[4];
#pragma unroll
    for (int j = 0; j < 4; j++) c[j] = in[j] ^ rk[j] ^ (m & d[j]);
#pragma unroll
    for (int r = 1; r < 9; r++)
        aes_round(T, c, rk[4 * r] ^ (m & d[4 * r]), rk[4 * r + 1] ^ (m & d[4 * r + 1]),
                  rk[4 * r + 2] ^ (m & d[4 * r + 2]), rk[4 * r + 3] ^ (m & d[4 * r + 3]));
    const uint32_t c0 = T.template lu<0, 0>(c[0]) ^ T.template lu<1, 1>(c[1]) ^ T.template lu<2, 2>(c[2]) ^
                        T.template lu<3, 3>(c[3]) ^ rk[36] ^ (m & d[36]);
    return (T.template lu<0, 3>(c0) ^ rk[40] ^ (m & d[40])) & 0xFFu;
}

}  // namespace ogm

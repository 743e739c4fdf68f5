// host_crypto.h -- host-side AES-128, FSS key generation and token parsing of
// the oblivgm library (client side of Sec. V-C and the servers' token intake).
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "oblivgm.h"

namespace ogm {

// AES-128 on 32-bit little-endian columns (column c = bytes 4c..4c+3 of the block).
struct RoundKeys { uint32_t w[44]; };

struct AesTables {
    uint8_t sbox[256];
    uint32_t te0[256];   // MixColumns(S[x]) contribution of row 0: bytes (2s, s, s, 3s)
};
const AesTables& aes_tables();
RoundKeys expand_key(const uint8_t key[16]);
void aes_encrypt(const RoundKeys& rk, const uint32_t in[4], uint32_t out[4]);

// the four fixed public PRG keys K_L, K_R, K_vL, K_vR: K_j[i] = 16 j + i
const RoundKeys& fixed_key(int j);

// Fixed-key round keys as the kernels take them (kernel parameter space).
struct AesParams {
    uint32_t rk_st[44];   // K_L round keys (seed / control-bit block, left child)
    uint32_t d_st[44];    // K_L ^ K_R   (right child = left ^ d under an all-ones mask)
    uint32_t rk_v[44];    // K_vL round keys (DCF value block)
    uint32_t d_v[44];     // K_vL ^ K_vR
};

constexpr uint32_t kBetaPrime = 0xAAAAAAABu;   // 3^{-1} mod 2^32
constexpr uint32_t kTokenMagic = 0x544D474Fu;
constexpr int kMaxPreds = 64;
constexpr int kMaxBits = 32;
constexpr int kMaxOnehotBits = 16;   // one-hot vectors of 2^n bits per element

inline size_t key_bytes(uint32_t kind, int n) { return 28u + (size_t)n * (kind == OBLIVGM_KEY_DPF ? 20u : 24u); }

// Device form of one key (repacked from the wire format), 16-byte aligned.
struct alignas(16) DevKey {
    uint32_t seed[4];
    uint32_t scw[kMaxBits][4];   // level i (1-based) at scw[i-1]
    uint32_t vcw[kMaxBits];      // DCF value correction words
    uint32_t tl, tr;             // bit i-1: t^L_CW / t^R_CW of level i
    uint32_t cw_final;           // CW_{n+1}
    uint32_t party;              // 0 or 1
    uint32_t n;
    uint32_t kind;
    uint32_t group;              // output group: 0 = Z_{2^32}, 1 = Z_2 (one-hot mode)
    uint32_t pad;
};
static_assert(sizeof(DevKey) == 688, "DevKey layout");
static_assert(sizeof(DevKey) % 16 == 0, "bulk copies need 16-byte multiples");

// One-hot mode keys (outputs in Z_2) stop the tree early: the last m = min(n, 7) input
// bits index a vector of 2^m <= 128 output bits that a leaf seed expands into, so a key
// has nu = n - m levels.  Wire layout: header 8 B, seed 16 B, per level s_CW 16 B,
// t^L_CW, t^R_CW, 2 zero bytes, (DCF) V_CW 16 B; the final CW 16 B.
constexpr int kEtLowBits = 7;
constexpr int kMaxEtLevels = kMaxOnehotBits - kEtLowBits;
inline int et_low_bits(int n) { return n < kEtLowBits ? n : kEtLowBits; }
inline size_t et_key_bytes(uint32_t kind, int n) {
    return 40u + (size_t)(n - et_low_bits(n)) * (kind == OBLIVGM_KEY_DPF ? 20u : 36u);
}

// Device form of an early-terminated key.  Vectors of 2^m bits are four 32-bit words,
// bit j in word j / 32 at bit j % 32.
struct alignas(16) EtKey {
    uint32_t seed[4];
    uint32_t scw[kMaxEtLevels][4];
    uint32_t vcw[kMaxEtLevels][4];   // DCF value corrections (2^m-bit vectors)
    uint32_t cw_final[4];
    uint32_t tl, tr;                 // bit i-1: t^L_CW / t^R_CW of level i
    uint32_t party, n, kind, low_bits, levels, pad;
};
static_assert(sizeof(EtKey) == 352, "EtKey layout");

// Gen of an early-terminated Z_2 key pair (beta = 1): [x == alpha] for a DPF,
// [x < alpha] for a DCF, in the wire layout above.
void gen_et(uint32_t kind, int n, uint32_t alpha, const uint8_t s0[16], const uint8_t s1[16], uint8_t* k0,
            uint8_t* k1);

// Wire key (early terminated) -> EtKey.  Returns false on a malformed key.
bool repack_key_et(const uint8_t* wire, size_t avail, uint32_t want_kind, int want_n, EtKey* out, std::string* err);

// Wire key -> DevKey.  Returns false on a malformed key.
bool repack_key(const uint8_t* wire, size_t avail, uint32_t want_kind, int want_n, DevKey* out, std::string* err);

// One predicate as the servers see it after parsing the three tokens.
struct ParsedPred {
    uint32_t kind, n, table, attr, group, step;
    uint32_t combine = 0;       // OBLIVGM_COMBINE_*: how the result joins the group's
    uint32_t r[3];        // <r>_1, <r>_2, <r>_3 (each server's own share)
    uint32_t cbeta;
    std::vector<DevKey> keys;   // [server][half][sub]: 6 (EQ) or 12 (RANGE); masked mode
    std::vector<EtKey> et_keys; // the same order, one-hot mode
};

// Fold of a group's result a with a predicate's result b (Sec. V-D), over 0/1 values in
// Z_{2^32}: w = lin (a + b) + prod a b, with (lin, prod) = AND (0, 1), XOR (1, -2),
// OR (1, -1).
inline void combine_coeffs(uint32_t op, uint32_t* lin, uint32_t* prod) {
    *lin = op == OBLIVGM_COMBINE_AND ? 0u : 1u;
    *prod = op == OBLIVGM_COMBINE_AND ? 1u : op == OBLIVGM_COMBINE_XOR ? 0xFFFFFFFEu : 0xFFFFFFFFu;
}

// Checks the combine fields of a predicate list: each at most OR, and AND on the
// first predicate of every group.  Returns false with *err set otherwise.
bool check_combine(const oblivgm_pred* preds, uint32_t n_preds, std::string* err);

struct ParsedQuery {
    uint32_t n_bits = 0;
    uint32_t out_group = 0;   // 0: masked mode over Z_{2^32}; 1: one-hot mode over Z_2
    std::vector<ParsedPred> preds;
};

// Parse and cross-check the three servers' tokens.
oblivgm_status parse_tokens(const uint8_t* const tok[3], const size_t tok_len[3], ParsedQuery* q, std::string* err);

// Client-side token generation; identical layout to the ABI description.
// onehot = false: masked mode; true: the one-hot mode of Sec. V-C (no mask, Z_2 keys, beta = 1).
oblivgm_status keygen(const oblivgm_pred* preds, uint32_t n_preds, uint32_t n_bits, const uint8_t seed[16],
                      uint8_t* const tok[3], size_t cap, size_t out_len[3], std::string* err, bool onehot = false);

// FSS Gen for one key pair in the wire format (exposed for tests through the ABI-free entry).
// group 0: outputs in Z_{2^32}; group 1: outputs in Z_2 (Convert = one bit, words stored mod 2)
void dpf_gen(int n, uint32_t alpha, uint32_t beta, const uint8_t s0[16], const uint8_t s1[16], uint8_t* k0,
             uint8_t* k1, int group = 0);
void dcf_gen(int n, uint32_t alpha, uint32_t beta, const uint8_t s0[16], const uint8_t s1[16], uint8_t* k0,
             uint8_t* k1, int group = 0);

}  // namespace ogm

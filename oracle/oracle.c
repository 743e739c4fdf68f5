/*
 * oracle.c -- plain, slow CPU oracle for the FSS predicate-evaluation path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py load this code.  The product
 * library (paper_2209_03526_gb300/) shares no code, table or header with it.
 *
 * What it computes (OblivGM, arXiv 2209.03526):
 *   - AES-128 exactly as FIPS-197 writes it, byte by byte; the S-box is derived
 *     at start-up from the GF(2^8) inverse and the affine map (Sec. VII-A fixes
 *     the security parameter lambda = 128; the paper is silent on the PRG).
 *   - the PRG  H_K(s) = AES_K(s) xor s  under four fixed public keys
 *     K_L, K_R, K_vL, K_vR with K_j[i] = 16 j + i   (reading P1 of the design).
 *   - DPF Gen/Eval for the point function f^=_{alpha,beta} (Sec. V-C; the
 *     tree construction of Boyle-Gilboa-Ishai, CCS'16, which the paper cites).
 *   - DCF Gen/Eval for the comparison function g^<_{alpha,beta} (Sec. V-C;
 *     the construction of Boyle et al., Eurocrypt'21, which the paper cites).
 *   - the secure query token of Sec. V-C: three independent key pairs per
 *     predicate, handed to CS1..CS3 as (k^1_1,k^2_1), (k^2_2,k^3_1), (k^3_2,k^1_2).
 *   - secEval (Alg. 3) on additively masked inputs (Sec. V-C, the masked-input
 *     approach), the per-server sum of Eq. (predEval), the PRF re-share of
 *     Sec. III-B and the aggregation of a target's predicates of Sec. V-D
 *     (all hold: the RSS product; "one of": the paper's XOR; or the inclusive
 *     OR), all over Z_{2^32}.
 *   - the one-hot mode of Sec. V-B/V-C: keys over Z_2 with beta = 1 that stop
 *     their trees early (BGI16's early termination for small output groups; the
 *     DCF the same over the vector group Z_2^(2^m)), evaluated at every position
 *     of a binary-RSS one-hot vector, re-shared with a PRF bit per element (one
 *     AES block per 128 elements) and folded in binary RSS.
 *
 * Every step is written in the order the construction states it; nothing is
 * blocked, fused or reordered.  Eval computes only the child the input bit
 * selects: the other half of G(s) is computed and then discarded by the
 * construction, so leaving it out changes no output.
 *
 * Parity unpinned (conventions the paper leaves open; they fix individual share
 * values, while every reconstructed result is pinned by the tests): the fixed
 * keys K_R, K_vL, K_vR (K_L is FIPS-pinned), the token byte layout, the keygen
 * random streams, the PRF counter layouts (the one-hot PRF's is pinned against
 * the FIPS-pinned AES), and secShuffle's derivation of each pair's permutation
 * and masks from its seed.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* GF(2^8) with the AES polynomial x^8 + x^4 + x^3 + x + 1 (FIPS-197 Sec. 4) */
/* ------------------------------------------------------------------------ */

static uint8_t gf_mul(uint8_t a, uint8_t b)
{
    uint8_t p = 0;
    for (int i = 0; i < 8; i++) {
        if (b & 1) p ^= a;
        uint8_t carry = (uint8_t)(a & 0x80);
        a = (uint8_t)(a << 1);
        if (carry) a ^= 0x1b;
        b >>= 1;
    }
    return p;
}

/* multiplicative inverse by exhaustive search; 0 maps to 0 (FIPS-197 Sec. 5.1.1) */
static uint8_t gf_inv(uint8_t a)
{
    if (a == 0) return 0;
    for (int x = 1; x < 256; x++)
        if (gf_mul(a, (uint8_t)x) == 1) return (uint8_t)x;
    return 0;
}

/* S-box entry: inverse followed by the affine map b'_i = b_i ^ b_{i+4} ^ b_{i+5} ^ b_{i+6} ^ b_{i+7} ^ c_i, c = 0x63 */
static uint8_t sbox_entry(uint8_t a)
{
    uint8_t b = gf_inv(a), s = 0;
    for (int i = 0; i < 8; i++) {
        int bit = ((b >> i) ^ (b >> ((i + 4) & 7)) ^ (b >> ((i + 5) & 7)) ^
                   (b >> ((i + 6) & 7)) ^ (b >> ((i + 7) & 7)) ^ (0x63 >> i)) & 1;
        s |= (uint8_t)(bit << i);
    }
    return s;
}

static uint8_t SBOX[256];

/* ------------------------------------------------------------------------ */
/* AES-128 (FIPS-197 Sec. 5.1 cipher, Sec. 5.2 key expansion)               */
/* ------------------------------------------------------------------------ */

typedef struct { uint8_t w[44][4]; } aes_ks;   /* 44 words of 4 bytes */

static void key_expansion(const uint8_t key[16], aes_ks* ks)
{
    uint8_t rcon = 0x01;
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) ks->w[i][j] = key[4 * i + j];
    for (int i = 4; i < 44; i++) {
        uint8_t temp[4];
        memcpy(temp, ks->w[i - 1], 4);
        if (i % 4 == 0) {
            uint8_t t0 = temp[0];                       /* RotWord */
            temp[0] = temp[1]; temp[1] = temp[2]; temp[2] = temp[3]; temp[3] = t0;
            for (int j = 0; j < 4; j++) temp[j] = SBOX[temp[j]];   /* SubWord */
            temp[0] ^= rcon;                            /* Rcon[i/4] = x^(i/4 - 1) */
            rcon = gf_mul(rcon, 0x02);
        }
        for (int j = 0; j < 4; j++) ks->w[i][j] = (uint8_t)(ks->w[i - 4][j] ^ temp[j]);
    }
}

static void add_round_key(uint8_t st[4][4], const aes_ks* ks, int round)
{
    for (int c = 0; c < 4; c++)
        for (int r = 0; r < 4; r++) st[r][c] ^= ks->w[4 * round + c][r];
}

static void sub_bytes(uint8_t st[4][4])
{
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) st[r][c] = SBOX[st[r][c]];
}

static void shift_rows(uint8_t st[4][4])
{
    for (int r = 1; r < 4; r++) {
        uint8_t row[4];
        for (int c = 0; c < 4; c++) row[c] = st[r][(c + r) % 4];
        for (int c = 0; c < 4; c++) st[r][c] = row[c];
    }
}

static void mix_columns(uint8_t st[4][4])
{
    for (int c = 0; c < 4; c++) {
        uint8_t a0 = st[0][c], a1 = st[1][c], a2 = st[2][c], a3 = st[3][c];
        st[0][c] = (uint8_t)(gf_mul(a0, 2) ^ gf_mul(a1, 3) ^ a2 ^ a3);
        st[1][c] = (uint8_t)(a0 ^ gf_mul(a1, 2) ^ gf_mul(a2, 3) ^ a3);
        st[2][c] = (uint8_t)(a0 ^ a1 ^ gf_mul(a2, 2) ^ gf_mul(a3, 3));
        st[3][c] = (uint8_t)(gf_mul(a0, 3) ^ a1 ^ a2 ^ gf_mul(a3, 2));
    }
}

/* Test instrumentation: the AES-128 blocks the calling thread has encrypted, so that the
 * tests can check the benchmark's algorithmic block counts against the oracle's own work. */
static __thread uint64_t AES_BLOCKS;

uint64_t orc_aes_blocks(void) { return AES_BLOCKS; }
void orc_aes_blocks_reset(void) { AES_BLOCKS = 0; }

/* Test instrumentation: a mistake the tests plant on purpose in the calling thread, so that
 * they can show that their uniformity pins fail on it (it never changes results otherwise).
 *   0  none (the default);
 *   1  every Convert and every mask word is the constant 0;
 *   2  Converts read the cleared control bit: a seed's Convert takes bytes 0..3 (Z_{2^32}) or
 *      bit 0 of byte 0 (Z_2), and a DCF value word is taken from the child seed block
 *      (whose bit 0 is cleared) instead of the value block;
 *   3  the mask share <r>_1 is read from the bytes of r itself. */
static __thread int PLANTED;
void orc_test_plant(int mode) { PLANTED = mode; }

/* S-box entry (test accessor; the table is built by orc_init) */
uint32_t orc_sbox(uint32_t x) { return SBOX[x & 0xFFu]; }

static void aes_encrypt(const aes_ks* ks, const uint8_t in[16], uint8_t out[16])
{
    uint8_t st[4][4];
    AES_BLOCKS++;
    for (int i = 0; i < 16; i++) st[i % 4][i / 4] = in[i];
    add_round_key(st, ks, 0);
    for (int round = 1; round < 10; round++) {
        sub_bytes(st);
        shift_rows(st);
        mix_columns(st);
        add_round_key(st, ks, round);
    }
    sub_bytes(st);
    shift_rows(st);
    add_round_key(st, ks, 10);
    for (int i = 0; i < 16; i++) out[i] = st[i % 4][i / 4];
}

/* ------------------------------------------------------------------------ */
/* PRG: H_K(s) = AES_K(s) xor s with fixed public keys K_j[i] = 16 j + i     */
/* ------------------------------------------------------------------------ */

enum { KEY_L = 0, KEY_R = 1, KEY_VL = 2, KEY_VR = 3 };
static aes_ks FIXED[4];
static int ready = 0;

void orc_init(void)
{
    if (ready) return;
    for (int a = 0; a < 256; a++) SBOX[a] = sbox_entry((uint8_t)a);
    for (int j = 0; j < 4; j++) {
        uint8_t k[16];
        for (int i = 0; i < 16; i++) k[i] = (uint8_t)(16 * j + i);
        key_expansion(k, &FIXED[j]);
    }
    ready = 1;
}

static void prg_h(int which, const uint8_t s[16], uint8_t out[16])
{
    uint8_t e[16];
    aes_encrypt(&FIXED[which], s, e);
    for (int i = 0; i < 16; i++) out[i] = (uint8_t)(e[i] ^ s[i]);
}

/* child seed and control bit: t = bit 0 of byte 0, seed = block with that bit cleared */
static void child(int dir, const uint8_t s[16], uint8_t cs[16], int* ct)
{
    prg_h(dir == 0 ? KEY_L : KEY_R, s, cs);
    *ct = cs[0] & 1;
    cs[0] &= 0xFE;
}

static uint32_t le32(const uint8_t* p)
{
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

static void put32(uint8_t* p, uint32_t v)
{
    p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); p[2] = (uint8_t)(v >> 16); p[3] = (uint8_t)(v >> 24);
}

/* Output groups: 0 = Z_{2^32}, 1 = Z_2 (the one-hot mode of Sec. V-B/V-C, beta = 1 in Z_2).
 * Convert of a seed: Z_{2^32} bytes 4..7 little-endian; Z_2 bit 1 of byte 0 (bit 0 of
 * byte 0 is the control bit).  Z_2 arithmetic is Z_{2^32} arithmetic reduced mod 2, so
 * the constructions below run unchanged and only stored words and outputs are masked. */
#define GROUP_Z2_32 0
#define GROUP_Z2 1
static uint32_t group_mask(int group) { return group == GROUP_Z2 ? 1u : 0xFFFFFFFFu; }

static uint32_t convert_seed_g(const uint8_t s[16], int group)
{
    if (PLANTED == 1) return 0u;
    if (PLANTED == 2) return group == GROUP_Z2 ? (uint32_t)(s[0] & 1) : le32(s);
    return group == GROUP_Z2 ? (uint32_t)((s[0] >> 1) & 1) : le32(s + 4);
}

/* DCF value of a child: Convert of H_{K_vL or K_vR}(s) -- bytes 0..3 (Z_{2^32}) or bit 0 of byte 0 (Z_2) */
static uint32_t value_word_g(int dir, const uint8_t s[16], int group)
{
    uint8_t v[16];
    if (PLANTED == 1) return 0u;
    prg_h(PLANTED == 2 ? (dir == 0 ? KEY_L : KEY_R) : (dir == 0 ? KEY_VL : KEY_VR), s, v);
    if (PLANTED == 2) v[0] &= 0xFE;   /* the child seed block, control bit cleared */
    return group == GROUP_Z2 ? (uint32_t)(v[0] & 1) : le32(v);
}

/* A predicate's mask r and its additive shares <r>_1, <r>_2, <r>_3 (mod 2^n) from one random
 * block: r = bytes 0..3, <r>_1 = bytes 4..7, <r>_2 = bytes 8..11, <r>_3 = r - <r>_1 - <r>_2. */
static uint32_t mask_words(const uint8_t blk[16], uint32_t m, uint32_t rs[3])
{
    uint32_t r = le32(blk) & m;
    rs[0] = le32(blk + (PLANTED == 3 ? 0 : 4)) & m;
    rs[1] = le32(blk + 8) & m;
    if (PLANTED == 1) r = rs[0] = rs[1] = 0u;
    rs[2] = (r - rs[0] - rs[1]) & m;
    return r;
}

/* i-th input bit, i = 1..n, most significant first */
static int bit_of(uint32_t x, int n, int i) { return (int)((x >> (n - i)) & 1u); }

/* ------------------------------------------------------------------------ */
/* Key wire format (little-endian):                                          */
/*   header  u8 kind (1 DPF, 2 DCF), u8 n, u8 party b, u8 group (0 = Z_2^32), */
/*           u32 0                                                            */
/*   seed    16 bytes                                                         */
/*   level i s_CW[16], u8 t^L_CW, u8 t^R_CW, u16 0, [DCF only: u32 V_CW]      */
/*   final   u32 CW_{n+1}                                                     */
/* ------------------------------------------------------------------------ */

#define KIND_DPF 1
#define KIND_DCF 2

static size_t level_bytes(int kind) { return kind == KIND_DPF ? 20u : 24u; }

size_t orc_key_len(int kind, int n) { return 24u + (size_t)n * level_bytes(kind) + 4u; }

static void write_header(uint8_t* k, int kind, int n, int b, const uint8_t seed[16], int group)
{
    memset(k, 0, 8);
    k[0] = (uint8_t)kind; k[1] = (uint8_t)n; k[2] = (uint8_t)b; k[3] = (uint8_t)group;
    memcpy(k + 8, seed, 16);
}

/* DPF Gen(1^lambda, alpha, beta): keys k0, k1 from the root seeds s0, s1, output group `group` */
void orc_dpf_gen_g(int n, uint32_t alpha, uint32_t beta, const uint8_t s0[16], const uint8_t s1[16],
                   uint8_t* k0, uint8_t* k1, int group)
{
    uint8_t s[2][16];
    int t[2] = {0, 1};
    memcpy(s[0], s0, 16);
    memcpy(s[1], s1, 16);
    write_header(k0, KIND_DPF, n, 0, s0, group);
    write_header(k1, KIND_DPF, n, 1, s1, group);
    for (int i = 1; i <= n; i++) {
        uint8_t sc[2][2][16];   /* [party][dir] */
        int tc[2][2];
        for (int b = 0; b < 2; b++)
            for (int dir = 0; dir < 2; dir++) child(dir, s[b], sc[b][dir], &tc[b][dir]);
        int a = bit_of(alpha, n, i);
        int keep = a, lose = 1 - a;
        uint8_t s_cw[16];
        for (int j = 0; j < 16; j++) s_cw[j] = (uint8_t)(sc[0][lose][j] ^ sc[1][lose][j]);
        int tl_cw = tc[0][0] ^ tc[1][0] ^ a ^ 1;
        int tr_cw = tc[0][1] ^ tc[1][1] ^ a;
        size_t off = 24 + (size_t)(i - 1) * level_bytes(KIND_DPF);
        for (int p = 0; p < 2; p++) {
            uint8_t* k = p ? k1 : k0;
            memcpy(k + off, s_cw, 16);
            k[off + 16] = (uint8_t)tl_cw;
            k[off + 17] = (uint8_t)tr_cw;
            k[off + 18] = 0; k[off + 19] = 0;
        }
        int t_keep_cw = keep == 0 ? tl_cw : tr_cw;
        for (int b = 0; b < 2; b++) {
            for (int j = 0; j < 16; j++) s[b][j] = (uint8_t)(sc[b][keep][j] ^ (t[b] ? s_cw[j] : 0));
            t[b] = tc[b][keep] ^ (t[b] & t_keep_cw);
        }
    }
    uint32_t cw = beta - convert_seed_g(s[0], group) + convert_seed_g(s[1], group);
    if (t[1]) cw = 0u - cw;
    cw &= group_mask(group);
    size_t off = 24 + (size_t)n * level_bytes(KIND_DPF);
    put32(k0 + off, cw);
    put32(k1 + off, cw);
}

void orc_dpf_gen(int n, uint32_t alpha, uint32_t beta, const uint8_t s0[16], const uint8_t s1[16],
                 uint8_t* k0, uint8_t* k1)
{
    orc_dpf_gen_g(n, alpha, beta, s0, s1, k0, k1, GROUP_Z2_32);
}

/* DPF Eval(b, k_b, x) -> share of beta * [x == alpha] */
uint32_t orc_dpf_eval(const uint8_t* key, uint32_t x)
{
    int n = key[1], b = key[2], group = key[3];
    uint8_t s[16];
    int t = b;
    memcpy(s, key + 8, 16);
    for (int i = 1; i <= n; i++) {
        const uint8_t* cw = key + 24 + (size_t)(i - 1) * level_bytes(KIND_DPF);
        int dir = bit_of(x, n, i);
        uint8_t ns[16];
        int nt;
        child(dir, s, ns, &nt);
        if (t) {
            for (int j = 0; j < 16; j++) ns[j] ^= cw[j];
            nt ^= dir == 0 ? cw[16] : cw[17];
        }
        memcpy(s, ns, 16);
        t = nt;
    }
    uint32_t y = convert_seed_g(s, group) + (t ? le32(key + 24 + (size_t)n * level_bytes(KIND_DPF)) : 0u);
    return (b ? 0u - y : y) & group_mask(group);
}

/* DCF Gen(1^lambda, alpha, beta): shares of beta * [x < alpha], output group `group` */
void orc_dcf_gen_g(int n, uint32_t alpha, uint32_t beta, const uint8_t s0[16], const uint8_t s1[16],
                   uint8_t* k0, uint8_t* k1, int group)
{
    uint8_t s[2][16];
    int t[2] = {0, 1};
    uint32_t v_alpha = 0;
    memcpy(s[0], s0, 16);
    memcpy(s[1], s1, 16);
    write_header(k0, KIND_DCF, n, 0, s0, group);
    write_header(k1, KIND_DCF, n, 1, s1, group);
    for (int i = 1; i <= n; i++) {
        uint8_t sc[2][2][16];
        int tc[2][2];
        uint32_t vc[2][2];
        for (int b = 0; b < 2; b++)
            for (int dir = 0; dir < 2; dir++) {
                child(dir, s[b], sc[b][dir], &tc[b][dir]);
                vc[b][dir] = value_word_g(dir, s[b], group);
            }
        int a = bit_of(alpha, n, i);
        int keep = a, lose = 1 - a;
        uint8_t s_cw[16];
        for (int j = 0; j < 16; j++) s_cw[j] = (uint8_t)(sc[0][lose][j] ^ sc[1][lose][j]);
        int neg = t[1];   /* (-1)^{t_1^{(i-1)}} */
        uint32_t v_cw = vc[1][lose] - vc[0][lose] - v_alpha;
        if (neg) v_cw = 0u - v_cw;
        if (lose == 0) v_cw += neg ? 0u - beta : beta;
        v_alpha = v_alpha - vc[1][keep] + vc[0][keep] + (neg ? 0u - v_cw : v_cw);
        int tl_cw = tc[0][0] ^ tc[1][0] ^ a ^ 1;
        int tr_cw = tc[0][1] ^ tc[1][1] ^ a;
        size_t off = 24 + (size_t)(i - 1) * level_bytes(KIND_DCF);
        for (int p = 0; p < 2; p++) {
            uint8_t* k = p ? k1 : k0;
            memcpy(k + off, s_cw, 16);
            k[off + 16] = (uint8_t)tl_cw;
            k[off + 17] = (uint8_t)tr_cw;
            k[off + 18] = 0; k[off + 19] = 0;
            put32(k + off + 20, v_cw & group_mask(group));
        }
        int t_keep_cw = keep == 0 ? tl_cw : tr_cw;
        for (int b = 0; b < 2; b++) {
            for (int j = 0; j < 16; j++) s[b][j] = (uint8_t)(sc[b][keep][j] ^ (t[b] ? s_cw[j] : 0));
            t[b] = tc[b][keep] ^ (t[b] & t_keep_cw);
        }
    }
    uint32_t cw = convert_seed_g(s[1], group) - convert_seed_g(s[0], group) - v_alpha;
    if (t[1]) cw = 0u - cw;
    cw &= group_mask(group);
    size_t off = 24 + (size_t)n * level_bytes(KIND_DCF);
    put32(k0 + off, cw);
    put32(k1 + off, cw);
}

void orc_dcf_gen(int n, uint32_t alpha, uint32_t beta, const uint8_t s0[16], const uint8_t s1[16],
                 uint8_t* k0, uint8_t* k1)
{
    orc_dcf_gen_g(n, alpha, beta, s0, s1, k0, k1, GROUP_Z2_32);
}

/* DCF Eval(b, k_b, x) -> share of beta * [x < alpha] */
uint32_t orc_dcf_eval(const uint8_t* key, uint32_t x)
{
    int n = key[1], b = key[2], group = key[3];
    uint8_t s[16];
    int t = b;
    uint32_t v = 0;
    memcpy(s, key + 8, 16);
    for (int i = 1; i <= n; i++) {
        const uint8_t* cw = key + 24 + (size_t)(i - 1) * level_bytes(KIND_DCF);
        int dir = bit_of(x, n, i);
        uint8_t ns[16];
        int nt;
        child(dir, s, ns, &nt);
        uint32_t vw = value_word_g(dir, s, group);
        uint32_t term = vw + (t ? le32(cw + 20) : 0u);
        v += b ? 0u - term : term;
        if (t) {
            for (int j = 0; j < 16; j++) ns[j] ^= cw[j];
            nt ^= dir == 0 ? cw[16] : cw[17];
        }
        memcpy(s, ns, 16);
        t = nt;
    }
    uint32_t term = convert_seed_g(s, group) + (t ? le32(key + 24 + (size_t)n * level_bytes(KIND_DCF)) : 0u);
    v += b ? 0u - term : term;
    return v & group_mask(group);
}

/* ------------------------------------------------------------------------ */
/* Z_2 keys with early termination (the one-hot mode's keys)                 */
/* ------------------------------------------------------------------------ */
/*
 * BGI16 (the DPF the paper cites in Sec. IV-B) stops the tree early when the output
 * group is small: a leaf seed of lambda = 128 bits expands into the outputs of many
 * consecutive inputs.  Over Z_2 the last m = min(n, 7) input bits index a vector of
 * 2^m <= 128 output bits, so the tree has nu = n - m levels, walked with the high
 * bits x_hi = x >> m; the low bits x_lo pick the output bit.
 *
 * Vectors of 2^m bits sit in 16 bytes, bit j at byte j / 8, bit j % 8; bits from 2^m
 * up are zero.  A leaf seed s converts to Conv(s) = H_{K_vL}(s) (the value block a
 * further level would compute; a leaf seed is never expanded, so the block is used
 * nowhere else), and a DCF value block to H_{K_vdir}(s), both cut to 2^m bits.
 *
 * DPF, f(x) = [x == alpha]: the nu levels on alpha_hi as in the full-depth DPF; the
 * final word CW = e_{alpha_lo} xor Conv(s_0) xor Conv(s_1), so that the parties'
 * leaf vectors Conv(s_b) xor t_b CW differ exactly in bit alpha_lo on alpha_hi's leaf
 * and agree everywhere else.
 *
 * DCF, f(x) = [x < alpha]: the BCG+21 tree over the vector group Z_2^(2^m) with
 * beta = the all-ones vector on the nu levels of alpha_hi (so a leaf left of
 * alpha_hi's carries all ones), and the final word chosen so that alpha_hi's own leaf
 * carries L_{alpha_lo} (bits j < alpha_lo set):
 *   V_CW  = v^lose_0 xor v^lose_1 xor V_alpha xor [lose = L] 1,
 *   V_alpha <- V_alpha xor v^keep_0 xor v^keep_1 xor V_CW,
 *   CW    = Conv(s_0) xor Conv(s_1) xor V_alpha xor L_{alpha_lo}.
 * Over Z_2 every sign of BCG+21 is +.  Key layout (group byte 1):
 *   header 8 B, seed 16 B, per level s_CW[16], u8 t^L_CW, u8 t^R_CW, u16 0,
 *   [DCF: V_CW[16]], final CW[16].
 */
static int et_low_bits(int n) { return n < 7 ? n : 7; }

static size_t et_level_bytes(int kind) { return kind == KIND_DPF ? 20u : 36u; }

size_t orc_key_len_et(int kind, int n)
{
    return 24u + (size_t)(n - et_low_bits(n)) * et_level_bytes(kind) + 16u;
}

static void vec_cut(uint8_t v[16], int m)
{
    int bits = 1 << m;
    for (int j = 0; j < 128; j++)
        if (j >= bits) v[j / 8] &= (uint8_t)~(1u << (j % 8));
}

static int vec_bit(const uint8_t v[16], uint32_t j) { return (v[j / 8] >> (j % 8)) & 1; }

/* Conv(s) of a leaf seed, 2^m bits */
static void leaf_vec(const uint8_t s[16], int m, uint8_t out[16])
{
    if (PLANTED == 1) { memset(out, 0, 16); return; }
    if (PLANTED == 2) memcpy(out, s, 16);       /* the seed itself, control bit cleared */
    else prg_h(KEY_VL, s, out);
    vec_cut(out, m);
}

/* value vector of child dir of node s (DCF), 2^m bits */
static void value_vec(int dir, const uint8_t s[16], int m, uint8_t out[16])
{
    if (PLANTED == 1) { memset(out, 0, 16); return; }
    prg_h(dir == 0 ? KEY_VL : KEY_VR, s, out);
    vec_cut(out, m);
}

static void et_header(uint8_t* k, int kind, int n, int b, const uint8_t seed[16])
{
    write_header(k, kind, n, b, seed, GROUP_Z2);
}

/* the nu tree levels shared by both kinds: seeds, control bits and, for the DCF, V_alpha */
static void et_levels(int kind, int n, uint32_t a_hi, uint8_t s[2][16], int t[2], uint8_t v_alpha[16],
                      uint8_t* k0, uint8_t* k1)
{
    const int m = et_low_bits(n), nu = n - m;
    for (int i = 1; i <= nu; i++) {
        uint8_t sc[2][2][16], vc[2][2][16];
        int tc[2][2];
        for (int b = 0; b < 2; b++)
            for (int dir = 0; dir < 2; dir++) {
                child(dir, s[b], sc[b][dir], &tc[b][dir]);
                if (kind == KIND_DCF) value_vec(dir, s[b], m, vc[b][dir]);
            }
        int a = bit_of(a_hi, nu, i);
        int keep = a, lose = 1 - a;
        uint8_t s_cw[16], v_cw[16];
        for (int j = 0; j < 16; j++) s_cw[j] = (uint8_t)(sc[0][lose][j] ^ sc[1][lose][j]);
        int tl_cw = tc[0][0] ^ tc[1][0] ^ a ^ 1;
        int tr_cw = tc[0][1] ^ tc[1][1] ^ a;
        if (kind == KIND_DCF) {
            for (int j = 0; j < 16; j++) v_cw[j] = (uint8_t)(vc[0][lose][j] ^ vc[1][lose][j] ^ v_alpha[j]);
            if (lose == 0)
                for (int j = 0; j < 16; j++) v_cw[j] ^= 0xFF;
            vec_cut(v_cw, m);
            for (int j = 0; j < 16; j++) v_alpha[j] ^= (uint8_t)(vc[0][keep][j] ^ vc[1][keep][j] ^ v_cw[j]);
        }
        size_t off = 24 + (size_t)(i - 1) * et_level_bytes(kind);
        for (int p = 0; p < 2; p++) {
            uint8_t* k = p ? k1 : k0;
            memcpy(k + off, s_cw, 16);
            k[off + 16] = (uint8_t)tl_cw;
            k[off + 17] = (uint8_t)tr_cw;
            k[off + 18] = 0; k[off + 19] = 0;
            if (kind == KIND_DCF) memcpy(k + off + 20, v_cw, 16);
        }
        int t_keep_cw = keep == 0 ? tl_cw : tr_cw;
        for (int b = 0; b < 2; b++) {
            for (int j = 0; j < 16; j++) s[b][j] = (uint8_t)(sc[b][keep][j] ^ (t[b] ? s_cw[j] : 0));
            t[b] = tc[b][keep] ^ (t[b] & t_keep_cw);
        }
    }
}

/* DPF Gen with early termination, f = [x == alpha] over Z_2 */
void orc_dpf_gen_et(int n, uint32_t alpha, const uint8_t s0[16], const uint8_t s1[16], uint8_t* k0, uint8_t* k1)
{
    const int m = et_low_bits(n);
    uint8_t s[2][16], unused[16] = {0};
    int t[2] = {0, 1};
    memcpy(s[0], s0, 16);
    memcpy(s[1], s1, 16);
    et_header(k0, KIND_DPF, n, 0, s0);
    et_header(k1, KIND_DPF, n, 1, s1);
    et_levels(KIND_DPF, n, alpha >> m, s, t, unused, k0, k1);
    uint8_t c0[16], c1[16], cw[16] = {0};
    leaf_vec(s[0], m, c0);
    leaf_vec(s[1], m, c1);
    uint32_t a_lo = alpha & ((1u << m) - 1u);
    cw[a_lo / 8] = (uint8_t)(1u << (a_lo % 8));
    for (int j = 0; j < 16; j++) cw[j] ^= (uint8_t)(c0[j] ^ c1[j]);
    size_t off = 24 + (size_t)(n - m) * et_level_bytes(KIND_DPF);
    memcpy(k0 + off, cw, 16);
    memcpy(k1 + off, cw, 16);
}

/* DCF Gen with early termination, f = [x < alpha] over Z_2 */
void orc_dcf_gen_et(int n, uint32_t alpha, const uint8_t s0[16], const uint8_t s1[16], uint8_t* k0, uint8_t* k1)
{
    const int m = et_low_bits(n);
    uint8_t s[2][16], v_alpha[16] = {0};
    int t[2] = {0, 1};
    memcpy(s[0], s0, 16);
    memcpy(s[1], s1, 16);
    et_header(k0, KIND_DCF, n, 0, s0);
    et_header(k1, KIND_DCF, n, 1, s1);
    et_levels(KIND_DCF, n, alpha >> m, s, t, v_alpha, k0, k1);
    uint8_t c0[16], c1[16], cw[16] = {0};
    leaf_vec(s[0], m, c0);
    leaf_vec(s[1], m, c1);
    uint32_t a_lo = alpha & ((1u << m) - 1u);
    for (uint32_t j = 0; j < a_lo; j++) cw[j / 8] |= (uint8_t)(1u << (j % 8));
    for (int j = 0; j < 16; j++) cw[j] ^= (uint8_t)(c0[j] ^ c1[j] ^ v_alpha[j]);
    size_t off = 24 + (size_t)(n - m) * et_level_bytes(KIND_DCF);
    memcpy(k0 + off, cw, 16);
    memcpy(k1 + off, cw, 16);
}

/* Eval of an early-terminated key: the 2^m-bit leaf vector of x_hi = x >> m
 * (the DCF's value terms included), of which the caller takes bit x_lo. */
static void et_leaf(const uint8_t* key, uint32_t x_hi, uint8_t y[16])
{
    int kind = key[0], n = key[1], b = key[2];
    const int m = et_low_bits(n), nu = n - m;
    uint8_t s[16], v[16] = {0};
    int t = b;
    memcpy(s, key + 8, 16);
    for (int i = 1; i <= nu; i++) {
        const uint8_t* cw = key + 24 + (size_t)(i - 1) * et_level_bytes(kind);
        int dir = bit_of(x_hi, nu, i);
        uint8_t ns[16];
        int nt;
        child(dir, s, ns, &nt);
        if (kind == KIND_DCF) {
            uint8_t vw[16];
            value_vec(dir, s, m, vw);
            for (int j = 0; j < 16; j++) v[j] ^= (uint8_t)(vw[j] ^ (t ? cw[20 + j] : 0));
        }
        if (t) {
            for (int j = 0; j < 16; j++) ns[j] ^= cw[j];
            nt ^= dir == 0 ? cw[16] : cw[17];
        }
        memcpy(s, ns, 16);
        t = nt;
    }
    const uint8_t* fin = key + 24 + (size_t)nu * et_level_bytes(kind);
    uint8_t c[16];
    leaf_vec(s, m, c);
    for (int j = 0; j < 16; j++) y[j] = (uint8_t)(v[j] ^ c[j] ^ (t ? fin[j] : 0));
}

uint32_t orc_eval_et(const uint8_t* key, uint32_t x)
{
    const int m = et_low_bits(key[1]);
    uint8_t y[16];
    et_leaf(key, x >> m, y);
    return (uint32_t)vec_bit(y, x & ((1u << m) - 1u));
}

void orc_aes128(const uint8_t key[16], const uint8_t in[16], uint8_t out[16])
{
    aes_ks ks;
    key_expansion(key, &ks);
    aes_encrypt(&ks, in, out);
}

void orc_prg(int which, const uint8_t s[16], uint8_t out[16]) { prg_h(which, s, out); }

/* ------------------------------------------------------------------------ */
/* Secure query token (Sec. V-C) over masked inputs                          */
/* ------------------------------------------------------------------------ */
/*
 * Token of server i (little-endian):
 *   header (16 B)  u32 magic 0x544D474F, u8 version 1, u8 server i (1..3),
 *                  u8 n, u8 group 0, u16 n_preds, u16 0, u32 total length
 *   per predicate  record (24 B): u8 kind (1 EQ, 2 RANGE), u8 n, u16 table,
 *                  u16 attr, u16 and-group, u32 <r>_i, u32 <r>_{i+1},
 *                  u32 c*beta' (RANGE) or 0, u32 0
 *                  then key half A and key half B of this server; a half is
 *                  one DPF key (EQ) or two DCF keys, a1 first then a0 (RANGE).
 * Halves held: CS1 (pair 1, party 0), (pair 2, party 0); CS2 (2,1), (3,0);
 * CS3 (3,1), (1,1)  -- the assignment of Sec. V-C.
 * beta' = 3^{-1} mod 2^32 for every pair, so the three pairs sum to f.
 * Randomness: AES-128 under the 16-byte seed in counter mode, counter block =
 * u64 index (LE) || 8 zero bytes; per predicate one block for the mask
 * (bytes 0..3 r, 4..7 <r>_1, 8..11 <r>_2, each reduced mod 2^n), then for
 * pair 1..3 and each key of the pair two blocks (root seeds s0, s1).
 */

#define TOKEN_MAGIC 0x544D474Fu
#define PRED_EQ 1
#define PRED_RANGE 2
#define BETA_PRIME 0xAAAAAAABu   /* 3 * 0xAAAAAAAB = 1 mod 2^32 */
#define MAX_HALF (2 * (24 + 32 * 24 + 4))   /* two DCF keys at n = 32 */

#define COMBINE_AND 0
#define COMBINE_XOR 1
#define COMBINE_OR 2

typedef struct {
    uint32_t kind, table, attr, group, lo, hi;
    uint32_t combine;   /* how the predicate's result joins its group's: COMBINE_* */
} orc_pred;

/* 1 if predicate p is the first of its group in list order */
static int first_of_group(const orc_pred* preds, uint32_t p)
{
    for (uint32_t e = 0; e < p; e++)
        if (preds[e].group == preds[p].group) return 0;
    return 1;
}

static const int HOLD_PAIR[3][2] = {{1, 2}, {2, 3}, {3, 1}};
static const int HOLD_PARTY[3][2] = {{0, 0}, {1, 0}, {1, 1}};

typedef struct { aes_ks ks; uint64_t ctr; } ctr_rng;

static void rng_block(ctr_rng* g, uint8_t out[16])
{
    uint8_t c[16] = {0};
    for (int i = 0; i < 8; i++) c[i] = (uint8_t)(g->ctr >> (8 * i));
    g->ctr++;
    aes_encrypt(&g->ks, c, out);
}

static uint32_t mask_n(int n) { return n >= 32 ? 0xFFFFFFFFu : ((1u << n) - 1u); }

size_t orc_key_len_et(int kind, int n);

/* key length of the mode: full depth over Z_{2^32} (masked), early terminated over Z_2 (one-hot) */
static size_t key_len_mode(int kind, int n, int onehot)
{
    return onehot ? orc_key_len_et(kind, n) : orc_key_len(kind, n);
}

static size_t token_len_mode(const orc_pred* preds, uint32_t n_preds, int n, int onehot)
{
    size_t len = 16;
    for (uint32_t p = 0; p < n_preds; p++) {
        len += 24;
        if (preds[p].kind == PRED_EQ) len += 2 * key_len_mode(KIND_DPF, n, onehot);
        else len += 4 * key_len_mode(KIND_DCF, n, onehot);
    }
    return len;
}

size_t orc_token_len(const orc_pred* preds, uint32_t n_preds, int n) { return token_len_mode(preds, n_preds, n, 0); }

size_t orc_token_len_onehot(const orc_pred* preds, uint32_t n_preds, int n)
{
    return token_len_mode(preds, n_preds, n, 1);
}

/*
 * Token generation for both modes.  Masked mode (onehot = 0): a fresh mask r per
 * predicate, keys for the shifted functions over Z_{2^32} with beta' = 3^{-1}.
 * One-hot mode (onehot = 1, Sec. V-C as written): no mask, keys for the predicate
 * itself over Z_2 with beta = 1, to be evaluated at every position of the one-hot
 * encoding; the token header's group byte is 1 and every <r> field is 0.  The random
 * stream then skips the mask block.  Returns 0, or -1 on an invalid predicate, -2 if a
 * buffer is too small.
 */
static int keygen_impl(const orc_pred* preds, uint32_t n_preds, int n, const uint8_t seed[16],
                       uint8_t* tok1, uint8_t* tok2, uint8_t* tok3, size_t cap, int onehot)
{
    uint8_t* tok[3] = {tok1, tok2, tok3};
    const int group = onehot ? GROUP_Z2 : GROUP_Z2_32;
    if (n < 1 || n > (onehot ? 16 : 32) || n_preds == 0 || n_preds > 64) return -1;
    uint32_t m = mask_n(n);
    for (uint32_t p = 0; p < n_preds; p++) {
        const orc_pred* q = &preds[p];
        if (q->kind == PRED_EQ) { if (q->lo > m) return -1; }
        else if (q->kind == PRED_RANGE) { if (q->lo > q->hi || q->hi > m) return -1; }
        else return -1;
        if (q->table > 0xFFFF || q->attr > 0xFFFF || q->group > 0xFFFF) return -1;
        if (q->combine > COMBINE_OR || (first_of_group(preds, p) && q->combine != COMBINE_AND)) return -1;
    }
    size_t total = token_len_mode(preds, n_preds, n, onehot);
    if (cap < total) return -2;
    ctr_rng g;
    key_expansion(seed, &g.ks);
    g.ctr = 0;
    size_t dpf_len = key_len_mode(KIND_DPF, n, onehot), dcf_len = key_len_mode(KIND_DCF, n, onehot);
    for (int i = 0; i < 3; i++) {
        uint8_t* h = tok[i];
        memset(h, 0, 16);
        put32(h, TOKEN_MAGIC);
        h[4] = 1; h[5] = (uint8_t)(i + 1); h[6] = (uint8_t)n; h[7] = (uint8_t)group;
        h[8] = (uint8_t)n_preds; h[9] = (uint8_t)(n_preds >> 8);
        put32(h + 12, (uint32_t)total);
    }
    size_t off = 16;
    for (uint32_t p = 0; p < n_preds; p++) {
        const orc_pred* q = &preds[p];
        uint32_t r = 0, rs[3] = {0, 0, 0};
        if (!onehot) {
            uint8_t blk[16];
            rng_block(&g, blk);
            r = mask_words(blk, m, rs);
        }
        const uint32_t beta = onehot ? 1u : BETA_PRIME;
        /* the functions of the three pairs */
        uint32_t a_eq = 0, a0 = 0, a1 = 0, cbeta = 0;
        if (q->kind == PRED_EQ) {
            a_eq = (q->lo + r) & m;
        } else {
            a0 = (q->lo + r) & m;
            a1 = (q->hi + 1u + r) & m;
            cbeta = a1 <= a0 ? beta : 0u;
        }
        /* keys of pair j, party b: one DPF key or two DCF keys (a1 then a0) */
        size_t half_len = q->kind == PRED_EQ ? dpf_len : 2 * dcf_len;
        uint8_t keys[3][2][MAX_HALF];   /* [pair][party][bytes of one key half] */
        for (int j = 0; j < 3; j++) {
            if (q->kind == PRED_EQ) {
                uint8_t s0[16], s1[16];
                rng_block(&g, s0);
                rng_block(&g, s1);
                if (onehot) orc_dpf_gen_et(n, a_eq, s0, s1, keys[j][0], keys[j][1]);
                else orc_dpf_gen_g(n, a_eq, beta, s0, s1, keys[j][0], keys[j][1], group);
            } else {
                uint8_t s0[16], s1[16];
                rng_block(&g, s0);
                rng_block(&g, s1);
                if (onehot) orc_dcf_gen_et(n, a1, s0, s1, keys[j][0], keys[j][1]);
                else orc_dcf_gen_g(n, a1, beta, s0, s1, keys[j][0], keys[j][1], group);
                rng_block(&g, s0);
                rng_block(&g, s1);
                /* over Z_2, -beta = beta = 1 */
                if (onehot) orc_dcf_gen_et(n, a0, s0, s1, keys[j][0] + dcf_len, keys[j][1] + dcf_len);
                else orc_dcf_gen_g(n, a0, 0u - beta, s0, s1, keys[j][0] + dcf_len, keys[j][1] + dcf_len, group);
            }
        }
        for (int i = 0; i < 3; i++) {
            uint8_t* rec = tok[i] + off;
            memset(rec, 0, 24);
            rec[0] = (uint8_t)q->kind; rec[1] = (uint8_t)n;
            rec[2] = (uint8_t)q->table; rec[3] = (uint8_t)(q->table >> 8);
            rec[4] = (uint8_t)q->attr; rec[5] = (uint8_t)(q->attr >> 8);
            rec[6] = (uint8_t)q->group; rec[7] = (uint8_t)(q->group >> 8);
            put32(rec + 8, rs[i]);
            put32(rec + 12, rs[(i + 1) % 3]);
            put32(rec + 16, cbeta);
            rec[20] = (uint8_t)q->combine;
            for (int h = 0; h < 2; h++) {
                int j = HOLD_PAIR[i][h] - 1, b = HOLD_PARTY[i][h];
                memcpy(rec + 24 + (size_t)h * half_len, keys[j][b], half_len);
            }
        }
        off += 24 + 2 * half_len;
    }
    return 0;
}

int orc_keygen(const orc_pred* preds, uint32_t n_preds, int n, const uint8_t seed[16],
               uint8_t* tok1, uint8_t* tok2, uint8_t* tok3, size_t cap)
{
    return keygen_impl(preds, n_preds, n, seed, tok1, tok2, tok3, cap, 0);
}

int orc_keygen_onehot(const orc_pred* preds, uint32_t n_preds, int n, const uint8_t seed[16],
                      uint8_t* tok1, uint8_t* tok2, uint8_t* tok3, size_t cap)
{
    return keygen_impl(preds, n_preds, n, seed, tok1, tok2, tok3, cap, 1);
}

/* ------------------------------------------------------------------------ */
/* Server-side evaluation: secEval (Alg. 3), re-share (Sec. III-B), AND fold  */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint64_t n_elems;
    uint32_t n_attrs;
    uint32_t n_bits;
    const uint32_t* share[3];   /* share[j][attr * n_elems + e], additive mod 2^n_bits */
} orc_table;

typedef struct {
    const uint8_t* rec[3];      /* the predicate's record in each server's token */
    int kind, n, table, attr, group;
    int combine;                /* COMBINE_* */
    int out_group;              /* 0 = Z_{2^32} (masked mode), 1 = Z_2 (one-hot mode) */
} pred_view;

static int parse_tokens(const uint8_t* const tok[3], const size_t tok_len[3], pred_view* pv, int max_preds)
{
    int np = -1, n = -1;
    for (int i = 0; i < 3; i++) {
        if (tok_len[i] < 16 || le32(tok[i]) != TOKEN_MAGIC || tok[i][4] != 1 || tok[i][5] != i + 1) return -1;
        if (tok[i][7] != tok[0][7] || tok[i][7] > GROUP_Z2) return -1;
        if (le32(tok[i] + 12) != tok_len[i]) return -1;
        int this_np = tok[i][8] | (tok[i][9] << 8);
        if (np < 0) { np = this_np; n = tok[i][6]; }
        else if (np != this_np || n != tok[i][6]) return -1;
    }
    if (np <= 0 || np > max_preds || n < 1 || n > 32) return -1;
    size_t off = 16;
    const int onehot = tok[0][7] == GROUP_Z2;
    if (onehot && n > 16) return -1;
    size_t dpf_len = key_len_mode(KIND_DPF, n, onehot), dcf_len = key_len_mode(KIND_DCF, n, onehot);
    for (int p = 0; p < np; p++) {
        if (off + 24 > tok_len[0]) return -1;
        const uint8_t* r0 = tok[0] + off;
        int kind = r0[0];
        if (kind != PRED_EQ && kind != PRED_RANGE) return -1;
        size_t half_len = kind == PRED_EQ ? dpf_len : 2 * dcf_len;
        if (off + 24 + 2 * half_len > tok_len[0]) return -1;
        pv[p].kind = kind;
        pv[p].n = r0[1];
        pv[p].table = r0[2] | (r0[3] << 8);
        pv[p].attr = r0[4] | (r0[5] << 8);
        pv[p].group = r0[6] | (r0[7] << 8);
        pv[p].combine = r0[20];
        pv[p].out_group = tok[0][7];
        if (r0[20] > COMBINE_OR || r0[21] || r0[22] || r0[23]) return -1;
        int first = 1;
        for (int e = 0; e < p; e++)
            if (pv[e].group == pv[p].group) first = 0;
        if (first && pv[p].combine != COMBINE_AND) return -1;
        for (int i = 0; i < 3; i++) {
            pv[p].rec[i] = tok[i] + off;
            if (memcmp(tok[i] + off, r0, 8) != 0 || memcmp(tok[i] + off + 20, r0 + 20, 4) != 0) return -1;
        }
        off += 24 + 2 * half_len;
    }
    if (off != tok_len[0]) return -1;
    return np;
}

/* F(k, ctr): bytes 0..3 of AES_k(ctr) with ctr = elem (u64) || step (u16) || table (u16) || query (u32) */
static uint32_t prf(const aes_ks* k, uint64_t elem, uint32_t step, uint32_t table, uint32_t query)
{
    uint8_t c[16], o[16];
    for (int i = 0; i < 8; i++) c[i] = (uint8_t)(elem >> (8 * i));
    c[8] = (uint8_t)step; c[9] = (uint8_t)(step >> 8);
    c[10] = (uint8_t)table; c[11] = (uint8_t)(table >> 8);
    put32(c + 12, query);
    aes_encrypt(k, c, o);
    return le32(o);
}

/* re-share a 3-out-of-3 additive sharing z into RSS: r_i = z_i + F(k_i, ctr) - F(k_{i-1}, ctr) */
static void reshare(const aes_ks prf_ks[3], const uint32_t z[3], uint32_t out[3],
                    uint64_t elem, uint32_t step, uint32_t table, uint32_t query)
{
    uint32_t f[3];
    for (int i = 0; i < 3; i++) f[i] = prf(&prf_ks[i], elem, step, table, query);
    for (int i = 0; i < 3; i++) out[i] = z[i] + f[i] - f[(i + 2) % 3];
}

/*
 * Aggregation of a target's predicates (Sec. V-D) over RSS shares of 0/1 values in
 * Z_{2^32}: acc = (a_i, a_{i+1}) and b = (b_i, b_{i+1}) held by CS_i.  Server i's
 * additive share of the product a b is a_i b_i + a_i b_{i+1} + a_{i+1} b_i (Sec. III-B).
 *   all predicates hold:   a b
 *   "one of" (paper's XOR): a XOR b = a + b - 2 a b
 *   at least one (OR):     a OR b  = a + b - a b
 * The result is 3-out-of-3 additive and is re-shared by the caller.
 */
static void fold_z2_32(int combine, const uint32_t a[3], const uint32_t b[3], uint32_t w[3])
{
    for (int i = 0; i < 3; i++) {
        int i1 = (i + 1) % 3;
        uint32_t ab = a[i] * b[i] + a[i] * b[i1] + a[i1] * b[i];
        if (combine == COMBINE_AND) w[i] = ab;
        else if (combine == COMBINE_XOR) w[i] = a[i] + b[i] - 2u * ab;
        else w[i] = a[i] + b[i] - ab;
    }
}

/* the same over binary RSS (one-hot mode, Z_2): a b, a ^ b, a ^ b ^ a b */
static void fold_z2(int combine, const uint32_t a[3], const uint32_t b[3], uint32_t w[3])
{
    for (int i = 0; i < 3; i++) {
        int i1 = (i + 1) % 3;
        uint32_t ab = (a[i] & b[i]) ^ (a[i] & b[i1]) ^ (a[i1] & b[i]);
        if (combine == COMBINE_AND) w[i] = ab;
        else if (combine == COMBINE_XOR) w[i] = a[i] ^ b[i];
        else w[i] = a[i] ^ b[i] ^ ab;
    }
}

/* y for one key half held by a server: DPF (EQ) or two DCFs plus c*beta' for party 0 (RANGE) */
static uint32_t eval_half(const pred_view* pv, int server, int h, uint32_t xhat)
{
    size_t dpf_len = orc_key_len(KIND_DPF, pv->n), dcf_len = orc_key_len(KIND_DCF, pv->n);
    const uint8_t* rec = pv->rec[server];
    if (pv->kind == PRED_EQ) {
        const uint8_t* key = rec + 24 + (size_t)h * dpf_len;
        return orc_dpf_eval(key, xhat);
    }
    const uint8_t* k_hi = rec + 24 + (size_t)h * 2 * dcf_len;
    const uint8_t* k_lo = k_hi + dcf_len;
    uint32_t y = orc_dcf_eval(k_hi, xhat) + orc_dcf_eval(k_lo, xhat);
    if (k_hi[2] == 0) y += le32(rec + 16);
    return y;
}

/*
 * Evaluate and-group `group` of the query on the listed elements of its table.
 * out is [3][n_sel]: the three RSS share sets of the AND of the group's predicates.
 * Returns 0, or a negative code on malformed input.
 */
int orc_filter(const uint8_t* tok1, const uint8_t* tok2, const uint8_t* tok3, const size_t tok_len[3],
               uint32_t query_id, const uint8_t prf_keys[48], const orc_table* tables, uint32_t n_tables,
               uint32_t group, const uint64_t* elems, uint64_t n_sel, uint32_t* out)
{
    const uint8_t* tok[3] = {tok1, tok2, tok3};
    pred_view pv[64];
    int np = parse_tokens(tok, tok_len, pv, 64);
    if (np < 0 || pv[0].out_group != GROUP_Z2_32) return -1;
    int members[64], nm = 0;
    for (int p = 0; p < np; p++)
        if ((uint32_t)pv[p].group == group) members[nm++] = p;
    if (nm == 0) return -2;
    int table = pv[members[0]].table;
    for (int k = 0; k < nm; k++) {
        const pred_view* q = &pv[members[k]];
        if (q->table != table || (uint32_t)q->table >= n_tables) return -3;
        if ((uint32_t)q->attr >= tables[table].n_attrs || (uint32_t)q->n != tables[table].n_bits) return -3;
    }
    const orc_table* T = &tables[table];
    aes_ks prf_ks[3];
    for (int i = 0; i < 3; i++) key_expansion(prf_keys + 16 * i, &prf_ks[i]);
    for (uint64_t s = 0; s < n_sel; s++) {
        uint64_t e = elems[s];
        if (e >= T->n_elems) return -4;
        uint32_t acc[3] = {0, 0, 0};
        for (int k = 0; k < nm; k++) {
            int p = members[k];
            const pred_view* q = &pv[p];
            uint32_t m = mask_n(q->n);
            /* open x^ = x + r: every server adds its own share of x and of r */
            uint32_t xhat = 0;
            for (int j = 0; j < 3; j++)
                xhat += T->share[j][(uint64_t)q->attr * T->n_elems + e] + le32(q->rec[j] + 8);
            xhat &= m;
            /* Eq. (predEval): CS_i sums its two key halves */
            uint32_t z[3];
            for (int i = 0; i < 3; i++) z[i] = eval_half(q, i, 0, xhat) + eval_half(q, i, 1, xhat);
            uint32_t bsh[3];
            reshare(prf_ks, z, bsh, e, (uint32_t)p, (uint32_t)table, query_id);
            if (k == 0) {
                memcpy(acc, bsh, sizeof acc);
            } else {
                uint32_t w[3];
                fold_z2_32(q->combine, acc, bsh, w);
                reshare(prf_ks, w, acc, e, 64u + (uint32_t)p, (uint32_t)table, query_id);
            }
        }
        for (int i = 0; i < 3; i++) out[(uint64_t)i * n_sel + s] = acc[i];
    }
    return 0;
}

/* the per-server additive shares z_1..z_3 of one predicate before the re-share (for invariant tests) */
int orc_pred_z(const uint8_t* tok1, const uint8_t* tok2, const uint8_t* tok3, const size_t tok_len[3],
               uint32_t pred, uint32_t xhat, uint32_t z_out[3], uint32_t y_out[6])
{
    const uint8_t* tok[3] = {tok1, tok2, tok3};
    pred_view pv[64];
    int np = parse_tokens(tok, tok_len, pv, 64);
    if (np < 0 || pred >= (uint32_t)np) return -1;
    for (int i = 0; i < 3; i++) {
        uint32_t y0 = eval_half(&pv[pred], i, 0, xhat), y1 = eval_half(&pv[pred], i, 1, xhat);
        y_out[2 * i] = y0;
        y_out[2 * i + 1] = y1;
        z_out[i] = y0 + y1;
    }
    return 0;
}

/* re-share on its own, for the zero-sharing invariant */
void orc_reshare(const uint8_t prf_keys[48], const uint32_t z[3], uint32_t out[3],
                 uint64_t elem, uint32_t step, uint32_t table, uint32_t query)
{
    aes_ks prf_ks[3];
    for (int i = 0; i < 3; i++) key_expansion(prf_keys + 16 * i, &prf_ks[i]);
    reshare(prf_ks, z, out, elem, step, table, query);
}

/* ------------------------------------------------------------------------ */
/* One-hot mode: secEval exactly as Eq. (predEval) writes it (Sec. V-D)      */
/* ------------------------------------------------------------------------ */
/*
 * A value v of an n-bit attribute is the one-hot vector e_v in {0,1}^(2^n), shared
 * in binary RSS: e_v = <e>_1 xor <e>_2 xor <e>_3 (Sec. V-B).  Storage: bit l of
 * the vector is bit (l mod 32) of 32-bit word l / 32; share[j] holds, per attribute
 * and element, W = max(1, 2^n / 32) words: share[j][(attr * n_elems + e) * W + w].
 * Server CS_i evaluates its key halves at every public position l and computes
 *   x = XOR_l Eval(k, l) AND <e>_j[l]
 * with j = i for its first half and j = i + 1 for its second (pair j meets share j),
 * XORs its two results, re-shares in binary RSS (F = prf_bit below) and the
 * group's predicates are ANDed with binary RSS multiplication.
 */
typedef struct {
    uint64_t n_elems;
    uint32_t n_attrs;
    uint32_t n_bits;
    const uint32_t* share[3];
} orc_onehot_table;

/* F(k, ctr) into Z_2: one AES block serves 128 consecutive elements.  The bit of element
 * e is bit e mod 128 (byte (e mod 128) / 8, bit e mod 8) of AES_k(c) with
 * c = u64 (e div 128) | 2^63 || u16 step || u16 table || u32 query; bit 63 of c keeps
 * these blocks apart from the masked mode's, whose element field stays below 2^63.
 * Distinct (e, step, table, query) read distinct bits of distinct blocks, so F stays a
 * PRF (Sec. III-B needs only that). */
static uint32_t prf_bit(const aes_ks* k, uint64_t elem, uint32_t step, uint32_t table, uint32_t query)
{
    uint8_t c[16], o[16];
    uint64_t blk = (elem >> 7) | (1ull << 63);
    uint32_t j = (uint32_t)(elem & 127u);
    for (int i = 0; i < 8; i++) c[i] = (uint8_t)(blk >> (8 * i));
    c[8] = (uint8_t)step; c[9] = (uint8_t)(step >> 8);
    c[10] = (uint8_t)table; c[11] = (uint8_t)(table >> 8);
    put32(c + 12, query);
    aes_encrypt(k, c, o);
    if (PLANTED == 1) return 0u;
    return (uint32_t)((o[j / 8] >> (j % 8)) & 1u);
}

uint32_t orc_prf_bit(const uint8_t key[16], uint64_t elem, uint32_t step, uint32_t table, uint32_t query)
{
    aes_ks ks;
    key_expansion(key, &ks);
    return prf_bit(&ks, elem, step, table, query);
}

static void reshare_bin(const aes_ks prf_ks[3], const uint32_t z[3], uint32_t out[3],
                        uint64_t elem, uint32_t step, uint32_t table, uint32_t query)
{
    uint32_t f[3];
    for (int i = 0; i < 3; i++) f[i] = prf_bit(&prf_ks[i], elem, step, table, query);
    for (int i = 0; i < 3; i++) out[i] = z[i] ^ f[i] ^ f[(i + 2) % 3];
}

/* value of server i's key half h at public position l (0/1) */
static uint32_t half_at(const pred_view* pv, int server, int h, uint32_t l)
{
    size_t dpf_len = orc_key_len_et(KIND_DPF, pv->n), dcf_len = orc_key_len_et(KIND_DCF, pv->n);
    const uint8_t* rec = pv->rec[server];
    if (pv->kind == PRED_EQ) return orc_eval_et(rec + 24 + (size_t)h * dpf_len, l);
    const uint8_t* k_hi = rec + 24 + (size_t)h * 2 * dcf_len;
    const uint8_t* k_lo = k_hi + dcf_len;
    uint32_t y = orc_eval_et(k_hi, l) ^ orc_eval_et(k_lo, l);
    if (k_hi[2] == 0) y ^= le32(rec + 16) & 1u;
    return y;
}

#include <stdlib.h>

int orc_filter_onehot(const uint8_t* tok1, const uint8_t* tok2, const uint8_t* tok3, const size_t tok_len[3],
                      uint32_t query_id, const uint8_t prf_keys[48], const orc_onehot_table* tables,
                      uint32_t n_tables, uint32_t group, const uint64_t* elems, uint64_t n_sel, uint32_t* out)
{
    const uint8_t* tok[3] = {tok1, tok2, tok3};
    pred_view pv[64];
    int np = parse_tokens(tok, tok_len, pv, 64);
    if (np < 0 || pv[0].out_group != GROUP_Z2) return -1;
    int members[64], nm = 0;
    for (int p = 0; p < np; p++)
        if ((uint32_t)pv[p].group == group) members[nm++] = p;
    if (nm == 0) return -2;
    int table = pv[members[0]].table;
    for (int k = 0; k < nm; k++) {
        const pred_view* q = &pv[members[k]];
        if (q->table != table || (uint32_t)q->table >= n_tables) return -3;
        if ((uint32_t)q->attr >= tables[table].n_attrs || (uint32_t)q->n != tables[table].n_bits) return -3;
    }
    const orc_onehot_table* T = &tables[table];
    const uint32_t D = 1u << T->n_bits;
    const uint32_t W = D >= 32 ? D / 32 : 1;
    /* Eval of every key half at every public position, once per predicate */
    uint8_t* ev = (uint8_t*)malloc((size_t)nm * 6 * D);
    if (!ev) return -5;
    for (int k = 0; k < nm; k++)
        for (int i = 0; i < 3; i++)
            for (int h = 0; h < 2; h++)
                for (uint32_t l = 0; l < D; l++)
                    ev[(((size_t)k * 3 + i) * 2 + h) * D + l] = (uint8_t)half_at(&pv[members[k]], i, h, l);
    aes_ks prf_ks[3];
    for (int i = 0; i < 3; i++) key_expansion(prf_keys + 16 * i, &prf_ks[i]);
    for (uint64_t s = 0; s < n_sel; s++) {
        uint64_t e = elems[s];
        if (e >= T->n_elems) { free(ev); return -4; }
        uint32_t acc[3] = {0, 0, 0};
        for (int k = 0; k < nm; k++) {
            int p = members[k];
            const pred_view* q = &pv[p];
            uint32_t z[3];
            for (int i = 0; i < 3; i++) {
                z[i] = 0;
                for (int h = 0; h < 2; h++) {
                    const uint32_t* d = T->share[(i + h) % 3] + ((uint64_t)q->attr * T->n_elems + e) * W;
                    const uint8_t* v = ev + (((size_t)k * 3 + i) * 2 + h) * D;
                    uint32_t x = 0;
                    for (uint32_t l = 0; l < D; l++) x ^= v[l] & ((d[l / 32] >> (l % 32)) & 1u);
                    z[i] ^= x;
                }
            }
            uint32_t bsh[3];
            reshare_bin(prf_ks, z, bsh, e, (uint32_t)p, (uint32_t)table, query_id);
            if (k == 0) {
                memcpy(acc, bsh, sizeof acc);
            } else {
                uint32_t w[3];
                fold_z2(q->combine, acc, bsh, w);
                reshare_bin(prf_ks, w, acc, e, 64u + (uint32_t)p, (uint32_t)table, query_id);
            }
        }
        for (int i = 0; i < 3; i++) out[(uint64_t)i * n_sel + s] = acc[i];
    }
    free(ev);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Fresh masks and keys per element (Sec. V-C, the basic masked approach)    */
/* ------------------------------------------------------------------------ */
/*
 * The masked-input approach as the paper first describes it: every attribute
 * value gets its own mask and its own keys.  For predicate p and element c of its
 * table the client's randomness is AES_K of the block B(c, p, tag, j) =
 * u64 c || u16 p || u16 tag || u32 j under the client seed K:
 *   tag 1, j 0: r = bytes 0..3, <r>_1 = bytes 4..7, <r>_2 = bytes 8..11 (each mod
 *               2^n), <r>_3 = r - <r>_1 - <r>_2 mod 2^n;
 *   tag 2, j = 4 pair + 2 sub + b: root seed of party b for key `sub` of `pair`.
 * The functions are those of the per-predicate token (EQ: DPF at lo + r; RANGE:
 * DCF at hi + 1 + r with beta', DCF at lo + r with -beta', c beta' with
 * c = [a1 <= a0]), and the servers combine, re-share and AND exactly as orc_filter.
 *
 * Token layout (per server i; little-endian; N4 = N rounded up to 4):
 *   64 B header: u32 0x464D474F, u8 1, u8 i, u8 n, u8 0, u16 n_preds, u16 0,
 *     u32 0, u64 total length, zeros;
 *   32 B per predicate: u8 kind, u8 n, u16 table, u16 attr, u16 group, u64 N,
 *     u64 offset of the data block, u64 0;
 *   data block: u32 rA[N4], u32 rB[N4], (RANGE) u32 cb[N4], then key blocks
 *     (A,0), (A,1), (B,0), (B,1) (sub 1 for RANGE only), each: 16-byte seed[N],
 *     16-byte scw[n][N], u32 tl[N4], u32 tr[N4], (DCF) u32 vcw[n][N4], u32 cw[N4].
 */
#define FRESH_MAGIC 0x464D474Fu
#define MAX_KEY (24 + 32 * 24 + 4)

static uint64_t round4(uint64_t x) { return (x + 3u) & ~(uint64_t)3u; }

static uint64_t fresh_key_block_len(int kind, int n, uint64_t N)
{
    uint64_t N4 = round4(N);
    uint64_t len = 16u * N + 16u * (uint64_t)n * N + 8u * N4 + 4u * N4;
    if (kind == KIND_DCF) len += 4u * (uint64_t)n * N4;
    return len;
}

static uint64_t fresh_data_len(int pred_kind, int n, uint64_t N)
{
    uint64_t N4 = round4(N);
    if (pred_kind == PRED_EQ) return 8u * N4 + 2u * fresh_key_block_len(KIND_DPF, n, N);
    return 12u * N4 + 4u * fresh_key_block_len(KIND_DCF, n, N);
}

static int fresh_check(const orc_pred* preds, uint32_t n_preds, int n, const uint64_t* table_elems, uint32_t n_tables)
{
    if (n < 1 || n > 32 || n_preds == 0 || n_preds > 64) return -1;
    uint32_t m = mask_n(n);
    for (uint32_t p = 0; p < n_preds; p++) {
        const orc_pred* q = &preds[p];
        if (q->kind == PRED_EQ) { if (q->lo > m) return -1; }
        else if (q->kind == PRED_RANGE) { if (q->lo > q->hi || q->hi > m) return -1; }
        else return -1;
        if (q->table >= n_tables || q->attr > 0xFFFF || q->group > 0xFFFF) return -1;
        if (q->combine > COMBINE_OR || (first_of_group(preds, p) && q->combine != COMBINE_AND)) return -1;
    }
    return 0;
}

uint64_t orc_fresh_token_len(const orc_pred* preds, uint32_t n_preds, int n, const uint64_t* table_elems,
                             uint32_t n_tables)
{
    if (fresh_check(preds, n_preds, n, table_elems, n_tables)) return 0;
    uint64_t len = 64u + 32u * n_preds;
    for (uint32_t p = 0; p < n_preds; p++) len += fresh_data_len((int)preds[p].kind, n, table_elems[preds[p].table]);
    return len;
}

static void client_block(const aes_ks* K, uint64_t c, uint32_t p, uint32_t tag, uint32_t j, uint8_t out[16])
{
    uint8_t b[16];
    for (int i = 0; i < 8; i++) b[i] = (uint8_t)(c >> (8 * i));
    b[8] = (uint8_t)p; b[9] = (uint8_t)(p >> 8);
    b[10] = (uint8_t)tag; b[11] = (uint8_t)(tag >> 8);
    put32(b + 12, j);
    aes_encrypt(K, b, out);
}

/* element c's mask shares, c*beta', and its key pairs in wire format:
 * keys[pair][sub][party] (sub 1 only for RANGE) */
static void fresh_element(const aes_ks* K, const orc_pred* q, uint32_t p, int n, uint64_t c, uint32_t rs[3],
                          uint32_t* cbeta, uint8_t keys[3][2][2][MAX_KEY])
{
    uint32_t m = mask_n(n);
    uint8_t blk[16];
    client_block(K, c, p, 1, 0, blk);
    uint32_t r = mask_words(blk, m, rs);
    *cbeta = 0;
    for (int pair = 0; pair < 3; pair++) {
        uint8_t s0[16], s1[16];
        if (q->kind == PRED_EQ) {
            client_block(K, c, p, 2, 4u * pair + 0, s0);
            client_block(K, c, p, 2, 4u * pair + 1, s1);
            orc_dpf_gen(n, (q->lo + r) & m, BETA_PRIME, s0, s1, keys[pair][0][0], keys[pair][0][1]);
        } else {
            uint32_t a0 = (q->lo + r) & m, a1 = (q->hi + 1u + r) & m;
            *cbeta = a1 <= a0 ? BETA_PRIME : 0u;
            client_block(K, c, p, 2, 4u * pair + 0, s0);
            client_block(K, c, p, 2, 4u * pair + 1, s1);
            orc_dcf_gen(n, a1, BETA_PRIME, s0, s1, keys[pair][0][0], keys[pair][0][1]);
            client_block(K, c, p, 2, 4u * pair + 2, s0);
            client_block(K, c, p, 2, 4u * pair + 3, s1);
            orc_dcf_gen(n, a0, 0u - BETA_PRIME, s0, s1, keys[pair][1][0], keys[pair][1][1]);
        }
    }
}

static void put_u64(uint8_t* p, uint64_t v)
{
    for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i));
}

static uint64_t get_u64(const uint8_t* p)
{
    uint64_t v = 0;
    for (int i = 0; i < 8; i++) v |= (uint64_t)p[i] << (8 * i);
    return v;
}

/* copy one wire-format key of element c into key block `blk` (layout above) */
static void scatter_key(uint8_t* blk, int kind, int n, uint64_t N, uint64_t c, const uint8_t* key)
{
    uint64_t N4 = round4(N);
    size_t lb = level_bytes(kind);
    memcpy(blk + 16u * c, key + 8, 16);
    uint8_t* scw = blk + 16u * N;
    uint8_t* tl = scw + 16u * (uint64_t)n * N;
    uint8_t* tr = tl + 4u * N4;
    uint8_t* vcw = tr + 4u * N4;
    uint8_t* cw = vcw + (kind == KIND_DCF ? 4u * (uint64_t)n * N4 : 0u);
    uint32_t tlw = 0, trw = 0;
    for (int l = 1; l <= n; l++) {
        const uint8_t* rec = key + 24 + (size_t)(l - 1) * lb;
        memcpy(scw + 16u * ((uint64_t)(l - 1) * N + c), rec, 16);
        tlw |= (uint32_t)(rec[16] & 1u) << (l - 1);
        trw |= (uint32_t)(rec[17] & 1u) << (l - 1);
        if (kind == KIND_DCF) memcpy(vcw + 4u * ((uint64_t)(l - 1) * N4 + c), rec + 20, 4);
    }
    put32(tl + 4u * c, tlw);
    put32(tr + 4u * c, trw);
    memcpy(cw + 4u * c, key + 24 + (size_t)n * lb, 4);
}

/*
 * Client key generation for the fresh-key mode, element by element.  Returns 0, -1
 * on an invalid predicate, -2 if cap is smaller than orc_fresh_token_len.
 */
int orc_keygen_fresh(const orc_pred* preds, uint32_t n_preds, int n, const uint64_t* table_elems, uint32_t n_tables,
                     const uint8_t seed[16], uint8_t* tok1, uint8_t* tok2, uint8_t* tok3, uint64_t cap)
{
    uint8_t* tok[3] = {tok1, tok2, tok3};
    if (fresh_check(preds, n_preds, n, table_elems, n_tables)) return -1;
    uint64_t total = orc_fresh_token_len(preds, n_preds, n, table_elems, n_tables);
    if (cap < total) return -2;
    aes_ks K;
    key_expansion(seed, &K);
    for (int i = 0; i < 3; i++) {
        memset(tok[i], 0, (size_t)total);
        put32(tok[i], FRESH_MAGIC);
        tok[i][4] = 1; tok[i][5] = (uint8_t)(i + 1); tok[i][6] = (uint8_t)n;
        tok[i][8] = (uint8_t)n_preds; tok[i][9] = (uint8_t)(n_preds >> 8);
        put_u64(tok[i] + 16, total);
    }
    uint8_t keys[3][2][2][MAX_KEY];
    uint64_t off = 64u + 32u * n_preds;
    for (uint32_t p = 0; p < n_preds; p++) {
        const orc_pred* q = &preds[p];
        uint64_t N = table_elems[q->table], N4 = round4(N);
        int eq = q->kind == PRED_EQ;
        int kkind = eq ? KIND_DPF : KIND_DCF, nsub = eq ? 1 : 2;
        uint64_t kb = fresh_key_block_len(kkind, n, N);
        for (int i = 0; i < 3; i++) {
            uint8_t* d = tok[i] + 64 + 32 * p;
            d[0] = (uint8_t)q->kind; d[1] = (uint8_t)n;
            d[2] = (uint8_t)q->table; d[3] = (uint8_t)(q->table >> 8);
            d[4] = (uint8_t)q->attr; d[5] = (uint8_t)(q->attr >> 8);
            d[6] = (uint8_t)q->group; d[7] = (uint8_t)(q->group >> 8);
            put_u64(d + 8, N);
            put_u64(d + 16, off);
            d[24] = (uint8_t)q->combine;
        }
        uint64_t keys_at = (eq ? 8u : 12u) * N4;
        for (uint64_t c = 0; c < N; c++) {
            uint32_t rs[3], cbeta;
            fresh_element(&K, q, p, n, c, rs, &cbeta, keys);
            for (int i = 0; i < 3; i++) {
                uint8_t* blk = tok[i] + off;
                put32(blk + 4u * c, rs[i]);
                put32(blk + 4u * N4 + 4u * c, rs[(i + 1) % 3]);
                if (!eq) put32(blk + 8u * N4 + 4u * c, cbeta);
                for (int h = 0; h < 2; h++) {
                    int pair = HOLD_PAIR[i][h] - 1, b = HOLD_PARTY[i][h];
                    for (int s = 0; s < nsub; s++)
                        scatter_key(blk + keys_at + (uint64_t)(h * nsub + s) * kb, kkind, n, N, c, keys[pair][s][b]);
                }
            }
        }
        off += fresh_data_len((int)q->kind, n, N);
    }
    return 0;
}

/* rebuild the wire-format key of element c from key block `blk` */
static void gather_key(const uint8_t* blk, int kind, int n, uint64_t N, uint64_t c, int party, uint8_t* key)
{
    uint64_t N4 = round4(N);
    size_t lb = level_bytes(kind);
    memset(key, 0, orc_key_len(kind, n));
    key[0] = (uint8_t)kind; key[1] = (uint8_t)n; key[2] = (uint8_t)party;
    memcpy(key + 8, blk + 16u * c, 16);
    const uint8_t* scw = blk + 16u * N;
    const uint8_t* tl = scw + 16u * (uint64_t)n * N;
    const uint8_t* tr = tl + 4u * N4;
    const uint8_t* vcw = tr + 4u * N4;
    const uint8_t* cw = vcw + (kind == KIND_DCF ? 4u * (uint64_t)n * N4 : 0u);
    uint32_t tlw = le32(tl + 4u * c), trw = le32(tr + 4u * c);
    for (int l = 1; l <= n; l++) {
        uint8_t* rec = key + 24 + (size_t)(l - 1) * lb;
        memcpy(rec, scw + 16u * ((uint64_t)(l - 1) * N + c), 16);
        rec[16] = (uint8_t)((tlw >> (l - 1)) & 1u);
        rec[17] = (uint8_t)((trw >> (l - 1)) & 1u);
        if (kind == KIND_DCF) memcpy(rec + 20, vcw + 4u * ((uint64_t)(l - 1) * N4 + c), 4);
    }
    memcpy(key + 24 + (size_t)n * lb, cw + 4u * c, 4);
}

/*
 * The servers' side on fresh tokens: and-group `group` on the listed elements, out
 * [3][n_sel] as orc_filter.  Element c reads its own mask shares and keys.
 * Returns 0 or a negative code on malformed input.
 */
int orc_filter_fresh(const uint8_t* tok1, const uint8_t* tok2, const uint8_t* tok3, uint32_t query_id,
                     const uint8_t prf_keys[48], const orc_table* tables, uint32_t n_tables, uint32_t group,
                     const uint64_t* elems, uint64_t n_sel, uint32_t* out)
{
    const uint8_t* tok[3] = {tok1, tok2, tok3};
    for (int i = 0; i < 3; i++) {
        if (le32(tok[i]) != FRESH_MAGIC || tok[i][4] != 1 || tok[i][5] != i + 1) return -1;
        if (memcmp(tok[i] + 6, tok[0] + 6, 4) != 0 || get_u64(tok[i] + 16) != get_u64(tok[0] + 16)) return -1;
    }
    int n = tok[0][6], np = tok[0][8] | (tok[0][9] << 8);
    if (n < 1 || n > 32 || np < 1 || np > 64) return -1;
    int members[64], nm = 0, table = -1;
    for (int p = 0; p < np; p++) {
        const uint8_t* d = tok[0] + 64 + 32 * p;
        for (int i = 1; i < 3; i++)
            if (memcmp(tok[i] + 64 + 32 * p, d, 32) != 0) return -1;
        if (d[24] > COMBINE_OR) return -1;
        for (int b = 25; b < 32; b++)
            if (d[b]) return -1;
        if ((uint32_t)(d[6] | (d[7] << 8)) != group) continue;
        if (nm == 0 && d[24] != COMBINE_AND) return -1;
        int t = d[2] | (d[3] << 8);
        if (table >= 0 && t != table) return -3;
        table = t;
        members[nm++] = p;
    }
    if (nm == 0) return -2;
    if ((uint32_t)table >= n_tables) return -3;
    const orc_table* T = &tables[table];
    aes_ks prf_ks[3];
    for (int i = 0; i < 3; i++) key_expansion(prf_keys + 16 * i, &prf_ks[i]);
    uint8_t key[MAX_KEY];
    for (uint64_t s = 0; s < n_sel; s++) {
        uint64_t e = elems[s];
        if (e >= T->n_elems) return -4;
        uint32_t acc[3] = {0, 0, 0};
        for (int k = 0; k < nm; k++) {
            int p = members[k];
            const uint8_t* d = tok[0] + 64 + 32 * p;
            int kind = d[0], attr = d[4] | (d[5] << 8);
            uint64_t N = get_u64(d + 8), off = get_u64(d + 16), N4 = round4(N);
            if (N != T->n_elems || (uint32_t)attr >= T->n_attrs || (uint32_t)n != T->n_bits) return -3;
            int eq = kind == PRED_EQ;
            int kkind = eq ? KIND_DPF : KIND_DCF, nsub = eq ? 1 : 2;
            uint64_t kb = fresh_key_block_len(kkind, n, N), keys_at = (eq ? 8u : 12u) * N4;
            /* open x^_e = x_e + r_e: server i contributes <x_e>_i + <r_e>_i */
            uint32_t xhat = 0;
            for (int i = 0; i < 3; i++)
                xhat += T->share[i][(uint64_t)attr * T->n_elems + e] + le32(tok[i] + off + 4u * e);
            xhat &= mask_n(n);
            uint32_t z[3];
            for (int i = 0; i < 3; i++) {
                const uint8_t* blk = tok[i] + off;
                z[i] = 0;
                for (int h = 0; h < 2; h++) {
                    int b = HOLD_PARTY[i][h];
                    for (int sb = 0; sb < nsub; sb++) {
                        gather_key(blk + keys_at + (uint64_t)(h * nsub + sb) * kb, kkind, n, N, e, b, key);
                        z[i] += eq ? orc_dpf_eval(key, xhat) : orc_dcf_eval(key, xhat);
                    }
                    if (!eq && b == 0) z[i] += le32(blk + 8u * N4 + 4u * e);
                }
            }
            uint32_t bsh[3];
            reshare(prf_ks, z, bsh, e, (uint32_t)p, (uint32_t)table, query_id);
            if (k == 0) {
                memcpy(acc, bsh, sizeof acc);
            } else {
                uint32_t w[3];
                fold_z2_32(d[24], acc, bsh, w);
                reshare(prf_ks, w, acc, e, 64u + (uint32_t)p, (uint32_t)table, query_id);
            }
        }
        for (int i = 0; i < 3; i++) out[(uint64_t)i * n_sel + s] = acc[i];
    }
    return 0;
}

/*
 * The same result computed straight from the client seed, without a token: element
 * e's keys are generated where they are used.  For sampled checks at sizes where a
 * whole token is too slow to build here.
 */
int orc_fresh_direct(const orc_pred* preds, uint32_t n_preds, int n, const uint64_t* table_elems,
                     uint32_t n_tables, const uint8_t seed[16], uint32_t query_id, const uint8_t prf_keys[48],
                     const orc_table* tables, uint32_t group, const uint64_t* elems, uint64_t n_sel, uint32_t* out)
{
    if (fresh_check(preds, n_preds, n, table_elems, n_tables)) return -1;
    int members[64], nm = 0, table = -1;
    for (uint32_t p = 0; p < n_preds; p++) {
        if (preds[p].group != group) continue;
        if (table >= 0 && (int)preds[p].table != table) return -3;
        table = (int)preds[p].table;
        members[nm++] = (int)p;
    }
    if (nm == 0) return -2;
    const orc_table* T = &tables[table];
    if (T->n_elems != table_elems[table] || (uint32_t)n != T->n_bits) return -3;
    aes_ks K, prf_ks[3];
    key_expansion(seed, &K);
    for (int i = 0; i < 3; i++) key_expansion(prf_keys + 16 * i, &prf_ks[i]);
    uint8_t keys[3][2][2][MAX_KEY];
    for (uint64_t s = 0; s < n_sel; s++) {
        uint64_t e = elems[s];
        if (e >= T->n_elems) return -4;
        uint32_t acc[3] = {0, 0, 0};
        for (int k = 0; k < nm; k++) {
            int p = members[k];
            const orc_pred* q = &preds[p];
            if (q->attr >= T->n_attrs) return -3;
            uint32_t rs[3], cbeta;
            fresh_element(&K, q, (uint32_t)p, n, e, rs, &cbeta, keys);
            uint32_t xhat = 0;
            for (int i = 0; i < 3; i++) xhat += T->share[i][(uint64_t)q->attr * T->n_elems + e] + rs[i];
            xhat &= mask_n(n);
            int eq = q->kind == PRED_EQ, nsub = eq ? 1 : 2;
            uint32_t z[3];
            for (int i = 0; i < 3; i++) {
                z[i] = 0;
                for (int h = 0; h < 2; h++) {
                    int pair = HOLD_PAIR[i][h] - 1, b = HOLD_PARTY[i][h];
                    for (int sb = 0; sb < nsub; sb++)
                        z[i] += eq ? orc_dpf_eval(keys[pair][sb][b], xhat) : orc_dcf_eval(keys[pair][sb][b], xhat);
                    if (!eq && b == 0) z[i] += cbeta;
                }
            }
            uint32_t bsh[3];
            reshare(prf_ks, z, bsh, e, (uint32_t)p, (uint32_t)table, query_id);
            if (k == 0) {
                memcpy(acc, bsh, sizeof acc);
            } else {
                uint32_t w[3];
                fold_z2_32(q->combine, acc, bsh, w);
                reshare(prf_ks, w, acc, e, 64u + (uint32_t)p, (uint32_t)table, query_id);
            }
        }
        for (int i = 0; i < 3; i++) out[(uint64_t)i * n_sel + s] = acc[i];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* secShuffle (Alg. 5, the protocol of Araki et al. the paper cites)         */
/* ------------------------------------------------------------------------ */
/*
 * A table D of n rows of W uint32 words, 3-out-of-3 shared as D = D1 op D2 op D3,
 * where op is XOR (binary RSS, as Alg. 5 is written) or addition mod 2^32 (the
 * arithmetic RSS the masked filter produces).  CS1/CS2 share seed s12, CS2/CS3
 * s23, CS3/CS1 s31.  From its seed a pair derives
 *   pi_ab  a pseudo-random permutation of [0, n): a 4-round balanced Feistel
 *          network on 2h bits (h = max(1, ceil(bits(n - 1) / 2))) with cycle
 *          walking; round r maps (L, R) to (R, L xor F_r(R)),
 *          F_r(R) = word 0 of AES_s(u64 R || u16 3 || u16 r || u32 n) mod 2^h;
 *   tables T_ab, R_a: word w of row i is word (w mod 4) of
 *          AES_s(u64 i || u16 tag || u16 (w / 4) || u32 0), tag 1 for T, 2 for R.
 * A permutation moves row i to row pi(i).  The steps, in the order Alg. 5 gives
 * them (X2 there is the X1 that CS2 receives), with "+"/"-" standing for XOR in
 * the binary case:
 *   CS1: X1 = pi31(pi12(D1 + D2 + T12) + T31)
 *   CS2: Y1 = pi12(D3 - T12);  C1 = pi23(X1 + T23) - R2
 *   CS3: C2 = pi23(pi31(Y1 - T31) - T23) - R1;  R3 = C1 + C2
 * Output shares (R1, R2, R3): R1 + R2 + R3 = pi23(pi31(pi12(D))).
 */
#define SHUF_XOR 1
#define SHUF_ADD 0

static int ceil_half_bits(uint64_t n)
{
    int b = 0;
    uint64_t v = n - 1;
    while (v) { b++; v >>= 1; }
    int h = (b + 1) / 2;
    return h < 1 ? 1 : h;
}

static uint32_t feistel_round(const aes_ks* K, uint32_t R, int r, uint64_t n, int h)
{
    uint8_t b[16], o[16];
    for (int i = 0; i < 8; i++) b[i] = (uint8_t)((uint64_t)R >> (8 * i));
    b[8] = 3; b[9] = 0;
    b[10] = (uint8_t)r; b[11] = 0;
    put32(b + 12, (uint32_t)n);
    aes_encrypt(K, b, o);
    return le32(o) & ((1u << h) - 1u);
}

static uint64_t feistel(const aes_ks* K, uint64_t x, uint64_t n, int h)
{
    uint32_t mask = (1u << h) - 1u;
    uint32_t L = (uint32_t)(x >> h) & mask, R = (uint32_t)x & mask;
    for (int r = 0; r < 4; r++) {
        uint32_t t = L ^ feistel_round(K, R, r, n, h);
        L = R;
        R = t;
    }
    return ((uint64_t)L << h) | R;
}

/* pi(x) for x < n: walk the Feistel cycle of x until it lands inside [0, n) */
static uint64_t prp_ks(const aes_ks* K, uint64_t n, uint64_t x)
{
    if (n <= 1) return 0;
    int h = ceil_half_bits(n);
    uint64_t y = feistel(K, x, n, h);
    while (y >= n) y = feistel(K, y, n, h);
    return y;
}

uint64_t orc_prp(const uint8_t seed[16], uint64_t n, uint64_t x)
{
    aes_ks K;
    key_expansion(seed, &K);
    return prp_ks(&K, n, x);
}

static uint32_t table_word(const aes_ks* K, int tag, uint64_t i, uint32_t w)
{
    uint8_t b[16], o[16];
    for (int k = 0; k < 8; k++) b[k] = (uint8_t)(i >> (8 * k));
    b[8] = (uint8_t)tag; b[9] = 0;
    b[10] = (uint8_t)(w / 4); b[11] = (uint8_t)(w / 4 >> 8);
    put32(b + 12, 0);
    aes_encrypt(K, b, o);
    return le32(o + 4 * (w % 4));
}

static uint32_t op_add(int g, uint32_t a, uint32_t b) { return g == SHUF_XOR ? a ^ b : a + b; }
static uint32_t op_sub(int g, uint32_t a, uint32_t b) { return g == SHUF_XOR ? a ^ b : a - b; }

/* dst[pi(i)] = src[i] for every row */
static void permute_rows(const uint64_t* pi, const uint32_t* src, uint32_t* dst, uint64_t n, uint32_t W)
{
    for (uint64_t i = 0; i < n; i++) memcpy(dst + pi[i] * W, src + i * W, W * sizeof(uint32_t));
}

static void fill_table(const aes_ks* K, int tag, uint32_t* t, uint64_t n, uint32_t W)
{
    for (uint64_t i = 0; i < n; i++)
        for (uint32_t w = 0; w < W; w++) t[i * W + w] = table_word(K, tag, i, w);
}

/*
 * in[j] / out[j]: share j+1 as n x W row-major words.  seeds: s12 || s23 || s31.
 * scratch: 8 n W words.  Returns 0.
 */
int orc_shuffle(int group, uint64_t n, uint32_t W, const uint32_t* in1, const uint32_t* in2, const uint32_t* in3,
                const uint8_t seeds[48], uint32_t* out1, uint32_t* out2, uint32_t* out3, uint32_t* scratch,
                uint64_t* perm_scratch)
{
    uint64_t NW = n * W;
    aes_ks K12, K23, K31;
    key_expansion(seeds, &K12);
    key_expansion(seeds + 16, &K23);
    key_expansion(seeds + 32, &K31);
    uint64_t* p12 = perm_scratch;
    uint64_t* p23 = perm_scratch + n;
    uint64_t* p31 = perm_scratch + 2 * n;
    for (uint64_t i = 0; i < n; i++) {
        p12[i] = prp_ks(&K12, n, i);
        p23[i] = prp_ks(&K23, n, i);
        p31[i] = prp_ks(&K31, n, i);
    }
    uint32_t* T12 = scratch;
    uint32_t* T23 = scratch + NW;
    uint32_t* T31 = scratch + 2 * NW;
    uint32_t* R1 = out1;   /* R1 and R2 are the final shares of CS1 (with CS3 / CS2) */
    uint32_t* R2 = out2;
    uint32_t* A = scratch + 3 * NW;
    uint32_t* X1 = scratch + 4 * NW;
    uint32_t* Y1 = scratch + 5 * NW;
    uint32_t* C1 = scratch + 6 * NW;
    uint32_t* C2 = scratch + 7 * NW;
    fill_table(&K12, 1, T12, n, W);   /* CS1, CS2 from s12: pi12, T12, R2 */
    fill_table(&K12, 2, R2, n, W);
    fill_table(&K23, 1, T23, n, W);   /* CS2, CS3 from s23: pi23, T23 */
    fill_table(&K31, 1, T31, n, W);   /* CS3, CS1 from s31: pi31, T31, R1 */
    fill_table(&K31, 2, R1, n, W);
    /* CS1: X1 = pi31(pi12(D1 + D2 + T12) + T31) */
    for (uint64_t k = 0; k < NW; k++) A[k] = op_add(group, op_add(group, in1[k], in2[k]), T12[k]);
    permute_rows(p12, A, X1, n, W);
    for (uint64_t k = 0; k < NW; k++) A[k] = op_add(group, X1[k], T31[k]);
    permute_rows(p31, A, X1, n, W);
    /* CS2: Y1 = pi12(D3 - T12); C1 = pi23(X1 + T23) - R2 */
    for (uint64_t k = 0; k < NW; k++) A[k] = op_sub(group, in3[k], T12[k]);
    permute_rows(p12, A, Y1, n, W);
    for (uint64_t k = 0; k < NW; k++) A[k] = op_add(group, X1[k], T23[k]);
    permute_rows(p23, A, C1, n, W);
    for (uint64_t k = 0; k < NW; k++) C1[k] = op_sub(group, C1[k], R2[k]);
    /* CS3: C2 = pi23(pi31(Y1 - T31) - T23) - R1; R3 = C1 + C2 */
    for (uint64_t k = 0; k < NW; k++) A[k] = op_sub(group, Y1[k], T31[k]);
    permute_rows(p31, A, C2, n, W);
    for (uint64_t k = 0; k < NW; k++) A[k] = op_sub(group, C2[k], T23[k]);
    permute_rows(p23, A, C2, n, W);
    for (uint64_t k = 0; k < NW; k++) {
        C2[k] = op_sub(group, C2[k], R1[k]);
        out3[k] = op_add(group, C1[k], C2[k]);
    }
    return 0;
}

/*
 * secFetch case II (Alg. 4): the candidates' records D_c = x_c || id_c || d_c are
 * shuffled (secShuffle over Z_{2^32}, additive shares as the masked filter gives
 * them), the shuffled x^ are opened, and the records whose x^ = 1 are kept, in
 * shuffled order, still shared.  id_c = c is shared as (c, 0, 0).
 * x[j]: filter result share j+1 (n values); attrs: the fetched attribute rows of T.
 * out[j]: share j+1 of the kept records, cap rows of (1 + n_attrs) words
 * (id, then the attributes).  Returns the number of kept records (it may exceed
 * cap; then only cap rows are written), or -1 on bad arguments.
 */
int64_t orc_fetch_multi(uint64_t n, const uint32_t* x1, const uint32_t* x2, const uint32_t* x3,
                        const orc_table* T, uint32_t n_attrs, const uint32_t* attrs, const uint8_t seeds[48],
                        uint32_t* out1, uint32_t* out2, uint32_t* out3, uint64_t cap, uint32_t* scratch,
                        uint64_t* perm_scratch)
{
    const uint32_t* x[3] = {x1, x2, x3};
    uint32_t* out[3] = {out1, out2, out3};
    if (T->n_elems != n) return -1;
    for (uint32_t a = 0; a < n_attrs; a++)
        if (attrs[a] >= T->n_attrs) return -1;
    uint32_t W = 2 + n_attrs;
    uint64_t NW = n * W;
    /* scratch: D[3] then S[3] then the shuffle's 8 n W words */
    uint32_t* D[3] = {scratch, scratch + NW, scratch + 2 * NW};
    uint32_t* S[3] = {scratch + 3 * NW, scratch + 4 * NW, scratch + 5 * NW};
    for (int j = 0; j < 3; j++)
        for (uint64_t c = 0; c < n; c++) {
            uint32_t* row = D[j] + c * W;
            row[0] = x[j][c];
            row[1] = j == 0 ? (uint32_t)c : 0u;
            for (uint32_t a = 0; a < n_attrs; a++) row[2 + a] = T->share[j][(uint64_t)attrs[a] * n + c];
        }
    orc_shuffle(SHUF_ADD, n, W, D[0], D[1], D[2], seeds, S[0], S[1], S[2], scratch + 6 * NW, perm_scratch);
    int64_t m = 0;
    for (uint64_t l = 0; l < n; l++) {
        uint32_t xh = S[0][l * W] + S[1][l * W] + S[2][l * W];
        if (xh != 1u) continue;
        if ((uint64_t)m < cap)
            for (int j = 0; j < 3; j++) memcpy(out[j] + (uint64_t)m * (W - 1), S[j] + l * W + 1, (W - 1) * 4);
        m++;
    }
    return m;
}

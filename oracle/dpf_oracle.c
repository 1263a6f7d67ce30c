/*
 * CPU oracle for two-server DPF-PIR over Z_2^32 — TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
 * this code.  It is a plain, slow, obviously correct restatement of the method
 * (Lam et al., "GPU-based Private Information Retrieval for On-Device Machine
 * Learning Inference", arXiv 2301.10904), written for checking by eye against
 * the paper and FIPS-197.  It shares no code with the CUDA library.
 *
 * What each function follows:
 *   - AES-128 (the PRF of Sec. 3.2.6): FIPS-197 Sec. 4 (GF(2^8)), Sec. 5.1
 *     (Cipher), Sec. 5.2 (KeyExpansion).  The S-box is derived from its
 *     definition (multiplicative inverse, then the affine map), not typed in.
 *   - PRF_s(x) = AES-128 under key s of the block (x, 0, ..., 0) (Sec. 3.1,
 *     text under Eq. p3: the PRF is a cipher keyed by s applied to x).
 *     Alternative PRF (Sec. 3.2.6, Table 5): ChaCha20 (RFC 8439 Sec. 2.1-2.3),
 *     block 0 under key s || 0^128 and an all-zero nonce, PRF_s(x) = its 16
 *     bytes at offset 16x.  The key header names the PRF.
 *   - Eval: the recurrence of Eqs. p1-p3 (Sec. 3.1), "+" read as XOR in
 *     F_{2^128}, "P mod 2" read as the node's least-significant bit, path bits
 *     most-significant first (parent of node j is floor(j/2)).
 *   - Leaf value and key generation: the paper defers Gen to BGI16 [dpf_1]
 *     (Sec. 3.1, end); the correction-word construction below is BGI16's,
 *     adapted to the codeword form C_t[b][d] of Eq. p3.  Output group Z_2^32.
 *   - Server answer: T x Eval(k, {0..L-1}) (Sec. 3.1, "Eval is the key
 *     evaluation process ...").
 *
 * Parity pins (see tests/test_oracle_*.py): FIPS-197 vectors, the DPF
 * correctness identity by brute force, tree-vs-branch equality, the paper's
 * L=4 dependency example, the key-size law of Table 4, linearity over index
 * ranges (Sec. 3.2.7) and reconstruction of T[alpha].
 *
 * Key wire format (little-endian), shared as an interface with the library:
 *   [0,4)   magic "DPFK"      [4] version = 1     [5] n      [6] party sigma
 *   [7]     PRF (0 AES-128, 1 ChaCha20)  [8,12) cw_out (u32) [12,16) 0
 *   [16,32) root seed of this party
 *   then for d = 1..n: C_0[0][d], C_0[1][d], C_1[0][d], C_1[1][d] (16 B each)
 *   total 32 + 64 n bytes.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* FIPS-197 Sec. 4: arithmetic in GF(2^8) modulo x^8 + x^4 + x^3 + x + 1 */

static uint8_t gf_mul(uint8_t a, uint8_t b)
{
    /* Sec. 4.2 / 4.2.1: repeated xtime() and conditional addition. */
    uint8_t product = 0;
    for (int bit = 0; bit < 8; bit++) {
        if (b & 1)
            product ^= a;
        uint8_t carry = (uint8_t)(a & 0x80);
        a = (uint8_t)(a << 1);
        if (carry)
            a ^= 0x1b;
        b >>= 1;
    }
    return product;
}

static uint8_t gf_inverse(uint8_t a)
{
    /* Sec. 5.1.1: {00} maps to itself; otherwise search for b with a*b = 1. */
    if (a == 0)
        return 0;
    for (int b = 1; b < 256; b++)
        if (gf_mul(a, (uint8_t)b) == 1)
            return (uint8_t)b;
    return 0; /* unreachable: every non-zero element is invertible */
}

static uint8_t SBOX[256];

static uint8_t sbox_from_definition(uint8_t x)
{
    /* Sec. 5.1.1 Eq. 5.1: b'_i = b_i ^ b_{i+4} ^ b_{i+5} ^ b_{i+6} ^ b_{i+7} ^ c_i,
       indices mod 8, c = {63}, applied to the multiplicative inverse b. */
    uint8_t b = gf_inverse(x);
    uint8_t out = 0;
    for (int i = 0; i < 8; i++) {
        int bit = ((b >> i) & 1) ^ ((b >> ((i + 4) % 8)) & 1) ^ ((b >> ((i + 5) % 8)) & 1) ^
                  ((b >> ((i + 6) % 8)) & 1) ^ ((b >> ((i + 7) % 8)) & 1) ^ ((0x63 >> i) & 1);
        out |= (uint8_t)(bit << i);
    }
    return out;
}

__attribute__((constructor)) static void oracle_init(void)
{
    for (int x = 0; x < 256; x++)
        SBOX[x] = sbox_from_definition((uint8_t)x);
}

void orc_sbox(uint8_t out[256]) { memcpy(out, SBOX, 256); }
uint8_t orc_gf_mul(uint8_t a, uint8_t b) { return gf_mul(a, b); }

/* ------------------------------------------------------------------ */
/* FIPS-197 Sec. 5.2: KeyExpansion for Nk = 4, Nr = 10 (44 words).     */

void orc_aes128_key_expansion(const uint8_t key[16], uint8_t w[44][4])
{
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++)
            w[i][j] = key[4 * i + j];
    uint8_t rcon = 0x01; /* Rcon[i/Nk] = (x^(i/Nk - 1), 0, 0, 0) */
    for (int i = 4; i < 44; i++) {
        uint8_t temp[4];
        memcpy(temp, w[i - 1], 4);
        if (i % 4 == 0) {
            uint8_t first = temp[0]; /* RotWord */
            temp[0] = temp[1];
            temp[1] = temp[2];
            temp[2] = temp[3];
            temp[3] = first;
            for (int j = 0; j < 4; j++) /* SubWord */
                temp[j] = SBOX[temp[j]];
            temp[0] ^= rcon;
            rcon = gf_mul(rcon, 0x02);
        }
        for (int j = 0; j < 4; j++)
            w[i][j] = (uint8_t)(w[i - 4][j] ^ temp[j]);
    }
}

/* ------------------------------------------------------------------ */
/* FIPS-197 Sec. 5.1: Cipher.  state[r][c] = in[r + 4c].                */

static void add_round_key(uint8_t state[4][4], const uint8_t w[44][4], int round)
{
    for (int c = 0; c < 4; c++)
        for (int r = 0; r < 4; r++)
            state[r][c] ^= w[round * 4 + c][r];
}

static void sub_bytes(uint8_t state[4][4])
{
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++)
            state[r][c] = SBOX[state[r][c]];
}

static void shift_rows(uint8_t state[4][4])
{
    /* Sec. 5.1.2: s'[r][c] = s[r][(c + shift(r)) mod 4], shift(r) = r. */
    uint8_t tmp[4][4];
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++)
            tmp[r][c] = state[r][(c + r) % 4];
    memcpy(state, tmp, 16);
}

/* Sec. 4.2.1: multiplication by {02} is xtime(); {03} = {02} + {01}. */
static uint8_t xtime(uint8_t a) { return (uint8_t)((a << 1) ^ ((a & 0x80) ? 0x1b : 0x00)); }
static uint8_t mul2(uint8_t a) { return xtime(a); }
static uint8_t mul3(uint8_t a) { return (uint8_t)(xtime(a) ^ a); }

static void mix_columns(uint8_t state[4][4])
{
    /* Sec. 5.1.3 Eq. 5.6: multiplication by {03}x^3 + {01}x^2 + {01}x + {02}. */
    for (int c = 0; c < 4; c++) {
        uint8_t s0 = state[0][c], s1 = state[1][c], s2 = state[2][c], s3 = state[3][c];
        state[0][c] = (uint8_t)(mul2(s0) ^ mul3(s1) ^ s2 ^ s3);
        state[1][c] = (uint8_t)(s0 ^ mul2(s1) ^ mul3(s2) ^ s3);
        state[2][c] = (uint8_t)(s0 ^ s1 ^ mul2(s2) ^ mul3(s3));
        state[3][c] = (uint8_t)(mul3(s0) ^ s1 ^ s2 ^ mul2(s3));
    }
}

void orc_aes128_encrypt(const uint8_t key[16], const uint8_t in[16], uint8_t out[16])
{
    uint8_t w[44][4];
    orc_aes128_key_expansion(key, w);
    uint8_t state[4][4];
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++)
            state[r][c] = in[r + 4 * c];
    add_round_key(state, w, 0);
    for (int round = 1; round < 10; round++) {
        sub_bytes(state);
        shift_rows(state);
        mix_columns(state);
        add_round_key(state, w, round);
    }
    sub_bytes(state);
    shift_rows(state);
    add_round_key(state, w, 10);
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++)
            out[r + 4 * c] = state[r][c];
}

/* ------------------------------------------------------------------ */
/* ChaCha20 (RFC 8439): Sec. 2.1 quarter round, Sec. 2.3 block function. */

static uint32_t rotl32(uint32_t v, int c) { return (v << c) | (v >> (32 - c)); }

void orc_chacha_quarter_round(uint32_t* a, uint32_t* b, uint32_t* c, uint32_t* d)
{
    *a += *b; *d ^= *a; *d = rotl32(*d, 16);
    *c += *d; *b ^= *c; *b = rotl32(*b, 12);
    *a += *b; *d ^= *a; *d = rotl32(*d, 8);
    *c += *d; *b ^= *c; *b = rotl32(*b, 7);
}

static void quarter_round_on(uint32_t x[16], int a, int b, int c, int d)
{
    orc_chacha_quarter_round(&x[a], &x[b], &x[c], &x[d]);
}

void orc_chacha20_block(const uint8_t key[32], uint32_t counter, const uint8_t nonce[12], uint8_t out[64])
{
    /* Sec. 2.3: constants "expand 32-byte k", key, block counter, nonce; all little-endian words */
    uint32_t state[16];
    state[0] = 0x61707865;
    state[1] = 0x3320646e;
    state[2] = 0x79622d32;
    state[3] = 0x6b206574;
    for (int i = 0; i < 8; i++)
        state[4 + i] = (uint32_t)key[4 * i] | ((uint32_t)key[4 * i + 1] << 8) | ((uint32_t)key[4 * i + 2] << 16) |
                       ((uint32_t)key[4 * i + 3] << 24);
    state[12] = counter;
    for (int i = 0; i < 3; i++)
        state[13 + i] = (uint32_t)nonce[4 * i] | ((uint32_t)nonce[4 * i + 1] << 8) |
                        ((uint32_t)nonce[4 * i + 2] << 16) | ((uint32_t)nonce[4 * i + 3] << 24);
    uint32_t x[16];
    memcpy(x, state, sizeof(x));
    for (int i = 0; i < 10; i++) { /* 20 rounds: column round then diagonal round */
        quarter_round_on(x, 0, 4, 8, 12);
        quarter_round_on(x, 1, 5, 9, 13);
        quarter_round_on(x, 2, 6, 10, 14);
        quarter_round_on(x, 3, 7, 11, 15);
        quarter_round_on(x, 0, 5, 10, 15);
        quarter_round_on(x, 1, 6, 11, 12);
        quarter_round_on(x, 2, 7, 8, 13);
        quarter_round_on(x, 3, 4, 9, 14);
    }
    for (int i = 0; i < 16; i++) {
        uint32_t v = x[i] + state[i];
        out[4 * i] = (uint8_t)v;
        out[4 * i + 1] = (uint8_t)(v >> 8);
        out[4 * i + 2] = (uint8_t)(v >> 16);
        out[4 * i + 3] = (uint8_t)(v >> 24);
    }
}

/* ------------------------------------------------------------------ */
/* The PRF of Eq. p3: PRF_s(x) encrypts message x under key s.          */
/* prf 0: AES-128 of the block (x, 0, ..., 0) under key s.              */
/* prf 1: ChaCha20 block 0 under key s || 0^128 with nonce 0; PRF_s(x)  */
/*        is its 16 bytes at offset 16x (one block serves both x).      */

enum { PRF_AES128 = 0, PRF_CHACHA20 = 1 };

void orc_prf(const uint8_t s[16], uint8_t x, uint8_t out[16])
{
    uint8_t msg[16] = {0};
    msg[0] = x;
    orc_aes128_encrypt(s, msg, out);
}

void orc_prf_id(int prf, const uint8_t s[16], uint8_t x, uint8_t out[16])
{
    if (prf == PRF_CHACHA20) {
        uint8_t key[32] = {0}, nonce[12] = {0}, block[64];
        memcpy(key, s, 16);
        orc_chacha20_block(key, 0, nonce, block);
        memcpy(out, block + 16 * x, 16);
    } else {
        orc_prf(s, x, out);
    }
}

/* ------------------------------------------------------------------ */
/* Key layout helpers (wire format in the header comment).             */

enum { KEY_HEADER = 32, ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_KEY = -3 };

size_t orc_key_bytes(uint32_t n) { return (size_t)KEY_HEADER + 64u * (size_t)n; }

static const uint8_t* codeword(const uint8_t* key, uint32_t d, int t, int b)
{
    /* C_t[b][d] for depth d in 1..n */
    return key + KEY_HEADER + 64u * (d - 1) + 32u * (uint32_t)t + 16u * (uint32_t)b;
}

static uint32_t get_u32(const uint8_t* p)
{
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

static void put_u32(uint8_t* p, uint32_t v)
{
    p[0] = (uint8_t)v;
    p[1] = (uint8_t)(v >> 8);
    p[2] = (uint8_t)(v >> 16);
    p[3] = (uint8_t)(v >> 24);
}

static int lsb(const uint8_t v[16]) { return v[0] & 1; }

/* Conv: the Z_2^32 element carried by a leaf = bytes 4..7, little-endian. */
static uint32_t conv(const uint8_t v[16]) { return get_u32(v + 4); }

int orc_key_parse(const uint8_t* key, uint32_t* n, uint32_t* party, uint32_t* cw_out)
{
    if (key[0] != 'D' || key[1] != 'P' || key[2] != 'F' || key[3] != 'K' || key[4] != 1)
        return ORC_ERR_KEY;
    if (key[5] < 1 || key[5] > 63 || key[6] > 1 || key[7] > PRF_CHACHA20)
        return ORC_ERR_KEY;
    *n = key[5];
    *party = key[6];
    *cw_out = get_u32(key + 8);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Gen (BGI16 construction in the codeword form of Eq. p3).             */
/* All randomness is an input: seed0/seed1 (roots, lsb forced to 0/1)   */
/* and rand_c0 = n x 2 x 16 bytes for the codewords C_0[b][d].          */

int orc_gen_prf(uint32_t n, uint64_t alpha, uint32_t beta, int prf, const uint8_t seed0[16],
                const uint8_t seed1[16], const uint8_t* rand_c0, uint8_t* key0, uint8_t* key1)
{
    if (prf != PRF_AES128 && prf != PRF_CHACHA20)
        return ORC_ERR_ARG;
    if (n < 1 || n > 63 || (n < 64 && (alpha >> n) != 0))
        return ORC_ERR_ARG;
    size_t kb = orc_key_bytes(n);
    memset(key0, 0, kb);
    memset(key1, 0, kb);

    uint8_t v[2][16];
    memcpy(v[0], seed0, 16);
    memcpy(v[1], seed1, 16);
    v[0][0] &= 0xfe; /* control bit of party 0's root is 0 */
    v[1][0] |= 0x01; /* control bit of party 1's root is 1 */

    for (uint32_t d = 1; d <= n; d++) {
        int a = (int)((alpha >> (n - d)) & 1); /* path bit toward alpha at this depth */
        int keep = a, lose = 1 - a;
        uint8_t c[2][2][16]; /* c[party][b] = PRF_{v_party}(b) */
        for (int p = 0; p < 2; p++)
            for (int b = 0; b < 2; b++)
                orc_prf_id(prf, v[p], (uint8_t)b, c[p][b]);

        /* seed correction: makes the off-path children equal */
        uint8_t s_cw[16];
        for (int i = 0; i < 16; i++)
            s_cw[i] = (uint8_t)(c[0][lose][i] ^ c[1][lose][i]);
        s_cw[0] &= 0xfe;
        /* control-bit corrections: off-path bits equal, on-path bits differ */
        int t_cw[2];
        t_cw[0] = lsb(c[0][0]) ^ lsb(c[1][0]) ^ a ^ 1;
        t_cw[1] = lsb(c[0][1]) ^ lsb(c[1][1]) ^ a;

        for (int b = 0; b < 2; b++) {
            uint8_t delta[16];
            memcpy(delta, s_cw, 16);
            delta[0] |= (uint8_t)t_cw[b];
            const uint8_t* c0_rand = rand_c0 + 32u * (d - 1) + 16u * (uint32_t)b;
            uint8_t* c0_k0 = (uint8_t*)codeword(key0, d, 0, b);
            uint8_t* c1_k0 = (uint8_t*)codeword(key0, d, 1, b);
            for (int i = 0; i < 16; i++) {
                c0_k0[i] = c0_rand[i];                       /* C_0[b][d]: shared random  */
                c1_k0[i] = (uint8_t)(c0_rand[i] ^ delta[i]); /* C_1[b][d] = C_0 ^ Delta^b */
            }
        }
        /* advance both parties along the path, selecting the codeword by the
           PARENT's control bit, exactly as Eval does (Eq. p3) */
        for (int p = 0; p < 2; p++) {
            const uint8_t* cw = codeword(key0, d, lsb(v[p]), keep);
            uint8_t next[16];
            for (int i = 0; i < 16; i++)
                next[i] = (uint8_t)(c[p][keep][i] ^ cw[i]);
            memcpy(v[p], next, 16);
        }
    }
    /* output correction: y_0 + y_1 = beta at alpha (leaf conversion below) */
    uint32_t diff = beta - conv(v[0]) + conv(v[1]);
    uint32_t cw_out = lsb(v[1]) ? (uint32_t)(0u - diff) : diff;

    memcpy(key1 + KEY_HEADER, key0 + KEY_HEADER, 64u * n); /* both keys carry C_0, C_1 */
    uint8_t* keys[2] = {key0, key1};
    for (int p = 0; p < 2; p++) {
        uint8_t* k = keys[p];
        k[0] = 'D';
        k[1] = 'P';
        k[2] = 'F';
        k[3] = 'K';
        k[4] = 1;
        k[5] = (uint8_t)n;
        k[6] = (uint8_t)p;
        k[7] = (uint8_t)prf;
        put_u32(k + 8, cw_out);
        memcpy(k + 16, p == 0 ? seed0 : seed1, 16);
        k[16] = p == 0 ? (uint8_t)(k[16] & 0xfe) : (uint8_t)(k[16] | 0x01);
    }
    return ORC_OK;
}

int orc_gen(uint32_t n, uint64_t alpha, uint32_t beta, const uint8_t seed0[16], const uint8_t seed1[16],
            const uint8_t* rand_c0, uint8_t* key0, uint8_t* key1)
{
    return orc_gen_prf(n, alpha, beta, PRF_AES128, seed0, seed1, rand_c0, key0, key1);
}

/* ------------------------------------------------------------------ */
/* Leaf -> Z_2^32 share: y = (-1)^sigma (Conv(v) + lsb(v) * cw_out).    */

static uint32_t leaf_share(const uint8_t v[16], uint32_t party, uint32_t cw_out)
{
    uint32_t y = conv(v) + (uint32_t)lsb(v) * cw_out;
    return party ? (uint32_t)(0u - y) : y;
}

/* Eval(k, j) = P(n, j) by walking the root-to-leaf path (branch form). */
int orc_eval(const uint8_t* key, uint64_t j, uint32_t* y)
{
    uint32_t n, party, cw_out;
    if (orc_key_parse(key, &n, &party, &cw_out) != ORC_OK)
        return ORC_ERR_KEY;
    if (n < 64 && (j >> n) != 0)
        return ORC_ERR_ARG;
    uint8_t v[16];
    memcpy(v, key + 16, 16); /* P(0, 0) */
    for (uint32_t d = 1; d <= n; d++) {
        int b = (int)((j >> (n - d)) & 1); /* "j mod 2" of the depth-d ancestor */
        uint8_t prf[16];
        orc_prf_id(key[7], v, (uint8_t)b, prf);
        const uint8_t* cw = codeword(key, d, lsb(v), b);
        for (int i = 0; i < 16; i++)
            v[i] = (uint8_t)(prf[i] ^ cw[i]);
    }
    *y = leaf_share(v, party, cw_out);
    return ORC_OK;
}

/* FullEval: every node computed once, level by level (Eq. p3 over all j). */
int orc_full_eval(const uint8_t* key, uint64_t L, uint32_t* y)
{
    uint32_t n, party, cw_out;
    if (orc_key_parse(key, &n, &party, &cw_out) != ORC_OK)
        return ORC_ERR_KEY;
    if (L == 0 || n > 40 || L > (1ull << n))
        return ORC_ERR_ARG;
    uint64_t width = 1ull << n;
    uint8_t* level = (uint8_t*)malloc(16);
    if (!level)
        return ORC_ERR_ARG;
    memcpy(level, key + 16, 16);
    for (uint32_t d = 1; d <= n; d++) {
        uint64_t count = 1ull << d;
        /* only ancestors of leaves < L are needed at the next depths */
        uint64_t needed = (L - 1) >> (n - d);
        uint64_t keep = needed + 1 < count ? needed + 1 : count;
        uint8_t* next = (uint8_t*)malloc(keep * 16);
        if (!next) {
            free(level);
            return ORC_ERR_ARG;
        }
        for (uint64_t jd = 0; jd < keep; jd++) {
            const uint8_t* parent = level + 16 * (jd >> 1); /* P(d-1, floor(j/2)) */
            int b = (int)(jd & 1);                         /* j mod 2 */
            uint8_t prf[16];
            orc_prf_id(key[7], parent, (uint8_t)b, prf);
            const uint8_t* cw = codeword(key, d, lsb(parent), b);
            for (int i = 0; i < 16; i++)
                next[16 * jd + i] = (uint8_t)(prf[i] ^ cw[i]);
        }
        free(level);
        level = next;
    }
    (void)width;
    for (uint64_t j = 0; j < L; j++)
        y[j] = leaf_share(level + 16 * j, party, cw_out);
    free(level);
    return ORC_OK;
}

/* Server answer: out[w] = sum_{lo <= j < hi} y(j) * T[j][w]  (mod 2^32).
   table points at row `lo`; rows are `stride` words apart. */
int orc_answer_range(const uint8_t* key, const uint32_t* table, uint64_t L, uint32_t W, uint64_t stride,
                     uint64_t lo, uint64_t hi, uint32_t* out)
{
    if (hi > L || lo > hi || W == 0 || stride < W)
        return ORC_ERR_ARG;
    uint32_t* y = (uint32_t*)malloc((size_t)(L ? L : 1) * 4);
    if (!y)
        return ORC_ERR_ARG;
    int rc = orc_full_eval(key, L, y);
    if (rc != ORC_OK) {
        free(y);
        return rc;
    }
    for (uint32_t w = 0; w < W; w++)
        out[w] = 0;
    for (uint64_t j = lo; j < hi; j++) {
        const uint32_t* row = table + (j - lo) * stride;
        for (uint32_t w = 0; w < W; w++)
            out[w] += y[j] * row[w];
    }
    free(y);
    return ORC_OK;
}

int orc_answer(const uint8_t* key, const uint32_t* table, uint64_t L, uint32_t W, uint64_t stride, uint32_t* out)
{
    return orc_answer_range(key, table, L, W, stride, 0, L, out);
}

/* Client-side reconstruction (Sec. 3.1): T[alpha] = share_0 + share_1. */
void orc_reconstruct(const uint32_t* s0, const uint32_t* s1, size_t w, uint32_t* out)
{
    for (size_t i = 0; i < w; i++)
        out[i] = s0[i] + s1[i];
}

/* Structural probe for tests: the node P(d, j) itself (16 bytes). */
int orc_node(const uint8_t* key, uint32_t d, uint64_t j, uint8_t out[16])
{
    uint32_t n, party, cw_out;
    if (orc_key_parse(key, &n, &party, &cw_out) != ORC_OK)
        return ORC_ERR_KEY;
    if (d > n || (d < 64 && (j >> d) != 0))
        return ORC_ERR_ARG;
    uint8_t v[16];
    memcpy(v, key + 16, 16);
    for (uint32_t e = 1; e <= d; e++) {
        int b = (int)((j >> (d - e)) & 1);
        uint8_t prf[16];
        orc_prf_id(key[7], v, (uint8_t)b, prf);
        const uint8_t* cw = codeword(key, e, lsb(v), b);
        for (int i = 0; i < 16; i++)
            v[i] = (uint8_t)(prf[i] ^ cw[i]);
    }
    memcpy(out, v, 16);
    return ORC_OK;
}

// Host AES-128 for client key generation (FIPS-197), 32-bit T-table form.
//
// The S-box is derived at first use from GF(2^8): inverses through the
// log/antilog tables of the generator {03}, then the affine map written as
// b ^ rotl(b,1) ^ rotl(b,2) ^ rotl(b,3) ^ rotl(b,4) ^ {63} (FIPS-197 Sec. 5.1.1).
#include <cstring>
#include <mutex>

#include "internal.h"

namespace pir {
namespace {

struct Tables {
    uint8_t sbox[256];
    uint32_t te0[256];  // column contribution of S(x): bytes (2S, S, S, 3S)
};

uint8_t xtime8(uint8_t a) { return (uint8_t)((a << 1) ^ ((a & 0x80) ? 0x1b : 0)); }
uint8_t rotl8(uint8_t a, int k) { return (uint8_t)((a << k) | (a >> (8 - k))); }

const Tables& tables() {
    static Tables t;
    static std::once_flag once;
    std::call_once(once, [] {
        uint8_t exp[256], log[256] = {0};
        uint8_t g = 1;
        for (int i = 0; i < 255; ++i) {  // powers of the generator {03}
            exp[i] = g;
            log[g] = (uint8_t)i;
            g = (uint8_t)(g ^ xtime8(g));
        }
        for (int x = 0; x < 256; ++x) {
            uint8_t inv = x == 0 ? 0 : exp[(255 - log[x]) % 255];
            uint8_t s = (uint8_t)(inv ^ rotl8(inv, 1) ^ rotl8(inv, 2) ^ rotl8(inv, 3) ^ rotl8(inv, 4) ^ 0x63);
            t.sbox[x] = s;
            uint8_t s2 = xtime8(s);
            t.te0[x] = (uint32_t)s2 | ((uint32_t)s << 8) | ((uint32_t)s << 16) | ((uint32_t)(s2 ^ s) << 24);
        }
    });
    return t;
}

inline uint32_t rotl32(uint32_t x, int k) { return (x << k) | (x >> (32 - k)); }
inline uint32_t load_le(const uint8_t* p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
inline void store_le(uint8_t* p, uint32_t v) {
    p[0] = (uint8_t)v;
    p[1] = (uint8_t)(v >> 8);
    p[2] = (uint8_t)(v >> 16);
    p[3] = (uint8_t)(v >> 24);
}

}  // namespace

const uint8_t* aes_sbox() { return tables().sbox; }

void Aes128::set_key(const uint8_t key[16]) {
    const uint8_t* s = tables().sbox;
    for (int i = 0; i < 4; ++i) rk[i] = load_le(key + 4 * i);
    uint8_t rcon = 1;
    for (int i = 4; i < 44; ++i) {
        uint32_t t = rk[i - 1];
        if (i % 4 == 0) {
            // SubWord(RotWord(t)) ^ Rcon, with byte 0 in the low bits
            uint32_t r = (t >> 8) | (t << 24);
            t = (uint32_t)s[r & 0xff] | ((uint32_t)s[(r >> 8) & 0xff] << 8) | ((uint32_t)s[(r >> 16) & 0xff] << 16) |
                ((uint32_t)s[r >> 24] << 24);
            t ^= rcon;
            rcon = xtime8(rcon);
        }
        rk[i] = rk[i - 4] ^ t;
    }
}

void Aes128::encrypt(const uint8_t in[16], uint8_t out[16]) const {
    const Tables& tb = tables();
    uint32_t s[4], o[4];
    for (int c = 0; c < 4; ++c) s[c] = load_le(in + 4 * c) ^ rk[c];
    for (int round = 1; round < 10; ++round) {
        for (int c = 0; c < 4; ++c) {
            o[c] = tb.te0[s[c] & 0xff] ^ rotl32(tb.te0[(s[(c + 1) & 3] >> 8) & 0xff], 8) ^
                   rotl32(tb.te0[(s[(c + 2) & 3] >> 16) & 0xff], 16) ^ rotl32(tb.te0[s[(c + 3) & 3] >> 24], 24) ^
                   rk[4 * round + c];
        }
        std::memcpy(s, o, sizeof(s));
    }
    for (int c = 0; c < 4; ++c) {
        o[c] = (uint32_t)tb.sbox[s[c] & 0xff] | ((uint32_t)tb.sbox[(s[(c + 1) & 3] >> 8) & 0xff] << 8) |
               ((uint32_t)tb.sbox[(s[(c + 2) & 3] >> 16) & 0xff] << 16) |
               ((uint32_t)tb.sbox[s[(c + 3) & 3] >> 24] << 24);
        store_le(out + 4 * c, o[c] ^ rk[40 + c]);
    }
}

}  // namespace pir

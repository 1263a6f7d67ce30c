// Client side of DPF-PIR: key generation, key validation, reconstruction.
//
// Gen follows Sec. 3.1 of the paper, which defers the construction to BGI16
// [dpf_1]: the two parties' roots differ in their control bit (the node's
// least-significant bit, which selects the codeword set C_0 or C_1 in Eq. p3);
// at every depth the correction Delta^b = C_1[b][d] ^ C_0[b][d] makes the two
// parties' children equal off the path to alpha and keeps their control bits
// different on it; a final output word makes the two leaf shares at alpha sum
// to beta in Z_2^32.
#include <algorithm>
#include <atomic>
#include <cerrno>
#include <cstdio>
#include <cstring>
#include <thread>
#include <vector>

#include <sys/random.h>

#include "internal.h"

namespace pir {
namespace {

inline void put_u32(uint8_t* p, uint32_t v) {
    p[0] = (uint8_t)v;
    p[1] = (uint8_t)(v >> 8);
    p[2] = (uint8_t)(v >> 16);
    p[3] = (uint8_t)(v >> 24);
}
inline uint32_t get_u32(const uint8_t* p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

// Deterministic byte source: AES-128 in counter mode keyed by seed[0..16),
// counter block starting at seed[16..32) read as a little-endian integer.
class CtrStream {
  public:
    explicit CtrStream(const uint8_t seed[32]) {
        aes_.set_key(seed);
        std::memcpy(ctr_, seed + 16, 16);
    }
    void fill(uint8_t* out, size_t len) {
        while (len) {
            if (used_ == 16) {
                aes_.encrypt(ctr_, buf_);
                for (int i = 0; i < 16 && ++ctr_[i] == 0; ++i) {
                }
                used_ = 0;
            }
            size_t take = 16 - used_ < len ? 16 - used_ : len;
            std::memcpy(out, buf_ + used_, take);
            used_ += take;
            out += take;
            len -= take;
        }
    }

  private:
    Aes128 aes_;
    uint8_t ctr_[16], buf_[16];
    size_t used_ = 16;
};

bool os_entropy(uint8_t* out, size_t len) {
    while (len) {
        ssize_t got = getrandom(out, len, 0);
        if (got < 0) {
            if (errno == EINTR) continue;
            return false;
        }
        out += got;
        len -= (size_t)got;
    }
    return true;
}

// ChaCha20 block 0 (RFC 8439) under key node || 0^128, nonce 0: the first
// 32 bytes are the two children.
void chacha_children(const uint8_t node[16], uint8_t out[2][16]) {
    uint32_t s[16] = {0x61707865u, 0x3320646eu, 0x79622d32u, 0x6b206574u};
    for (int i = 0; i < 4; ++i) s[4 + i] = get_u32(node + 4 * i);
    uint32_t x[16];
    std::memcpy(x, s, sizeof(x));
    auto rotl = [](uint32_t v, int c) { return (v << c) | (v >> (32 - c)); };
    auto qr = [&](int a, int b, int c, int d) {
        x[a] += x[b]; x[d] = rotl(x[d] ^ x[a], 16);
        x[c] += x[d]; x[b] = rotl(x[b] ^ x[c], 12);
        x[a] += x[b]; x[d] = rotl(x[d] ^ x[a], 8);
        x[c] += x[d]; x[b] = rotl(x[b] ^ x[c], 7);
    };
    for (int r = 0; r < 10; ++r) {
        qr(0, 4, 8, 12); qr(1, 5, 9, 13); qr(2, 6, 10, 14); qr(3, 7, 11, 15);
        qr(0, 5, 10, 15); qr(1, 6, 11, 12); qr(2, 7, 8, 13); qr(3, 4, 9, 14);
    }
    for (int i = 0; i < 8; ++i) put_u32(out[i >> 2] + 4 * (i & 3), x[i] + s[i]);
}

// Both children of a node: out[b] = PRF_node(b) for the key's PRF.
void prf_pair(const uint8_t node[16], uint32_t prf, uint8_t out[2][16]) {
    if (prf == PIR_PRF_CHACHA20) {
        chacha_children(node, out);
        return;
    }
    Aes128 a;
    a.set_key(node);
    uint8_t msg[16] = {0};
    a.encrypt(msg, out[0]);
    msg[0] = 1;
    a.encrypt(msg, out[1]);
}

}  // namespace
}  // namespace pir

extern "C" {

size_t pir_key_bytes(uint32_t n) { return pir::key_bytes(n); }

uint32_t pir_domain_bits(uint64_t rows) {
    if (rows == 0 || rows > (1ull << PIR_MAX_DOMAIN_BITS)) return 0;
    uint32_t n = 1;
    while ((1ull << n) < rows) ++n;
    return n;
}

int pir_keygen(uint32_t n, uint64_t alpha, uint32_t beta, const uint8_t* seed, uint8_t* key0, uint8_t* key1) {
    return pir_keygen_prf(n, alpha, beta, PIR_PRF_AES128, seed, key0, key1);
}

int pir_keygen_prf(uint32_t n, uint64_t alpha, uint32_t beta, uint32_t prf, const uint8_t* seed, uint8_t* key0,
                   uint8_t* key1) {
    using namespace pir;
    if (!key0 || !key1 || n == 0 || n > PIR_MAX_DOMAIN_BITS) return PIR_ERR_ARG;
    if (prf != PIR_PRF_AES128 && prf != PIR_PRF_CHACHA20) return PIR_ERR_ARG;
    if ((alpha >> n) != 0) return PIR_ERR_DOMAIN;

    // randomness: two roots and the shared codeword set C_0
    const size_t rand_len = 32 + 32 * (size_t)n;
    uint8_t* rnd = new uint8_t[rand_len];
    if (seed) {
        CtrStream(seed).fill(rnd, rand_len);
    } else if (!os_entropy(rnd, rand_len)) {
        delete[] rnd;
        return PIR_ERR_ARG;
    }

    const size_t kb = key_bytes(n);
    std::memset(key0, 0, kb);
    uint8_t node[2][16];
    std::memcpy(node[0], rnd, 16);
    std::memcpy(node[1], rnd + 16, 16);
    node[0][0] &= 0xfe;
    node[1][0] |= 0x01;
    std::memcpy(key0 + 16, node[0], 16);
    uint8_t root1[16];
    std::memcpy(root1, node[1], 16);

    for (uint32_t d = 1; d <= n; ++d) {
        const uint32_t on = (uint32_t)(alpha >> (n - d)) & 1u;  // child bit on the path
        const uint32_t off = on ^ 1u;
        uint8_t ch[2][2][16];  // ch[party][b]
        prf_pair(node[0], prf, ch[0]);
        prf_pair(node[1], prf, ch[1]);
        uint8_t delta[2][16];
        for (int i = 0; i < 16; ++i) delta[0][i] = delta[1][i] = ch[0][off][i] ^ ch[1][off][i];
        delta[0][0] &= 0xfe;
        delta[1][0] &= 0xfe;
        // control-bit corrections: equal off the path, different on it
        const uint32_t tl = (ch[0][0][0] ^ ch[1][0][0] ^ on ^ 1u) & 1u;
        const uint32_t tr = (ch[0][1][0] ^ ch[1][1][0] ^ on) & 1u;
        delta[0][0] |= (uint8_t)tl;
        delta[1][0] |= (uint8_t)tr;
        const uint8_t* c0rand = rnd + 32 + 32 * (size_t)(d - 1);
        for (uint32_t b = 0; b < 2; ++b) {
            uint8_t* c0 = key0 + codeword_offset(d, 0, b);
            uint8_t* c1 = key0 + codeword_offset(d, 1, b);
            for (int i = 0; i < 16; ++i) {
                c0[i] = c0rand[16 * b + i];
                c1[i] = (uint8_t)(c0rand[16 * b + i] ^ delta[b][i]);
            }
        }
        for (int p = 0; p < 2; ++p) {
            const uint8_t* cw = key0 + codeword_offset(d, node[p][0] & 1u, on);
            for (int i = 0; i < 16; ++i) node[p][i] = (uint8_t)(ch[p][on][i] ^ cw[i]);
        }
    }
    // leaf value in Z_2^32: word 1 of the leaf, plus cw_out when its control bit is set,
    // negated for party 1
    const uint32_t v0 = get_u32(node[0] + 4), v1 = get_u32(node[1] + 4);
    uint32_t corr = beta - v0 + v1;
    if (node[1][0] & 1u) corr = 0u - corr;

    std::memcpy(key1, key0, kb);
    for (int p = 0; p < 2; ++p) {
        uint8_t* k = p ? key1 : key0;
        put_u32(k, kKeyMagic);
        k[4] = (uint8_t)kKeyVersion;
        k[5] = (uint8_t)n;
        k[6] = (uint8_t)p;
        k[7] = (uint8_t)prf;
        put_u32(k + 8, corr);
        put_u32(k + 12, 0);
    }
    std::memcpy(key1 + 16, root1, 16);
    delete[] rnd;
    return PIR_OK;
}

int pir_keygen_batch(uint32_t n, size_t count, const uint64_t* alphas, const uint32_t* betas, uint32_t prf,
                     const uint8_t* seed, uint8_t* keys0, uint8_t* keys1, uint32_t threads) {
    using namespace pir;
    if (count == 0) return PIR_OK;
    if (!alphas || !keys0 || !keys1 || n == 0 || n > PIR_MAX_DOMAIN_BITS) return PIR_ERR_ARG;
    if (prf != PIR_PRF_AES128 && prf != PIR_PRF_CHACHA20) return PIR_ERR_ARG;
    for (size_t i = 0; i < count; ++i)
        if ((alphas[i] >> n) != 0) return PIR_ERR_DOMAIN;
    NvtxRange range("pir_keygen_batch");
    // one 32-byte seed per key, drawn in key order from the master seed's stream
    uint8_t master[32];
    if (seed) {
        std::memcpy(master, seed, 32);
    } else if (!os_entropy(master, 32)) {
        return PIR_ERR_ARG;
    }
    std::vector<uint8_t> seeds(32 * count);
    CtrStream(master).fill(seeds.data(), seeds.size());
    const size_t kb = key_bytes(n);
    unsigned nt = threads ? threads : std::max(1u, std::thread::hardware_concurrency());
    nt = (unsigned)std::min<size_t>(nt, count);
    std::atomic<size_t> next{0};
    std::atomic<int> rc{PIR_OK};
    auto work = [&] {
        for (size_t i; (i = next.fetch_add(1)) < count;) {
            const int r = pir_keygen_prf(n, alphas[i], betas ? betas[i] : 1u, prf, seeds.data() + 32 * i,
                                         keys0 + i * kb, keys1 + i * kb);
            if (r != PIR_OK) rc.store(r);
        }
    };
    std::vector<std::thread> pool;
    for (unsigned t = 1; t < nt; ++t) pool.emplace_back(work);
    work();
    for (auto& t : pool) t.join();
    return rc.load();
}

int pir_pbr_keygen(uint64_t rows, uint64_t bin_rows, const uint64_t* indices, size_t count, uint32_t prf,
                   const uint8_t* seed, uint8_t* keys0, uint8_t* keys1, uint8_t* kept) {
    using namespace pir;
    if (!keys0 || !keys1 || (count && (!indices || !kept)) || bin_rows < 2 || rows == 0) return PIR_ERR_ARG;
    const uint32_t nb = pir_domain_bits(bin_rows);
    if (nb == 0) return PIR_ERR_ARG;
    const uint64_t nbins = (rows + bin_rows - 1) / bin_rows;
    std::vector<uint64_t> alpha(nbins, 0);
    std::vector<uint32_t> beta(nbins, 0);  // bins nobody asked for: dummy queries with beta = 0
    for (size_t i = 0; i < count; ++i) {
        if (indices[i] >= rows) return PIR_ERR_DOMAIN;
        const uint64_t b = indices[i] / bin_rows;
        kept[i] = beta[b] == 0 ? 1 : 0;  // one entry per bin: the first index that falls in it
        if (kept[i]) {
            alpha[b] = indices[i] - b * bin_rows;
            beta[b] = 1;
        }
    }
    return pir_keygen_batch(nb, nbins, alpha.data(), beta.data(), prf, seed, keys0, keys1, 0);
}

int pir_hotfull_keygen(uint64_t full_rows, const uint64_t* hot_rows, uint64_t hot_count, const uint64_t* indices,
                       size_t count, uint32_t q_hot, uint32_t q_full, uint32_t prf, const uint8_t* seed,
                       uint8_t* hot_keys0, uint8_t* hot_keys1, uint8_t* full_keys0, uint8_t* full_keys1,
                       int64_t* slot) {
    using namespace pir;
    if (full_rows < 2 || hot_count < 2 || hot_count > full_rows || !hot_rows || (count && (!indices || !slot)))
        return PIR_ERR_ARG;
    if ((q_hot && (!hot_keys0 || !hot_keys1)) || (q_full && (!full_keys0 || !full_keys1))) return PIR_ERR_ARG;
    for (uint64_t h = 0; h < hot_count; ++h)
        if (hot_rows[h] >= full_rows || (h && hot_rows[h] <= hot_rows[h - 1])) return PIR_ERR_ARG;
    // fixed budgets: exactly q_hot queries to the hot table and q_full to the full one
    std::vector<uint64_t> ha(q_hot, 0), fa(q_full, 0);
    std::vector<uint32_t> hb(q_hot, 0), fb(q_full, 0);  // beta 0: dummy queries
    uint32_t nh = 0, nf = 0;
    for (size_t i = 0; i < count; ++i) {
        if (indices[i] >= full_rows) return PIR_ERR_DOMAIN;
        const uint64_t* it = std::lower_bound(hot_rows, hot_rows + hot_count, indices[i]);
        const bool hot = it != hot_rows + hot_count && *it == indices[i];
        if (hot && nh < q_hot) {
            ha[nh] = (uint64_t)(it - hot_rows);
            hb[nh] = 1;
            slot[i] = nh++;
        } else if (nf < q_full) {
            fa[nf] = indices[i];
            fb[nf] = 1;
            slot[i] = (int64_t)q_hot + nf++;
        } else {
            slot[i] = -1;  // over both budgets: dropped
        }
    }
    // the hot and the full keys come from two seeds drawn from `seed`'s stream
    uint8_t masters[64];
    if (seed) {
        CtrStream(seed).fill(masters, 64);
    } else if (!os_entropy(masters, 64)) {
        return PIR_ERR_ARG;
    }
    int rc = q_hot ? pir_keygen_batch(pir_domain_bits(hot_count), q_hot, ha.data(), hb.data(), prf, masters,
                                      hot_keys0, hot_keys1, 0)
                   : PIR_OK;
    if (rc == PIR_OK && q_full)
        rc = pir_keygen_batch(pir_domain_bits(full_rows), q_full, fa.data(), fb.data(), prf, masters + 32, full_keys0,
                              full_keys1, 0);
    return rc;
}

int pir_key_check(const uint8_t* key, size_t len, uint32_t* n, uint32_t* party) {
    using namespace pir;
    if (!key || len < PIR_KEY_HEADER_BYTES) return PIR_ERR_ARG;
    if (get_u32(key) != kKeyMagic || key[4] != kKeyVersion || key[7] > PIR_PRF_CHACHA20) return PIR_ERR_KEY;
    const uint32_t kn = key[5], kp = key[6];
    if (kn == 0 || kn > PIR_MAX_DOMAIN_BITS || kp > 1) return PIR_ERR_KEY;
    if (len != key_bytes(kn)) return PIR_ERR_KEY;
    if (n) *n = kn;
    if (party) *party = kp;
    return PIR_OK;
}

int pir_reconstruct(const uint32_t* s0, const uint32_t* s1, size_t w, uint32_t* out) {
    if (!s0 || !s1 || !out) return PIR_ERR_ARG;
    for (size_t i = 0; i < w; ++i) out[i] = s0[i] + s1[i];
    return PIR_OK;
}

}  // extern "C"

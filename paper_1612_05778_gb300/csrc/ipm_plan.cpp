// ipm_plan.cpp -- host planner: DetermineBase and RecoveryPrime (§2, §2.1),
// in the several-word-size-primes form of §4, plus the twiddle and CRT
// tables the kernels read.
//
// Choices (the paper leaves them to table look-up, §2.4):
//  * K is a power of two (2-way FFTs, §2.1) and N = K*M >= max(bits)+1 so
//    that every coefficient is an N-bit two's-complement number (Eq.
//    definingN).  M >= 2 and K >= 2 (Theorem 1 asks K, M > 1).
//  * The primes p_t satisfy 2^29 < p_t < 2^30 and 2^21 | p_t - 1, so they
//    hold primitive roots of every power-of-two order up to 2^21 (Eq.
//    HavingAppropriatePrimitiveRootsOfUnity, with Y = 2^ceil(log2(nc)) in
//    place of 2d-1 and 2K for theta's order).
//  * The modulus m = prod p_t must exceed 4H (the m > 4H of §1), with H the
//    largest |c_{i,j}|.  Digits satisfy |a_{i,j}| <= 2^(M-1), and a
//    coefficient c_{i,j} sums at most min(na,nb)*K products, so
//    H <= min(na,nb) * K * 2^(2M-2) and the test is m > min(na,nb)*K*2^(2M).
//  * Among the valid (K, M, r) the planner takes the cheapest by a simple
//    work estimate: r transforms of Y x 2K points (the complexity of §4 has
//    the same shape, O(dKM log(dK)(log(dK) + 2M))).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "ipm_internal.h"

namespace ipm {
namespace {

uint64_t powmod(uint64_t b, uint64_t e, uint64_t m) {
    uint64_t r = 1 % m;
    b %= m;
    while (e) {
        if (e & 1) r = r * b % m;
        b = b * b % m;
        e >>= 1;
    }
    return r;
}

// Deterministic Miller-Rabin for n < 4,759,123,141 (bases 2, 7, 61).
bool is_prime32(uint64_t n) {
    if (n < 2) return false;
    for (uint64_t q : {2ull, 3ull, 5ull, 7ull, 11ull, 13ull, 61ull})
        if (n % q == 0) return n == q;
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; ++s; }
    for (uint64_t a : {2ull, 7ull, 61ull}) {
        uint64_t x = powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < s; ++i) {
            x = x * x % n;
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

// Primes p = c*2^21 + 1 with 2^29 < p < 2^30, largest first.
const std::vector<uint32_t> &prime_table() {
    static std::vector<uint32_t> table;
    static std::once_flag once;
    std::call_once(once, [] {
        for (uint64_t c = (1ull << (30 - PRIME_ORDER_LOG2)) - 1; c >= (1ull << (29 - PRIME_ORDER_LOG2)); --c) {
            uint64_t p = (c << PRIME_ORDER_LOG2) + 1;
            if (p < (1ull << 30) && p > (1ull << 29) && is_prime32(p)) table.push_back((uint32_t)p);
        }
    });
    return table;
}

// A generator of (Z/p)^*: g with g^((p-1)/q) != 1 for every prime q | p-1.
uint32_t generator(uint32_t p) {
    std::vector<uint64_t> fac;
    uint64_t n = p - 1;
    for (uint64_t q = 2; q * q <= n; ++q) {
        if (n % q == 0) {
            fac.push_back(q);
            while (n % q == 0) n /= q;
        }
    }
    if (n > 1) fac.push_back(n);
    for (uint64_t g = 2;; ++g) {
        bool ok = true;
        for (uint64_t q : fac)
            if (powmod(g, (p - 1) / q, p) == 1) { ok = false; break; }
        if (ok) return (uint32_t)g;
    }
}

// Primitive root of unity of order 2^lg modulo p.
uint32_t root_of_unity(uint32_t p, int lg) {
    uint32_t g = generator(p);
    return (uint32_t)powmod(g, (uint64_t)(p - 1) >> lg, p);
}

uint32_t shoup_q(uint32_t w, uint32_t p) { return (uint32_t)(((uint64_t)w << 32) / p); }
uint32_t invmod(uint32_t x, uint32_t p) { return (uint32_t)powmod(x, p - 2, p); }

int ilog2(uint64_t x) {
    int l = 0;
    while ((1ull << l) < x) ++l;
    return l;
}

// Multiword (little-endian 32-bit) helpers for the exact m > 4H test.
struct Big {
    uint32_t w[10];
};
Big big_from_u64(uint64_t v) {
    Big b{};
    b.w[0] = (uint32_t)v;
    b.w[1] = (uint32_t)(v >> 32);
    return b;
}
Big big_mul_u32(const Big &a, uint32_t m) {
    Big r{};
    uint64_t carry = 0;
    for (int i = 0; i < 10; ++i) {
        uint64_t t = (uint64_t)a.w[i] * m + carry;
        r.w[i] = (uint32_t)t;
        carry = t >> 32;
    }
    return r;
}
Big big_shl(const Big &a, int s) {
    Big r{};
    int ws = s / 32, bs = s % 32;
    for (int i = 9; i >= 0; --i) {
        int src = i - ws;
        if (src < 0) continue;
        uint64_t v = (uint64_t)a.w[src] << bs;
        r.w[i] |= (uint32_t)v;
        if (i + 1 < 10) r.w[i + 1] |= (uint32_t)(v >> 32);
    }
    return r;
}
int big_cmp(const Big &a, const Big &b) {
    for (int i = 9; i >= 0; --i)
        if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
    return 0;
}

struct Tiles {
    int64_t Y2;
    int32_t S;
    bool mid_tables;
    int64_t Y1b;   // outer split of the middle transform (1 = none)
    int32_t S2;    // outer pass tile width W (words)
    size_t smem_fwd, smem_mid, smem_inv, smem_outer;
};

size_t fwd_smem(int64_t Y2, int K) {
    // digits, two sets of twist / row / x / y twiddles, signs, tile
    return (size_t)Y2 * K * 8 + 4 * ((size_t)K + (size_t)Y2) * 8 + (((size_t)Y2 + 15) & ~(size_t)15) +
           (size_t)Y2 * (2 * K + 1) * 4;
}
size_t inv_smem(int64_t Y2, int K, int r, int lc) {
    size_t sources = ((size_t)lc + 1) * 16;  // one uint4 per limb
    size_t tables = (size_t)r * (2 * (size_t)Y2 + (size_t)K) * 8;  // per prime: row / x / y twiddles
    return (((size_t)r * Y2 * (2 * K + 1) * 4 + 15) & ~(size_t)15) + sources + tables;
}
// tiles of A and B (for S < 32 rows of S words with one empty row after
// every 2^pl, for S >= 32 unpadded rows of S words), plus (tables) one twiddle block per
// register stage of the length-Y1 transform, 2 (Lc_i + R_i) entries for the
// stage's sub-block length Lc_i and radix R_i (ntt_stages.cuh,
// stage_blocks; passes.cuh, mid_tile)
size_t mid_smem(int64_t Y1, int S, bool tables) {
    const int logY1 = ilog2((uint64_t)Y1);
    const int pl = mid_pad_log(logY1, S);
    const size_t tile = (size_t)(pl ? Y1 + (Y1 >> pl) : Y1) * mid_pitch(S, pl);
    size_t tab = 0;
    if (tables) {
        int off[8];
        tab = (size_t)stage_blocks(logY1, off);
    }
    return (2 * tile + 16) * 4 + tab * 8;
}
// outer pass: Y1b rows x W consecutive words of one operand (W a power of
// two >= 4, about OUTER_TILE_WORDS words per tile)
int64_t outer_width(int64_t Y1a, int K, int64_t Y1b) {
    return std::min<int64_t>(Y1a * 2 * K, std::max<int64_t>(4, OUTER_TILE_WORDS / Y1b));
}
size_t outer_smem(int64_t Y1b, int64_t W) { return (size_t)Y1b * (size_t)W * 4; }

// Tile shapes: Y2 rows per forward/inverse tile, S columns per middle tile
// (Y1 = Y / Y2 is the middle pass's column length).  Hard limit: every pass
// fits one block's shared memory.  Preferences, in order: middle slices of
// at least 4 columns (one 16-byte copy per row; 8 columns fill a 32-byte
// DRAM sector and are preferred slightly), an inverse tile small enough
// for two CTAs per SM, a forward tile small enough for three, no split of
// the middle transform (a split costs an extra pass over the data), and Y2
// close to max(32, Y / 2048).  When Y1 is long, the middle transform may be
// split as Y1 = Y1a * Y1b (Y1a <= 2048) with an outer pass over Y1b.  Slices
// wider than 32 columns are used only when asked for (s).
bool choose_tiles(int64_t Y, int K, int r, int lc, int64_t y2_force, int s_force, int64_t y1b_force,
                  Tiles &t) {
    const int64_t target = std::max<int64_t>(std::min<int64_t>(32, Y), Y / 2048);
    bool found = false;
    double best = 0;
    auto widest = [&](int64_t rows, bool tab, int force) {
        for (int s = std::min(2 * K, force ? force : 32); s >= 1; s >>= 1) {
            if (force && s != force) continue;
            if (mid_smem(rows, s, tab) <= SMEM_MID_MAX) return s;
        }
        return 0;
    };
    for (int64_t Y2 = 1; Y2 <= Y && Y2 <= 8192; Y2 <<= 1) {
        if (y2_force && Y2 != y2_force) continue;
        const size_t fw = fwd_smem(Y2, K), iv = inv_smem(Y2, K, r, lc);
        if (fw > SMEM_FWD_MAX || iv > SMEM_INV_MAX) continue;
        const int64_t Y1 = Y / Y2;
        for (int64_t Y1b = 1; Y1b <= Y1; Y1b <<= 1) {
            if (y1b_force ? Y1b != y1b_force : (Y1b > 1 && Y1 / Y1b < 512)) continue;
            const int64_t Y1a = Y1 / Y1b;
            if (Y1b > 1 && Y1a > 2048) continue;
            if (Y1b > 1 && Y1a < 2) continue;
            // middle slice, with the twiddle tables in shared memory if possible
            // (the per-stage blocks of the length-Y1a column transform, split
            // or not)
            bool tab = true;
            int S = tab ? widest(Y1a, true, s_force) : 0;
            if (S > 0 && S < 8 && S < 2 * K && !s_force) {
                const int s2 = widest(Y1a, false, 0);  // wider without the tables
                if (s2 > S) { S = s2; tab = false; }
            }
            if (S == 0) {
                tab = false;
                S = widest(Y1a, false, s_force);
            }
            if (s_force && (s_force > 2 * K || (s_force & (s_force - 1)))) S = 0;
            if (S == 0) continue;
            const int64_t S2 = Y1b > 1 ? outer_width(Y1a, K, Y1b) : 0;
            if (Y1b > 1 && outer_smem(Y1b, S2) > SMEM_MID_MAX) continue;
            // slices narrower than 4 words fill less than a 16-byte copy per row
            const double score = (S >= 8 || S == 2 * K ? 0 : S >= 4 ? 1 : 8) + (iv <= SMEM_INV_2PERSM ? 0 : 4) +
                                 (fw <= SMEM_FWD_3PERSM ? 0 : 2) + (tab ? 0 : 1) + (Y1b > 1 ? 3 : 0) +
                                 0.1 * std::abs(ilog2((uint64_t)Y2) - ilog2((uint64_t)target));
            if (!found || score < best) {
                found = true;
                best = score;
                t.Y2 = Y2;
                t.S = S;
                t.mid_tables = tab;
                t.Y1b = Y1b;
                t.S2 = S2 ? (int32_t)S2 : 1;
                t.smem_fwd = fw;
                t.smem_mid = mid_smem(Y1a, S, tab);
                t.smem_inv = iv;
                t.smem_outer = Y1b > 1 ? outer_smem(Y1b, S2) : 0;
            }
        }
    }
    return found;
}

}  // namespace

TableLayout table_layout(int64_t Y, int64_t Y1, int32_t K) {
    TableLayout L;
    L.ty_f = 0;
    L.ty_i = L.ty_f + (size_t)Y;
    L.t1_f = L.ty_i + (size_t)Y;
    L.t1_i = L.t1_f + (size_t)Y1;
    L.tx_f = L.t1_i + (size_t)Y1;
    L.tx_i = L.tx_f + 2 * (size_t)K;
    L.untw = L.tx_i + 2 * (size_t)K;
    L.total = L.untw + (size_t)K;
    L.total = (L.total + 1) & ~(size_t)1;  // keep blocks 16-byte aligned
    return L;
}

namespace {
// The plan of the transform product itself (no packing).
ipm_status choose_plan_direct(const ipm_shape &sh, const ipm_params *prm, ShapePlan &sp) {
    if (sh.deg_a < 0 || sh.deg_b < 0 || sh.bits_a < 1 || sh.bits_b < 1 ||
        sh.bits_a > 65536 || sh.bits_b > 65536)
        return IPM_ERR_ARG;
    if (sh.deg_a >= (1ll << 40) || sh.deg_b >= (1ll << 40)) return IPM_ERR_UNSUPPORTED;
    ipm_params P{};
    if (prm) P = *prm;
    if (P.K < 0 || P.M < 0 || P.r < 0 || P.y2 < 0 || P.s < 0 || P.y1b < 0) return IPM_ERR_ARG;
    if (P.y1b == 1 || (P.y1b & (P.y1b - 1))) return IPM_ERR_ARG;
    if (P.K && (P.K < 2 || (P.K & (P.K - 1)) || P.K > (1 << KMAX_LOG2))) return IPM_ERR_ARG;
    if (P.M && (P.M < 2 || P.M > MMAX)) return IPM_ERR_ARG;
    if (P.r && P.r > RMAX) return IPM_ERR_ARG;

    const int64_t na = sh.deg_a + 1, nb = sh.deg_b + 1, nc = na + nb - 1;
    const int64_t mn = std::min(na, nb);
    const uint32_t nmag = std::max(sh.bits_a, sh.bits_b);
    const int la = (int)((sh.bits_a + 31) / 32), lb = (int)((sh.bits_b + 31) / 32);
    const int lgmin = ilog2((uint64_t)mn);
    const int lc = (int)((sh.bits_a + sh.bits_b + (uint32_t)lgmin + 31) / 32);
    const int logY = ilog2((uint64_t)nc);
    const int64_t Y = 1ll << logY;
    if (logY > PRIME_ORDER_LOG2) return IPM_ERR_UNSUPPORTED;
    const auto &primes = prime_table();

    bool found = false;
    double best_cost = 0;
    ShapePlan best{};
    for (int logK = 1; logK <= KMAX_LOG2; ++logK) {
        const int K = 1 << logK;
        if (P.K && K != P.K) continue;
        if (logK + 1 > PRIME_ORDER_LOG2) continue;
        int M = (int)((nmag + 1 + K - 1) / K);
        if (M < 2) M = 2;
        if (P.M) {
            if ((int64_t)P.M * K < (int64_t)nmag + 1) continue;
            M = P.M;
        }
        if (M > MMAX) continue;
        // 4H bound: mn * K * 2^(2M)
        Big bound = big_shl(big_from_u64((uint64_t)mn * (uint64_t)K), 2 * M);
        Big m = big_from_u64(1);
        int r = 0;
        for (int t = 1; t <= RMAX; ++t) {
            m = big_mul_u32(m, primes[t - 1]);
            if (P.r ? t == P.r : big_cmp(m, bound) > 0) {
                r = t;
                break;
            }
        }
        if (!r || big_cmp(m, bound) <= 0) continue;
        Tiles tl;
        if (!choose_tiles(Y, K, r, lc, P.y2, P.s, P.y1b, tl)) continue;
        const double pts = (double)r * (double)Y * 2.0 * K;
        const double cost = pts * (3.0 * (logY + logK + 1) + 2.0 * r + 4.0);
        if (found && cost >= best_cost) continue;
        found = true;
        best_cost = cost;
        ShapePlan s{};
        ipm_plan_info &I = s.info;
        I.na = na; I.nb = nb; I.nc = nc;
        I.la = la; I.lb = lb; I.lc = lc;
        I.K = K; I.M = M; I.N = K * M; I.r = r;
        I.Y = Y; I.Y2 = tl.Y2; I.Y1 = Y / tl.Y2; I.S = tl.S;
        double lm = 0;
        for (int t = 0; t < r; ++t) { I.primes[t] = primes[t]; lm += std::log2((double)primes[t]); }
        I.log2_modulus = lm;
        I.log2_bound = std::log2((double)mn) + logK + 2.0 * M;
        s.smem_fwd = tl.smem_fwd;
        s.smem_mid = tl.smem_mid;
        s.smem_inv = tl.smem_inv;
        s.smem_outer = tl.smem_outer;
        I.Y1b = tl.Y1b;
        s.z_words = (size_t)r * 2 * (size_t)Y * 2 * K;
        s.table_words = table_layout(Y, Y / tl.Y2, K).total;
        I.workspace_bytes = s.z_words * 4 + (size_t)r * s.table_words * 8;
        KParams &kp = s.kp;
        std::memset(&kp, 0, sizeof(kp));
        kp.na = na; kp.nb = nb; kp.nc = nc;
        kp.la = la; kp.lb = lb; kp.lc = lc;
        kp.bits_a = sh.bits_a; kp.bits_b = sh.bits_b;
        kp.K = K; kp.logK = logK; kp.M = M; kp.N = K * M; kp.r = r;
        kp.Y = Y; kp.Y2 = tl.Y2; kp.Y1 = Y / tl.Y2;
        kp.logY = logY; kp.logY2 = ilog2((uint64_t)tl.Y2); kp.logY1 = logY - kp.logY2;
        kp.S = tl.S; kp.logS = ilog2((uint64_t)tl.S);
        kp.mid_tables_in_smem = tl.mid_tables ? 1 : 0;
        kp.Y1b = tl.Y1b;
        kp.Y1a = kp.Y1 / tl.Y1b;
        kp.logY1b = ilog2((uint64_t)tl.Y1b);
        kp.logY1a = kp.logY1 - kp.logY1b;
        kp.S2 = tl.S2;
        kp.logS2 = ilog2((uint64_t)tl.S2);
        best = s;
    }
    if (!found) return (P.K || P.M || P.r || P.y2 || P.s || P.y1b) ? IPM_ERR_ARG : IPM_ERR_UNSUPPORTED;
    sp = best;
    return IPM_OK;
}

size_t round4(size_t w) { return (w + 3) & ~(size_t)3; }

}  // namespace

// Kronecker slot width for a shape: bits_a + bits_b + ceil(log2 min(na, nb)) + 1.
int kron_slot_width(const ipm_shape &sh) {
    const int64_t mn = std::min(sh.deg_a, sh.deg_b) + 1;
    return (int)(sh.bits_a + sh.bits_b) + ilog2((uint64_t)mn) + 1;
}

ipm_status choose_plan(const ipm_shape &sh, const ipm_params *prm, ShapePlan &sp) {
    ipm_params P{};
    if (prm) P = *prm;
    if (P.kron < 0) return IPM_ERR_ARG;
    if (sh.deg_a < 0 || sh.deg_b < 0 || sh.bits_a < 1 || sh.bits_b < 1 || sh.bits_a > 65536 ||
        sh.bits_b > 65536)
        return IPM_ERR_ARG;
    const int64_t na = sh.deg_a + 1, nb = sh.deg_b + 1;
    KronPlan kr{};
    kr.s = 1;
    kr.na = na;
    kr.nb = nb;
    kr.nc = na + nb - 1;
    kr.la = (int)((sh.bits_a + 31) / 32);
    kr.lb = (int)((sh.bits_b + 31) / 32);
    kr.lc = (int)((sh.bits_a + sh.bits_b + (uint32_t)ilog2((uint64_t)std::min(na, nb)) + 31) / 32);
    kr.bits_a = sh.bits_a;
    kr.bits_b = sh.bits_b;
    if (P.school < 0 || P.school > 1 || P.ks < 0 || P.ks > 1 || P.kara < 0) return IPM_ERR_ARG;
    if (P.ks) {  // Kronecker substitution: the digit polynomials' product
        if (P.kron > 1 || P.school || P.kara) return IPM_ERR_ARG;
        const int w = kr.lc + 3;
        const int64_t nA = na * w, nB = nb * w;
        if (nA + nB - 1 > (1ll << PRIME_ORDER_LOG2)) return IPM_ERR_UNSUPPORTED;
        const ipm_shape inner{nA - 1, nB - 1, 32, 32};
        ipm_params Q = P;
        Q.ks = 0;
        Q.kron = 0;
        const ipm_status st = choose_plan_direct(inner, &Q, sp);
        if (st != IPM_OK) return st;
        sp.school = false;
        sp.kr = kr;
        KsPlan &k = sp.ks;
        k.on = 1;
        k.w = w;
        k.na = na;
        k.nb = nb;
        k.nc = kr.nc;
        k.la = kr.la;
        k.lb = kr.lb;
        k.lc = kr.lc;
        k.bits_a = sh.bits_a;
        k.bits_b = sh.bits_b;
        const KParams &kp = sp.kp;
        const int64_t nslots = kr.nc + 1;
        size_t at = round4(sp.z_words);
        k.off_a = at;  at = round4(at + (size_t)nA);
        k.off_an = at; at = round4(at + ((size_t)nA + 3) / 4);
        k.off_b = at;  at = round4(at + (size_t)nB);
        k.off_bn = at; at = round4(at + ((size_t)nB + 3) / 4);
        k.off_c = at;  at = round4(at + (size_t)kp.nc * kp.lc);
        k.off_cn = at; at = round4(at + ((size_t)kp.nc + 3) / 4);
        k.off_L = at;  at = round4(at + (size_t)nslots * w);
        k.off_H = at;  at = round4(at + 2 * (size_t)nslots);
        k.off_g = at;  at = round4(at + ((size_t)nslots + 3) / 4);
        ipm_plan_info &I = sp.info;
        I.workspace_bytes += (at - sp.z_words) * 4;
        sp.z_words = at;
        I.na = na;
        I.nb = nb;
        I.nc = kr.nc;
        I.la = kr.la;
        I.lb = kr.lb;
        I.lc = kr.lc;
        I.kron = 1;
        I.kron_w = 0;
        I.kron_na = na;
        I.kron_nb = nb;
        I.kron_bits_a = sh.bits_a;
        I.kron_bits_b = sh.bits_b;
        I.school = 0;
        I.ks = 1;
        I.ks_w = w;
        I.kara = 0;
        return IPM_OK;
    }
    if (P.bigp < 0 || P.bigp > 1) return IPM_ERR_ARG;
    if (P.bigp) {  // one generalized Fermat prime, no CRT
        if (P.M || P.r || P.y2 || P.s || P.y1b || P.kron > 1 || P.school || P.ks || P.kara) return IPM_ERR_ARG;
        if (P.K && (P.K < 2 || (P.K & (P.K - 1)) || P.K > (1 << KMAX_LOG2))) return IPM_ERR_ARG;
        const int64_t mn = std::min(na, nb);
        const uint32_t nmag = std::max(sh.bits_a, sh.bits_b);
        const int logY = ilog2((uint64_t)kr.nc);
        if (logY > PRIME_ORDER_LOG2) return IPM_ERR_UNSUPPORTED;
        int K = 0, M = 0;
        for (int logK = 1; logK <= KMAX_LOG2 && !K; ++logK) {
            const int k = 1 << logK;
            if (P.K && k != P.K) continue;
            int m = (int)((nmag + 1 + k - 1) / k);
            if (m < 2) m = 2;
            if (m <= MMAX && bigp_bound_ok(mn, k, m)) { K = k; M = m; }
        }
        if (!K) return P.K ? IPM_ERR_ARG : IPM_ERR_UNSUPPORTED;
        BigpPlan b{};
        b.on = 1;
        b.K = K;
        b.logK = ilog2((uint64_t)K);
        b.M = M;
        b.N = K * M;
        b.logY = logY;
        b.Y = 1ll << logY;
        b.na = na; b.nb = nb; b.nc = kr.nc;
        b.la = kr.la; b.lb = kr.lb; b.lc = kr.lc;
        b.bits_a = sh.bits_a; b.bits_b = sh.bits_b;
        const size_t cells = (size_t)b.Y * 2 * K;  // 128-bit cells per operand
        b.off_xa = 0;
        b.off_xb = cells;
        b.tab_theta = 0;
        b.tab_untw = b.tab_theta + K;
        b.tab_wk = b.tab_untw + K;
        b.tab_wk_i = b.tab_wk + K / 2;
        b.tab_wy = b.tab_wk_i + K / 2;
        b.tab_wy_i = b.tab_wy + (size_t)(b.Y / 2);
        b.table_entries = b.tab_wy_i + (size_t)(b.Y / 2);
        ShapePlan s{};
        s.school = false;
        s.kr = kr;
        s.bp = b;
        s.z_words = 2 * cells * 4;
        ipm_plan_info &I = s.info;
        I.na = na; I.nb = nb; I.nc = kr.nc;
        I.la = kr.la; I.lb = kr.lb; I.lc = kr.lc;
        I.K = K; I.M = M; I.N = K * M; I.r = 1;
        I.Y = b.Y; I.Y1 = b.Y; I.Y2 = 1; I.Y1b = 1;
        I.log2_bound = std::log2((double)mn) + std::log2((double)K) + 2.0 * M;
        I.log2_modulus = 126.00282;  // log2((2^63 + 2^53)^2 + 1)
        I.kron = 1;
        I.kron_na = na;
        I.kron_nb = nb;
        I.kron_bits_a = sh.bits_a;
        I.kron_bits_b = sh.bits_b;
        I.bigp = 1;
        I.workspace_bytes = s.z_words * 4 + b.table_entries * 16;
        std::memset(&s.kp, 0, sizeof(s.kp));
        s.kp.na = na; s.kp.nb = nb; s.kp.nc = kr.nc;
        s.kp.la = kr.la; s.kp.lb = kr.lb; s.kp.lc = kr.lc;
        s.kp.Y1b = 1;
        sp = s;
        return IPM_OK;
    }
    if (P.kara) {  // the Karatsuba family over y with schoolbook leaves
        if (P.kara > KARA_MAX_LEVELS || P.K || P.M || P.r || P.y2 || P.s || P.y1b || P.kron > 1 || P.school)
            return IPM_ERR_ARG;
        const int L = P.kara;
        const int64_t n = std::max(na, nb);
        const int64_t m = (n + (1ll << L) - 1) >> L, n2 = m << L;
        KaraPlan k{};
        k.levels = L;
        k.n2 = n2;
        k.m = m;
        k.na = na;
        k.nb = nb;
        k.nc = kr.nc;
        k.la = kr.la;
        k.lb = kr.lb;
        k.lc = kr.lc;
        k.bits_a = sh.bits_a;
        k.bits_b = sh.bits_b;
        k.lla = (int)((sh.bits_a + L + 31) / 32);
        k.llb = (int)((sh.bits_b + L + 31) / 32);
        // every node product at depth d is below len 2^(bits_a + d) 2^(bits_b + d) <= n2 2^(bits_a + bits_b + 2L)
        k.lci = (int)((sh.bits_a + sh.bits_b + 2 * L + ilog2((uint64_t)n2) + 1 + 31) / 32);
        if (k.lla + k.llb > SCHOOL_MAX_COLUMNS) return IPM_ERR_ARG;
        if ((double)m * (double)m * k.lla * k.llb > SCHOOL_MAX_LIMB_PRODUCTS) return IPM_ERR_ARG;
        int64_t leaves = 1;
        for (int d = 0; d < L; ++d) leaves *= 3;
        size_t at = 0;
        k.off_a = at;  at = round4(at + (size_t)(leaves * m) * k.lla);
        k.off_an = at; at = round4(at + ((size_t)(leaves * m) + 3) / 4);
        k.off_b = at;  at = round4(at + (size_t)(leaves * m) * k.llb);
        k.off_bn = at; at = round4(at + ((size_t)(leaves * m) + 3) / 4);
        int64_t nodes = 1;
        for (int d = 0; d <= L; ++d) {
            const int64_t len = n2 >> d, cnt = nodes * (2 * len - 1);
            if (d > 0) {
                k.off_lev[d] = at;  at = round4(at + (size_t)cnt * k.lci);
                k.off_levn[d] = at; at = round4(at + ((size_t)cnt + 3) / 4);
            }
            nodes *= 3;
        }
        ShapePlan s{};
        s.school = false;
        s.kr = kr;
        s.ka = k;
        s.z_words = at;
        ipm_plan_info &I = s.info;
        I.na = na; I.nb = nb; I.nc = kr.nc;
        I.la = kr.la; I.lb = kr.lb; I.lc = kr.lc;
        I.Y1b = 1;
        I.kron = 1;
        I.kron_na = na;
        I.kron_nb = nb;
        I.kron_bits_a = sh.bits_a;
        I.kron_bits_b = sh.bits_b;
        I.kara = L;
        I.workspace_bytes = at * 4;
        KParams &kp = s.kp;  // one leaf product (schoolbook)
        std::memset(&kp, 0, sizeof(kp));
        kp.na = m; kp.nb = m; kp.nc = 2 * m - 1;
        kp.la = k.lla; kp.lb = k.llb; kp.lc = k.lci;
        kp.bits_a = sh.bits_a + (uint32_t)L; kp.bits_b = sh.bits_b + (uint32_t)L;
        kp.Y1b = 1;
        sp = s;
        return IPM_OK;
    }
    if (P.school) {
        if (P.K || P.M || P.r || P.y2 || P.s || P.y1b || P.kron > 1) return IPM_ERR_ARG;
        if (kr.la + kr.lb > SCHOOL_MAX_COLUMNS) return IPM_ERR_ARG;
        if ((double)na * (double)nb * kr.la * kr.lb > SCHOOL_MAX_LIMB_PRODUCTS) return IPM_ERR_ARG;
        ShapePlan s{};
        s.school = true;
        s.kr = kr;
        ipm_plan_info &I = s.info;
        I.na = na; I.nb = nb; I.nc = kr.nc;
        I.la = kr.la; I.lb = kr.lb; I.lc = kr.lc;
        I.Y1b = 1;
        I.kron = 1;
        I.kron_na = na;
        I.kron_nb = nb;
        I.kron_bits_a = sh.bits_a;
        I.kron_bits_b = sh.bits_b;
        I.school = 1;
        KParams &kp = s.kp;
        std::memset(&kp, 0, sizeof(kp));
        kp.na = na; kp.nb = nb; kp.nc = kr.nc;
        kp.la = kr.la; kp.lb = kr.lb; kp.lc = kr.lc;
        kp.bits_a = sh.bits_a; kp.bits_b = sh.bits_b;
        kp.Y1b = 1;
        sp = s;
        return IPM_OK;
    }
    if (P.kron <= 1) {
        P.kron = 0;
        const ipm_status st = choose_plan_direct(sh, &P, sp);
        if (st != IPM_OK) return st;
        sp.school = false;
        sp.info.school = 0;
        sp.kr = kr;
        sp.info.kron = 1;
        sp.info.kron_w = 0;
        sp.info.kron_na = na;
        sp.info.kron_nb = nb;
        sp.info.kron_bits_a = sh.bits_a;
        sp.info.kron_bits_b = sh.bits_b;
        return IPM_OK;
    }
    if ((P.kron & (P.kron - 1)) || P.kron > KRON_MAX) return IPM_ERR_ARG;
    const int w = kron_slot_width(sh);
    if (w > KRON_WMAX) return IPM_ERR_ARG;
    kr.s = P.kron;
    kr.w = w;
    const int64_t na2 = (na + kr.s - 1) / kr.s, nb2 = (nb + kr.s - 1) / kr.s;
    // |A'_k| < 2^(bits_a + (s-1) w + 1): the slots hold disjoint bit ranges
    const ipm_shape inner{na2 - 1, nb2 - 1, sh.bits_a + (uint32_t)((kr.s - 1) * w + 1),
                          sh.bits_b + (uint32_t)((kr.s - 1) * w + 1)};
    ipm_params Q = P;
    Q.kron = 0;
    const ipm_status st = choose_plan_direct(inner, &Q, sp);
    if (st != IPM_OK) return st;
    sp.school = false;
    sp.info.school = 0;
    // packed operands and product after the transform workspace (16-byte aligned)
    const KParams &kp = sp.kp;
    size_t at = round4(sp.z_words);
    kr.off_a = at;  at = round4(at + (size_t)kp.na * kp.la);
    kr.off_an = at; at = round4(at + ((size_t)kp.na + 3) / 4);
    kr.off_b = at;  at = round4(at + (size_t)kp.nb * kp.lb);
    kr.off_bn = at; at = round4(at + ((size_t)kp.nb + 3) / 4);
    kr.off_c = at;  at = round4(at + (size_t)kp.nc * kp.lc);
    kr.off_cn = at; at = round4(at + ((size_t)kp.nc + 3) / 4);
    ipm_plan_info &I = sp.info;
    I.workspace_bytes += (at - sp.z_words) * 4;
    sp.z_words = at;
    sp.kr = kr;
    I.kron = kr.s;
    I.kron_w = w;
    I.kron_na = na2;
    I.kron_nb = nb2;
    I.kron_bits_a = inner.bits_a;
    I.kron_bits_b = inner.bits_b;
    I.na = na;
    I.nb = nb;
    I.nc = kr.nc;
    I.la = kr.la;
    I.lb = kr.lb;
    I.lc = kr.lc;
    return IPM_OK;
}

void build_tables(ShapePlan &sp, uint2 *tab) {
    KParams &kp = sp.kp;
    const int64_t Y = kp.Y;
    const int K = kp.K;
    const TableLayout L = table_layout(Y, kp.Y1, K);
    for (int t = 0; t < kp.r; ++t) {
        const uint32_t p = sp.info.primes[t];
        uint2 *blk = tab + (size_t)t * L.total;
        const uint32_t w = root_of_unity(p, kp.logY);          // order Y
        const uint32_t th = root_of_unity(p, kp.logK + 1);     // order 2K
        const uint32_t wi = invmod(w, p), thi = invmod(th, p);
        uint64_t x = 1, xi = 1;
        for (int64_t e = 0; e < Y; ++e) {
            blk[L.ty_f + e] = make_uint2((uint32_t)x, shoup_q((uint32_t)x, p));
            blk[L.ty_i + e] = make_uint2((uint32_t)xi, shoup_q((uint32_t)xi, p));
            x = x * w % p;
            xi = xi * wi % p;
        }
        for (int64_t e = 0; e < kp.Y1; ++e) {  // omega_Y1 = omega_Y^Y2
            blk[L.t1_f + e] = blk[L.ty_f + e * kp.Y2];
            blk[L.t1_i + e] = blk[L.ty_i + e * kp.Y2];
        }
        // scale = 2^32 * (2 Y K)^{-1} mod p
        const uint64_t two32 = (1ull << 32) % p;
        const uint64_t denom = (2ull * (uint64_t)(Y % p) % p) * (uint64_t)K % p;
        const uint32_t scale = (uint32_t)(two32 * invmod((uint32_t)denom, p) % p);
        x = 1;
        xi = 1;
        for (int e = 0; e < 2 * K; ++e) {
            blk[L.tx_f + e] = make_uint2((uint32_t)x, shoup_q((uint32_t)x, p));
            blk[L.tx_i + e] = make_uint2((uint32_t)xi, shoup_q((uint32_t)xi, p));
            if (e < K) {
                uint32_t u = (uint32_t)((uint64_t)scale * xi % p);
                blk[L.untw + e] = make_uint2(u, shoup_q(u, p));
            }
            x = x * th % p;
            xi = xi * thi % p;
        }
        PrimeConst &pc = kp.pc[t];
        pc.p = p;
        pc.p2 = 2 * p;
        uint32_t inv = p;  // Newton iteration for p^{-1} mod 2^32
        for (int i = 0; i < 5; ++i) inv *= 2u - p * inv;
        pc.mont = 0u - inv;
        pc.one_s = shoup_q(1, p);
        pc.c32 = (uint32_t)two32;
        pc.c32_s = shoup_q(pc.c32, p);
        pc.scale = scale;
        pc.scale_s = shoup_q(scale, p);
    }
    for (int t = 0; t < kp.r; ++t)
        for (int s = 0; s < t; ++s) {
            uint32_t pt = kp.pc[t].p;
            uint32_t g = invmod(kp.pc[s].p % pt, pt);
            kp.ginv[t][s] = g;
            kp.ginv_s[t][s] = shoup_q(g, pt);
        }
    // m = prod p_t in r words (each p < 2^30 so r words suffice)
    uint32_t mw[RMAX + 1] = {1};
    for (int t = 0; t < kp.r; ++t) {
        uint64_t carry = 0;
        for (int i = 0; i <= RMAX; ++i) {
            uint64_t v = (uint64_t)mw[i] * kp.pc[t].p + carry;
            mw[i] = (uint32_t)v;
            carry = v >> 32;
        }
    }
    for (int i = 0; i < RMAX; ++i) kp.m_words[i] = i < kp.r ? mw[i] : 0;
}

// Byte-slice fragments of the radix-16 DFT matrices for the tensor-core
// stages (layout and arithmetic: stage_tc16 in ntt_stages.cuh).  omega is
// omega_16 = g^((p-1)/16) for the generator g every table of the plan uses,
// so it is the root every radix-16 register stage uses too.
void build_tc_fragments(const uint32_t *primes, int r, uint32_t *out) {
    auto brev4 = [](int x) { return ((x & 1) << 3) | ((x & 2) << 1) | ((x & 4) >> 1) | ((x & 8) >> 3); };
    for (int t = 0; t < r; ++t) {
        const uint32_t p = primes[t];
        const uint64_t w = root_of_unity(p, 4), wi = invmod((uint32_t)w, p);
        uint64_t pw[16], pwi[16], cs[4];
        pw[0] = pwi[0] = 1;
        for (int e = 1; e < 16; ++e) {
            pw[e] = pw[e - 1] * w % p;
            pwi[e] = pwi[e - 1] * wi % p;
        }
        cs[0] = (1ull << 32) % p;  // 2^(8s) 2^32 mod p
        for (int s = 1; s < 4; ++s) cs[s] = (cs[s - 1] << 8) % p;
        for (int dir = 0; dir < 2; ++dir) {
            uint32_t *frag = out + (size_t)t * TC_FRAG_WORDS + (size_t)dir * (TC_FRAG_WORDS / 2);
            // C[j][k][s] = E[j][k] 2^(8s) 2^32 mod p
            uint32_t C[16][16][4];
            for (int j = 0; j < 16; ++j)
                for (int k = 0; k < 16; ++k) {
                    const uint64_t e = dir == 0 ? pw[(brev4(j) * k) & 15] : pwi[(j * brev4(k)) & 15];
                    for (int s = 0; s < 4; ++s) C[j][k][s] = (uint32_t)(e * cs[s] % p);
                }
            for (int l = 0; l < 4; ++l)
                for (int lane = 0; lane < 32; ++lane) {
                    const int g = lane >> 2, q = lane & 3;
                    for (int c = 0; c < 2; ++c)
                        for (int i = 0; i < 4; ++i) {
                            // register i: rows g (i even) or g + 8 (i odd),
                            // inputs 8c + q (i < 2) or 8c + 4 + q (i >= 2)
                            const int j = g + 8 * (i & 1), k = 8 * c + q + 4 * (i >> 1);
                            uint32_t word = 0;
                            for (int s = 0; s < 4; ++s) word |= ((C[j][k][s] >> (8 * l)) & 0xffu) << (8 * s);
                            frag[(l * 32 + lane) * 8 + c * 4 + i] = word;
                        }
                }
        }
    }
}

}  // namespace ipm

namespace ipm {

// Cost-model features of one candidate plan (the layout is given with
// IPM_FEATURES in ipm.h).
void candidate_features(const ipm_shape &sh, const ShapePlan &sp, float *f) {
    const ipm_plan_info &I = sp.info;
    auto lg = [](double x) { return (float)std::log2(std::max(1.0, x)); };
    f[0] = lg((double)I.na);
    f[1] = lg((double)I.nb);
    f[2] = lg((double)sh.bits_a);
    f[3] = lg((double)sh.bits_b);
    f[4] = lg((double)I.K);
    f[5] = (float)I.M / 32.0f;
    f[6] = (float)I.r;
    f[7] = lg((double)I.Y);
    f[8] = lg((double)I.Y2);
    f[9] = lg((double)I.S);
    f[10] = lg((double)I.Y1b);
    f[11] = sp.school ? lg((double)I.na * (double)I.nb * I.la * I.lb) : lg((double)I.r * (double)I.Y * 2.0 * I.K);
    f[12] = lg((double)sp.kp.Y1a);
    f[13] = lg((double)I.na * sh.bits_a + (double)I.nb * sh.bits_b);
    f[14] = !sp.school && sp.smem_fwd <= SMEM_FWD_3PERSM ? 1.0f : 0.0f;
    f[15] = !sp.school && sp.smem_inv <= SMEM_INV_2PERSM ? 1.0f : 0.0f;
    f[16] = lg((double)sp.kr.s);
    f[17] = sp.school ? 1.0f : 0.0f;
    f[18] = 0.0f;  // log2(min(batch size, 16)): set by the dispatcher
}

}  // namespace ipm

extern "C" int32_t ipm_candidates(const ipm_shape *shape, ipm_candidate *out, int32_t max) {
    if (!shape || max < 0 || (max > 0 && !out)) return -(int32_t)IPM_ERR_ARG;
    ipm::ShapePlan base;
    ipm_status st = ipm::choose_plan(*shape, nullptr, base);
    if (st != IPM_OK) return -(int32_t)st;
    std::vector<std::pair<ipm_params, ipm::ShapePlan>> found;
    auto add = [&](const ipm_params &prm) {
        ipm::ShapePlan sp;
        if (ipm::choose_plan(*shape, &prm, sp) != IPM_OK) return;
        for (auto &f : found) {
            const ipm_plan_info &a = f.second.info, &b = sp.info;
            if (a.K == b.K && a.M == b.M && a.r == b.r && a.Y2 == b.Y2 && a.S == b.S && a.Y1b == b.Y1b &&
                a.kron == b.kron && a.school == b.school)
                return;
        }
        found.emplace_back(prm, sp);
    };
    // digit splits from half to eight times the planner's K (the range in
    // which the measured best plans lie), each with its tile variants
    for (int logK = 1; logK <= ipm::KMAX_LOG2; ++logK) {
        if ((1 << logK) < base.info.K / 2 || (1 << logK) > base.info.K * 8) continue;
        ipm_params prm{};
        prm.K = 1 << logK;
        ipm::ShapePlan sp;
        if (ipm::choose_plan(*shape, &prm, sp) != IPM_OK) continue;
        add(prm);
        for (int64_t y2 : {sp.info.Y2 / 2, sp.info.Y2 * 2, sp.info.Y2 * 4}) {
            if (y2 < 1) continue;
            ipm_params v = prm;
            v.y2 = (int32_t)y2;
            add(v);
        }
        for (int32_t sl : {sp.info.S / 2, sp.info.S * 2}) {  // narrower and wider middle slices
            if (sl < 1) continue;
            ipm_params v = prm;
            v.s = sl;
            add(v);
        }
    }
    // Kronecker balancing: each packing factor with the planner's plan of
    // the packed product and its K halved and doubled
    if (ipm::kron_slot_width(*shape) <= ipm::KRON_WMAX) {
        for (int s = 2; s <= ipm::KRON_MAX; s *= 2) {
            if (shape->deg_a + 1 < s && shape->deg_b + 1 < s) break;
            ipm_params prm{};
            prm.kron = s;
            ipm::ShapePlan sp;
            if (ipm::choose_plan(*shape, &prm, sp) != IPM_OK) continue;
            add(prm);
            for (int32_t k : {sp.info.K / 2, sp.info.K * 2}) {
                ipm_params v = prm;
                v.K = k;
                if (k >= 2) add(v);
            }
        }
    }
    {  // the schoolbook family, where its limits allow it
        ipm_params prm{};
        prm.school = 1;
        add(prm);
    }
    const int32_t n = (int32_t)found.size();
    for (int32_t i = 0; i < n && i < max; ++i) {
        out[i].params = found[(size_t)i].first;
        out[i].info = found[(size_t)i].second.info;
        ipm::candidate_features(*shape, found[(size_t)i].second, out[i].features);
    }
    return n;
}

extern "C" ipm_status ipm_choose(const ipm_shape *shape, const ipm_params *params,
                                 ipm_plan_info *out) {
    if (!shape || !out) return IPM_ERR_ARG;
    ipm::ShapePlan sp;
    ipm_status st = ipm::choose_plan(*shape, params, sp);
    if (st != IPM_OK) return st;
    *out = sp.info;
    return IPM_OK;
}

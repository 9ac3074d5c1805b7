/*
 * ipm_oracle.c -- CPU oracle for dense integer polynomial multiplication.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  The CUDA
 * library never links, includes or calls it, and it shares no code with it.
 *
 * What it computes is the plain definition of the problem (§1, §2 of
 * "Parallel Integer Polynomial Multiplication", arXiv 1612.05778):
 *
 *     c(y) = a(y) b(y),   c_k = sum_{i+j=k} a_i b_j   over Z,
 *
 * with a of na coefficients and b of nb coefficients, so c has na+nb-1.
 * The method of the paper reaches this exact result (the recovery identity,
 * Eq. (recoveringC), is exact), so the oracle is this definition written out
 * with its own arbitrary-precision integers: schoolbook limb products summed
 * into two non-negative accumulators (terms with positive and with negative
 * sign), subtracted at the end.
 *
 * Number format (the library's operand format): coefficient i occupies
 * 32-bit little-endian limbs [i*L, (i+1)*L) holding |a_i|; neg[i] = 1 marks
 * a negative coefficient.  Output zero is always written with sign 0.
 *
 * Pins (tests/test_oracle_pins.py): brute force against Python's own
 * integers on tiny inputs; Kronecker substitution through one big Python
 * integer product on mid sizes; the closed form for constant polynomials;
 * the exact identities C(1)=A(1)B(1) and C(-1)=A(-1)B(-1); evaluation modulo
 * independent 61-bit primes.  The `mutation` argument of orc_polymul_mut
 * plants known mistakes so that the tests can show each pin catches them;
 * the public entry points always pass 0.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ---- bigint helpers (non-negative, little-endian u32 limbs) ------------ */

/* acc[0..len) += x[0..lx) * y[0..ly); acc must have room for the carry.   */
static void mul_acc(uint32_t *acc, int64_t len, const uint32_t *x, int32_t lx,
                    const uint32_t *y, int32_t ly, int drop_top_carry) {
    for (int32_t i = 0; i < lx; ++i) {
        uint64_t xi = x[i];
        if (xi == 0) continue;
        uint64_t carry = 0;
        for (int32_t j = 0; j < ly; ++j) {
            uint64_t t = xi * (uint64_t)y[j] + acc[i + j] + carry;
            acc[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        if (drop_top_carry) continue;           /* planted mistake (mutation 4) */
        for (int64_t k = (int64_t)i + ly; carry != 0 && k < len; ++k) {
            uint64_t t = (uint64_t)acc[k] + carry;
            acc[k] = (uint32_t)t;
            carry = t >> 32;
        }
    }
}

/* returns -1, 0, 1 as x <, =, > y (both len limbs) */
static int cmp_n(const uint32_t *x, const uint32_t *y, int64_t len) {
    for (int64_t k = len - 1; k >= 0; --k) {
        if (x[k] != y[k]) return x[k] < y[k] ? -1 : 1;
    }
    return 0;
}

/* out = x - y, requires x >= y */
static void sub_n(uint32_t *out, const uint32_t *x, const uint32_t *y, int64_t len) {
    uint64_t borrow = 0;
    for (int64_t k = 0; k < len; ++k) {
        uint64_t t = (uint64_t)x[k] - y[k] - borrow;
        out[k] = (uint32_t)t;
        borrow = (t >> 63) & 1;
    }
}

/* ---- one output coefficient ------------------------------------------- */

typedef struct {
    int64_t na, nb;
    int32_t la, lb, lc;
    const uint32_t *a, *b;
    const uint8_t *an, *bn;
    uint32_t *c;
    uint8_t *cn;
    int mutation;
    int64_t k0, k1;       /* coefficient range of a worker */
    int status;
} job_t;

/*
 * c_k = sum over i of a_i * b_{k-i}, 0 <= i < na, 0 <= k-i < nb.
 * pos/neg are scratch accumulators of `width` limbs.
 */
static int one_coeff(const job_t *J, int64_t k, uint32_t *pos, uint32_t *neg,
                     int64_t width, uint32_t *out, uint8_t *out_neg) {
    memset(pos, 0, (size_t)width * 4);
    memset(neg, 0, (size_t)width * 4);
    int64_t ilo = k - (J->nb - 1);
    if (ilo < 0) ilo = 0;
    int64_t ihi = k < J->na - 1 ? k : J->na - 1;
    if (J->mutation == 1) ilo += 1;             /* planted mistake: drop a term */
    for (int64_t i = ilo; i <= ihi; ++i) {
        int64_t j = k - i;
        if (J->mutation == 3 && j + 1 < J->nb) j += 1;   /* planted: wrong index */
        const uint32_t *ai = J->a + (size_t)i * J->la;
        const uint32_t *bj = J->b + (size_t)j * J->lb;
        int sb = J->bn[j];
        if (J->mutation == 2) sb = 0;           /* planted: drop b's sign */
        int s = J->an[i] ^ sb;
        if (J->mutation == 5) {                 /* planted: limbs read big-endian */
            uint32_t tmp[64];
            int32_t la = J->la < 64 ? J->la : 64;
            for (int32_t q = 0; q < la; ++q) tmp[q] = ai[la - 1 - q];
            mul_acc(s ? neg : pos, width, tmp, la, bj, J->lb, 0);
        } else {
            mul_acc(s ? neg : pos, width, ai, J->la, bj, J->lb, J->mutation == 4);
        }
    }
    int sign = 0;
    int c = cmp_n(pos, neg, width);
    if (c >= 0) {
        sub_n(pos, pos, neg, width);
    } else {
        sub_n(pos, neg, pos, width);
        sign = 1;
    }
    /* the result must fit in lc limbs */
    for (int64_t q = J->lc; q < width; ++q)
        if (pos[q] != 0) return -2;
    int nz = 0;
    for (int32_t q = 0; q < J->lc; ++q) {
        out[q] = pos[q];
        nz |= pos[q] != 0;
    }
    *out_neg = (uint8_t)(nz ? sign : 0);
    return 0;
}

static int64_t acc_width(const job_t *J) {
    /* |c_k| < min(na,nb) * 2^(32 la + 32 lb): la+lb limbs plus 2 for the count */
    int64_t w = (int64_t)J->la + J->lb + 2;
    if (w < J->lc) w = J->lc;
    return w;
}

static void *worker(void *arg) {
    job_t *J = (job_t *)arg;
    int64_t width = acc_width(J);
    uint32_t *pos = (uint32_t *)malloc((size_t)width * 4);
    uint32_t *neg = (uint32_t *)malloc((size_t)width * 4);
    if (!pos || !neg) { J->status = -3; free(pos); free(neg); return NULL; }
    for (int64_t k = J->k0; k < J->k1; ++k) {
        int st = one_coeff(J, k, pos, neg, width, J->c + (size_t)k * J->lc, J->cn + k);
        if (st) { J->status = st; break; }
    }
    free(pos);
    free(neg);
    return NULL;
}

/*
 * Full product.  Returns 0 on success, -1 on bad arguments, -2 when a
 * coefficient does not fit in lc limbs, -3 when out of memory.
 */
int orc_polymul_mut(int64_t na, int32_t la, const uint32_t *a, const uint8_t *an,
                    int64_t nb, int32_t lb, const uint32_t *b, const uint8_t *bn,
                    int32_t lc, uint32_t *c, uint8_t *cn, int32_t nthreads, int mutation) {
    if (na < 1 || nb < 1 || la < 1 || lb < 1 || lc < 1 || !a || !b || !an || !bn || !c || !cn)
        return -1;
    if (mutation == 5 && la > 64) return -1;
    int64_t nc = na + nb - 1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nthreads > nc) nthreads = (int32_t)nc;
    job_t jobs[256];
    pthread_t tids[256];
    double total = (double)na * (double)nb;
    for (int32_t t = 0; t < nthreads; ++t) {
        job_t *J = &jobs[t];
        J->na = na; J->nb = nb; J->la = la; J->lb = lb; J->lc = lc;
        J->a = a; J->b = b; J->an = an; J->bn = bn; J->c = c; J->cn = cn;
        J->mutation = mutation; J->status = 0;
    }
    /* split by the cumulative number of terms so that threads finish together */
    {
        int64_t kk = 0;
        double cum = 0;
        for (int32_t t = 0; t < nthreads; ++t) {
            jobs[t].k0 = kk;
            double target = total * (double)(t + 1) / nthreads;
            while (kk < nc && (cum < target || t == nthreads - 1)) {
                int64_t lo = kk - (nb - 1) < 0 ? 0 : kk - (nb - 1);
                int64_t hi = kk < na - 1 ? kk : na - 1;
                cum += (double)(hi - lo + 1);
                ++kk;
            }
            jobs[t].k1 = kk;
        }
        jobs[nthreads - 1].k1 = nc;
    }
    if (nthreads == 1) {
        worker(&jobs[0]);
        return jobs[0].status;
    }
    int started = 0;
    for (int32_t t = 0; t < nthreads; ++t) {
        if (pthread_create(&tids[t], NULL, worker, &jobs[t]) != 0) break;
        ++started;
    }
    for (int32_t t = 0; t < started; ++t) pthread_join(tids[t], NULL);
    for (int32_t t = started; t < nthreads; ++t) worker(&jobs[t]);
    for (int32_t t = 0; t < nthreads; ++t)
        if (jobs[t].status) return jobs[t].status;
    return 0;
}

int orc_polymul(int64_t na, int32_t la, const uint32_t *a, const uint8_t *an,
                int64_t nb, int32_t lb, const uint32_t *b, const uint8_t *bn,
                int32_t lc, uint32_t *c, uint8_t *cn, int32_t nthreads) {
    return orc_polymul_mut(na, la, a, an, nb, lb, b, bn, lc, c, cn, nthreads, 0);
}

/*
 * A chosen list of output coefficients (the full-size checks sample these).
 * ks[0..nk) are coefficient indices; row q of c/cn receives c_{ks[q]}.
 */
typedef struct {
    job_t base;
    const int64_t *ks;
    int64_t q0, q1;
} sjob_t;

static void *sample_worker(void *arg) {
    sjob_t *S = (sjob_t *)arg;
    job_t *J = &S->base;
    int64_t width = acc_width(J);
    uint32_t *pos = (uint32_t *)malloc((size_t)width * 4);
    uint32_t *neg = (uint32_t *)malloc((size_t)width * 4);
    if (!pos || !neg) { J->status = -3; free(pos); free(neg); return NULL; }
    for (int64_t q = S->q0; q < S->q1; ++q) {
        int st = one_coeff(J, S->ks[q], pos, neg, width, J->c + (size_t)q * J->lc, J->cn + q);
        if (st) { J->status = st; break; }
    }
    free(pos);
    free(neg);
    return NULL;
}

int orc_coeffs(int64_t nk, const int64_t *ks,
               int64_t na, int32_t la, const uint32_t *a, const uint8_t *an,
               int64_t nb, int32_t lb, const uint32_t *b, const uint8_t *bn,
               int32_t lc, uint32_t *c, uint8_t *cn, int32_t nthreads) {
    if (na < 1 || nb < 1 || la < 1 || lb < 1 || lc < 1 || nk < 0) return -1;
    for (int64_t q = 0; q < nk; ++q)
        if (ks[q] < 0 || ks[q] >= na + nb - 1) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nk == 0) return 0;
    if (nthreads > nk) nthreads = (int32_t)nk;
    sjob_t jobs[256];
    pthread_t tids[256];
    for (int32_t t = 0; t < nthreads; ++t) {
        job_t *J = &jobs[t].base;
        J->na = na; J->nb = nb; J->la = la; J->lb = lb; J->lc = lc;
        J->a = a; J->b = b; J->an = an; J->bn = bn; J->c = c; J->cn = cn;
        J->mutation = 0; J->status = 0;
        jobs[t].ks = ks;
        jobs[t].q0 = nk * t / nthreads;
        jobs[t].q1 = nk * (t + 1) / nthreads;
    }
    int started = 0;
    for (int32_t t = 0; t < nthreads; ++t) {
        if (pthread_create(&tids[t], NULL, sample_worker, &jobs[t]) != 0) break;
        ++started;
    }
    for (int32_t t = 0; t < started; ++t) pthread_join(tids[t], NULL);
    for (int32_t t = started; t < nthreads; ++t) sample_worker(&jobs[t]);
    for (int32_t t = 0; t < nthreads; ++t)
        if (jobs[t].base.status) return jobs[t].base.status;
    return 0;
}

/* ---- evaluation modulo a prime q < 2^62 -------------------------------- */

static uint64_t mulmod64(uint64_t x, uint64_t y, uint64_t q) {
    return (uint64_t)(((unsigned __int128)x * y) % q);
}

/* sum_k s_k |c_k| t^k mod q, where s_k = -1 if neg[k] else +1 */
uint64_t orc_eval_mod(int64_t n, int32_t l, const uint32_t *x, const uint8_t *neg,
                      uint64_t t, uint64_t q) {
    uint64_t w32 = (uint64_t)(((unsigned __int128)1 << 32) % q);
    uint64_t acc = 0;
    t %= q;
    for (int64_t k = n - 1; k >= 0; --k) {
        const uint32_t *xk = x + (size_t)k * l;
        uint64_t v = 0;
        for (int32_t r = l - 1; r >= 0; --r) v = (mulmod64(v, w32, q) + xk[r]) % q;
        if (neg[k] && v) v = q - v;
        acc = (mulmod64(acc, t, q) + v) % q;
    }
    return acc;
}

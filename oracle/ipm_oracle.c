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

/* ======================================================================
 * Full outputs at large sizes: Kronecker substitution (§1: the product of
 * two polynomials is read off the product of the integers a(2^s), b(2^s))
 * with the oracle's own Karatsuba integer multiplication (A. Karatsuba,
 * Yu. Ofman, "Multiplication of multidigit numbers on automata", 1962).
 *
 *   A = a(2^s) = sum_i a_i 2^(s i),  B = b(2^s),  C = A B = sum_k c_k 2^(s k)
 *
 * with slots of s = 32 (lc + 1) bits: |c_k| < 2^(32 lc) <= 2^(s-1), so the
 * signed slots of C are read back exactly (a slot value t, plus the
 * borrow of the slot below, is c_k when below 2^(s-1) and c_k + 2^s with a
 * borrow of one into the next slot otherwise).  Schoolbook on the full
 * cfg sizes is out of reach (about 10^13 limb products); this is the
 * definition of c evaluated at 2^s, with the integer product done by
 * Karatsuba's three half-size products.  Pinned against the schoolbook
 * oracle and Python integers in tests/test_oracle_pins.py.
 * ====================================================================== */

typedef unsigned __int128 u128;
#define KARA_BASE 32   /* schoolbook below this many 64-bit limbs */

/* r[0..2n) = a[0..n) * b[0..n), schoolbook on 64-bit limbs */
static void school64(uint64_t *r, const uint64_t *a, const uint64_t *b, int64_t n) {
    memset(r, 0, (size_t)(2 * n) * 8);
    for (int64_t i = 0; i < n; ++i) {
        uint64_t carry = 0;
        const u128 ai = a[i];
        for (int64_t j = 0; j < n; ++j) {
            u128 t = ai * b[j] + r[i + j] + carry;
            r[i + j] = (uint64_t)t;
            carry = (uint64_t)(t >> 64);
        }
        r[i + n] = carry;
    }
}

/* r[0..n) = x[0..n) + y[0..n); returns the carry */
static uint64_t add64(uint64_t *r, const uint64_t *x, const uint64_t *y, int64_t n) {
    uint64_t c = 0;
    for (int64_t k = 0; k < n; ++k) {
        u128 t = (u128)x[k] + y[k] + c;
        r[k] = (uint64_t)t;
        c = (uint64_t)(t >> 64);
    }
    return c;
}

/* r[0..n) = x[0..n) - y[0..n); returns the borrow */
static uint64_t sub64(uint64_t *r, const uint64_t *x, const uint64_t *y, int64_t n) {
    uint64_t b = 0;
    for (int64_t k = 0; k < n; ++k) {
        uint64_t xk = x[k], yk = y[k];
        uint64_t d = xk - yk - b;
        b = (xk < yk) || (xk == yk && b) ? 1 : 0;
        r[k] = d;
    }
    return b;
}

/* adds x[0..n) into r[0..len) (len >= n), carrying upward */
static void add_into(uint64_t *r, int64_t len, const uint64_t *x, int64_t n) {
    uint64_t c = add64(r, r, x, n);
    for (int64_t k = n; c && k < len; ++k) {
        r[k] += 1;
        c = r[k] == 0;
    }
}

/* |x - y| for x of nx limbs and y of ny limbs (nx, ny <= n), zero-extended
 * to n limbs, into d[0..n); returns 1 when x < y */
static int absdiff(uint64_t *d, const uint64_t *x, int64_t nx, const uint64_t *y, int64_t ny, int64_t n) {
    int64_t k;
    int cmp = 0;
    for (k = n - 1; k >= 0; --k) {
        uint64_t xk = k < nx ? x[k] : 0, yk = k < ny ? y[k] : 0;
        if (xk != yk) { cmp = xk < yk ? -1 : 1; break; }
    }
    const uint64_t *hi = cmp < 0 ? y : x, *lo = cmp < 0 ? x : y;
    int64_t nh = cmp < 0 ? ny : nx, nl = cmp < 0 ? nx : ny;
    uint64_t b = 0;
    for (k = 0; k < n; ++k) {
        uint64_t hk = k < nh ? hi[k] : 0, lk = k < nl ? lo[k] : 0;
        uint64_t dk = hk - lk - b;
        b = (hk < lk) || (hk == lk && b) ? 1 : 0;
        d[k] = dk;
    }
    return cmp < 0;
}

typedef struct {
    uint64_t *r;
    const uint64_t *a, *b;
    int64_t n;
    int depth;  /* levels that still run their three products on threads */
    int status;
} kara_job;

static int kara(uint64_t *r, const uint64_t *a, const uint64_t *b, int64_t n, uint64_t *tmp, int depth);

static void *kara_thread(void *arg) {
    kara_job *J = (kara_job *)arg;
    uint64_t *tmp = (uint64_t *)malloc((size_t)(4 * J->n + 256) * 8);
    if (!tmp) { J->status = -3; return NULL; }
    J->status = kara(J->r, J->a, J->b, J->n, tmp, J->depth);
    free(tmp);
    return NULL;
}

/*
 * r[0..2n) = a[0..n) * b[0..n).  With h = floor(n/2), m = n - h and
 * a = a0 + a1 W^h, b = b0 + b1 W^h (W = 2^64):
 *     a b = z0 + (z0 + z2 + s |a0 - a1| |b1 - b0|) W^h + z2 W^(2h),
 * z0 = a0 b0, z2 = a1 b1, s the sign of (a0 - a1)(b1 - b0): the middle
 * term is a0 b1 + a1 b0 >= 0.  tmp holds at least 4 n + 64 limbs.
 */
static int kara(uint64_t *r, const uint64_t *a, const uint64_t *b, int64_t n, uint64_t *tmp, int depth) {
    if (n <= KARA_BASE) {
        school64(r, a, b, n);
        return 0;
    }
    const int64_t h = n / 2, m = n - h;
    uint64_t *da = tmp, *db = tmp + m, *p = tmp + 2 * m, *rest = tmp + 4 * m;
    const int na_neg = absdiff(da, a, h, a + h, m, m);   /* |a0 - a1| */
    const int nb_neg = absdiff(db, b + h, m, b, h, m);   /* |b1 - b0| */
    const int neg = na_neg ^ nb_neg;
    int st = 0;
    if (depth > 0) {
        kara_job J[3] = {{r, a, b, h, depth - 1, 0}, {r + 2 * h, a + h, b + h, m, depth - 1, 0},
                         {p, da, db, m, depth - 1, 0}};
        pthread_t tid[2];
        int started[2] = {0, 0};
        for (int q = 0; q < 2; ++q) started[q] = pthread_create(&tid[q], NULL, kara_thread, &J[q]) == 0;
        kara_thread(&J[2]);
        for (int q = 0; q < 2; ++q) {
            if (started[q]) pthread_join(tid[q], NULL);
            else kara_thread(&J[q]);
        }
        for (int q = 0; q < 3; ++q) if (J[q].status) st = J[q].status;
        if (st) return st;
    } else {
        st = kara(r, a, b, h, rest, 0);                 /* z0 in r[0, 2h) */
        if (!st) st = kara(r + 2 * h, a + h, b + h, m, rest, 0);  /* z2 in r[2h, 2n) */
        if (!st) st = kara(p, da, db, m, rest, 0);      /* |a0-a1| |b1-b0| */
        if (st) return st;
    }
    /* t = z0 + z2 +- p, 2m + 1 limbs (non-negative) */
    uint64_t *t = rest;
    memcpy(t, r + 2 * h, (size_t)(2 * m) * 8);
    t[2 * m] = 0;
    add_into(t, 2 * m + 1, r, 2 * h);
    if (neg) {
        uint64_t bw = sub64(t, t, p, 2 * m);
        t[2 * m] -= bw;
    } else {
        add_into(t, 2 * m + 1, p, 2 * m);
    }
    add_into(r + h, 2 * n - h, t, 2 * m + 1 <= 2 * n - h ? 2 * m + 1 : 2 * n - h);
    return 0;
}

/* Product of two non-negative integers of n 32-bit limbs each (n even),
 * r of 2n limbs: Karatsuba over 64-bit limbs (little-endian pairs). */
int orc_kara_mul(int64_t n32, const uint32_t *a, const uint32_t *b, uint32_t *r, int32_t nthreads) {
    if (n32 < 1 || (n32 & 1)) return -1;
    const int64_t n = n32 / 2;
    uint64_t *A = (uint64_t *)malloc((size_t)n * 8), *B = (uint64_t *)malloc((size_t)n * 8);
    uint64_t *R = (uint64_t *)malloc((size_t)(2 * n) * 8);
    uint64_t *tmp = (uint64_t *)malloc((size_t)(4 * n + 256) * 8);
    int st = -3;
    if (A && B && R && tmp) {
        memcpy(A, a, (size_t)n32 * 4);  /* little-endian u32 pairs are u64 limbs */
        memcpy(B, b, (size_t)n32 * 4);
        int depth = 0;
        for (int64_t w = 1; w < nthreads && depth < 5; w *= 3) ++depth;
        st = kara(R, A, B, n, tmp, depth);
        if (!st) memcpy(r, R, (size_t)(2 * n32) * 4);
    }
    free(A); free(B); free(R); free(tmp);
    return st;
}

/* Packs the signed coefficients x (n rows of l limbs, signs xn) into
 * X = sum_i x_i 2^(32 w i) as a sign-magnitude integer of `len` 32-bit
 * limbs (len >= n w + 1, even); returns the sign (1 negative). */
static int pack_signed(uint32_t *X, int64_t len, const uint32_t *x, const uint8_t *xn, int64_t n, int32_t l,
                       int32_t w, uint32_t *scratch) {
    uint32_t *P = X, *N = scratch;
    memset(P, 0, (size_t)len * 4);
    memset(N, 0, (size_t)len * 4);
    for (int64_t i = 0; i < n; ++i)
        memcpy((xn[i] ? N : P) + (size_t)i * w, x + (size_t)i * l, (size_t)l * 4);
    if (cmp_n(P, N, len) >= 0) {
        sub_n(P, P, N, len);
        return 0;
    }
    sub_n(P, N, P, len);
    return 1;
}

/*
 * Full product by Kronecker substitution and Karatsuba.  Same arguments and
 * results as orc_polymul.  Returns 0, -1 (bad arguments), -2 (a
 * coefficient does not fit lc limbs, or the packed product is not
 * consistent), -3 (out of memory).
 */
int orc_polymul_kron(int64_t na, int32_t la, const uint32_t *a, const uint8_t *an,
                     int64_t nb, int32_t lb, const uint32_t *b, const uint8_t *bn,
                     int32_t lc, uint32_t *c, uint8_t *cn, int32_t nthreads) {
    if (na < 1 || nb < 1 || la < 1 || lb < 1 || lc < 1 || !a || !b || !an || !bn || !c || !cn) return -1;
    const int32_t w = lc + 1;                  /* slot: s = 32 w bits */
    if (la > w || lb > w) return -1;
    const int64_t nmax = na > nb ? na : nb, nc = na + nb - 1;
    int64_t len = nmax * w + 2;                /* limbs of each packed operand */
    len += len & 1;
    uint32_t *A = (uint32_t *)malloc((size_t)len * 4), *B = (uint32_t *)malloc((size_t)len * 4);
    uint32_t *S = (uint32_t *)malloc((size_t)len * 4), *R = (uint32_t *)malloc((size_t)(2 * len) * 4);
    int st = -3;
    if (!A || !B || !S || !R) goto done;
    const int sa = pack_signed(A, len, a, an, na, la, w, S);
    const int sbg = pack_signed(B, len, b, bn, nb, lb, w, S);
    st = orc_kara_mul(len, A, B, R, nthreads);
    if (st) goto done;
    const int64_t rlen = 2 * len;
    if (sa ^ sbg) {                            /* two's complement of the product */
        uint64_t cy = 1;
        for (int64_t k = 0; k < rlen; ++k) {
            uint64_t v = (uint64_t)(uint32_t)~R[k] + cy;
            R[k] = (uint32_t)v;
            cy = v >> 32;
        }
    }
    /* read the signed slots back, lowest first */
    uint32_t borrow = 0;
    for (int64_t k = 0; k < nc; ++k) {
        uint32_t *slot = R + (size_t)k * w;
        uint64_t cy = borrow;                  /* t = slot + borrow, in place */
        for (int32_t q = 0; q < w && cy; ++q) {
            uint64_t v = (uint64_t)slot[q] + cy;
            slot[q] = (uint32_t)v;
            cy = v >> 32;
        }
        /* cy = 1 only when slot was all ones and borrow 1: t = 2^s, i.e. 0 with a borrow out */
        const int negative = cy || (slot[w - 1] >> 31);
        borrow = negative ? 1u : 0u;
        uint32_t *out = c + (size_t)k * lc;
        int nz = 0;
        if (negative && !cy) {                 /* |c_k| = 2^s - t */
            uint64_t b2 = 1;
            for (int32_t q = 0; q < w; ++q) {
                uint64_t v = (uint64_t)(uint32_t)~slot[q] + b2;
                slot[q] = (uint32_t)v;
                b2 = v >> 32;
            }
        } else if (cy) {
            memset(slot, 0, (size_t)w * 4);
        }
        if (slot[w - 1] != 0) { st = -2; goto done; }  /* beyond lc limbs */
        for (int32_t q = 0; q < lc; ++q) { out[q] = slot[q]; nz |= slot[q] != 0; }
        cn[k] = (uint8_t)(nz && negative);
    }
    /* the rest of the product must be the sign extension the borrow cancels */
    for (int64_t q = nc * w; q < rlen; ++q)
        if (R[q] != (borrow ? 0xffffffffu : 0u)) { st = -2; goto done; }
    st = 0;
done:
    free(A); free(B); free(S); free(R);
    return st;
}

/*
 * hwc_oracle.c -- plain CPU oracle for point counts of hyperelliptic curves.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker for the
 * GPU library: only the test suite, the smoke check and the timed CPU
 * baseline of the benchmark may build, load or call it.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * What it computes (the plain definition, no Zech logarithms anywhere):
 *   For every polynomial f in a slice of a coefficient family over F_q and
 *   every k = 1..g, the number of points of C_f : y^2 = f(x) over F_{q^k},
 *       #C_f(E) = r^0(f,E) + 2 r^sq(f,E) + (1 + chi_E(f(inf)))      (Sec. 1.1)
 *   with r^0 the number of x in E with f(x) = 0, r^sq the number of x with
 *   f(x) a NONZERO square (Algorithm 1 counts them in an else-branch), and
 *   f(inf) := c_{2g+2} (zero when deg f = 2g+1).  Each f is also tested for
 *   square-freeness (Sec. 1.1: C_f is smooth when f is square-free) by
 *   Euclid's algorithm on gcd(f, f').
 *
 * Field arithmetic is the polynomial-basis representation of Sec. 2.2:
 *   F_q   = F_p[T] / m(T),  m the first monic irreducible of degree e in the
 *           order of the index sum_i m_i p^i (m_choice > 0 takes a later one);
 *   F_Q   = F_q[U] / h(U),  Q = q^k, h the first monic irreducible of degree k
 *           over F_q in the order of sum_i h_i q^i (h_choice likewise).
 * Elements of F_q are the integers c = sum_i b_i p^i <-> sum_i b_i T^i, so 0
 * and 1 are the field's 0 and 1.  Elements of F_Q are integers
 * y = sum_i y_i q^i <-> sum_i y_i U^i with digits y_i in F_q; an element of
 * F_q sits in F_Q as its own integer value (digit 0).
 * The quadratic character of F_Q comes from a bitmap of all squares z^2;
 * orc_chi_euler gives Euler's criterion y^((Q-1)/2) for cross-checking.
 *
 * Families (index -> coefficients c_0..c_d, base-q digits, little endian):
 *   ORC_ALL     : exact degree d, any lead: c_i = digit i of (idx mod q^d),
 *                 c_d = 1 + floor(idx / q^d); (q-1) q^d members.
 *   ORC_MZ      : monic, c_{d-1} = 0, (c_0..c_{d-2}) = digits of idx; q^(d-1).
 *   ORC_MZ_SAMP : sample j of the MZ family: idx = floor(z_j * q^(d-1) / 2^64),
 *                 z_j = SplitMix64 output for state seed + (j+1)*gamma
 *                 (Steele, Lea, Flood, OOPSLA 2014).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXE 16
#define ORC_MAXK 4
#define ORC_MAXD 10
#define ORC_MAXQ (1L << 24)

enum { ORC_ALL = 0, ORC_MZ = 1, ORC_MZ_SAMP = 2 };

typedef struct {
    int p, e, q;
    int m[ORC_MAXE + 1];       /* modulus of F_q over F_p, m[e] = 1 */
    int k;
    long Q;
    int h[ORC_MAXK + 1];       /* modulus of F_Q over F_q (F_q digits), h[k] = 1 */
    int *add, *mul;            /* F_q tables q*q, filled from the definitions */
    int *neg, *inv;            /* F_q tables q */
    signed char *chi;          /* quadratic character of F_Q, length Q */
} orc_field;

/* ------------------------------------------------------------------ */
/* integers                                                            */

static long ipow(long b, int e)
{
    long r = 1;
    while (e-- > 0) r *= b;
    return r;
}

/* q = p^e with p an odd prime; returns 0 on success. */
static int prime_power(int q, int *p, int *e)
{
    if (q < 3 || (q % 2) == 0) return -1;
    int s = 0;
    for (int d = 3; d * d <= q; d += 2)
        if (q % d == 0) { s = d; break; }
    if (s == 0) s = q;
    int x = q, n = 0;
    while (x % s == 0) { x /= s; ++n; }
    if (x != 1) return -1;
    *p = s;
    *e = n;
    return 0;
}

/* ------------------------------------------------------------------ */
/* F_p[T]: remainder and irreducibility by trial division              */

/* a (degree da, not necessarily monic) mod b (monic, degree db) over F_p;
 * the remainder overwrites a[0..db-1].  Returns 1 if the remainder is 0. */
static int fp_rem_is_zero(int *a, int da, const int *b, int db, int p)
{
    for (int t = da; t >= db; --t) {
        int c = a[t] % p;
        if (c == 0) continue;
        for (int i = 0; i <= db; ++i) {
            int v = a[t - db + i] - c * b[i];
            v %= p;
            if (v < 0) v += p;
            a[t - db + i] = v;
        }
    }
    for (int i = 0; i < db; ++i)
        if (a[i] % p) return 0;
    return 1;
}

/* monic a of degree n over F_p is irreducible iff no monic b of degree
 * 1..n/2 divides it. */
static int fp_irreducible(const int *a, int n, int p)
{
    int tmp[2 * ORC_MAXE + 2], b[ORC_MAXE + 1];
    for (int t = 1; 2 * t <= n; ++t) {
        long nb = ipow(p, t);
        for (long idx = 0; idx < nb; ++idx) {
            long r = idx;
            for (int i = 0; i < t; ++i) { b[i] = (int)(r % p); r /= p; }
            b[t] = 1;
            memcpy(tmp, a, sizeof(int) * (n + 1));
            if (fp_rem_is_zero(tmp, n, b, t, p)) return 0;
        }
    }
    return 1;
}

/* ------------------------------------------------------------------ */
/* F_q = F_p[T]/m(T) from the definition (Sec. 2.2)                    */

static int fq_add_def(const orc_field *F, int a, int b)
{
    int r = 0, w = 1;
    for (int i = 0; i < F->e; ++i) {
        int da = a % F->p, db = b % F->p;
        a /= F->p;
        b /= F->p;
        r += ((da + db) % F->p) * w;
        w *= F->p;
    }
    return r;
}

static int fq_mul_def(const orc_field *F, int a, int b)
{
    int p = F->p, e = F->e;
    int da[ORC_MAXE], db[ORC_MAXE], r[2 * ORC_MAXE];
    for (int i = 0; i < e; ++i) { da[i] = a % p; a /= p; db[i] = b % p; b /= p; }
    for (int i = 0; i < 2 * e; ++i) r[i] = 0;
    for (int i = 0; i < e; ++i)
        for (int j = 0; j < e; ++j)
            r[i + j] = (r[i + j] + da[i] * db[j]) % p;
    /* T^e = -(m_0 + ... + m_{e-1} T^{e-1}) */
    for (int t = 2 * e - 2; t >= e; --t) {
        int c = r[t];
        if (!c) continue;
        r[t] = 0;
        for (int i = 0; i < e; ++i) {
            int v = (r[t - e + i] - c * F->m[i]) % p;
            if (v < 0) v += p;
            r[t - e + i] = v;
        }
    }
    int v = 0, w = 1;
    for (int i = 0; i < e; ++i) { v += r[i] * w; w *= p; }
    return v;
}

/* ------------------------------------------------------------------ */
/* F_q[U]: remainder and irreducibility over F_q (tables)              */

static int fqx_rem_is_zero(const orc_field *F, int *a, int da, const int *b, int db)
{
    int q = F->q;
    for (int t = da; t >= db; --t) {
        int c = a[t];
        if (c == 0) continue;
        for (int i = 0; i <= db; ++i) {
            int prod = F->mul[c * q + b[i]];
            a[t - db + i] = F->add[a[t - db + i] * q + F->neg[prod]];
        }
    }
    for (int i = 0; i < db; ++i)
        if (a[i]) return 0;
    return 1;
}

static int fqx_irreducible(const orc_field *F, const int *a, int n)
{
    int tmp[2 * ORC_MAXK + 2], b[ORC_MAXK + 1];
    for (int t = 1; 2 * t <= n; ++t) {
        long nb = ipow(F->q, t);
        for (long idx = 0; idx < nb; ++idx) {
            long r = idx;
            for (int i = 0; i < t; ++i) { b[i] = (int)(r % F->q); r /= F->q; }
            b[t] = 1;
            memcpy(tmp, a, sizeof(int) * (n + 1));
            if (fqx_rem_is_zero(F, tmp, n, b, t)) return 0;
        }
    }
    return 1;
}

/* ------------------------------------------------------------------ */
/* F_Q = F_q[U]/h(U), elements as digit vectors                        */

static void fQ_to_digits(const orc_field *F, long y, int *d)
{
    for (int i = 0; i < F->k; ++i) { d[i] = (int)(y % F->q); y /= F->q; }
}

static long fQ_from_digits(const orc_field *F, const int *d)
{
    long y = 0;
    for (int i = F->k - 1; i >= 0; --i) y = y * F->q + d[i];
    return y;
}

/* out = a * b mod h */
static void fQ_mul_d(const orc_field *F, const int *a, const int *b, int *out)
{
    int q = F->q, k = F->k;
    int r[2 * ORC_MAXK];
    for (int i = 0; i < 2 * k; ++i) r[i] = 0;
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j)
            r[i + j] = F->add[r[i + j] * q + F->mul[a[i] * q + b[j]]];
    /* U^k = -(h_0 + ... + h_{k-1} U^{k-1}) */
    for (int t = 2 * k - 2; t >= k; --t) {
        int c = r[t];
        if (!c) continue;
        r[t] = 0;
        for (int i = 0; i < k; ++i)
            r[t - k + i] = F->add[r[t - k + i] * q + F->neg[F->mul[c * q + F->h[i]]]];
    }
    for (int i = 0; i < k; ++i) out[i] = r[i];
}

/* ------------------------------------------------------------------ */
/* field construction                                                  */

void orc_field_free(void *hdl)
{
    orc_field *F = (orc_field *)hdl;
    if (!F) return;
    free(F->add);
    free(F->mul);
    free(F->neg);
    free(F->inv);
    free(F->chi);
    free(F);
}

void *orc_field_new(int q, int k, int m_choice, int h_choice)
{
    int p, e;
    if (prime_power(q, &p, &e) || e > ORC_MAXE || k < 1 || k > ORC_MAXK) return NULL;
    long Q = ipow(q, k);
    if (Q > ORC_MAXQ) return NULL;
    orc_field *F = (orc_field *)calloc(1, sizeof(orc_field));
    if (!F) return NULL;
    F->p = p; F->e = e; F->q = q; F->k = k; F->Q = Q;

    /* m: the (m_choice)-th monic irreducible of degree e over F_p */
    {
        long n = ipow(p, e), found = -1;
        int cand[ORC_MAXE + 1];
        for (long idx = 0; idx < n; ++idx) {
            long r = idx;
            for (int i = 0; i < e; ++i) { cand[i] = (int)(r % p); r /= p; }
            cand[e] = 1;
            if (fp_irreducible(cand, e, p)) {
                if (++found == m_choice) { memcpy(F->m, cand, sizeof(int) * (e + 1)); break; }
            }
        }
        if (found != m_choice) { orc_field_free(F); return NULL; }
    }

    F->add = (int *)malloc(sizeof(int) * q * q);
    F->mul = (int *)malloc(sizeof(int) * q * q);
    F->neg = (int *)malloc(sizeof(int) * q);
    F->inv = (int *)malloc(sizeof(int) * q);
    F->chi = (signed char *)malloc((size_t)Q);
    if (!F->add || !F->mul || !F->neg || !F->inv || !F->chi) { orc_field_free(F); return NULL; }
    for (int a = 0; a < q; ++a)
        for (int b = 0; b < q; ++b) {
            F->add[a * q + b] = fq_add_def(F, a, b);
            F->mul[a * q + b] = fq_mul_def(F, a, b);
        }
    for (int a = 0; a < q; ++a) {
        F->neg[a] = -1;
        F->inv[a] = -1;
        for (int b = 0; b < q; ++b) {
            if (F->add[a * q + b] == 0) F->neg[a] = b;
            if (F->mul[a * q + b] == 1) F->inv[a] = b;
        }
    }

    /* h: the (h_choice)-th monic irreducible of degree k over F_q */
    {
        long n = ipow(q, k), found = -1;
        int cand[ORC_MAXK + 1];
        for (long idx = 0; idx < n; ++idx) {
            long r = idx;
            for (int i = 0; i < k; ++i) { cand[i] = (int)(r % q); r /= q; }
            cand[k] = 1;
            if (fqx_irreducible(F, cand, k)) {
                if (++found == h_choice) { memcpy(F->h, cand, sizeof(int) * (k + 1)); break; }
            }
        }
        if (found != h_choice) { orc_field_free(F); return NULL; }
    }

    /* quadratic character from the set of squares */
    memset(F->chi, -1, (size_t)Q);
    F->chi[0] = 0;
    {
        int dz[ORC_MAXK], dy[ORC_MAXK];
        for (long z = 1; z < Q; ++z) {
            fQ_to_digits(F, z, dz);
            fQ_mul_d(F, dz, dz, dy);
            F->chi[fQ_from_digits(F, dy)] = 1;
        }
    }
    return F;
}

/* out: p, e, q, k, Q, m_0..m_e, h_0..h_k */
int orc_field_info(void *hdl, int32_t *out)
{
    orc_field *F = (orc_field *)hdl;
    if (!F) return -1;
    int n = 0;
    out[n++] = F->p; out[n++] = F->e; out[n++] = F->q; out[n++] = F->k; out[n++] = (int32_t)F->Q;
    for (int i = 0; i <= F->e; ++i) out[n++] = F->m[i];
    for (int i = 0; i <= F->k; ++i) out[n++] = F->h[i];
    return n;
}

int orc_fq_add(void *hdl, int a, int b) { orc_field *F = (orc_field *)hdl; return F->add[a * F->q + b]; }
int orc_fq_mul(void *hdl, int a, int b) { orc_field *F = (orc_field *)hdl; return F->mul[a * F->q + b]; }

long orc_fQ_add(void *hdl, long y, long z)
{
    orc_field *F = (orc_field *)hdl;
    int dy[ORC_MAXK] = {0}, dz[ORC_MAXK] = {0};
    fQ_to_digits(F, y, dy);
    fQ_to_digits(F, z, dz);
    for (int i = 0; i < F->k; ++i) dy[i] = F->add[dy[i] * F->q + dz[i]];
    return fQ_from_digits(F, dy);
}

long orc_fQ_mul(void *hdl, long y, long z)
{
    orc_field *F = (orc_field *)hdl;
    int dy[ORC_MAXK] = {0}, dz[ORC_MAXK] = {0}, dr[ORC_MAXK];
    fQ_to_digits(F, y, dy);
    fQ_to_digits(F, z, dz);
    fQ_mul_d(F, dy, dz, dr);
    return fQ_from_digits(F, dr);
}

int orc_chi(void *hdl, long y) { orc_field *F = (orc_field *)hdl; return F->chi[y]; }

/* Euler's criterion: y^((Q-1)/2) is 1 for nonzero squares, -1 otherwise. */
int orc_chi_euler(void *hdl, long y)
{
    orc_field *F = (orc_field *)hdl;
    if (y == 0) return 0;
    int base[ORC_MAXK], acc[ORC_MAXK], t[ORC_MAXK];
    fQ_to_digits(F, y, base);
    for (int i = 0; i < F->k; ++i) acc[i] = 0;
    acc[0] = 1;
    long ex = (F->Q - 1) / 2;
    while (ex) {
        if (ex & 1) { fQ_mul_d(F, acc, base, t); memcpy(acc, t, sizeof(int) * F->k); }
        fQ_mul_d(F, base, base, t);
        memcpy(base, t, sizeof(int) * F->k);
        ex >>= 1;
    }
    long v = fQ_from_digits(F, acc);
    if (v == 1) return 1;
    if (v == F->neg[1]) return -1;
    return 99; /* not +-1: the arithmetic is broken */
}

/* f(x) for f = sum c_i X^i (c_i in F_q), x in F_Q, by Horner's rule. */
static long eval_d(const orc_field *F, int d, const int32_t *c, const int *dx)
{
    int acc[ORC_MAXK], t[ORC_MAXK];
    for (int i = 0; i < F->k; ++i) acc[i] = 0;
    acc[0] = c[d];
    for (int i = d - 1; i >= 0; --i) {
        fQ_mul_d(F, acc, dx, t);
        t[0] = F->add[t[0] * F->q + c[i]];
        memcpy(acc, t, sizeof(int) * F->k);
    }
    return fQ_from_digits(F, acc);
}

long orc_eval(void *hdl, int d, const int32_t *c, long x)
{
    orc_field *F = (orc_field *)hdl;
    int dx[ORC_MAXK];
    fQ_to_digits(F, x, dx);
    return eval_d(F, d, c, dx);
}

/* gcd(f, f') over F_q is a nonzero constant  <=>  f square-free. */
int orc_squarefree(void *hdl, int d, const int32_t *c)
{
    orc_field *F = (orc_field *)hdl;
    int q = F->q, p = F->p;
    int a[ORC_MAXD + 1], b[ORC_MAXD + 1];
    int da = d, db = d - 1;
    for (int i = 0; i <= d; ++i) a[i] = c[i];
    /* f' = sum i c_i X^(i-1); the integer i is (i mod p) in F_p, inside F_q */
    for (int i = 1; i <= d; ++i) b[i - 1] = F->mul[(i % p) * q + c[i]];
    while (da >= 0 && a[da] == 0) --da;
    while (db >= 0 && b[db] == 0) --db;
    if (db < 0) return 0;               /* f' = 0: f is a p-th power */
    while (db >= 0) {
        /* a <- a mod b */
        int il = F->inv[b[db]];
        for (int t = da; t >= db; --t) {
            int cf = F->mul[a[t] * q + il];
            if (!cf) continue;
            for (int i = 0; i <= db; ++i)
                a[t - db + i] = F->add[a[t - db + i] * q + F->neg[F->mul[cf * q + b[i]]]];
        }
        da = db - 1;
        while (da >= 0 && a[da] == 0) --da;
        /* swap a, b */
        int tmp[ORC_MAXD + 1];
        memcpy(tmp, a, sizeof(a));
        memcpy(a, b, sizeof(a));
        memcpy(b, tmp, sizeof(a));
        int td = da; da = db; db = td;
    }
    return da == 0;
}

/* ------------------------------------------------------------------ */
/* factorisation pattern lambda(f) (Sec. 1.1, eq. 1.2)                  */
/* by distinct-degree factorisation: for monic square-free f over F_q, */
/* gcd(f, X^(q^m) - X) is the product of the irreducible factors of    */
/* f whose degree divides m; removing them degree by degree leaves the */
/* factors of each exact degree m.                                     */

/* r = a * b mod f over F_q; f monic of degree n, a and b of degree < n */
static void fqx_mulmod(const orc_field *F, const int *a, const int *b, const int *f, int n, int *r)
{
    int q = F->q, t[2 * ORC_MAXD];
    for (int i = 0; i < 2 * n - 1; ++i) t[i] = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            t[i + j] = F->add[t[i + j] * q + F->mul[a[i] * q + b[j]]];
    for (int i = 2 * n - 2; i >= n; --i) {   /* X^i = X^(i-n) * (X^n - f) */
        int c = t[i];
        if (!c) continue;
        t[i] = 0;
        for (int j = 0; j < n; ++j) t[i - n + j] = F->add[t[i - n + j] * q + F->neg[F->mul[c * q + f[j]]]];
    }
    for (int i = 0; i < n; ++i) r[i] = t[i];
}

/* degree of a (array of n+1 coefficients), -1 for the zero polynomial */
static int fqx_deg(const int *a, int n)
{
    while (n >= 0 && a[n] == 0) --n;
    return n;
}

/* g = gcd(a, b) made monic; a and b are overwritten; returns deg g */
static int fqx_gcd(const orc_field *F, int *a, int da, int *b, int db, int *g)
{
    int q = F->q;
    da = fqx_deg(a, da);
    db = fqx_deg(b, db);
    while (db >= 0) {
        int il = F->inv[b[db]];
        for (int t = da; t >= db; --t) {
            int cf = F->mul[a[t] * q + il];
            if (!cf) continue;
            for (int i = 0; i <= db; ++i) a[t - db + i] = F->add[a[t - db + i] * q + F->neg[F->mul[cf * q + b[i]]]];
        }
        da = fqx_deg(a, db - 1);
        int *tp = a; a = b; b = tp;
        int td = da; da = db; db = td;
    }
    if (da < 0) return -1;
    int il = F->inv[a[da]];
    for (int i = 0; i <= da; ++i) g[i] = F->mul[a[i] * q + il];
    return da;
}

/* a <- a / b (exact division by monic b) */
static int fqx_divexact(const orc_field *F, int *a, int da, const int *b, int db, int *quo)
{
    int q = F->q;
    for (int i = 0; i <= da - db; ++i) quo[i] = 0;
    for (int t = da; t >= db; --t) {
        int c = a[t];
        quo[t - db] = c;
        if (!c) continue;
        for (int i = 0; i <= db; ++i) a[t - db + i] = F->add[a[t - db + i] * q + F->neg[F->mul[c * q + b[i]]]];
    }
    return da - db;
}

/* n_by_deg[m] (m = 0..d) = number of irreducible factors of degree m of the
 * square-free f = sum c_i X^i of degree d over F_q (F: any field of this
 * oracle with this q; its F_q tables are used).  Returns 0, -1 if f is not
 * square-free of degree d. */
int orc_factor_degrees(void *hdl, int d, const int32_t *c, int32_t *n_by_deg)
{
    orc_field *F = (orc_field *)hdl;
    int q = F->q;
    if (d < 1 || d > ORC_MAXD || c[d] == 0 || !orc_squarefree(hdl, d, c)) return -1;
    for (int m = 0; m <= d; ++m) n_by_deg[m] = 0;
    int f[ORC_MAXD + 1], rest[ORC_MAXD + 1];
    int il = F->inv[c[d]];
    for (int i = 0; i <= d; ++i) f[i] = F->mul[c[i] * q + il];   /* monic */
    memcpy(rest, f, sizeof(int) * (d + 1));
    int drest = d;
    /* h = X^(q^m) mod f, by q-th powers of the previous h */
    int h[ORC_MAXD], x[ORC_MAXD];
    for (int i = 0; i < d; ++i) h[i] = x[i] = 0;
    if (d == 1) {
        n_by_deg[1] = 1;
        return 0;
    }
    h[1] = x[1] = 1;
    for (int m = 1; 2 * m <= drest; ++m) {
        int base[ORC_MAXD], acc[ORC_MAXD], t[ORC_MAXD];
        memcpy(base, h, sizeof(int) * d);
        for (int i = 0; i < d; ++i) acc[i] = 0;
        acc[0] = 1;
        for (long ex = q; ex; ex >>= 1) {
            if (ex & 1) { fqx_mulmod(F, acc, base, f, d, t); memcpy(acc, t, sizeof(int) * d); }
            fqx_mulmod(F, base, base, f, d, t);
            memcpy(base, t, sizeof(int) * d);
        }
        memcpy(h, acc, sizeof(int) * d);
        /* gcd(rest, h - X) */
        int a[ORC_MAXD + 1], b[ORC_MAXD + 1], g[ORC_MAXD + 1];
        memcpy(a, rest, sizeof(int) * (drest + 1));
        for (int i = 0; i < d; ++i) b[i] = F->add[h[i] * q + F->neg[x[i]]];
        b[d] = 0;
        int dg = fqx_gcd(F, a, drest, b, d - 1, g);
        if (dg >= 1) {
            n_by_deg[m] = dg / m;
            int quo[ORC_MAXD + 1];
            drest = fqx_divexact(F, rest, drest, g, dg, quo);
            memcpy(rest, quo, sizeof(int) * (drest + 1));
        }
    }
    if (drest >= 1) n_by_deg[drest] += 1;   /* what is left is irreducible */
    return 0;
}

/* ------------------------------------------------------------------ */
/* families                                                            */

static uint64_t splitmix64_at(uint64_t seed, uint64_t j)
{
    uint64_t z = seed + (j + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_family_size(int q, int kind, int d, uint64_t sample_count)
{
    if (kind == ORC_ALL) return (uint64_t)(q - 1) * (uint64_t)ipow(q, d);
    if (kind == ORC_MZ) return (uint64_t)ipow(q, d - 1);
    if (kind == ORC_MZ_SAMP) return sample_count;
    return 0;
}

/* Coefficients c_0..c_d of member idx (or sample idx) of the family. */
int orc_decode(int q, int kind, int d, uint64_t seed, uint64_t idx, int32_t *c)
{
    if (kind == ORC_MZ_SAMP) {
        unsigned __int128 z = splitmix64_at(seed, idx);
        idx = (uint64_t)((z * (unsigned __int128)ipow(q, d - 1)) >> 64);
        kind = ORC_MZ;
    }
    if (kind == ORC_ALL) {
        uint64_t r = idx;
        for (int i = 0; i < d; ++i) { c[i] = (int32_t)(r % (uint64_t)q); r /= (uint64_t)q; }
        c[d] = (int32_t)(1 + r);
        return 0;
    }
    if (kind == ORC_MZ) {
        uint64_t r = idx;
        for (int i = 0; i <= d - 2; ++i) { c[i] = (int32_t)(r % (uint64_t)q); r /= (uint64_t)q; }
        c[d - 1] = 0;
        c[d] = 1;
        return 0;
    }
    return -1;
}

/* ------------------------------------------------------------------ */
/* the count                                                           */

/* counts[i*g + k-1] = #C_f(F_{q^k}) for member first+i; sqf[i] = square-free.
 * filter != 0: non-square-free members get counts 0 and are not evaluated.
 * Returns 0, or -1 (bad argument), -2 (range), -3 (field too large / alloc). */
int orc_count_polys(int g, int q, int kind, int d, uint64_t seed, uint64_t sample_count,
                    uint64_t first, uint64_t count, int filter, int m_choice, int h_choice,
                    int nthreads, int32_t *counts, uint8_t *sqf)
{
    int p, e;
    if (g < 1 || g > ORC_MAXK || prime_power(q, &p, &e)) return -1;
    if (d != 2 * g + 1 && d != 2 * g + 2) return -1;
    if (kind < ORC_ALL || kind > ORC_MZ_SAMP) return -1;
    uint64_t n = orc_family_size(q, kind, d, sample_count);
    if (first > n || count > n - first) return -2;
    orc_field *F[ORC_MAXK + 1];
    for (int k = 1; k <= g; ++k) {
        F[k] = (orc_field *)orc_field_new(q, k, m_choice, h_choice);
        if (!F[k]) {
            for (int j = 1; j < k; ++j) orc_field_free(F[j]);
            return -3;
        }
    }
    if (nthreads <= 0) nthreads = 1;

#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (long i = 0; i < (long)count; ++i) {
        int32_t c[ORC_MAXD + 1];
        orc_decode(q, kind, d, seed, first + (uint64_t)i, c);
        int s = orc_squarefree(F[1], d, c);
        sqf[i] = (uint8_t)s;
        for (int k = 1; k <= g; ++k) {
            if (filter && !s) { counts[i * g + (k - 1)] = 0; continue; }
            const orc_field *Fk = F[k];
            long r0 = 0, rsq = 0;
            int dx[ORC_MAXK];
            for (long x = 0; x < Fk->Q; ++x) {
                fQ_to_digits(Fk, x, dx);
                long y = eval_d(Fk, d, c, dx);
                if (y == 0) ++r0;
                else if (Fk->chi[y] == 1) ++rsq;
            }
            /* f(inf) := c_{2g+2}, an element of F_q inside F_Q */
            int finf = (d == 2 * g + 2) ? c[d] : 0;
            long pts = r0 + 2 * rsq + (1 + Fk->chi[finf]);
            counts[i * g + (k - 1)] = (int32_t)pts;
        }
    }
    for (int k = 1; k <= g; ++k) orc_field_free(F[k]);
    return 0;
}

/* Point counts of an explicit list of polynomials: coeffs[i*(d+1) + n] = c_n
 * of polynomial i (F_q digits, c_d != 0); counts[i*g + k-1] = #C(F_{q^k}),
 * sqf[i] = square-free, codes[i] = lambda code (as orc_lambda_codes; 0 if
 * not square-free).  Non-square-free entries get counts 0, unless nthreads is
 * negative (then every entry is counted, with -nthreads threads).  Returns 0,
 * -1 (bad argument), -3 (field). */
int orc_count_list(int g, int q, int d, uint64_t n, const int32_t *coeffs, int nthreads, int32_t *counts,
                   uint8_t *sqf, uint64_t *codes)
{
    int p, e;
    if (g < 1 || g > ORC_MAXK || prime_power(q, &p, &e) || d < 1 || d > ORC_MAXD) return -1;
    orc_field *F[ORC_MAXK + 1];
    for (int k = 1; k <= g; ++k) {
        F[k] = (orc_field *)orc_field_new(q, k, 0, 0);
        if (!F[k]) {
            for (int j = 1; j < k; ++j) orc_field_free(F[j]);
            return -3;
        }
    }
    const int all = nthreads < 0;
    if (nthreads < 0) nthreads = -nthreads;
    if (nthreads == 0) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (long i = 0; i < (long)n; ++i) {
        const int32_t *c = coeffs + i * (d + 1);
        int32_t nd[ORC_MAXD + 1];
        int s = c[d] != 0 && orc_squarefree(F[1], d, c);
        sqf[i] = (uint8_t)s;
        uint64_t code = 0;
        if (s && orc_factor_degrees(F[1], d, c, nd) == 0) {
            if (d == 2 * g + 1) nd[1] += 1;
            for (int m = 1; m <= d; ++m) code += (uint64_t)nd[m] << (4 * (m - 1));
        }
        codes[i] = code;
        for (int k = 1; k <= g; ++k) {
            if (!s && !all) { counts[i * g + (k - 1)] = 0; continue; }
            const orc_field *Fk = F[k];
            long r0 = 0, rsq = 0;
            int dx[ORC_MAXK];
            for (long x = 0; x < Fk->Q; ++x) {
                fQ_to_digits(Fk, x, dx);
                long y = eval_d(Fk, d, c, dx);
                if (y == 0) ++r0;
                else if (Fk->chi[y] == 1) ++rsq;
            }
            /* points at infinity: one for odd degree, 1 + chi(c_d) for even degree */
            int finf = (d % 2 == 0) ? c[d] : 0;
            counts[i * g + (k - 1)] = (int32_t)(r0 + 2 * rsq + (1 + Fk->chi[finf]));
        }
    }
    for (int k = 1; k <= g; ++k) orc_field_free(F[k]);
    return 0;
}

/* lambda(f) of eq. 1.2 for members [first, first+count): the partition of
 * 2g+2 given by the degrees of the irreducible factors of f, with one more
 * part 1 when deg f = 2g+1; coded as sum_m n_m 16^(m-1), n_m the number of
 * parts equal to m.  0 for members that are not square-free.  Returns 0, or
 * -1 / -2 / -3 as orc_count_polys. */
int orc_lambda_codes(int g, int q, int kind, int d, uint64_t seed, uint64_t sample_count, uint64_t first,
                     uint64_t count, int nthreads, uint64_t *codes)
{
    int p, e;
    if (g < 1 || g > ORC_MAXK || prime_power(q, &p, &e)) return -1;
    if (d != 2 * g + 1 && d != 2 * g + 2) return -1;
    uint64_t n = orc_family_size(q, kind, d, sample_count);
    if (first > n || count > n - first) return -2;
    orc_field *F = (orc_field *)orc_field_new(q, 1, 0, 0);
    if (!F) return -3;
    if (nthreads <= 0) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
    for (long i = 0; i < (long)count; ++i) {
        int32_t c[ORC_MAXD + 1], nd[ORC_MAXD + 1];
        orc_decode(q, kind, d, seed, first + (uint64_t)i, c);
        uint64_t code = 0;
        if (orc_factor_degrees(F, d, c, nd) == 0) {
            if (d == 2 * g + 1) nd[1] += 1;   /* the extra part 1 of odd degree */
            for (int m = 1; m <= d; ++m) code += (uint64_t)nd[m] << (4 * (m - 1));
        }
        codes[i] = code;
    }
    orc_field_free(F);
    return 0;
}

/* ------------------------------------------------------------------ */
/* the histogram                                                       */

/* lexicographic order of #C tuples; the tuple width is set per call */
static int g_cmp_width;

static int cmp_tuple(const void *a, const void *b)
{
    const int32_t *x = (const int32_t *)a, *y = (const int32_t *)b;
    for (int k = 0; k < g_cmp_width; ++k)
        if (x[k] != y[k]) return x[k] < y[k] ? -1 : 1;
    return 0;
}

/* hwc_cpu_count: the histogram of (#C(F_q), ..., #C(F_{q^g})) over the
 * square-free members [first, first+count) of a family, computed by this
 * oracle (the same job arguments as the GPU library's hwc_count, the family
 * given as kind, degree, seed, sample_count; no stream).  Algorithm 1's
 * histogram with weight 1 per member.
 *   counts[max_entries * g]: distinct tuples, sorted lexicographically;
 *   mult[max_entries]: their multiplicities;
 *   *n_entries: number of distinct tuples; *n_squarefree: square-free members.
 * Members are counted in slices of at most 2^20 (bounded memory); slice
 * histograms are merged.  Returns 0; -1 bad argument, -2 range, -3 field or
 * allocation failure, -4 more than max_entries tuples (*n_entries then holds
 * the number needed).  Not thread-safe (one call at a time). */
int hwc_cpu_count(uint32_t g, uint32_t q, uint32_t kind, uint32_t degree, uint64_t seed,
                  uint64_t sample_count, uint64_t first, uint64_t count, int nthreads,
                  uint64_t max_entries, int32_t *counts, uint64_t *mult, uint64_t *n_entries,
                  uint64_t *n_squarefree)
{
    if (!n_entries || !n_squarefree || (max_entries && (!counts || !mult))) return -1;
    if (g < 1 || g > ORC_MAXK) return -1;
    const uint64_t slice = 1u << 20;
    const int G = (int)g;
    int32_t *pc = NULL, *tup = NULL, *acc = NULL, *nxt = NULL;
    uint8_t *ps = NULL;
    uint64_t *accm = NULL, *nxtm = NULL, *tm = NULL;
    uint64_t nacc = 0, nsq = 0;
    int rc = 0;
    const uint64_t cap = count < slice ? (count ? count : 1) : slice;
    pc = (int32_t *)malloc(sizeof(int32_t) * cap * G);
    tup = (int32_t *)malloc(sizeof(int32_t) * cap * G);
    tm = (uint64_t *)malloc(sizeof(uint64_t) * cap);
    ps = (uint8_t *)malloc(cap);
    if (!pc || !tup || !tm || !ps) { rc = -3; goto out; }
    for (uint64_t s0 = 0; s0 < count || (count == 0 && s0 == 0); s0 += slice) {
        const uint64_t n = count - s0 < slice ? count - s0 : slice;
        rc = orc_count_polys(G, (int)q, (int)kind, (int)degree, seed, sample_count, first + s0, n, 1, 0, 0,
                             nthreads, pc, ps);
        if (rc) goto out;
        if (count == 0) break;
        /* this slice's square-free tuples, sorted and run-length encoded */
        uint64_t m = 0;
        for (uint64_t i = 0; i < n; ++i)
            if (ps[i]) { memcpy(tup + m * G, pc + i * G, sizeof(int32_t) * G); ++m; }
        nsq += m;
        g_cmp_width = G;
        qsort(tup, m, sizeof(int32_t) * G, cmp_tuple);
        uint64_t u = 0;
        for (uint64_t i = 0; i < m; ++i) {
            if (u && cmp_tuple(tup + (u - 1) * G, tup + i * G) == 0) { ++tm[u - 1]; continue; }
            memmove(tup + u * G, tup + i * G, sizeof(int32_t) * G);
            tm[u++] = 1;
        }
        /* merge with the running histogram */
        nxt = (int32_t *)malloc(sizeof(int32_t) * (nacc + u) * G + 1);
        nxtm = (uint64_t *)malloc(sizeof(uint64_t) * (nacc + u) + 1);
        if (!nxt || !nxtm) { rc = -3; goto out; }
        uint64_t a = 0, b = 0, o = 0;
        while (a < nacc || b < u) {
            int c = a == nacc ? 1 : (b == u ? -1 : cmp_tuple(acc + a * G, tup + b * G));
            if (c <= 0) {
                memcpy(nxt + o * G, acc + a * G, sizeof(int32_t) * G);
                nxtm[o] = accm[a] + (c == 0 ? tm[b] : 0);
                ++a;
                if (c == 0) ++b;
            } else {
                memcpy(nxt + o * G, tup + b * G, sizeof(int32_t) * G);
                nxtm[o] = tm[b];
                ++b;
            }
            ++o;
        }
        free(acc);
        free(accm);
        acc = nxt;
        accm = nxtm;
        nxt = NULL;
        nxtm = NULL;
        nacc = o;
    }
    *n_entries = nacc;
    *n_squarefree = nsq;
    if (nacc > max_entries) { rc = -4; goto out; }
    if (nacc) {
        memcpy(counts, acc, sizeof(int32_t) * nacc * G);
        memcpy(mult, accm, sizeof(uint64_t) * nacc);
    }
out:
    free(pc);
    free(tup);
    free(tm);
    free(ps);
    free(acc);
    free(accm);
    free(nxt);
    free(nxtm);
    return rc;
}

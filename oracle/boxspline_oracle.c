/*
 * boxspline_oracle.c -- plain, slow FP64 CPU oracle for the lattice convolution sum
 *
 *     f(x) = sum_k sum_i c_k[i] * phi(x - (D*i + l_k)),   phi(x) = |det L| * M_Xi(x + sum(Xi)/2)
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call this file:
 * only tests/, __graft_entry__.smoke() and the cpu_baseline / reference leg of bench.py use it.
 * It shares no code with the CUDA path (no headers, no tables, no helpers).
 *
 * What it follows (Horacsek & Alim, arXiv 2102.08514):
 *   - Sec. 3, the convolution-sum space V(phi, L, h) with h = 1 (Eq. 1) and the box spline M_Xi:
 *     base case 1/|det Xi| on Xi[0,1)^s, support = zonotope sum a_k xi_k (Sec. 3).
 *   - Sec. 4.1, the Cartesian coset split of the sum (Eq. "coset form"): L Z^s = U_k (D Z^s + l_k).
 *   - M_Xi is evaluated with de Boor's recurrence
 *         (n - s) M_Xi(x) = sum_xi [ t_xi M_{Xi\xi}(x) + (1 - t_xi) M_{Xi\xi}(x - xi) ],  Xi t = x,
 *     which is the textbook form of the paper's recursive integral (Sec. 3); sub-matrices that do
 *     not span R^s are singular measures and contribute 0.
 *   - Sec. 2 notes that this recurrence is unstable unless every decision on the separating planes
 *     is taken consistently.  Here every point is carried EXACTLY as an integer numerator over 2^64
 *     (query points are FP32/FP64 dyadic rationals, Xi is integer), and every base-case decision
 *     "Xi_B^{-1} x in [0,1)^s" is taken exactly, as the one-sided limit x + eps*v, eps -> 0+, for a
 *     fixed generic direction v.  Every config spline is continuous (order >= 2), so this gives
 *     the value of M_Xi itself at every x; only the weights t and the sums are FP64.
 *
 * Derivatives: D_xi M_Xi = M_{Xi\xi} - M_{Xi\xi}(. - xi) (closed form), the gradient solved from s
 * independent non-bridge directions.  Adjoint: dL/dc_n = sum_q g_q phi(x_q - n) by brute force.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXS 4
#define ORC_MAXN 12
#define ORC_F 64 /* fixed-point fraction bits of every exact coordinate */

typedef __int128 i128;

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_EINEXACT = 2, ORC_ENOMEM = 3 };

typedef struct {
    int s, n;
    int xi[ORC_MAXN][ORC_MAXS]; /* column j is xi[j][0..s-1] */
    double scale;               /* |det L|: makes phi a partition of unity on L Z^s */
    int tmode;                  /* 0: t = pseudo-inverse solution, 1: t supported on a basis */
    int nmask;
    int8_t *spans;              /* [mask] 1 if the columns in mask span R^s */
    double *tmat;               /* [mask][j][a]: t_j = sum_a tmat * x_a, for |mask| > s */
    int *det;                   /* [mask] det of the s columns, for |mask| == s */
    int *adj;                   /* [mask][a][b] adjugate, for |mask| == s */
    int64_t *bblo, *bbhi;       /* [mask][a] closed bounding box of the zonotope of mask */
    int64_t pow3[ORC_MAXN + 1];
    i128 vdir[ORC_MAXS];        /* generic perturbation direction for boundary decisions */
} orc_spline;

typedef struct {
    double *val;
    uint32_t *stamp;
    uint32_t gen;
    int64_t size;
} orc_memo;

/* ---------------------------------------------------------------- small exact linear algebra */

static int64_t idet(const int64_t *a, int m) /* Laplace expansion, m <= 4 */
{
    if (m == 1) return a[0];
    int64_t sum = 0;
    int64_t sub[16];
    for (int c = 0; c < m; ++c) {
        int k = 0;
        for (int r = 1; r < m; ++r)
            for (int cc = 0; cc < m; ++cc)
                if (cc != c) sub[k++] = a[r * m + cc];
        int64_t d = idet(sub, m - 1);
        sum += ((c & 1) ? -1 : 1) * a[c] * d;
    }
    return sum;
}

/* rows of B are the coordinates a, columns are the chosen directions: B[a][c] = xi[col_c][a] */
static void iadj(const int64_t *B, int m, int64_t *adj)
{
    /* adj[c][a] = (-1)^(a+c) * minor(a, c)  so that adj * B = det * I */
    int64_t sub[16];
    for (int a = 0; a < m; ++a)
        for (int c = 0; c < m; ++c) {
            if (m == 1) { adj[0] = 1; return; }
            int k = 0;
            for (int r = 0; r < m; ++r) {
                if (r == a) continue;
                for (int cc = 0; cc < m; ++cc)
                    if (cc != c) sub[k++] = B[r * m + cc];
            }
            adj[c * m + a] = (((a + c) & 1) ? -1 : 1) * idet(sub, m - 1);
        }
}

static int rank_of(const orc_spline *sp, unsigned mask) /* exact rank via fraction-free elimination */
{
    int s = sp->s;
    int64_t m[ORC_MAXN][ORC_MAXS];
    int rows = 0;
    for (int j = 0; j < sp->n; ++j)
        if (mask >> j & 1u) {
            for (int a = 0; a < s; ++a) m[rows][a] = sp->xi[j][a];
            ++rows;
        }
    int rank = 0;
    for (int col = 0; col < s && rank < rows; ++col) {
        int piv = -1;
        for (int r = rank; r < rows; ++r)
            if (m[r][col] != 0) { piv = r; break; }
        if (piv < 0) continue;
        for (int a = 0; a < s; ++a) { int64_t t = m[rank][a]; m[rank][a] = m[piv][a]; m[piv][a] = t; }
        for (int r = 0; r < rows; ++r) {
            if (r == rank || m[r][col] == 0) continue;
            int64_t f1 = m[rank][col], f2 = m[r][col];
            for (int a = 0; a < s; ++a) m[r][a] = m[r][a] * f1 - m[rank][a] * f2;
            /* keep entries small */
            int64_t g = 0;
            for (int a = 0; a < s; ++a) { int64_t v = llabs(m[r][a]); while (v) { int64_t t = g % v; g = v; v = t; } }
            if (g > 1) for (int a = 0; a < s; ++a) m[r][a] /= g;
        }
        ++rank;
    }
    return rank;
}

static int solve_fp64(double *A, double *b, int m) /* Gauss-Jordan with partial pivoting, A m x m */
{
    for (int c = 0; c < m; ++c) {
        int p = c;
        for (int r = c + 1; r < m; ++r) if (fabs(A[r * m + c]) > fabs(A[p * m + c])) p = r;
        if (A[p * m + c] == 0.0) return -1;
        if (p != c) {
            for (int k = 0; k < m; ++k) { double t = A[c * m + k]; A[c * m + k] = A[p * m + k]; A[p * m + k] = t; }
            double t = b[c]; b[c] = b[p]; b[p] = t;
        }
        for (int r = 0; r < m; ++r) {
            if (r == c) continue;
            double f = A[r * m + c] / A[c * m + c];
            for (int k = 0; k < m; ++k) A[r * m + k] -= f * A[c * m + k];
            b[r] -= f * b[c];
        }
    }
    for (int c = 0; c < m; ++c) b[c] /= A[c * m + c];
    return 0;
}

/* ---------------------------------------------------------------- exact coordinates */

/* x (double) -> x * 2^64 as an exact 128-bit integer; fails if x is not a multiple of 2^-64
 * or |x| >= 2^40 */
static int to_fixed(double x, i128 *out)
{
    if (x == 0.0) { *out = 0; return 0; }
    if (!isfinite(x) || fabs(x) >= 1099511627776.0) return ORC_EINEXACT;
    int e;
    double m = frexp(x, &e);                /* x = m * 2^e, 0.5 <= |m| < 1 */
    int64_t mant = (int64_t)ldexp(m, 53);   /* exact */
    int sh = e - 53 + ORC_F;
    if (sh >= 0) {
        *out = ((i128)mant) << sh;
    } else {
        int r = -sh;
        if (r >= 63) return ORC_EINEXACT;
        if (mant & ((((int64_t)1) << r) - 1)) return ORC_EINEXACT;
        *out = (i128)(mant >> r);
    }
    return 0;
}

static double fixed_to_double(i128 v) { return ldexp((double)v, -ORC_F); }

/* ---------------------------------------------------------------- spline set-up */

int orc_create(int s, int n, const int *xi_cols, double scale, int tmode, void **out)
{
    if (s < 1 || s > ORC_MAXS || n < s || n > ORC_MAXN || !out) return ORC_EINVAL;
    orc_spline *sp = (orc_spline *)calloc(1, sizeof(orc_spline));
    if (!sp) return ORC_ENOMEM;
    sp->s = s; sp->n = n; sp->scale = scale; sp->tmode = tmode;
    for (int j = 0; j < n; ++j)
        for (int a = 0; a < s; ++a) sp->xi[j][a] = xi_cols[j * s + a];
    sp->nmask = 1 << n;
    sp->pow3[0] = 1;
    for (int j = 1; j <= n; ++j) sp->pow3[j] = sp->pow3[j - 1] * 3;
    /* v = (K^(s-1), ..., K, 1): a dot product with any integer row of entries below K/2 in
     * magnitude is nonzero unless the row is zero, so no exact tie survives the perturbation. */
    {
        i128 K = 1 << 12, p = 1;
        for (int a = s - 1; a >= 0; --a) { sp->vdir[a] = p; p *= K; }
    }
    int nm = sp->nmask;
    sp->spans = (int8_t *)calloc(nm, 1);
    sp->tmat = (double *)calloc((size_t)nm * ORC_MAXN * ORC_MAXS, sizeof(double));
    sp->det = (int *)calloc(nm, sizeof(int));
    sp->adj = (int *)calloc((size_t)nm * ORC_MAXS * ORC_MAXS, sizeof(int));
    sp->bblo = (int64_t *)calloc((size_t)nm * ORC_MAXS, sizeof(int64_t));
    sp->bbhi = (int64_t *)calloc((size_t)nm * ORC_MAXS, sizeof(int64_t));
    if (!sp->spans || !sp->tmat || !sp->det || !sp->adj || !sp->bblo || !sp->bbhi) return ORC_ENOMEM;

    for (unsigned mask = 0; mask < (unsigned)nm; ++mask) {
        int cnt = __builtin_popcount(mask);
        for (int a = 0; a < s; ++a) {
            int64_t lo = 0, hi = 0;
            for (int j = 0; j < n; ++j)
                if (mask >> j & 1u) {
                    if (sp->xi[j][a] < 0) lo += sp->xi[j][a]; else hi += sp->xi[j][a];
                }
            sp->bblo[mask * ORC_MAXS + a] = lo;
            sp->bbhi[mask * ORC_MAXS + a] = hi;
        }
        if (cnt < s) continue;
        sp->spans[mask] = (int8_t)(rank_of(sp, mask) == s);
        if (!sp->spans[mask]) continue;
        if (cnt == s) {
            int64_t B[16], A[16];
            int c = 0;
            for (int j = 0; j < n; ++j)
                if (mask >> j & 1u) { for (int a = 0; a < s; ++a) B[a * s + c] = sp->xi[j][a]; ++c; }
            sp->det[mask] = (int)idet(B, s);
            iadj(B, s, A);
            for (int k = 0; k < s * s; ++k) sp->adj[mask * ORC_MAXS * ORC_MAXS + k] = (int)A[k];
            continue;
        }
        double *T = sp->tmat + (size_t)mask * ORC_MAXN * ORC_MAXS;
        if (tmode == 0) {
            /* t = Xi'^T (Xi' Xi'^T)^{-1} x : the minimum-norm solution of Xi' t = x */
            double G[16];
            for (int a = 0; a < s; ++a)
                for (int b = 0; b < s; ++b) {
                    double acc = 0;
                    for (int j = 0; j < n; ++j) if (mask >> j & 1u) acc += (double)sp->xi[j][a] * sp->xi[j][b];
                    G[a * s + b] = acc;
                }
            /* invert G column by column */
            double Ginv[16];
            for (int b = 0; b < s; ++b) {
                double Gc[16], e[4] = {0, 0, 0, 0};
                memcpy(Gc, G, sizeof(double) * s * s);
                e[b] = 1.0;
                if (solve_fp64(Gc, e, s)) return ORC_EINVAL;
                for (int a = 0; a < s; ++a) Ginv[a * s + b] = e[a];
            }
            for (int j = 0; j < n; ++j) {
                if (!(mask >> j & 1u)) continue;
                for (int a = 0; a < s; ++a) {
                    double acc = 0;
                    for (int b = 0; b < s; ++b) acc += sp->xi[j][b] * Ginv[b * s + a];
                    T[j * ORC_MAXS + a] = acc;
                }
            }
        } else {
            /* t supported on the first basis (in column order) found inside mask: t_B = B^{-1} x */
            int cols[ORC_MAXS];
            int found = 0;
            unsigned sub;
            for (sub = mask; sub; sub = (sub - 1) & mask) {
                if (__builtin_popcount(sub) != s) continue;
                if (rank_of(sp, sub) == s) { found = 1; break; }
            }
            if (!found) return ORC_EINVAL;
            int c = 0;
            int64_t B[16], A[16];
            for (int j = 0; j < n; ++j)
                if (sub >> j & 1u) { cols[c] = j; for (int a = 0; a < s; ++a) B[a * s + c] = sp->xi[j][a]; ++c; }
            double d = (double)idet(B, s);
            iadj(B, s, A);
            for (int k = 0; k < s; ++k)
                for (int a = 0; a < s; ++a) T[cols[k] * ORC_MAXS + a] = (double)A[k * s + a] / d;
        }
    }
    *out = sp;
    return ORC_OK;
}

void orc_destroy(void *h)
{
    orc_spline *sp = (orc_spline *)h;
    if (!sp) return;
    free(sp->spans); free(sp->tmat); free(sp->det); free(sp->adj); free(sp->bblo); free(sp->bbhi);
    free(sp);
}

static int memo_init(orc_memo *mm, const orc_spline *sp)
{
    mm->size = sp->pow3[sp->n];
    mm->val = (double *)malloc(sizeof(double) * mm->size);
    mm->stamp = (uint32_t *)calloc(mm->size, sizeof(uint32_t));
    mm->gen = 0;
    return (mm->val && mm->stamp) ? 0 : ORC_ENOMEM;
}

static void memo_free(orc_memo *mm) { free(mm->val); free(mm->stamp); }

static void memo_next(orc_memo *mm)
{
    if (++mm->gen == 0) { memset(mm->stamp, 0, sizeof(uint32_t) * mm->size); mm->gen = 1; }
}

/* ---------------------------------------------------------------- the box spline */

/* Base case (Sec. 3): M_B(x) = 1/|det B| if B^{-1} x in [0,1)^s, decided exactly as the limit of
 * x + eps*v. */
static double base_case(const orc_spline *sp, unsigned mask, const i128 *X)
{
    int s = sp->s;
    int d = sp->det[mask];
    const int *A = sp->adj + (size_t)mask * ORC_MAXS * ORC_MAXS;
    int sg = d > 0 ? 1 : -1;
    i128 upper = (i128)(d * sg) << ORC_F;
    for (int c = 0; c < s; ++c) {
        i128 a = 0, b = 0;
        for (int k = 0; k < s; ++k) { a += (i128)A[c * s + k] * X[k]; b += (i128)A[c * s + k] * sp->vdir[k]; }
        a *= sg; b *= sg;
        int ge0 = (a > 0) || (a == 0 && b > 0);
        int lt1 = (a < upper) || (a == upper && b < 0);
        if (!(ge0 && lt1)) return 0.0;
    }
    return 1.0 / (double)(d * sg);
}

/* M_{Xi_mask}(X) with X = x * 2^64 exact; key identifies (removed columns, shifted columns)
 * relative to the evaluation's start, so equal keys mean equal points. */
static double M_rec(const orc_spline *sp, orc_memo *mm, unsigned mask, int64_t key, const i128 *X)
{
    int s = sp->s;
    for (int a = 0; a < s; ++a) {
        if (X[a] < ((i128)sp->bblo[mask * ORC_MAXS + a] << ORC_F)) return 0.0;
        if (X[a] > ((i128)sp->bbhi[mask * ORC_MAXS + a] << ORC_F)) return 0.0;
    }
    if (!sp->spans[mask]) return 0.0;
    int cnt = __builtin_popcount(mask);
    if (cnt == s) return base_case(sp, mask, X);
    if (mm->stamp[key] == mm->gen) return mm->val[key];

    double x[ORC_MAXS];
    for (int a = 0; a < s; ++a) x[a] = fixed_to_double(X[a]);
    const double *T = sp->tmat + (size_t)mask * ORC_MAXN * ORC_MAXS;
    double acc = 0.0;
    for (int j = 0; j < sp->n; ++j) {
        if (!(mask >> j & 1u)) continue;
        unsigned sub = mask & ~(1u << j);
        if (!sp->spans[sub]) continue; /* singular measure: 0 off a plane */
        double t = 0.0;
        for (int a = 0; a < s; ++a) t += T[j * ORC_MAXS + a] * x[a];
        i128 X1[ORC_MAXS];
        for (int a = 0; a < s; ++a) X1[a] = X[a] - ((i128)sp->xi[j][a] << ORC_F);
        double m0 = (t != 0.0) ? M_rec(sp, mm, sub, key + sp->pow3[j], X) : 0.0;
        double m1 = (t != 1.0) ? M_rec(sp, mm, sub, key + 2 * sp->pow3[j], X1) : 0.0;
        acc += t * m0 + (1.0 - t) * m1;
    }
    double v = acc / (double)(cnt - s);
    mm->val[key] = v;
    mm->stamp[key] = mm->gen;
    return v;
}

static double M_eval(const orc_spline *sp, orc_memo *mm, unsigned mask, const i128 *X)
{
    memo_next(mm);
    return M_rec(sp, mm, mask, 0, X);
}

/* D_xi_j M_mask(X) = M_{mask\j}(X) - M_{mask\j}(X - xi_j)  (closed form of the directional derivative) */
static double dir_deriv(const orc_spline *sp, orc_memo *mm, unsigned mask, int j, const i128 *X)
{
    unsigned sub = mask & ~(1u << j);
    i128 X1[ORC_MAXS];
    for (int a = 0; a < sp->s; ++a) X1[a] = X[a] - ((i128)sp->xi[j][a] << ORC_F);
    return M_eval(sp, mm, sub, X) - M_eval(sp, mm, sub, X1);
}

/* gradient of M_mask at X from s independent non-bridge directions */
static int grad_M(const orc_spline *sp, orc_memo *mm, unsigned mask, const i128 *X, double *g)
{
    int s = sp->s;
    int cols[ORC_MAXS], c = 0;
    /* greedily collect independent columns whose removal keeps the rest spanning */
    for (int j = 0; j < sp->n && c < s; ++j) {
        if (!(mask >> j & 1u)) continue;
        if (!sp->spans[mask & ~(1u << j)]) continue;
        unsigned trial = 0;
        for (int k = 0; k < c; ++k) trial |= 1u << cols[k];
        trial |= 1u << j;
        if (rank_of(sp, trial) == c + 1) cols[c++] = j;
    }
    if (c < s) return ORC_EINVAL;
    double A[16], b[4];
    for (int k = 0; k < s; ++k) {
        for (int a = 0; a < s; ++a) A[k * s + a] = sp->xi[cols[k]][a];
        b[k] = dir_deriv(sp, mm, mask, cols[k], X);
    }
    if (solve_fp64(A, b, s)) return ORC_EINVAL;
    for (int a = 0; a < s; ++a) g[a] = b[a];
    return ORC_OK;
}

/* ---------------------------------------------------------------- exported point-wise functions */

static unsigned full_mask(const orc_spline *sp) { return (sp->n == 32) ? 0xffffffffu : ((1u << sp->n) - 1u); }

/* raw (uncentred, unscaled) M_{Xi_mask}(w) at npts points w (npts x s, row-major) */
int orc_M(void *h, unsigned mask, int64_t npts, const double *w, double *out)
{
    orc_spline *sp = (orc_spline *)h;
    int err = 0;
#pragma omp parallel
    {
        orc_memo mm;
        int lerr = memo_init(&mm, sp);
#pragma omp for schedule(dynamic, 16)
        for (int64_t q = 0; q < npts; ++q) {
            if (lerr) continue;
            i128 X[ORC_MAXS];
            int bad = 0;
            for (int a = 0; a < sp->s; ++a) bad |= to_fixed(w[q * sp->s + a], &X[a]);
            if (bad) { out[q] = NAN; lerr = ORC_EINEXACT; continue; }
            out[q] = M_eval(sp, &mm, mask, X);
        }
        memo_free(&mm);
#pragma omp critical
        if (lerr) err = lerr;
    }
    return err;
}

/* phi(z) = |det L| M_Xi(z + sum(Xi)/2) and optionally its gradient */
static int phi_fixed(const orc_spline *sp, orc_memo *mm, const i128 *Z, double *val, double *grad)
{
    i128 W[ORC_MAXS];
    for (int a = 0; a < sp->s; ++a) {
        i128 c2 = 0;
        for (int j = 0; j < sp->n; ++j) c2 += sp->xi[j][a];
        W[a] = Z[a] + (c2 << (ORC_F - 1));
    }
    unsigned full = full_mask(sp);
    *val = sp->scale * M_eval(sp, mm, full, W);
    if (grad) {
        int e = grad_M(sp, mm, full, W, grad);
        if (e) return e;
        for (int a = 0; a < sp->s; ++a) grad[a] *= sp->scale;
    }
    return ORC_OK;
}

int orc_phi(void *h, int64_t npts, const double *z, double *out, double *grad)
{
    orc_spline *sp = (orc_spline *)h;
    int err = 0;
#pragma omp parallel
    {
        orc_memo mm;
        int lerr = memo_init(&mm, sp);
#pragma omp for schedule(dynamic, 16)
        for (int64_t q = 0; q < npts; ++q) {
            if (lerr) continue;
            i128 Z[ORC_MAXS];
            int bad = 0;
            for (int a = 0; a < sp->s; ++a) bad |= to_fixed(z[q * sp->s + a], &Z[a]);
            if (bad) { lerr = ORC_EINEXACT; continue; }
            int e = phi_fixed(sp, &mm, Z, &out[q], grad ? &grad[q * sp->s] : NULL);
            if (e) lerr = e;
        }
        memo_free(&mm);
#pragma omp critical
        if (lerr) err = lerr;
    }
    return err;
}

/* support half-width per axis of the centred phi: sum_j |xi_ja| / 2, as a double */
static double halfwidth(const orc_spline *sp, int a)
{
    double h = 0;
    for (int j = 0; j < sp->n; ++j) h += abs(sp->xi[j][a]);
    return 0.5 * h;
}

/* ---------------------------------------------------------------- the convolution sum (O1) */

typedef struct {
    int D, M;
    const int *lk;    /* M x s coset shifts */
    const int *dims;  /* s: N per axis of every coset array */
} orc_layout;

static int64_t lin_index(const int *i, const int *dims, int s)
{
    int64_t idx = 0;
    for (int a = 0; a < s; ++a) idx = idx * dims[a] + i[a];
    return idx;
}

/* Calls fn(site index k, linear index, phi, grad phi) for every stored site with phi != 0.
 * Brute force over the index box that covers the support's bounding box around x. */
typedef void (*site_fn)(void *ctx, int k, int64_t lin, double phi, const double *gphi);

static int for_each_site(const orc_spline *sp, orc_memo *mm, const orc_layout *ly, const double *x,
                         int want_grad, site_fn fn, void *ctx)
{
    int s = sp->s;
    i128 X[ORC_MAXS];
    for (int a = 0; a < s; ++a) if (to_fixed(x[a], &X[a])) return ORC_EINEXACT;
    int64_t sitesz = 1;
    for (int a = 0; a < s; ++a) sitesz *= ly->dims[a];
    for (int k = 0; k < ly->M; ++k) {
        int lo[ORC_MAXS], hi[ORC_MAXS];
        int empty = 0;
        for (int a = 0; a < s; ++a) {
            double h = halfwidth(sp, a);
            double u = x[a] - ly->lk[k * s + a];
            lo[a] = (int)floor((u - h) / ly->D);
            hi[a] = (int)ceil((u + h) / ly->D);
            if (lo[a] < 0) lo[a] = 0;
            if (hi[a] > ly->dims[a] - 1) hi[a] = ly->dims[a] - 1;
            if (lo[a] > hi[a]) empty = 1;
        }
        if (empty) continue;
        int i[ORC_MAXS];
        for (int a = 0; a < s; ++a) i[a] = lo[a];
        for (;;) {
            i128 Z[ORC_MAXS];
            for (int a = 0; a < s; ++a)
                Z[a] = X[a] - ((i128)(ly->D * (int64_t)i[a] + ly->lk[k * s + a]) << ORC_F);
            double phi, g[ORC_MAXS] = {0, 0, 0, 0};
            /* the gradient is the limit along x + eps*v like every decision, also where phi = 0
             * exactly: on the boundary of the support a continuous but not C^1 phi has a nonzero
             * one-sided gradient pointing into the support */
            int e = phi_fixed(sp, mm, Z, &phi, want_grad ? g : NULL);
            if (e) return e;
            int nz = phi != 0.0;
            for (int a = 0; a < s; ++a) nz |= g[a] != 0.0;
            if (nz) fn(ctx, k, (int64_t)k * sitesz + lin_index(i, ly->dims, s), phi, g);
            int a = s - 1;
            while (a >= 0) {
                if (++i[a] <= hi[a]) break;
                i[a] = lo[a];
                --a;
            }
            if (a < 0) break;
        }
    }
    return ORC_OK;
}

typedef struct { const double *c; double f; double g[ORC_MAXS]; int s; } eval_ctx;

static void eval_fn(void *vctx, int k, int64_t lin, double phi, const double *gphi)
{
    (void)k;
    eval_ctx *ctx = (eval_ctx *)vctx;
    double c = ctx->c[lin];
    ctx->f += c * phi;
    for (int a = 0; a < ctx->s; ++a) ctx->g[a] += c * gphi[a];
}

/* f(x_q) (and grad f) for npts points; coeffs are M arrays of prod(dims) doubles, coset-major,
 * row-major inside a coset (last axis fastest). */
int orc_eval(void *h, int D, int M, const int *lk, const int *dims, const double *coeffs,
             int64_t npts, const double *pts, double *out, double *grad, int nthreads)
{
    orc_spline *sp = (orc_spline *)h;
    orc_layout ly = {D, M, lk, dims};
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        orc_memo mm;
        int lerr = memo_init(&mm, sp);
#pragma omp for schedule(dynamic, 4)
        for (int64_t q = 0; q < npts; ++q) {
            if (lerr) continue;
            eval_ctx ctx;
            memset(&ctx, 0, sizeof(ctx));
            ctx.c = coeffs; ctx.s = sp->s;
            int e = for_each_site(sp, &mm, &ly, pts + q * sp->s, grad != NULL, eval_fn, &ctx);
            if (e) { lerr = e; continue; }
            out[q] = ctx.f;
            if (grad) for (int a = 0; a < sp->s; ++a) grad[q * sp->s + a] = ctx.g[a];
        }
        memo_free(&mm);
#pragma omp critical
        if (lerr) err = lerr;
    }
    return err;
}

typedef struct { double *d; double g; } adj_ctx;

static void adj_fn(void *vctx, int k, int64_t lin, double phi, const double *gphi)
{
    (void)k; (void)gphi;
    adj_ctx *ctx = (adj_ctx *)vctx;
    ctx->d[lin] += ctx->g * phi;
}

/* dcoeffs[n] += sum_q g_q phi(x_q - n).  Each thread sums its share of the queries into its own
 * array; the arrays are then added into dcoeffs. */
int orc_adjoint(void *h, int D, int M, const int *lk, const int *dims, int64_t npts,
                const double *pts, const double *g, double *dcoeffs)
{
    orc_spline *sp = (orc_spline *)h;
    orc_layout ly = {D, M, lk, dims};
    int64_t total = M;
    for (int a = 0; a < sp->s; ++a) total *= dims[a];
    int err = 0;
#pragma omp parallel
    {
        orc_memo mm;
        int lerr = memo_init(&mm, sp);
        double *mine = (double *)calloc((size_t)total, sizeof(double));
        if (!mine) lerr = ORC_ENOMEM;
#pragma omp for schedule(dynamic, 16)
        for (int64_t q = 0; q < npts; ++q) {
            if (lerr) continue;
            adj_ctx ctx = {mine, g[q]};
            lerr = for_each_site(sp, &mm, &ly, pts + q * sp->s, 0, adj_fn, &ctx);
        }
#pragma omp critical
        {
            if (lerr) err = lerr;
            else for (int64_t i = 0; i < total; ++i) dcoeffs[i] += mine[i];
        }
        free(mine);
        memo_free(&mm);
    }
    return err;
}

/* ---------------------------------------------------------------- exact cell reduction (O7) */

/* For every point and coset k: the nearest coset site index i = floor((x - l_k)/D + 1/2) and the
 * offset y = x - l_k - D i in [-D/2, D/2)^s, both exact (Sec. 4.1, the shift rho to the region of
 * evaluation, here the cube centred on the coset site). */
int orc_cells(int s, int D, int M, const int *lk, int64_t npts, const double *pts,
              int32_t *cells, double *offs)
{
    for (int64_t q = 0; q < npts; ++q)
        for (int k = 0; k < M; ++k)
            for (int a = 0; a < s; ++a) {
                i128 X;
                if (to_fixed(pts[q * s + a], &X)) return ORC_EINEXACT;
                i128 U = X - ((i128)lk[k * s + a] << ORC_F) + (((i128)D) << (ORC_F - 1));
                i128 den = ((i128)D) << ORC_F;
                i128 fl = U / den;
                if (U % den != 0 && U < 0) fl -= 1; /* floor division */
                cells[(q * M + k) * s + a] = (int32_t)fl;
                i128 Y = X - ((i128)lk[k * s + a] << ORC_F) - fl * den;
                offs[(q * M + k) * s + a] = fixed_to_double(Y);
            }
    return ORC_OK;
}

/*
 * FP64 CPU oracle of one two-fluid SPH (TFSPH) time step with the implicit
 * "drag in cell" (SPH-IDIC) interphase drag of Stoyanovskaya et al.,
 * "Monodisperse gas-solid mixtures with intense interphase interaction in
 * two-fluid SPH" (arXiv:1908.01682).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the independent checker of the GPU
 * library: only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark load it. It shares no code, header, table or constant with
 * the CUDA path, and the product path never calls it.
 *
 * Everything is a plain loop in double precision, following the method in the
 * paper's order:
 *   - two-fluid momentum equations in K form (Sec. 2, Eq. 7), gas pressure
 *     acceleration as the symmetric SPH sum of the first term of Eq. 19;
 *   - decomposition of the domain into disjoint Euler cells holding N gas and
 *     L dust particles (Sec. 2.3), eps* = m_d L / (m_g N) (Eq. 17),
 *     K* = rho*_d / t*_stop and rho*_g = rho*_d / eps* (Eq. 18);
 *   - gas and dust velocity equations with drag taken implicitly against the
 *     cell-mean velocity of the other phase (Eqs. 19-20), cell means v_*, u_*
 *     (Eq. 21), first-order time discretisation (the "parsimonious" solve the
 *     paper states but does not print; see orc_step).
 *
 * Readings of points the paper leaves open (each one is listed in the design
 * notes of the repository):
 *   - summation density with the self term, fixed h; M4 cubic spline kernel
 *     with support 2h (the paper names no kernel);
 *   - isothermal p = cs^2 rho, or adiabatic p = (gamma-1) rho e with the
 *     standard SPH energy equation and Monaghan artificial viscosity;
 *   - t*_stop = arithmetic mean of the per-particle stopping times of the
 *     cell's dust (harmonic mean selectable); rho*_d cancels out;
 *   - cells with N = 0 or L = 0 get no drag this step;
 *   - positions advance with the new velocities, x' = x + tau v';
 *   - particles are ordered by (cell key, particle id).
 *
 * Cell keys and neighbour membership are integer decisions taken from
 * floating point. Both are taken exactly, over the real numbers, from their
 * definitions (orc_axis_cell, orc_pair_band); every value is computed in
 * binary64. Pairs within a few units in the last place of the support
 * radius, in the precision of the path under test (path_fp32), are flagged
 * so that a checker can report them instead of failing on them.
 *
 * Build with -ffp-contract=off so that every binary64 expression is rounded
 * as written (no fused multiply-add).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_E_ARG 1
#define ORC_E_OOM 2

typedef struct {
    int32_t dim;          /* 1, 2 or 3 */
    int32_t path_fp32;    /* 1: the path under test computes in binary32 (width of the reported pair band) */
    int32_t eos;          /* 0 isothermal, 1 adiabatic */
    int32_t tstar_mode;   /* 0 arithmetic mean of t_j, 1 harmonic mean */
    int32_t periodic[3];
    int32_t brute;        /* 1: all-pairs neighbour search, 0: cell lists */
    double lo[3], hi[3];
    double h, cell_size;
    double m_gas, m_dust;
    double cs, gamma;
    double av_alpha, av_beta;
} orc_params;

/* ------------------------------------------------------------------------ */
/* Smoothing kernel: M4 cubic spline, support 2h.                            */
/* W(r,h) = sigma_d / h^d * { 1 - 3/2 q^2 + 3/4 q^3   (0 <= q < 1)           */
/*                            1/4 (2 - q)^3           (1 <= q < 2)           */
/*                            0                       (q >= 2) }, q = r/h    */
/* sigma_1 = 2/3, sigma_2 = 10/(7 pi), sigma_3 = 1/pi (unit integral).      */
/* ------------------------------------------------------------------------ */
static double orc_sigma(int dim)
{
    if (dim == 1) return 2.0 / 3.0;
    if (dim == 2) return 10.0 / (7.0 * M_PI);
    return 1.0 / M_PI;
}

double orc_W(int dim, double h, double r)
{
    double q = r / h;
    double norm = orc_sigma(dim) / pow(h, dim);
    if (q < 1.0) return norm * (1.0 - 1.5 * q * q + 0.75 * q * q * q);
    if (q < 2.0) return norm * 0.25 * (2.0 - q) * (2.0 - q) * (2.0 - q);
    return 0.0;
}

/* dW/dr */
double orc_dWdr(int dim, double h, double r)
{
    double q = r / h;
    double norm = orc_sigma(dim) / pow(h, dim + 1);
    if (q < 1.0) return norm * (-3.0 * q + 2.25 * q * q);
    if (q < 2.0) return norm * (-0.75 * (2.0 - q) * (2.0 - q));
    return 0.0;
}

/* ------------------------------------------------------------------------ */
/* Euler cells: uniform axis-aligned grid from lo, n_d = floor(L_d / size).  */
/* ------------------------------------------------------------------------ */
int orc_ncell(const orc_params *P, int32_t ncell[3])
{
    for (int d = 0; d < 3; ++d) {
        if (d >= P->dim) { ncell[d] = 1; continue; }
        double L = P->hi[d] - P->lo[d];
        double n = floor(L / P->cell_size);
        if (n < 1.0) n = 1.0;
        ncell[d] = (int32_t)n;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Integer decisions, taken exactly from their definitions.                 */
/*                                                                          */
/* A cell index and a neighbour membership are integers decided from        */
/* floating-point data. Both are decided here over the real numbers, on the */
/* stored values (the binary32 positions of the FP32 path are exact         */
/* binary64 values):                                                        */
/*   cell index along axis d: floor((x - lo) n / L), L = hi - lo in         */
/*     binary64, clamped to [0, n-1] (Sec. 2.3: disjoint volumes);          */
/*   membership: r^2 < 4 h^2 with r^2 = sum over axes of s^2, s = x_a - x_b */
/*     shifted by -+L when |x_a - x_b| > L/2 on a periodic axis (support of */
/*     the kernel in the sums of Eq. 19).                                   */
/* A binary64 estimate settles every case whose margin exceeds the          */
/* estimate's rounding error; the others are settled with integers.         */
/* ------------------------------------------------------------------------ */

/* |v| = m 2^e with an integer m < 2^53 (m = 0 for v = 0). */
static void orc_split(double v, uint64_t *m, int *e)
{
    int ex = 0;
    double f = frexp(fabs(v), &ex); /* |v| = f 2^ex, 1/2 <= f < 1 */
    *m = (uint64_t)ldexp(f, 53);
    *e = ex - 53;
}

/* Multi-word two's-complement integer, value = sum_j w[j] 2^(32 j + E0).   */
/* Every binary64 value times an integer below 2^31 is an integer multiple  */
/* of 2^E0 (E0 = -1126, the last bit of the smallest subnormal written with */
/* a 53-bit m) below 2^(1024 + 31); 72 words hold a sum of three of them.   */
#define ORC_BN_WORDS 72
#define ORC_BN_E0 (-1126)
typedef struct {
    uint32_t w[ORC_BN_WORDS];
} orc_bn;

/* A += m k 2^e (negative = 0) or A -= m k 2^e (negative = 1); m < 2^53, k < 2^31. */
static void orc_bn_add(orc_bn *A, int negative, uint64_t m, uint64_t k, int e)
{
    int s = e - ORC_BN_E0;
    unsigned __int128 t = ((unsigned __int128)m * k) << (s % 32); /* < 2^115 */
    uint32_t add[ORC_BN_WORDS];
    memset(add, 0, sizeof add);
    for (int j = 0; j < 4; ++j) add[s / 32 + j] = (uint32_t)(t >> (32 * j));
    int64_t carry = 0;
    for (int j = 0; j < ORC_BN_WORDS; ++j) {
        int64_t v = (int64_t)A->w[j] + (negative ? -(int64_t)add[j] : (int64_t)add[j]) + carry;
        A->w[j] = (uint32_t)v;                                     /* v mod 2^32 */
        carry = (v - (int64_t)(uint32_t)v) / ((int64_t)1 << 32);   /* exact */
    }
}

static int orc_bn_sign(const orc_bn *A)
{
    if (A->w[ORC_BN_WORDS - 1] & 0x80000000u) return -1;
    for (int j = 0; j < ORC_BN_WORDS; ++j)
        if (A->w[j]) return 1;
    return 0;
}

/* A += sign * v * k for a binary64 v and an integer 0 <= k < 2^31. */
static void orc_bn_term(orc_bn *A, double v, int64_t k, int sign)
{
    uint64_t m;
    int e;
    orc_split(v, &m, &e);
    orc_bn_add(A, (v < 0.0) != (sign < 0), m, (uint64_t)k, e);
}

/* Sign of (x - lo) n - i L over the reals: where x lies against the face   */
/* between cells i - 1 and i.                                               */
static int orc_face_sign(double x, double lo, double L, int64_t n, int64_t i)
{
    orc_bn A;
    memset(&A, 0, sizeof A);
    orc_bn_term(&A, x, n, +1);
    orc_bn_term(&A, lo, n, -1);
    orc_bn_term(&A, L, i, -1);
    return orc_bn_sign(&A);
}

/* Cell index of one position along axis d: floor((x - lo) n / L), clamped */
/* to [0, n-1]; NaN goes to cell 0.                                          */
static int64_t orc_axis_cell(const orc_params *P, int d, int32_t n, double x)
{
    if (x != x) return 0;
    if (isinf(x)) return x > 0.0 ? n - 1 : 0;
    double lo = P->lo[d], L = P->hi[d] - P->lo[d];
    /* estimate: three correctly rounded operations, relative error below 2^-50 */
    double q = (x - lo) * (double)n / L;
    double f = floor(q);
    int64_t i = !(f >= 0.0) ? 0 : (f > (double)(n - 1) ? n - 1 : (int64_t)f);
    /* no integer within the estimate's error: its floor is the exact one */
    if (fabs(q - nearbyint(q)) > 1e-12 * (1.0 + fabs(q))) return i;
    /* otherwise settle the cell face exactly */
    while (i > 0 && orc_face_sign(x, lo, L, n, i) < 0) --i;
    while (i < n - 1 && orc_face_sign(x, lo, L, n, i + 1) >= 0) ++i;
    return i;
}

/* key = ix + nx (iy + ny iz); x is the position of one particle, x[d]. */
static int64_t orc_key(const orc_params *P, const int32_t nc[3], const double x[3])
{
    int64_t c[3] = {0, 0, 0};
    for (int d = 0; d < P->dim; ++d) c[d] = orc_axis_cell(P, d, nc[d], x[d]);
    return c[0] + (int64_t)nc[0] * (c[1] + (int64_t)nc[1] * c[2]);
}

/* |v| = m 2^e with an odd integer m (m = 0 for v = 0): e is v's last bit. */
static void orc_split_odd(double v, uint64_t *m, int *e)
{
    orc_split(v, m, e);
    while (*m && !(*m & 1u)) {
        *m >>= 1;
        *e += 1;
    }
}

static int orc_bits(uint64_t m)
{
    int b = 0;
    while (m) {
        ++b;
        m >>= 1;
    }
    return b;
}

/* r^2 < 4 h^2 over the reals for the periodic image shifts chosen (shift[k] */
/* L subtracted along axis k), with 128-bit integers: every coordinate, box */
/* edge and h is an integer multiple of 2^g, g the smallest last bit among  */
/* them. Returns 1 or 0, or -1 when the scaled values do not fit.           */
static int orc_exact_lt(const orc_params *P, const double xa[3], const double xb[3], const int shift[3])
{
    uint64_t mh;
    int eh;
    orc_split_odd(P->h, &mh, &eh);
    uint64_t m[3][3];
    int e[3][3], neg[3][3];
    int g = eh;
    for (int k = 0; k < P->dim; ++k) {
        double v[3] = {xa[k], -xb[k], -(double)shift[k] * (P->hi[k] - P->lo[k])};
        for (int t = 0; t < 3; ++t) {
            orc_split_odd(v[t], &m[k][t], &e[k][t]);
            neg[k][t] = v[t] < 0.0;
            if (m[k][t] && e[k][t] < g) g = e[k][t];
        }
    }
    unsigned __int128 r2 = 0;
    for (int k = 0; k < P->dim; ++k) {
        __int128 S = 0;
        for (int t = 0; t < 3; ++t) {
            if (!m[k][t]) continue;
            int sh = e[k][t] - g;
            if (orc_bits(m[k][t]) + sh > 124) return -1;
            __int128 term = (__int128)((unsigned __int128)m[k][t] << sh);
            S += neg[k][t] ? -term : term;
        }
        if (S < 0) S = -S;
        if (S >= ((__int128)1 << 62)) return -1;
        r2 += (unsigned __int128)S * (unsigned __int128)S;
    }
    /* 4 h^2 = mh^2 2^(2 (eh - g) + 2) */
    int sh = 2 * (eh - g) + 2;
    if (2 * orc_bits(mh) + sh > 127) return -1;
    unsigned __int128 H = ((unsigned __int128)mh * mh) << sh;
    return r2 < H;
}

/* Neighbour decision of a pair: 1 if r^2 < 4 h^2 over the reals, else 0.   */
/* d[] receives x_a - x_b (minimum image on periodic axes) and *r2 its      */
/* squared norm, in binary64. *band is set when r^2 lies within 8 units in  */
/* the last place of 4 h^2, in the precision of the path under test, of    */
/* 4 h^2 (the GPU path may decide such a pair either way; the kernel there  */
/* is below 1e-17 of its peak), or when the decision could not be          */
/* certified (the 128-bit form overflows: only for a coordinate within      */
/* about 2^-15 of zero in a pair within 2^-49 of the boundary).            */
static int orc_pair_band(const orc_params *P, const double xa[3], const double xb[3], double d[3], double *r2,
                         int *band)
{
    const double u = 0x1p-53;
    int shift[3] = {0, 0, 0};
    double slack = 0.0; /* an image choice within rounding of L/2 */
    double s2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        d[k] = 0.0;
        if (k >= P->dim) continue;
        double L = P->hi[k] - P->lo[k];
        double s = xa[k] - xb[k];
        if (P->periodic[k]) {
            if (fabs(fabs(s) - 0.5 * L) <= 4.0 * u * L) slack += 32.0 * u * L * L;
            if (s > 0.5 * L) {
                s -= L;
                shift[k] = 1;
            } else if (s < -0.5 * L) {
                s += L;
                shift[k] = -1;
            }
        }
        d[k] = s;
        s2 += s * s;
    }
    *r2 = s2;
    const double H = 4.0 * P->h * P->h;
    const double err = 16.0 * u * (s2 + H) + slack; /* bounds |s2 - r^2| + |H - 4h^2| */
    const double ulp_path = ldexp(1.0, ilogb(H) - (P->path_fp32 ? 23 : 52));
    *band = fabs(s2 - H) <= 8.0 * ulp_path + err;
    if (fabs(s2 - H) > err) return s2 < H;
    int exact = slack > 0.0 ? -1 : orc_exact_lt(P, xa, xb, shift);
    if (exact < 0) {
        *band = 1;
        return s2 < H;
    }
    return exact;
}

static int orc_pair(const orc_params *P, const double xa[3], const double xb[3], double d[3], double *r2)
{
    int band;
    return orc_pair_band(P, xa, xb, d, r2, &band);
}

/* The membership decision of one pair, for the tests: 1 if r^2 < 4 h^2, else */
/* 0; *band as in orc_pair_band.                                              */
int orc_neighbour(const orc_params *P, const double *xa, const double *xb, int32_t *band)
{
    double pa[3] = {0, 0, 0}, pb[3] = {0, 0, 0}, d[3], r2;
    int b = 0;
    for (int k = 0; k < P->dim; ++k) {
        pa[k] = xa[k];
        pb[k] = xb[k];
    }
    int in = orc_pair_band(P, pa, pb, d, &r2, &b);
    if (band) *band = b;
    return in;
}

/* The cell index of one position along axis d, for the tests. */
int64_t orc_cell_index(const orc_params *P, int d, double x)
{
    int32_t nc[3];
    orc_ncell(P, nc);
    return orc_axis_cell(P, d, nc[d], x);
}

/* ------------------------------------------------------------------------ */
/* Sorting into cells: ascending (key, id).                                  */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t key; int64_t id; } orc_kv;

static int orc_kv_cmp(const void *a, const void *b)
{
    const orc_kv *x = (const orc_kv *)a, *y = (const orc_kv *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

static void orc_get_pos(int dim, int64_t n, const double *x, int64_t i, double p[3])
{
    p[0] = p[1] = p[2] = 0.0;
    for (int d = 0; d < dim; ++d) p[d] = x[(int64_t)d * n + i];
}

/* keys[i] per particle (id order); perm[s] = id at sorted slot s;
 * cstart[c] = first slot of cell c, cstart[ncells] = n. */
int orc_bin(const orc_params *P, int64_t n, const double *x,
            int64_t *keys, int64_t *perm, int64_t *cstart)
{
    int32_t nc[3];
    orc_ncell(P, nc);
    int64_t ncells = (int64_t)nc[0] * nc[1] * nc[2];
    orc_kv *kv = (orc_kv *)malloc(sizeof(orc_kv) * (size_t)(n > 0 ? n : 1));
    if (!kv) return ORC_E_OOM;
    for (int64_t i = 0; i < n; ++i) {
        double p[3];
        orc_get_pos(P->dim, n, x, i, p);
        kv[i].key = orc_key(P, nc, p);
        kv[i].id = i;
        if (keys) keys[i] = kv[i].key;
    }
    qsort(kv, (size_t)n, sizeof(orc_kv), orc_kv_cmp);
    if (perm) for (int64_t s = 0; s < n; ++s) perm[s] = kv[s].id;
    if (cstart) {
        for (int64_t c = 0; c <= ncells; ++c) cstart[c] = 0;
        for (int64_t s = 0; s < n; ++s) cstart[kv[s].key + 1] += 1;
        for (int64_t c = 0; c < ncells; ++c) cstart[c + 1] += cstart[c];
    }
    free(kv);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Neighbour candidates. Brute force: every particle. Cell lists: every      */
/* distinct cell within +-R of the particle's cell, R = floor(2h/w) + 2,     */
/* which is wider than any pair within 2h can reach. The membership test     */
/* decides; the candidate set only has to contain the neighbours.           */
/* ------------------------------------------------------------------------ */
typedef struct {
    const orc_params *P;
    int32_t nc[3];
    int64_t n;
    const double *x;
    const int64_t *perm;    /* sorted slot -> id */
    const int64_t *cstart;  /* cell -> first slot */
} orc_grid;

/* Distinct cell coordinates along axis d around cell c; returns count. */
static int orc_axis_window(const orc_grid *G, int d, int64_t c, int64_t *out)
{
    int32_t n = G->nc[d];
    if (d >= G->P->dim) { out[0] = 0; return 1; }
    double w = (G->P->hi[d] - G->P->lo[d]) / (double)n;
    int64_t R = (int64_t)floor(2.0 * G->P->h / w) + 2;
    int cnt = 0;
    if (G->P->periodic[d]) {
        if (2 * R + 1 >= n) {
            for (int64_t k = 0; k < n; ++k) out[cnt++] = k;
        } else {
            for (int64_t o = -R; o <= R; ++o) out[cnt++] = ((c + o) % n + n) % n;
        }
    } else {
        for (int64_t o = -R; o <= R; ++o) {
            int64_t k = c + o;
            if (k >= 0 && k < n) out[cnt++] = k;
        }
    }
    return cnt;
}

/* Calls visit(ctx, b) for every candidate b of particle position p. */
typedef void (*orc_visit_fn)(void *ctx, int64_t b);

static void orc_foreach_candidate(const orc_grid *G, const double p[3],
                                  orc_visit_fn visit, void *ctx)
{
    if (G->P->brute) {
        for (int64_t b = 0; b < G->n; ++b) visit(ctx, b);
        return;
    }
    int64_t cc[3] = {0, 0, 0};
    for (int d = 0; d < G->P->dim; ++d) cc[d] = orc_axis_cell(G->P, d, G->nc[d], p[d]);
    int64_t *wx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(G->nc[0] + 8));
    int64_t *wy = (int64_t *)malloc(sizeof(int64_t) * (size_t)(G->nc[1] + 8));
    int64_t *wz = (int64_t *)malloc(sizeof(int64_t) * (size_t)(G->nc[2] + 8));
    int nx = orc_axis_window(G, 0, cc[0], wx);
    int ny = orc_axis_window(G, 1, cc[1], wy);
    int nz = orc_axis_window(G, 2, cc[2], wz);
    for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
            for (int ix = 0; ix < nx; ++ix) {
                int64_t key = wx[ix] + (int64_t)G->nc[0] * (wy[iy] + (int64_t)G->nc[1] * wz[iz]);
                for (int64_t s = G->cstart[key]; s < G->cstart[key + 1]; ++s) visit(ctx, G->perm[s]);
            }
    free(wx);
    free(wy);
    free(wz);
}

/* ------------------------------------------------------------------------ */
/* Summation density rho_a = sum_b m W(|r_ab|, h), self term included.       */
/* Also the neighbour statistics a checker compares with: the count and an  */
/* order-free fingerprint of the neighbours outside the reported band (sum  */
/* over them of (id_b + 1) * 0x9E3779B97F4A7C15 mod 2^64), the number of    */
/* candidate pairs inside the band and the ids of the first ORC_NBAND.      */
/* ------------------------------------------------------------------------ */
#define ORC_NBAND 4

typedef struct {
    const orc_grid *G;
    double pa[3];
    double m;
    double rho;
    int64_t count;
    uint64_t fprint;
    int64_t nband;
    int64_t band_id[ORC_NBAND];
} orc_dens_ctx;

static void orc_dens_visit(void *vctx, int64_t b)
{
    orc_dens_ctx *c = (orc_dens_ctx *)vctx;
    double pb[3], d[3], r2;
    int band = 0;
    orc_get_pos(c->G->P->dim, c->G->n, c->G->x, b, pb);
    int inside = orc_pair_band(c->G->P, c->pa, pb, d, &r2, &band);
    if (band) {
        if (c->nband < ORC_NBAND) c->band_id[c->nband] = b;
        c->nband += 1;
    }
    if (!inside) return;
    c->rho += c->m * orc_W(c->G->P->dim, c->G->P->h, sqrt(r2));
    if (band) return;
    c->count += 1;
    c->fprint += (uint64_t)(b + 1) * 0x9E3779B97F4A7C15ull;
}

static int orc_make_grid(const orc_params *P, int64_t n, const double *x, orc_grid *G,
                         int64_t **perm, int64_t **cstart)
{
    G->P = P;
    orc_ncell(P, G->nc);
    G->n = n;
    G->x = x;
    int64_t ncells = (int64_t)G->nc[0] * G->nc[1] * G->nc[2];
    *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    *cstart = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncells + 1));
    if (!*perm || !*cstart) return ORC_E_OOM;
    orc_bin(P, n, x, NULL, *perm, *cstart);
    G->perm = *perm;
    G->cstart = *cstart;
    return ORC_OK;
}

/* Density of one particle set (gas or dust) of particle mass m. */
/* count, fprint, nband (each [n]) and band_ids ([ORC_NBAND n], -1 beyond  */
/* nband) are nullable.                                                     */
int orc_density(const orc_params *P, int64_t n, const double *x, double m,
                double *rho, int64_t *count, uint64_t *fprint, int64_t *nband, int64_t *band_ids)
{
    orc_grid G;
    int64_t *perm = NULL, *cstart = NULL;
    if (orc_make_grid(P, n, x, &G, &perm, &cstart) != ORC_OK) { free(perm); free(cstart); return ORC_E_OOM; }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t a = 0; a < n; ++a) {
        orc_dens_ctx c;
        c.G = &G;
        orc_get_pos(P->dim, n, x, a, c.pa);
        c.m = m;
        c.rho = 0.0;
        c.count = 0;
        c.fprint = 0;
        c.nband = 0;
        for (int k = 0; k < ORC_NBAND; ++k) c.band_id[k] = -1;
        orc_foreach_candidate(&G, c.pa, orc_dens_visit, &c);
        rho[a] = c.rho;
        if (count) count[a] = c.count;
        if (fprint) fprint[a] = c.fprint;
        if (nband) nband[a] = c.nband;
        if (band_ids)
            for (int k = 0; k < ORC_NBAND; ++k) band_ids[(int64_t)ORC_NBAND * a + k] = c.band_id[k];
    }
    free(perm);
    free(cstart);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Equation of state.                                                        */
/* ------------------------------------------------------------------------ */
static double orc_pressure(const orc_params *P, double rho, double e)
{
    if (P->eos == 1) return (P->gamma - 1.0) * rho * e;
    return P->cs * P->cs * rho;
}

static double orc_sound(const orc_params *P, double e)
{
    if (P->eos == 1) return sqrt(P->gamma * (P->gamma - 1.0) * e);
    return P->cs;
}

/* ------------------------------------------------------------------------ */
/* Gas pressure acceleration (first term of Eq. 19) and, with artificial    */
/* viscosity on, Monaghan's Pi_ab; energy rate of the adiabatic gas.         */
/*   A_a   = - sum_b m (p_a/rho_a^2 + p_b/rho_b^2 + Pi_ab) grad_a W_ab       */
/*   de_a  =   sum_b m (p_a/rho_a^2 + Pi_ab / 2) (v_a - v_b) . grad_a W_ab    */
/*   grad_a W_ab = (r_a - r_b) / r * dW/dr                                   */
/*   Pi_ab = (-alpha cbar mu + beta mu^2) / rhobar  if (v_ab . r_ab) < 0      */
/*   mu = h (v_ab . r_ab) / (r^2 + 0.01 h^2)                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    const orc_grid *G;
    int64_t a;
    double pa[3], va[3];
    const double *v, *rho, *pr, *cs;
    double acc[3];
    double dedt;
    double scale;  /* sum over pairs of |pair coefficient| |grad W|: the condition scale of A */
} orc_force_ctx;

static void orc_force_visit(void *vctx, int64_t b)
{
    orc_force_ctx *c = (orc_force_ctx *)vctx;
    const orc_params *P = c->G->P;
    int64_t n = c->G->n;
    double pb[3], d[3], r2;
    if (b == c->a) return;
    orc_get_pos(P->dim, n, c->G->x, b, pb);
    if (!orc_pair(P, c->pa, pb, d, &r2)) return;
    double r = sqrt(r2);
    if (r <= 0.0) return; /* coincident particles exert no pressure force */
    double dw = orc_dWdr(P->dim, P->h, r);
    double grad[3];
    for (int k = 0; k < 3; ++k) grad[k] = d[k] / r * dw;
    double vab[3] = {0, 0, 0};
    double vr = 0.0;
    for (int k = 0; k < P->dim; ++k) {
        vab[k] = c->va[k] - c->v[(int64_t)k * n + b];
        vr += vab[k] * d[k];
    }
    double qa = c->pr[c->a] / (c->rho[c->a] * c->rho[c->a]);
    double qb = c->pr[b] / (c->rho[b] * c->rho[b]);
    double pi = 0.0;
    if ((P->av_alpha > 0.0 || P->av_beta > 0.0) && vr < 0.0) {
        double mu = P->h * vr / (r2 + 0.01 * P->h * P->h);
        double cbar = 0.5 * (c->cs[c->a] + c->cs[b]);
        double rbar = 0.5 * (c->rho[c->a] + c->rho[b]);
        pi = (-P->av_alpha * cbar * mu + P->av_beta * mu * mu) / rbar;
    }
    double m = P->m_gas;
    double vg = 0.0, g2 = 0.0;
    for (int k = 0; k < P->dim; ++k) {
        c->acc[k] -= m * (qa + qb + pi) * grad[k];
        vg += vab[k] * grad[k];
        g2 += grad[k] * grad[k];
    }
    c->dedt += m * (qa + 0.5 * pi) * vg;
    c->scale += m * fabs(qa + qb + pi) * sqrt(g2);
}

/* acc[dim*n], dedt[n] (nullable) and scale[n] (nullable: the magnitude sum
 * of the pair terms, a diagnostic for tests) for every gas particle. */
int orc_accel(const orc_params *P, int64_t n, const double *x, const double *v,
              const double *e, const double *rho, double *acc, double *dedt, double *scale)
{
    orc_grid G;
    int64_t *perm = NULL, *cstart = NULL;
    double *pr = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *cs = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!pr || !cs || orc_make_grid(P, n, x, &G, &perm, &cstart) != ORC_OK) {
        free(pr); free(cs); free(perm); free(cstart);
        return ORC_E_OOM;
    }
    for (int64_t a = 0; a < n; ++a) {
        double ea = e ? e[a] : 0.0;
        pr[a] = orc_pressure(P, rho[a], ea);
        cs[a] = orc_sound(P, ea);
    }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t a = 0; a < n; ++a) {
        orc_force_ctx c;
        c.G = &G;
        c.a = a;
        orc_get_pos(P->dim, n, x, a, c.pa);
        for (int k = 0; k < 3; ++k) c.va[k] = k < P->dim ? v[(int64_t)k * n + a] : 0.0;
        c.v = v;
        c.rho = rho;
        c.pr = pr;
        c.cs = cs;
        c.acc[0] = c.acc[1] = c.acc[2] = 0.0;
        c.dedt = 0.0;
        c.scale = 0.0;
        orc_foreach_candidate(&G, c.pa, orc_force_visit, &c);
        for (int k = 0; k < P->dim; ++k) acc[(int64_t)k * n + a] = c.acc[k];
        if (dedt) dedt[a] = c.dedt;
        if (scale) scale[a] = c.scale;
    }
    free(pr);
    free(cs);
    free(perm);
    free(cstart);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Courant time step (Eq. 4): tau = CFL h / max over moving gas of           */
/* max(|v_a|, c_a).                                                           */
/* ------------------------------------------------------------------------ */
double orc_max_dt(const orc_params *P, int64_t n, const double *v, const double *e,
                  const uint8_t *frozen, double cfl)
{
    double vmax = 0.0;
    for (int64_t a = 0; a < n; ++a) {
        if (frozen && frozen[a]) continue;
        double s = 0.0;
        for (int k = 0; k < P->dim; ++k) s += v[(int64_t)k * n + a] * v[(int64_t)k * n + a];
        double sp = sqrt(s);
        double c = orc_sound(P, e ? e[a] : 0.0);
        double m = sp > c ? sp : c;
        if (m > vmax) vmax = m;
    }
    return cfl * P->h / vmax;
}

/* ------------------------------------------------------------------------ */
/* One SPH-IDIC step (Sec. 2.3, Eqs. 17-21), in place.                       */
/*                                                                           */
/* With K^/rho^_g = eps^/t^ and K^/rho^_d = 1/t^ (Eq. 18; ^ marks a cell    */
/* value), the first-order                                                   */
/* implicit scheme for a cell with N > 0 gas and L > 0 dust reads            */
/*   (v_a' - v_a)/tau = A_a + g - (eps^/t^) (v_a' - u_^')      (Eq. 19)      */
/*   (u_j' - u_j)/tau = g + (1/t^) (v_^' - u_j')               (Eq. 20)      */
/* with v_^, u_^ the cell means (Eq. 21). Averaging the first over the       */
/* cell's gas and the second over its dust gives two equations for the     */
/* new means; their difference fixes the new slip w' = v_^' - u_^':         */
/*   w' (1 + tau (1 + eps^)/t^) = w + tau Abar,    w = v_^ - u_^            */
/*   u_^' = u_^ + tau g + (tau/t^) w',   v_^' = u_^' + w'                  */
/* after which each particle equation is linear in its own new velocity.   */
/* ------------------------------------------------------------------------ */
/* Periodic image of x in [lo, hi), whatever the number of periods crossed. */
static double orc_wrap(double x, double lo, double hi)
{
    double L = hi - lo;
    double y = x - lo;
    y -= L * floor(y / L);
    double r = lo + y;
    if (r >= hi) r = lo;
    if (r < lo) r = lo;
    return r;
}

typedef struct {
    /* outputs, each nullable */
    double *rho_g;          /* [ng] density used in the step */
    double *acc_g;          /* [dim*ng] pressure (+viscous) acceleration */
    double *dedt_g;         /* [ng] */
    double *acc_scale_g;    /* [ng] magnitude sum of the pair terms of A (diagnostic) */
    int64_t *nb_count;      /* [ng] neighbours outside the reported band */
    uint64_t *nb_fprint;    /* [ng] their fingerprint */
    int64_t *nb_band;       /* [ng] candidate pairs inside the band */
    int64_t *nb_band_ids;   /* [ORC_NBAND ng] ids of the first of them, -1 beyond */
    int64_t *keys_g, *keys_d;     /* [ng], [nd] per particle (id order) */
    int64_t *perm_g, *perm_d;     /* [ng], [nd] id at sorted slot */
    int64_t *cstart_g, *cstart_d; /* [ncells+1] */
    int64_t n_drag_cells;         /* cells with N > 0 and L > 0 */
} orc_step_out;

int orc_step(const orc_params *P, int64_t ng, int64_t nd,
             double *gx, double *gv, double *ge, const uint8_t *gfrozen,
             double *dx, double *du, const double *tstop,
             double tau, const double g[3], const double *acc_override,
             orc_step_out *out)
{
    int dim = P->dim;
    int32_t nc[3];
    orc_ncell(P, nc);
    int64_t ncells = (int64_t)nc[0] * nc[1] * nc[2];
    if (dim < 1 || dim > 3 || tau <= 0.0) return ORC_E_ARG;

    /* 1. Cells and sorting. */
    int64_t *kg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ng > 0 ? ng : 1));
    int64_t *kd = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nd > 0 ? nd : 1));
    int64_t *pg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ng > 0 ? ng : 1));
    int64_t *pd = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nd > 0 ? nd : 1));
    int64_t *sg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncells + 1));
    int64_t *sd = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncells + 1));
    double *rho = (double *)malloc(sizeof(double) * (size_t)(ng > 0 ? ng : 1));
    double *acc = (double *)calloc((size_t)(dim * (ng > 0 ? ng : 1)), sizeof(double));
    double *dedt = (double *)calloc((size_t)(ng > 0 ? ng : 1), sizeof(double));
    /* per-cell: N, L, sum v, sum u, sum A, sum t (or sum 1/t) */
    double *cN = (double *)calloc((size_t)ncells, sizeof(double));
    double *cL = (double *)calloc((size_t)ncells, sizeof(double));
    double *cv = (double *)calloc((size_t)(3 * ncells), sizeof(double));
    double *cu = (double *)calloc((size_t)(3 * ncells), sizeof(double));
    double *cA = (double *)calloc((size_t)(3 * ncells), sizeof(double));
    double *ct = (double *)calloc((size_t)ncells, sizeof(double));
    int rc = ORC_OK;
    if (!kg || !kd || !pg || !pd || !sg || !sd || !rho || !acc || !dedt || !cN || !cL || !cv ||
        !cu || !cA || !ct) {
        rc = ORC_E_OOM;
        goto done;
    }
    orc_bin(P, ng, gx, kg, pg, sg);
    orc_bin(P, nd, dx, kd, pd, sd);

    /* 2. Gas summation density and pressure. */
    if (ng > 0) orc_density(P, ng, gx, P->m_gas, rho, out ? out->nb_count : NULL,
                            out ? out->nb_fprint : NULL, out ? out->nb_band : NULL,
                            out ? out->nb_band_ids : NULL);

    /* 3. Gas pressure (+ viscous) acceleration and energy rate. */
    if (ng > 0) orc_accel(P, ng, gx, gv, ge, rho, acc, dedt, out ? out->acc_scale_g : NULL);
    if (acc_override) memcpy(acc, acc_override, sizeof(double) * (size_t)(dim * ng));

    /* 4. Cell aggregates (Eqs. 17, 21), summed in sorted order. */
    for (int64_t s = 0; s < ng; ++s) {
        int64_t a = pg[s];
        if (gfrozen && gfrozen[a]) continue;
        int64_t c = kg[a];
        cN[c] += 1.0;
        for (int k = 0; k < dim; ++k) {
            cv[3 * c + k] += gv[(int64_t)k * ng + a];
            cA[3 * c + k] += acc[(int64_t)k * ng + a];
        }
    }
    for (int64_t s = 0; s < nd; ++s) {
        int64_t j = pd[s];
        int64_t c = kd[j];
        cL[c] += 1.0;
        for (int k = 0; k < dim; ++k) cu[3 * c + k] += du[(int64_t)k * nd + j];
        ct[c] += (P->tstar_mode == 1) ? 1.0 / tstop[j] : tstop[j];
    }

    /* 5. Per-cell implicit solve for the new mean velocities. */
    double *ustar = (double *)calloc((size_t)(3 * ncells), sizeof(double));
    double *vstar = (double *)calloc((size_t)(3 * ncells), sizeof(double));
    double *eps_c = (double *)calloc((size_t)ncells, sizeof(double));
    double *tst_c = (double *)calloc((size_t)ncells, sizeof(double));
    if (!ustar || !vstar || !eps_c || !tst_c) {
        free(ustar); free(vstar); free(eps_c); free(tst_c);
        rc = ORC_E_OOM;
        goto done;
    }
    int64_t ndrag = 0;
    for (int64_t c = 0; c < ncells; ++c) {
        if (cN[c] <= 0.0 || cL[c] <= 0.0) continue;
        ++ndrag;
        double N = cN[c], L = cL[c];
        double eps = P->m_dust * L / (P->m_gas * N);                 /* Eq. 17 */
        double tst = (P->tstar_mode == 1) ? L / ct[c] : ct[c] / L;   /* t*_stop */
        eps_c[c] = eps;
        tst_c[c] = tst;
        for (int k = 0; k < dim; ++k) {
            double vs = cv[3 * c + k] / N;                            /* Eq. 21 */
            double us = cu[3 * c + k] / L;
            double Abar = cA[3 * c + k] / N;
            double w = vs - us;
            double wn = (w + tau * Abar) / (1.0 + tau * (1.0 + eps) / tst);
            double un = us + tau * g[k] + (tau / tst) * wn;
            ustar[3 * c + k] = un;
            vstar[3 * c + k] = un + wn;
        }
    }

    /* 6. Particle velocities (Eqs. 19-20) and energies; 7. positions. */
    for (int64_t a = 0; a < ng; ++a) {
        if (gfrozen && gfrozen[a]) continue;
        int64_t c = kg[a];
        int drag = cN[c] > 0.0 && cL[c] > 0.0;
        for (int k = 0; k < dim; ++k) {
            double va = gv[(int64_t)k * ng + a];
            double rhs = va + tau * (acc[(int64_t)k * ng + a] + g[k]);
            double vn;
            if (drag) {
                double kg_ = eps_c[c] / tst_c[c];   /* K^/rho^_g */
                vn = (rhs + tau * kg_ * ustar[3 * c + k]) / (1.0 + tau * kg_);
            } else {
                vn = rhs;
            }
            gv[(int64_t)k * ng + a] = vn;
        }
        if (P->eos == 1 && ge) ge[a] += tau * dedt[a];
    }
    for (int64_t j = 0; j < nd; ++j) {
        int64_t c = kd[j];
        int drag = cN[c] > 0.0 && cL[c] > 0.0;
        for (int k = 0; k < dim; ++k) {
            double uj = du[(int64_t)k * nd + j];
            double rhs = uj + tau * g[k];
            double un;
            if (drag) {
                double kd_ = 1.0 / tst_c[c];        /* K^/rho^_d */
                un = (rhs + tau * kd_ * vstar[3 * c + k]) / (1.0 + tau * kd_);
            } else {
                un = rhs;
            }
            du[(int64_t)k * nd + j] = un;
        }
    }
    for (int64_t a = 0; a < ng; ++a) {
        if (gfrozen && gfrozen[a]) continue;
        for (int k = 0; k < dim; ++k) {
            double xn = gx[(int64_t)k * ng + a] + tau * gv[(int64_t)k * ng + a];
            if (P->periodic[k]) xn = orc_wrap(xn, P->lo[k], P->hi[k]);
            gx[(int64_t)k * ng + a] = xn;
        }
    }
    for (int64_t j = 0; j < nd; ++j) {
        for (int k = 0; k < dim; ++k) {
            double xn = dx[(int64_t)k * nd + j] + tau * du[(int64_t)k * nd + j];
            if (P->periodic[k]) xn = orc_wrap(xn, P->lo[k], P->hi[k]);
            dx[(int64_t)k * nd + j] = xn;
        }
    }

    if (out) {
        if (out->rho_g) memcpy(out->rho_g, rho, sizeof(double) * (size_t)ng);
        if (out->acc_g) memcpy(out->acc_g, acc, sizeof(double) * (size_t)(dim * ng));
        if (out->dedt_g) memcpy(out->dedt_g, dedt, sizeof(double) * (size_t)ng);
        if (out->keys_g) memcpy(out->keys_g, kg, sizeof(int64_t) * (size_t)ng);
        if (out->keys_d) memcpy(out->keys_d, kd, sizeof(int64_t) * (size_t)nd);
        if (out->perm_g) memcpy(out->perm_g, pg, sizeof(int64_t) * (size_t)ng);
        if (out->perm_d) memcpy(out->perm_d, pd, sizeof(int64_t) * (size_t)nd);
        if (out->cstart_g) memcpy(out->cstart_g, sg, sizeof(int64_t) * (size_t)(ncells + 1));
        if (out->cstart_d) memcpy(out->cstart_d, sd, sizeof(int64_t) * (size_t)(ncells + 1));
        out->n_drag_cells = ndrag;
    }
    free(ustar);
    free(vstar);
    free(eps_c);
    free(tst_c);
done:
    free(kg); free(kd); free(pg); free(pd); free(sg); free(sd);
    free(rho); free(acc); free(dedt);
    free(cN); free(cL); free(cv); free(cu); free(cA); free(ct);
    return rc;
}

/* ======================================================================== */
/* The two other drag schemes the paper compares (Sec. 2.1, 2.2), on the    */
/* same gas pressure force and binning.                                     */
/*                                                                          */
/* Drag coefficient: the path takes the stopping time t_j of every dust     */
/* particle as input, so K = rho_d / t_stop (the definition of Eq. 7) is    */
/* used throughout, with rho_d the dust summation density:                  */
/*   MK:   K_aj = rho_j,d / t_j, so K_aj / (rho_a,g rho_j,d) = 1/(rho_a,g t_j) */
/*   ISPH: at a dust particle K_j = rho_j,d / t_j; at a gas particle K is   */
/*         SPH-interpolated like any dust field (Eq. 11 form):              */
/*         K_a = m_d sum_j (K_j / rho_j,d) W_aj = m_d sum_j W_aj / t_j.     */
/* Frozen (wall) gas particles enter the density and pressure sums and take */
/* no part in the drag (they are at rest and never move).                   */
/* ======================================================================== */

/* Cross-phase candidate walk: the neighbours, among the particles of the   */
/* grid G (the other phase), of a point p; membership as for gas pairs.     */
typedef struct {
    const orc_grid *G;
    double p[3];
    void (*pair)(void *ctx, int64_t b, const double d[3], double r2);
    void *ctx;
} orc_cross_ctx;

static void orc_cross_visit(void *vctx, int64_t b)
{
    orc_cross_ctx *c = (orc_cross_ctx *)vctx;
    double pb[3], d[3], r2;
    orc_get_pos(c->G->P->dim, c->G->n, c->G->x, b, pb);
    if (!orc_pair(c->G->P, c->p, pb, d, &r2)) return;
    c->pair(c->ctx, b, d, r2);  /* d = p - x_b */
}

static void orc_cross_walk(const orc_grid *G, const double p[3],
                           void (*pair)(void *, int64_t, const double *, double), void *ctx)
{
    orc_cross_ctx c;
    c.G = G;
    for (int k = 0; k < 3; ++k) c.p[k] = p[k];
    c.pair = pair;
    c.ctx = ctx;
    orc_foreach_candidate(G, p, orc_cross_visit, &c);
}

/* --- MK (Eqs. 8-10), explicit in the drag:                               */
/*   D_a = - sigma m_d sum_j K_aj/(rho_a,g rho_j,d) ((v_a - u_j).r_ja)       */
/*                          / (r_ja^2 + eta^2) r_ja W_ja                     */
/*   D_j = + sigma m_g sum_a (same pair factor)                              */
/* r_ja = r_j - r_a (the product ((v_a - u_j).r) r is even in r), eta^2 =    */
/* 0.001 h^2, sigma = the dimension (1 in 1D, as the paper states).          */
typedef struct {
    const orc_params *P;
    int64_t nsrc;
    const double *vsrc;       /* other phase velocities (dim x nsrc) */
    const double *coef_src;   /* per source: 1/t_j (gas target) or 1/rho_a,g (dust target) */
    const uint8_t *skip_src;  /* frozen gas sources (dust target), nullable */
    double vt[3];             /* target velocity */
    double coef_t;            /* per target: 1/rho_a,g (gas target) or 1/t_j (dust target) */
    double sign;              /* v_gas - u_dust = sign * (v_target - v_source) */
    double sum[3];
    double scale;
} orc_mk_ctx;

static void orc_mk_pair(void *vctx, int64_t b, const double d[3], double r2)
{
    orc_mk_ctx *c = (orc_mk_ctx *)vctx;
    const orc_params *P = c->P;
    if (c->skip_src && c->skip_src[b]) return;
    double rel = 0.0;
    for (int k = 0; k < P->dim; ++k)
        rel += c->sign * (c->vt[k] - c->vsrc[(int64_t)k * c->nsrc + b]) * d[k];
    double w = orc_W(P->dim, P->h, sqrt(r2));
    double f = c->coef_t * c->coef_src[b] * rel / (r2 + 0.001 * P->h * P->h) * w;
    double dn = 0.0;
    for (int k = 0; k < P->dim; ++k) {
        c->sum[k] += f * d[k];
        dn += d[k] * d[k];
    }
    c->scale += fabs(f) * sqrt(dn);
}

/* --- ISPH interpolation at a gas particle a over dust j (Eq. 11 form):   */
/*   rho^d_a = m_d sum_j W_aj,  K_a = m_d sum_j W_aj / t_j,                 */
/*   u_a = m_d sum_j u_j / rho_j,d W_aj.                                    */
typedef struct {
    const orc_params *P;
    int64_t nd;
    const double *du, *tstop, *rho_d;
    double rho, K, u[3];
    double uscale;   /* m_d sum_j |u_j| / rho_j,d W_aj */
} orc_isph_g_ctx;

static void orc_isph_g_pair(void *vctx, int64_t j, const double d[3], double r2)
{
    orc_isph_g_ctx *c = (orc_isph_g_ctx *)vctx;
    const orc_params *P = c->P;
    (void)d;
    double w = P->m_dust * orc_W(P->dim, P->h, sqrt(r2));
    c->rho += w;
    c->K += w / c->tstop[j];
    double un = 0.0;
    for (int k = 0; k < P->dim; ++k) {
        double uk = c->du[(int64_t)k * c->nd + j];
        c->u[k] += w * uk / c->rho_d[j];
        un += uk * uk;
    }
    c->uscale += w * sqrt(un) / c->rho_d[j];
}

/* --- ISPH interpolation at a dust particle j over gas a (Eqs. 11, 14):   */
/*   rho^g_j = m_g sum_a W_aj,  v_j = m_g sum_{a moving} v_a / rho_a W_aj,  */
/*   e_j = m_g sum_a e_a / rho_a W_aj (adiabatic gas),                      */
/*   G_j = m_g sum_a grad_j W_aj,  Q_j = m_g sum_a q_a grad_j W_aj,         */
/* q_a = p_a / rho_a^2; then the pressure acceleration at j (Eq. 14) is     */
/*   A_j = - (Q_j + q_j G_j),  q_j = p_j / (rho^g_j)^2.                     */
typedef struct {
    const orc_params *P;
    int64_t ng;
    const double *gv, *ge, *rho_g, *q;
    const uint8_t *frozen;
    double rho, e, v[3], Gs[3], Qs[3];
    double vscale, gscale, qscale;
} orc_isph_d_ctx;

static void orc_isph_d_pair(void *vctx, int64_t a, const double d[3], double r2)
{
    orc_isph_d_ctx *c = (orc_isph_d_ctx *)vctx;
    const orc_params *P = c->P;
    double r = sqrt(r2);
    double w = P->m_gas * orc_W(P->dim, P->h, r);
    c->rho += w;
    if (P->eos == 1 && c->ge) c->e += w * c->ge[a] / c->rho_g[a];
    if (!(c->frozen && c->frozen[a])) {
        double vn = 0.0;
        for (int k = 0; k < P->dim; ++k) {
            double vk = c->gv[(int64_t)k * c->ng + a];
            c->v[k] += w * vk / c->rho_g[a];
            vn += vk * vk;
        }
        c->vscale += w * sqrt(vn) / c->rho_g[a];
    }
    if (r > 0.0) {
        /* d = x_j - x_a: grad_j W_aj = d / r dW/dr */
        double dw = P->m_gas * orc_dWdr(P->dim, P->h, r) / r;
        double gn = 0.0;
        for (int k = 0; k < P->dim; ++k) {
            c->Gs[k] += dw * d[k];
            c->Qs[k] += c->q[a] * dw * d[k];
            gn += d[k] * d[k];
        }
        c->gscale += fabs(dw) * sqrt(gn);
        c->qscale += fabs(c->q[a] * dw) * sqrt(gn);
    }
}

typedef struct {
    /* outputs, each nullable (id order) */
    double *rho_g;       /* [ng] gas density */
    double *rho_d;       /* [nd] dust density */
    double *acc_g;       /* [dim*ng] gas pressure (+viscous) acceleration */
    double *acc_scale_g; /* [ng] */
    double *drag_g;      /* [dim*ng] MK: D_a; ISPH: interpolated dust velocity u_a */
    double *drag_d;      /* [dim*nd] MK: D_j; ISPH: interpolated gas velocity v_j */
    double *scale_g;     /* [ng] MK: magnitude sum of D_a's terms; ISPH: of u_a's */
    double *scale_d;     /* [nd] MK: of D_j's terms; ISPH: of v_j's */
    double *isph_acc_d;  /* [dim*nd] ISPH: pressure acceleration at the dust particle (Eq. 14) */
    double *isph_acc_scale_d; /* [nd] ISPH: its condition scale */
    double *isph_rho_dg; /* [ng] ISPH: interpolated dust density at gas particles */
    double *isph_K_g;    /* [ng] ISPH: interpolated K at gas particles */
    double *isph_rho_gd; /* [nd] ISPH: interpolated gas density at dust particles */
} orc_xstep_out;

/* One step with drag scheme 1 (ISPH, Eqs. 11-16) or 2 (MK, Eqs. 8-10), in  */
/* place; binning, densities, gas pressure force and the position update as */
/* in orc_step.                                                              */
/*   ISPH, each particle with neighbours of the other phase: the 2x2 system  */
/*     (v' - v)/tau = A + g - alpha (v' - u'),  (u' - u)/tau = g + beta (v' - u') */
/*   in (own velocity, interpolated velocity of the other phase), alpha =    */
/*   K / rho_g, beta = K / rho_d at the particle (Eqs. 12-16), solved by      */
/*     w' = (v - u + tau A) / (1 + tau (alpha + beta)),                      */
/*     v' = v + tau (A + g) - tau alpha w',   u' = u + tau g + tau beta w';   */
/*   a gas particle keeps v', a dust particle keeps u'. The paper's Eq. 15    */
/*   divides by rho^n_{a,d} where the dust density at j, rho^n_{j,d}, is      */
/*   meant (Eq. 15 is the equation of dust particle j).                       */
/*   MK: v_a' = v_a + tau (A_a + D_a + g), u_j' = u_j + tau (D_j + g).        */
int orc_step_x(const orc_params *P, int scheme, int64_t ng, int64_t nd,
               double *gx, double *gv, double *ge, const uint8_t *gfrozen,
               double *dx, double *du, const double *tstop,
               double tau, const double g[3], orc_xstep_out *out)
{
    int dim = P->dim;
    if (dim < 1 || dim > 3 || tau <= 0.0 || (scheme != 1 && scheme != 2)) return ORC_E_ARG;
    size_t sg = (size_t)(ng > 0 ? ng : 1), sd = (size_t)(nd > 0 ? nd : 1);
    double *rho_g = (double *)calloc(sg, sizeof(double));
    double *rho_d = (double *)calloc(sd, sizeof(double));
    double *acc = (double *)calloc((size_t)dim * sg, sizeof(double));
    double *dedt = (double *)calloc(sg, sizeof(double));
    double *ascale = (double *)calloc(sg, sizeof(double));
    double *q = (double *)calloc(sg, sizeof(double));
    double *Xg = (double *)calloc((size_t)dim * sg, sizeof(double));  /* D_a or u_a */
    double *Xd = (double *)calloc((size_t)dim * sd, sizeof(double));  /* D_j or v_j */
    double *Sg = (double *)calloc(sg, sizeof(double));
    double *Sd = (double *)calloc(sd, sizeof(double));
    double *Ad = (double *)calloc((size_t)dim * sd, sizeof(double));  /* ISPH A_j */
    double *ASd = (double *)calloc(sd, sizeof(double));
    double *rdg = (double *)calloc(sg, sizeof(double));               /* ISPH rho^d_a */
    double *Kg = (double *)calloc(sg, sizeof(double));                /* ISPH K_a */
    double *rgd = (double *)calloc(sd, sizeof(double));               /* ISPH rho^g_j */
    double *inv_t = (double *)calloc(sd, sizeof(double));
    double *inv_rho = (double *)calloc(sg, sizeof(double));
    orc_grid Gg, Gd;
    int64_t *pg = NULL, *cg = NULL, *pd = NULL, *cd = NULL;
    int rc = ORC_OK;
    if (!rho_g || !rho_d || !acc || !dedt || !ascale || !q || !Xg || !Xd || !Sg || !Sd || !Ad || !ASd ||
        !rdg || !Kg || !rgd || !inv_t || !inv_rho || orc_make_grid(P, ng, gx, &Gg, &pg, &cg) != ORC_OK ||
        orc_make_grid(P, nd, dx, &Gd, &pd, &cd) != ORC_OK) {
        rc = ORC_E_OOM;
        goto done;
    }
    /* densities, pressure and the gas pressure force */
    if (ng > 0) orc_density(P, ng, gx, P->m_gas, rho_g, NULL, NULL, NULL, NULL);
    if (nd > 0) orc_density(P, nd, dx, P->m_dust, rho_d, NULL, NULL, NULL, NULL);
    if (ng > 0) orc_accel(P, ng, gx, gv, ge, rho_g, acc, dedt, ascale);
    for (int64_t a = 0; a < ng; ++a) {
        q[a] = orc_pressure(P, rho_g[a], ge ? ge[a] : 0.0) / (rho_g[a] * rho_g[a]);
        inv_rho[a] = 1.0 / rho_g[a];
    }
    for (int64_t j = 0; j < nd; ++j) inv_t[j] = 1.0 / tstop[j];

    /* cross-phase sums at every gas particle (over dust) and every dust     */
    /* particle (over gas)                                                   */
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t a = 0; a < ng; ++a) {
        if (gfrozen && gfrozen[a]) continue;
        double pa[3];
        orc_get_pos(dim, ng, gx, a, pa);
        if (scheme == 2) {
            orc_mk_ctx c;
            memset(&c, 0, sizeof c);
            c.P = P;
            c.nsrc = nd;
            c.vsrc = du;
            c.coef_src = inv_t;
            c.skip_src = NULL;
            for (int k = 0; k < dim; ++k) c.vt[k] = gv[(int64_t)k * ng + a];
            c.coef_t = inv_rho[a];
            c.sign = 1.0;
            orc_cross_walk(&Gd, pa, orc_mk_pair, &c);
            for (int k = 0; k < dim; ++k) Xg[(int64_t)k * ng + a] = -(double)dim * P->m_dust * c.sum[k];
            Sg[a] = (double)dim * P->m_dust * c.scale;
        } else {
            orc_isph_g_ctx c;
            memset(&c, 0, sizeof c);
            c.P = P;
            c.nd = nd;
            c.du = du;
            c.tstop = tstop;
            c.rho_d = rho_d;
            orc_cross_walk(&Gd, pa, orc_isph_g_pair, &c);
            for (int k = 0; k < dim; ++k) Xg[(int64_t)k * ng + a] = c.u[k];
            Sg[a] = c.uscale;
            rdg[a] = c.rho;
            Kg[a] = c.K;
        }
    }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t j = 0; j < nd; ++j) {
        double pj[3];
        orc_get_pos(dim, nd, dx, j, pj);
        if (scheme == 2) {
            orc_mk_ctx c;
            memset(&c, 0, sizeof c);
            c.P = P;
            c.nsrc = ng;
            c.vsrc = gv;
            c.coef_src = inv_rho;
            c.skip_src = gfrozen;
            for (int k = 0; k < dim; ++k) c.vt[k] = du[(int64_t)k * nd + j];
            c.coef_t = inv_t[j];
            c.sign = -1.0;
            orc_cross_walk(&Gg, pj, orc_mk_pair, &c);
            for (int k = 0; k < dim; ++k) Xd[(int64_t)k * nd + j] = (double)dim * P->m_gas * c.sum[k];
            Sd[j] = (double)dim * P->m_gas * c.scale;
        } else {
            orc_isph_d_ctx c;
            memset(&c, 0, sizeof c);
            c.P = P;
            c.ng = ng;
            c.gv = gv;
            c.ge = ge;
            c.rho_g = rho_g;
            c.q = q;
            c.frozen = gfrozen;
            orc_cross_walk(&Gg, pj, orc_isph_d_pair, &c);
            rgd[j] = c.rho;
            double qj = 0.0;
            if (c.rho > 0.0) {
                /* p_j / rho_j^2: isothermal cs^2 / rho; adiabatic (gamma-1) e_j / rho */
                qj = P->eos == 1 ? (P->gamma - 1.0) * c.e / c.rho : P->cs * P->cs / c.rho;
            }
            double an = 0.0;
            for (int k = 0; k < dim; ++k) {
                Xd[(int64_t)k * nd + j] = c.v[k];
                Ad[(int64_t)k * nd + j] = -(c.Qs[k] + qj * c.Gs[k]);
            }
            (void)an;
            Sd[j] = c.vscale;
            ASd[j] = c.qscale + fabs(qj) * c.gscale;
        }
    }

    /* velocity updates */
    for (int64_t a = 0; a < ng; ++a) {
        if (gfrozen && gfrozen[a]) continue;
        for (int k = 0; k < dim; ++k) {
            double v = gv[(int64_t)k * ng + a], A = acc[(int64_t)k * ng + a];
            double vn;
            if (scheme == 2) {
                vn = v + tau * (A + Xg[(int64_t)k * ng + a] + g[k]);
            } else if (rdg[a] > 0.0) {
                double alpha = Kg[a] / rho_g[a], beta = Kg[a] / rdg[a];
                double wn = (v - Xg[(int64_t)k * ng + a] + tau * A) / (1.0 + tau * (alpha + beta));
                vn = v + tau * (A + g[k]) - tau * alpha * wn;
            } else {
                vn = v + tau * (A + g[k]);
            }
            gv[(int64_t)k * ng + a] = vn;
        }
        if (P->eos == 1 && ge) ge[a] += tau * dedt[a];
    }
    for (int64_t j = 0; j < nd; ++j) {
        for (int k = 0; k < dim; ++k) {
            double u = du[(int64_t)k * nd + j];
            double un;
            if (scheme == 2) {
                un = u + tau * (Xd[(int64_t)k * nd + j] + g[k]);
            } else if (rgd[j] > 0.0) {
                double alpha = rho_d[j] / (rgd[j] * tstop[j]), beta = 1.0 / tstop[j];
                double wn = (Xd[(int64_t)k * nd + j] - u + tau * Ad[(int64_t)k * nd + j]) /
                            (1.0 + tau * (alpha + beta));
                un = u + tau * g[k] + tau * beta * wn;
            } else {
                un = u + tau * g[k];
            }
            du[(int64_t)k * nd + j] = un;
        }
    }
    /* positions */
    for (int64_t a = 0; a < ng; ++a) {
        if (gfrozen && gfrozen[a]) continue;
        for (int k = 0; k < dim; ++k) {
            double xn = gx[(int64_t)k * ng + a] + tau * gv[(int64_t)k * ng + a];
            if (P->periodic[k]) xn = orc_wrap(xn, P->lo[k], P->hi[k]);
            gx[(int64_t)k * ng + a] = xn;
        }
    }
    for (int64_t j = 0; j < nd; ++j) {
        for (int k = 0; k < dim; ++k) {
            double xn = dx[(int64_t)k * nd + j] + tau * du[(int64_t)k * nd + j];
            if (P->periodic[k]) xn = orc_wrap(xn, P->lo[k], P->hi[k]);
            dx[(int64_t)k * nd + j] = xn;
        }
    }
    if (out) {
        size_t bg = sizeof(double) * (size_t)ng, bd = sizeof(double) * (size_t)nd;
        if (out->rho_g) memcpy(out->rho_g, rho_g, bg);
        if (out->rho_d) memcpy(out->rho_d, rho_d, bd);
        if (out->acc_g) memcpy(out->acc_g, acc, bg * dim);
        if (out->acc_scale_g) memcpy(out->acc_scale_g, ascale, bg);
        if (out->drag_g) memcpy(out->drag_g, Xg, bg * dim);
        if (out->drag_d) memcpy(out->drag_d, Xd, bd * dim);
        if (out->scale_g) memcpy(out->scale_g, Sg, bg);
        if (out->scale_d) memcpy(out->scale_d, Sd, bd);
        if (out->isph_acc_d) memcpy(out->isph_acc_d, Ad, bd * dim);
        if (out->isph_acc_scale_d) memcpy(out->isph_acc_scale_d, ASd, bd);
        if (out->isph_rho_dg) memcpy(out->isph_rho_dg, rdg, bg);
        if (out->isph_K_g) memcpy(out->isph_K_g, Kg, bg);
        if (out->isph_rho_gd) memcpy(out->isph_rho_gd, rgd, bd);
    }
done:
    free(rho_g); free(rho_d); free(acc); free(dedt); free(ascale); free(q); free(Xg); free(Xd);
    free(Sg); free(Sd); free(Ad); free(ASd); free(rdg); free(Kg); free(rgd); free(inv_t); free(inv_rho);
    free(pg); free(cg); free(pd); free(cd);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Binned dust density (the profile the differentiable rollout's loss is    */
/* taken on; the paper's test problems compare dust-density profiles,       */
/* Sec. 3). Cloud in cell on nbins[k] bins per axis over the box: a         */
/* particle's mass goes to the two bin centres that bracket it along each   */
/* axis, in proportion to its nearness (linear weights), with the product   */
/* of the per-axis weights in 2D and 3D; bin indices wrap on periodic axes  */
/* and are clamped to the end bins on walled axes. rho = mass / bin volume. */
/* ------------------------------------------------------------------------ */
int orc_dust_profile(const orc_params *P, const int32_t nbins[3], int64_t n, const double *x, double m,
                     double *rho)
{
    int64_t nb[3] = {1, 1, 1};
    double width[3] = {1.0, 1.0, 1.0};
    int64_t total = 1;
    double vol = 1.0;
    for (int k = 0; k < P->dim; ++k) {
        if (nbins[k] < 1) return ORC_E_ARG;
        nb[k] = nbins[k];
        width[k] = (P->hi[k] - P->lo[k]) / (double)nb[k];
        total *= nb[k];
        vol *= width[k];
    }
    for (int64_t b = 0; b < total; ++b) rho[b] = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        int64_t lower[3] = {0, 0, 0}, upper[3] = {0, 0, 0};
        double wl[3] = {1.0, 1.0, 1.0}, wu[3] = {0.0, 0.0, 0.0};
        int skip = 0;
        for (int k = 0; k < P->dim; ++k) {
            double xk = x[(int64_t)k * n + j];
            if (xk != xk) skip = 1;
            if (skip) break;
            /* position in units of bins, measured from the first bin centre */
            double s = (xk - P->lo[k]) / width[k] - 0.5;
            double below = floor(s);
            double frac = s - below;
            int64_t i0 = (int64_t)below, i1 = i0 + 1;
            if (P->periodic[k]) {
                i0 = ((i0 % nb[k]) + nb[k]) % nb[k];
                i1 = ((i1 % nb[k]) + nb[k]) % nb[k];
            } else {
                i0 = i0 < 0 ? 0 : (i0 > nb[k] - 1 ? nb[k] - 1 : i0);
                i1 = i1 < 0 ? 0 : (i1 > nb[k] - 1 ? nb[k] - 1 : i1);
            }
            lower[k] = i0;
            upper[k] = i1;
            wl[k] = 1.0 - frac;
            wu[k] = frac;
        }
        if (skip) continue;
        for (int cz = 0; cz < (P->dim > 2 ? 2 : 1); ++cz)
            for (int cy = 0; cy < (P->dim > 1 ? 2 : 1); ++cy)
                for (int cx = 0; cx < 2; ++cx) {
                    int64_t bx = cx ? upper[0] : lower[0];
                    int64_t by = cy ? upper[1] : lower[1];
                    int64_t bz = cz ? upper[2] : lower[2];
                    double wgt = (cx ? wu[0] : wl[0]) * (cy ? wu[1] : wl[1]) * (cz ? wu[2] : wl[2]);
                    rho[bx + nb[0] * (by + nb[1] * bz)] += m * wgt;
                }
    }
    for (int64_t b = 0; b < total; ++b) rho[b] /= vol;
    return ORC_OK;
}

/* Threads of the OpenMP loops (n >= 1); returns the number now in use. For
 * timing the oracle on one core and on all cores. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

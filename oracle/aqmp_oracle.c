/*
 * aqmp_oracle.c -- plain FP64 CPU oracle for the AQMP encoder hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code with the CUDA library.
 *
 * Everything here is the slow, obviously-correct restatement of what the
 * paper defines, in double precision, with sums taken in ascending index
 * order and no fused multiply-add (build with -ffp-contract=off so x86 and
 * Arm give identical bits):
 *
 *   - 1-D DCT-II matrix, Section 2.1, Eq. (1)-(2).
 *   - 2-D atoms as outer products of two 1-D rows, Section 2.1.
 *   - Haar atoms concatenated to the DCT atoms, Section 2.3 and Appendix A
 *     (the paper does not print the Haar construction; the standard
 *     tensor-product Haar basis is used, rows ordered scale by scale).
 *   - unravel = concatenation of the block's columns (Appendix A).
 *   - Matching Pursuit steps (a)-(d) of Section 2.2 with the stopping rule
 *     Eq. (3): stop when ||Dx - y||_2 < eps or after k steps.
 *   - Orthogonal Matching Pursuit (the solver the authors ran, Section 2.2):
 *     the same selection, with a least-squares re-fit of the support.
 *   - mp_encoder_rec, Algorithm 2: a block that misses the tolerance within
 *     its budget is replaced by its four quadrants of the ORIGINAL pixels.
 *   - mp_decoder, Algorithm 3: y = D_N x, un-ravel, place.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   eps^2 = tol^2 * b^2 on the 0-255 scale (a per-block RMSE tolerance),
 *   strict "<"; the budget counts MP steps; ties go to the lowest atom index,
 *   equality being decided to 2^-32 of the block norm (see TIE_REL);
 *   a zero correlation vector ends the pursuit; children are visited TL, TR,
 *   BL, BR and leaves are emitted in that depth-first order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------- 1-D bases */

/* Section 2.1, Eq. (1)-(2): C[k][m] = alpha_k cos(pi/N (m + 1/2) k). */
void oracle_dct_1d(int b, double *C)
{
    for (int k = 0; k < b; ++k) {
        double alpha = (k == 0) ? sqrt(1.0 / b) : sqrt(2.0 / b);
        for (int m = 0; m < b; ++m)
            C[k * b + m] = alpha * cos(M_PI / b * (m + 0.5) * k);
    }
}

/* Standard orthonormal Haar basis of length b = 2^J (Section 2.3 names the
 * Haar wavelets without printing them).  Row 0 is the scaling function
 * sqrt(1/b); then for scale j = 0..J-1 and shift t = 0..2^j-1, row 2^j + t is
 * +sqrt(2^j/b) on the first half of [t b/2^j, (t+1) b/2^j) and -sqrt(2^j/b)
 * on the second half.  Returns -1 if b is not a power of two. */
int oracle_haar_1d(int b, double *H)
{
    if (b < 1 || (b & (b - 1)) != 0) return -1;
    memset(H, 0, sizeof(double) * (size_t)b * b);
    for (int m = 0; m < b; ++m) H[m] = sqrt(1.0 / b);
    int row = 1;
    for (int scale = 1; scale < b; scale *= 2) {          /* scale = 2^j */
        int len = b / scale;                               /* support length */
        double v = sqrt((double)scale / b);
        for (int t = 0; t < scale; ++t, ++row) {
            for (int m = t * len; m < t * len + len / 2; ++m) H[row * b + m] = v;
            for (int m = t * len + len / 2; m < (t + 1) * len; ++m) H[row * b + m] = -v;
        }
    }
    return 0;
}

/* Number of atoms of dictionary `dict_id` at block side b:
 * 0 = DCT followed by Haar (2 b^2), 1 = DCT only (b^2), 2 = Haar only (b^2). */
int oracle_num_atoms(int b, int dict_id)
{
    int n = b * b;
    return dict_id == 0 ? 2 * n : n;
}

/* Dictionary D_N as an n x M matrix stored atom by atom (D[j*n + v]).
 * 2-D atom (p, q) of a family with 1-D matrix B has pixel (row i, column m)
 * equal to B[p][i] * B[q][m]; unravel concatenates columns, so that pixel sits
 * at v = m*b + i; the atom has index q*b + p inside its family; DCT atoms come
 * before Haar atoms. */
int oracle_dictionary(int b, int dict_id, double *D)
{
    int n = b * b;
    double *C = malloc(sizeof(double) * n);
    double *H = malloc(sizeof(double) * n);
    if (!C || !H) { free(C); free(H); return -2; }
    oracle_dct_1d(b, C);
    if (oracle_haar_1d(b, H) != 0) { free(C); free(H); return -1; }
    int nfam = dict_id == 0 ? 2 : 1;
    for (int f = 0; f < nfam; ++f) {
        const double *B = (dict_id == 2 || f == 1) ? H : C;
        for (int q = 0; q < b; ++q)
            for (int p = 0; p < b; ++p) {
                double *col = D + (size_t)(f * n + q * b + p) * n;
                for (int m = 0; m < b; ++m)
                    for (int i = 0; i < b; ++i)
                        col[m * b + i] = B[p * b + i] * B[q * b + m];
            }
    }
    free(C); free(H);
    return 0;
}

/* ------------------------------------------------------- Matching Pursuit */

/* Equality in finite precision.  "Ties go to the lowest atom index" is a
 * statement about exact values; two magnitudes that are equal in exact
 * arithmetic come out of any floating-point evaluation a few units of
 * rounding apart, in an order that depends on the evaluation.  So both this
 * oracle and the library treat correlations within TIE_REL * ||y|| of the
 * largest as tied (the lowest index among them wins), and an energy within
 * TIE_REL * ||y||^2 of eps^2 as equal to it (not below it: the test stays
 * strict).  TIE_REL = 2^-32 is far above either side's rounding error and
 * far below any difference that matters for the image. */
#define TIE_REL 0x1p-32

/* MP(D, y, eps, k), Section 2.2 steps (a)-(d) with the stop rule Eq. (3).
 * r^0 = y.  Before every step the residual energy E = sum r^2 is recomputed;
 * E < eps2 ends the pursuit as converged; after k steps it ends unconverged.
 * Each step computes every correlation <r, phi_j> from scratch, takes the
 * lowest index of largest magnitude, stores (j, alpha = <r, phi_j>) and sets
 * r <- r - alpha phi_j.  A step whose largest |correlation| is exactly zero
 * ends the pursuit unconverged (nothing can be removed).
 *
 * Outputs (capacity k): out_j, out_alpha, out_margin[t] = distance of the
 * nearest other atom's |c| to the tie boundary max|c| - TIE_REL ||y||
 * (atoms identical to the chosen one excluded), out_energy[t] for
 * t = 0..steps (capacity k+1).  Any output pointer may be NULL.
 * Returns the number of steps taken. */
int oracle_mp(const double *D, int n, int M, const double *y, double eps2, int k,
              int32_t *out_j, double *out_alpha, double *out_margin,
              double *out_energy, int *converged)
{
    double *r = malloc(sizeof(double) * n);
    double *c = malloc(sizeof(double) * M);
    if (!r || !c) { free(r); free(c); return -2; }
    memcpy(r, y, sizeof(double) * n);
    double S2 = 0.0;
    for (int v = 0; v < n; ++v) S2 += y[v] * y[v];
    const double tie_c = TIE_REL * sqrt(S2), tie_e = TIE_REL * S2;
    int t = 0;
    *converged = 0;
    for (;;) {
        double E = 0.0;
        for (int v = 0; v < n; ++v) E += r[v] * r[v];
        if (out_energy) out_energy[t] = E;
        if (E < eps2 - tie_e) { *converged = 1; break; }
        if (t == k) break;
        /* c[j] = <r, phi_j>, summed over ascending v.  Eight atoms are summed
         * side by side only to keep the CPU's adders busy: each c[j] is the
         * same sequence of roundings as a loop over that atom alone. */
        int j = 0;
        for (; j + 8 <= M; j += 8) {
            const double *p0 = D + (size_t)j * n;
            double s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0, s6 = 0, s7 = 0;
            for (int v = 0; v < n; ++v) {
                double rv = r[v];
                s0 += p0[v] * rv;          s1 += p0[n + v] * rv;
                s2 += p0[2 * n + v] * rv;  s3 += p0[3 * n + v] * rv;
                s4 += p0[4 * n + v] * rv;  s5 += p0[5 * n + v] * rv;
                s6 += p0[6 * n + v] * rv;  s7 += p0[7 * n + v] * rv;
            }
            c[j] = s0; c[j + 1] = s1; c[j + 2] = s2; c[j + 3] = s3;
            c[j + 4] = s4; c[j + 5] = s5; c[j + 6] = s6; c[j + 7] = s7;
        }
        for (; j < M; ++j) {
            const double *phi = D + (size_t)j * n;
            double s = 0.0;
            for (int v = 0; v < n; ++v) s += phi[v] * r[v];
            c[j] = s;
        }
        /* largest magnitude, then the lowest index tied with it */
        double cmax = 0.0;
        for (j = 0; j < M; ++j)
            if (fabs(c[j]) > cmax) cmax = fabs(c[j]);
        if (cmax == 0.0) break;
        const double edge = cmax - tie_c;
        int best = 0;
        while (fabs(c[best]) < edge) ++best;
        double alpha = c[best];
        /* decision margin: nearest other atom to the tie boundary (an atom
         * listed twice, such as the DCT DC atom and the Haar scaling atom,
         * always ties with itself and is left out) */
        const double *pb = D + (size_t)best * n;
        double margin = INFINITY;
        for (j = 0; j < M; ++j) {
            if (j == best) continue;
            double d = fabs(fabs(c[j]) - edge);
            if (d >= margin) continue;
            if (memcmp(D + (size_t)j * n, pb, sizeof(double) * n) == 0) continue;
            margin = d;
        }
        if (out_j) out_j[t] = best;
        if (out_alpha) out_alpha[t] = alpha;
        if (out_margin) out_margin[t] = margin;
        for (int v = 0; v < n; ++v) r[v] -= alpha * pb[v];
        ++t;
    }
    free(r); free(c);
    return t;
}

/* OMP(D, y, eps, k): Orthogonal Matching Pursuit, the solver the authors
 * ran (Section 2.2 names it in place of plain MP and cites the
 * scikit-learn implementation).  Selection, tie rule and stop rule are those
 * of oracle_mp; after each selection every coefficient on the support S is
 * re-fitted by least squares, x_S = argmin ||y - D_S x||, through the normal
 * equations G_SS x = D_S^T y (G_SS = D_S^T D_S), solved by a Cholesky
 * factorisation computed afresh each step; the residual r = y - D_S x_S is
 * then formed explicitly.  Readings: a new atom whose Cholesky pivot (the
 * squared norm of its part outside span(D_S)) is <= 2^-40 ends the pursuit
 * unconverged (scikit-learn also stops on linear dependence); so does a
 * residual whose largest |correlation| is <= TIE_REL ||y|| (zero to the
 * precision of the tie rule).  Outputs: the support in selection order
 * (out_j) and the final coefficients (out_alpha[t] belongs to out_j[t]),
 * per-step margins and energies as oracle_mp.  Returns |S|. */
#define PIVOT_MIN 0x1p-40

int oracle_omp(const double *D, int n, int M, const double *y, double eps2, int k,
               int32_t *out_j, double *out_alpha, double *out_margin,
               double *out_energy, int *converged)
{
    double *r = malloc(sizeof(double) * n);
    double *c = malloc(sizeof(double) * M);
    double *G = malloc(sizeof(double) * (size_t)(k + 1) * (k + 1));
    double *L = malloc(sizeof(double) * (size_t)(k + 1) * (k + 1));
    double *rhs = malloc(sizeof(double) * (k + 1));
    double *x = malloc(sizeof(double) * (k + 1));
    int32_t *S = malloc(sizeof(int32_t) * (k + 1));
    if (!r || !c || !G || !L || !rhs || !x || !S) {
        free(r); free(c); free(G); free(L); free(rhs); free(x); free(S);
        return -2;
    }
    memcpy(r, y, sizeof(double) * n);
    double S2 = 0.0;
    for (int v = 0; v < n; ++v) S2 += y[v] * y[v];
    const double tie_c = TIE_REL * sqrt(S2), tie_e = TIE_REL * S2;
    int t = 0;
    *converged = 0;
    for (;;) {
        double E = 0.0;
        for (int v = 0; v < n; ++v) E += r[v] * r[v];
        if (out_energy) out_energy[t] = E;
        if (E < eps2 - tie_e) { *converged = 1; break; }
        if (t == k) break;
        for (int j = 0; j < M; ++j) {                 /* c = D^T r */
            const double *phi = D + (size_t)j * n;
            double s = 0.0;
            for (int v = 0; v < n; ++v) s += phi[v] * r[v];
            c[j] = s;
        }
        double cmax = 0.0;
        for (int j = 0; j < M; ++j)
            if (fabs(c[j]) > cmax) cmax = fabs(c[j]);
        if (cmax <= tie_c) break;
        const double edge = cmax - tie_c;
        int best = 0;
        while (fabs(c[best]) < edge) ++best;
        const double *pb = D + (size_t)best * n;
        double margin = INFINITY;
        for (int j = 0; j < M; ++j) {
            if (j == best) continue;
            double d = fabs(fabs(c[j]) - edge);
            if (d >= margin) continue;
            if (memcmp(D + (size_t)j * n, pb, sizeof(double) * n) == 0) continue;
            margin = d;
        }
        /* normal equations of the enlarged support, factorised afresh */
        S[t] = best;
        const int m = t + 1;
        for (int a = 0; a < m; ++a) {
            const double *pa = D + (size_t)S[a] * n;
            for (int b = 0; b < m; ++b) {
                const double *pbb = D + (size_t)S[b] * n;
                double s = 0.0;
                for (int v = 0; v < n; ++v) s += pa[v] * pbb[v];
                G[a * m + b] = s;
            }
            double s = 0.0;
            for (int v = 0; v < n; ++v) s += pa[v] * y[v];
            rhs[a] = s;
        }
        int dependent = 0;
        for (int a = 0; a < m && !dependent; ++a) {   /* G = L L^T */
            for (int b = 0; b <= a; ++b) {
                double s = G[a * m + b];
                for (int q = 0; q < b; ++q) s -= L[a * m + q] * L[b * m + q];
                if (a == b) {
                    if (s <= PIVOT_MIN) { dependent = 1; break; }
                    L[a * m + a] = sqrt(s);
                } else {
                    L[a * m + b] = s / L[b * m + b];
                }
            }
        }
        if (dependent) break;
        for (int a = 0; a < m; ++a) {                 /* L z = rhs */
            double s = rhs[a];
            for (int q = 0; q < a; ++q) s -= L[a * m + q] * x[q];
            x[a] = s / L[a * m + a];
        }
        for (int a = m - 1; a >= 0; --a) {            /* L^T x = z */
            double s = x[a];
            for (int q = a + 1; q < m; ++q) s -= L[q * m + a] * x[q];
            x[a] = s / L[a * m + a];
        }
        for (int v = 0; v < n; ++v) {                 /* r = y - D_S x_S */
            double s = y[v];
            for (int a = 0; a < m; ++a) s -= x[a] * D[(size_t)S[a] * n + v];
            r[v] = s;
        }
        if (out_margin) out_margin[t] = margin;
        ++t;
    }
    for (int a = 0; a < t; ++a) {
        if (out_j) out_j[a] = S[a];
        if (out_alpha) out_alpha[a] = x[a];
    }
    free(r); free(c); free(G); free(L); free(rhs); free(x); free(S);
    return t;
}

/* ----------------------------------------------------- quadtree encoder */

typedef struct {
    int32_t plane, b, y, x;      /* block position and side */
    int32_t atom_off, n_atoms;   /* slice of the atom arrays */
    int32_t converged;
    double min_margin;           /* smallest top-2 margin over the steps */
} oracle_leaf;

typedef struct {
    const uint8_t *pix; long pitch;
    double tol; int cap_num, cap_den, min_block, dict_id, plane, alg;   /* alg: 0 MP, 1 OMP */
    double *const *dicts;        /* dicts[log2 b] */
    oracle_leaf *leaves; long n_leaves, cap_leaves;
    int32_t *atom_j; double *atom_alpha; long n_atoms, cap_atoms;
    long attempts, steps;        /* work counters (failed attempts included) */
    int err;
} enc_ctx;

static int ilog2(int b) { int l = 0; while ((1 << l) < b) ++l; return l; }

/* Algorithm 2 (mp_encoder_rec) for one block. */
static void rec(enc_ctx *c, int y0, int x0, int b)
{
    if (c->err) return;
    int n = b * b, M = oracle_num_atoms(b, c->dict_id);
    long kk = (long)n * c->cap_num / c->cap_den;
    int k = kk < 1 ? 1 : (int)kk;
    double eps2 = c->tol * c->tol * (double)n;
    const double *D = c->dicts[ilog2(b)];
    double *y = malloc(sizeof(double) * n);
    int32_t *js = malloc(sizeof(int32_t) * k);
    double *al = malloc(sizeof(double) * k);
    double *mg = malloc(sizeof(double) * k);
    if (!y || !js || !al || !mg) { c->err = -2; goto out; }
    for (int m = 0; m < b; ++m)                    /* unravel: columns */
        for (int i = 0; i < b; ++i)
            y[m * b + i] = (double)c->pix[(long)(y0 + i) * c->pitch + x0 + m];
    int conv = 0;
    int steps = c->alg ? oracle_omp(D, n, M, y, eps2, k, js, al, mg, NULL, &conv)
                       : oracle_mp(D, n, M, y, eps2, k, js, al, mg, NULL, &conv);
    if (steps < 0) { c->err = steps; goto out; }
    c->attempts += 1;
    c->steps += steps;
    if (!conv && b > c->min_block) {               /* split: original pixels */
        int h = b / 2;
        rec(c, y0, x0, h);
        rec(c, y0, x0 + h, h);
        rec(c, y0 + h, x0, h);
        rec(c, y0 + h, x0 + h, h);
    } else {
        if (c->n_leaves >= c->cap_leaves || c->n_atoms + steps > c->cap_atoms) { c->err = -3; goto out; }
        oracle_leaf *L = &c->leaves[c->n_leaves++];
        L->plane = c->plane; L->b = b; L->y = y0; L->x = x0;
        L->atom_off = (int32_t)c->n_atoms; L->n_atoms = steps; L->converged = conv;
        double mm = INFINITY;
        for (int t = 0; t < steps; ++t) {
            c->atom_j[c->n_atoms + t] = js[t];
            c->atom_alpha[c->n_atoms + t] = al[t];
            if (mg[t] < mm) mm = mg[t];
        }
        L->min_margin = mm;
        c->n_atoms += steps;
    }
out:
    free(y); free(js); free(al); free(mg);
}

/* Encode the root blocks [root_begin, root_end) of one plane (roots in
 * row-major order, side max_block).  `dicts[l]` must hold the dictionary for
 * side 2^l for every side between min_block and max_block.  Leaves are
 * written depth-first (TL, TR, BL, BR).  Returns 0, or -1 on bad arguments,
 * -2 on allocation failure, -3 when an output capacity is too small. */
int oracle_encode_roots(const uint8_t *pix, long pitch, int h, int w, int plane,
                        double tol, int cap_num, int cap_den, int min_block,
                        int max_block, int dict_id, double *const *dicts,
                        long root_begin, long root_end,
                        oracle_leaf *leaves, long cap_leaves, long *n_leaves,
                        int32_t *atom_j, double *atom_alpha, long cap_atoms,
                        long *n_atoms, long *attempts, long *steps, int alg)
{
    if (max_block < min_block || h % max_block || w % max_block || cap_den <= 0)
        return -1;
    enc_ctx c = {pix, pitch, tol, cap_num, cap_den, min_block, dict_id, plane, alg, dicts,
                 leaves, 0, cap_leaves, atom_j, atom_alpha, 0, cap_atoms, 0, 0, 0};
    long roots_x = w / max_block;
    for (long r = root_begin; r < root_end && !c.err; ++r)
        rec(&c, (int)(r / roots_x) * max_block, (int)(r % roots_x) * max_block, max_block);
    *n_leaves = c.n_leaves; *n_atoms = c.n_atoms;
    if (attempts) *attempts = c.attempts;
    if (steps) *steps = c.steps;
    return c.err;
}

/* ------------------------------------------------------------- decoder */

/* Algorithm 3 (mp_decoder) for one leaf: y = D_N x, un-ravel, place into
 * out (row-major, pitch in elements).  Atoms selected twice add up. */
void oracle_decode_leaf(const double *D, int b, int y0, int x0,
                        const int32_t *atom_j, const double *atom_alpha, int n_atoms,
                        double *out, long pitch)
{
    int n = b * b;
    for (int m = 0; m < b; ++m)
        for (int i = 0; i < b; ++i) {
            double s = 0.0;
            for (int t = 0; t < n_atoms; ++t)
                s += atom_alpha[t] * D[(size_t)atom_j[t] * n + m * b + i];
            out[(long)(y0 + i) * pitch + x0 + m] = s;
        }
}

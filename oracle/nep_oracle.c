/*
 * FP64 CPU oracle for the NEP energy, forces, virials and the E/F/W loss gradient.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow statement of what the
 * hot path computes.  Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it; the product library never links or calls it.
 * It shares no code, header or table with the CUDA sources.
 *
 * What it follows (TorchNEP paper, arXiv 2606.19557):
 *   Eq. 1          E = sum_i E_i
 *   Eq. "norm"     q~_nu = q_nu / (q_nu^max - q_nu^min)   (scale vector is an input)
 *   Eq. "ann"      E_i = sum_mu w1_{t,mu} tanh(sum_nu w0_{t,mu,nu} q~_nu - b0_{t,mu}) - b1
 *   Eq. "loss"     L = lE*DE + lF*DF + lV*DV with the per-atom-normalised MSE terms
 *   Methods, "NEP descriptors":
 *                  q_n = sum_j g_n(r_ij),  g_n = sum_k c^{ti tj}_{nk} f_k(r_ij)
 *                  f_k = 1/2 (T_k(2 (r/rc - 1)^2 - 1) + 1) f_c(r),
 *                  f_c = 1/2 (cos(pi r / rc) + 1) for r <= rc, else 0
 *                  A_nlm = sum_j g^A_n(r_ij) Y_lm(r^_ij),  q_nl = sum_m A_nlm^2  (Eq. "q3b")
 *                  higher-body terms: "higher-order contractions" of A (forms not printed).
 *
 * Readings where the paper is silent (also listed in the design notes):
 *   - Y_lm are the orthonormal REAL spherical harmonics, l = 1..l_max.
 *   - 4-body (one per n, from the l = 2 moments):
 *       q4_n = sum_{m1+m2+m3=0} (2 2 2; m1 m2 m3) A_{n2m1} A_{n2m2} A_{n2m3}
 *     with complex orthonormal harmonics.  The cubic invariant of one l = 2 irrep is
 *     unique up to scale, so it is computed here in Cartesian form as
 *       q4_n = KAPPA * tr(M_n^3),  M_n = sum_j g^A_n(r_ij) (r^ r^T - I/3),
 *     KAPPA = -(9/2) sqrt(2/35) (5/(4 pi))^{3/2}   (fixed by one bond along z).
 *   - 5-body (one per n, from the l = 1 moments): q5_n = (sum_m A_{n1m}^2)^2.
 *   - Virial W = -dE/d(eps) under r -> (I + eps) r for positions and cell, i.e.
 *     W_ab = -sum_pairs G_a d_b with G = dE_i/d(d_ij) and d_ij = r_j + S.h - r_i.
 *   - Pair inclusion: d is formed as ((double)r_j - (double)r_i) + S.h in double
 *     (fixed order, no fused multiply-add), rounded once to float, and the pair
 *     is kept iff the float dot product d.d < rc*rc (float).  This integer
 *     decision is taken in the GPU kernel's precision; the physics below then
 *     uses the unrounded double displacement.
 *
 * Derivatives: F = -dE/dr and W come from hand-written reverse mode over the
 * per-pair Jacobians dq/dd, which are themselves obtained with 3-component
 * forward-mode dual numbers.  The parameter gradient of the loss is the
 * gradient of  J = sum_s eb_s E_s + sum_i fb_i.F_i + sum_s Wb_s:W_s  with the
 * loss cotangents (eb, fb, Wb) held fixed.  The force/virial part equals
 * sum_i e_i . (s * dq_i), dq_i being the derivative of q_i along the pair
 * displacements lambda_p = fb_i - fb_j - Wb d_p; q and dq are linear (radial)
 * or polynomial (angular) in the c coefficients, so their c-derivatives are
 * sums of per-(species, k) moments.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int n_types;
    double rc_R, rc_A;
    int n_max_R, n_max_A, basis_R, basis_A;
    int l_max, has_4b, has_5b;
    int n_neu;
    /* optional ZBL short-range term (zbl != 0): switch from zbl_r1 to zbl_r2, atomic
     * numbers of the species */
    int zbl;
    double zbl_r1, zbl_r2;
    double zbl_Z[16];
} orc_cfg;

/* ------------------------------------------------------------------ sizes */
typedef struct {
    int T, NR, KR, NA, KA, L, L3, H4, H5, NN, ND;
    int64_t o_w0, o_b0, o_w1, o_b1, o_cR, o_cA, P;
} sizes;

static sizes get_sizes(const orc_cfg *c) {
    sizes s;
    s.T = c->n_types;
    s.NR = c->n_max_R + 1;
    s.KR = c->basis_R + 1;
    s.NA = c->n_max_A + 1;
    s.KA = c->basis_A + 1;
    s.L = c->l_max;
    s.L3 = s.L * (s.L + 2);
    s.H4 = c->has_4b ? 1 : 0;
    s.H5 = c->has_5b ? 1 : 0;
    s.NN = c->n_neu;
    s.ND = s.NR + s.NA * (s.L + s.H4 + s.H5);
    s.o_w0 = 0;
    s.o_b0 = s.o_w0 + (int64_t)s.T * s.NN * s.ND;
    s.o_w1 = s.o_b0 + (int64_t)s.T * s.NN;
    s.o_b1 = s.o_w1 + (int64_t)s.T * s.NN;
    s.o_cR = s.o_b1 + 1;
    s.o_cA = s.o_cR + (int64_t)s.T * s.T * s.NR * s.KR;
    s.P = s.o_cA + (int64_t)s.T * s.T * s.NA * s.KA;
    return s;
}

int64_t orc_num_params(const orc_cfg *c) { return get_sizes(c).P; }
int orc_num_descriptors(const orc_cfg *c) { return get_sizes(c).ND; }

static int cfg_ok(const orc_cfg *c) {
    if (c->n_types < 1 || c->n_max_R < 0 || c->n_max_A < 0 || c->basis_R < 0 || c->basis_A < 0) return 0;
    if (c->zbl) {
        if (c->n_types > 16 || !(c->zbl_r1 >= 0) || !(c->zbl_r2 > c->zbl_r1) || c->zbl_r2 > c->rc_R) return 0;
        for (int t = 0; t < c->n_types; t++) if (!(c->zbl_Z[t] > 0)) return 0;
    }
    if (c->l_max < 0 || c->l_max > 4 || c->n_neu < 1) return 0;
    if (c->has_4b && c->l_max < 2) return 0;
    if (c->has_5b && c->l_max < 1) return 0;
    if (!(c->rc_R > 0) || !(c->rc_A > 0) || c->rc_A > c->rc_R) return 0;
    return 1;
}

/* ------------------------------------------------ dual numbers over d (R^3) */
typedef struct { double v, g[3]; } dl;

static dl D(double c) { dl r = {c, {0.0, 0.0, 0.0}}; return r; }
static dl add(dl a, dl b) { dl r; r.v = a.v + b.v; for (int k = 0; k < 3; k++) r.g[k] = a.g[k] + b.g[k]; return r; }
static dl sub(dl a, dl b) { dl r; r.v = a.v - b.v; for (int k = 0; k < 3; k++) r.g[k] = a.g[k] - b.g[k]; return r; }
static dl mul(dl a, dl b) {
    dl r; r.v = a.v * b.v;
    for (int k = 0; k < 3; k++) r.g[k] = a.g[k] * b.v + a.v * b.g[k];
    return r;
}
static dl scl(dl a, double s) { dl r; r.v = a.v * s; for (int k = 0; k < 3; k++) r.g[k] = a.g[k] * s; return r; }
static dl dsqrt(dl a) { dl r; r.v = sqrt(a.v); for (int k = 0; k < 3; k++) r.g[k] = a.g[k] / (2.0 * r.v); return r; }
static dl dcos(dl a) { dl r; r.v = cos(a.v); double s = -sin(a.v); for (int k = 0; k < 3; k++) r.g[k] = s * a.g[k]; return r; }
static dl ddiv(dl a, dl b) {
    dl r; r.v = a.v / b.v;
    for (int k = 0; k < 3; k++) r.g[k] = (a.g[k] * b.v - a.v * b.g[k]) / (b.v * b.v);
    return r;
}
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ------------------------------------------------------- basis functions
 * Methods, "NEP descriptors": f_k(r) = 1/2 (T_k[2 (r/rc - 1)^2 - 1] + 1) f_c(r),
 * f_c(r) = 1/2 [cos(pi r / rc) + 1] for r <= rc and 0 beyond, k = 0..N_bas.
 * T_k are Chebyshev polynomials of the first kind: T_0 = 1, T_1 = x,
 * T_{k+1} = 2 x T_k - T_{k-1}. */
static void basis(dl r, double rc, int K, dl *f) {
    dl fc = (r.v <= rc) ? scl(add(dcos(scl(r, M_PI / rc)), D(1.0)), 0.5) : D(0.0);
    dl y = sub(scl(r, 1.0 / rc), D(1.0));
    dl x = sub(scl(mul(y, y), 2.0), D(1.0));
    dl tm1 = D(1.0), t = x;
    for (int k = 0; k < K; k++) {
        dl Tk;
        if (k == 0) Tk = D(1.0);
        else if (k == 1) Tk = x;
        else {
            dl tn = sub(scl(mul(x, t), 2.0), tm1);
            tm1 = t;
            t = tn;
            Tk = tn;
        }
        f[k] = mul(scl(add(Tk, D(1.0)), 0.5), fc);
    }
}

/* ------------------------------------------------- real spherical harmonics
 * Orthonormal real harmonics of the unit vector u, l = 1..lmax, stored at
 * index (l*l - 1) + (m + l).  Built from C_m + i S_m = (x + i y)^m and the
 * associated-Legendre polynomials Pi_l^m(z) = d^m P_l / dz^m (no Condon-Shortley
 * phase), which obey Pi_m^m = (2m-1)!!, Pi_{m+1}^m = (2m+1) z Pi_m^m and
 * (l-m) Pi_l^m = (2l-1) z Pi_{l-1}^m - (l+m-1) Pi_{l-2}^m on the unit sphere.
 * Y_l0 = sqrt((2l+1)/(4 pi)) Pi_l^0,
 * Y_{l,+-m} = sqrt(2 (2l+1)/(4 pi) (l-m)!/(l+m)!) Pi_l^m {C_m, S_m}. */
static double factorial(int n) { double f = 1.0; for (int i = 2; i <= n; i++) f *= i; return f; }

static void real_ylm(dl ux, dl uy, dl uz, int lmax, dl *Y) {
    dl C[5], S[5], Pi[5][5];
    C[0] = D(1.0);
    S[0] = D(0.0);
    for (int m = 1; m <= lmax; m++) {
        C[m] = sub(mul(ux, C[m - 1]), mul(uy, S[m - 1]));
        S[m] = add(mul(ux, S[m - 1]), mul(uy, C[m - 1]));
    }
    for (int m = 0; m <= lmax; m++) {
        double df = 1.0;
        for (int i = 2 * m - 1; i > 1; i -= 2) df *= i;
        Pi[m][m] = D(df);
        if (m + 1 <= lmax) Pi[m + 1][m] = scl(mul(uz, Pi[m][m]), 2.0 * m + 1.0);
        for (int l = m + 2; l <= lmax; l++)
            Pi[l][m] = scl(sub(scl(mul(uz, Pi[l - 1][m]), 2.0 * l - 1.0), scl(Pi[l - 2][m], l + m - 1.0)),
                           1.0 / (l - m));
    }
    for (int l = 1; l <= lmax; l++) {
        int base = l * l - 1 + l;
        Y[base] = scl(Pi[l][0], sqrt((2.0 * l + 1.0) / (4.0 * M_PI)));
        for (int m = 1; m <= l; m++) {
            double nrm = sqrt(2.0 * (2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - m) / factorial(l + m));
            Y[base + m] = scl(mul(Pi[l][m], C[m]), nrm);
            Y[base - m] = scl(mul(Pi[l][m], S[m]), nrm);
        }
    }
}

/* 4-body scale (reading of "higher-order contractions", see header). */
static double kappa4(void) { return -4.5 * sqrt(2.0 / 35.0) * pow(5.0 / (4.0 * M_PI), 1.5); }

static void mat_mul3(const double *a, const double *b, double *c) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += a[3 * i + k] * b[3 * k + j];
            c[3 * i + j] = s;
        }
}
static double tr_mul(const double *a, const double *b) {  /* tr(A B) */
    double s = 0.0;
    for (int i = 0; i < 3; i++)
        for (int k = 0; k < 3; k++) s += a[3 * i + k] * b[3 * k + i];
    return s;
}

/* ------------------------------------------------------------- pair list */
typedef struct {
    int i, j;
    int S[3];
    double d[3];
    int ang;
} opair;

/* Displacement and inclusion predicate of the pair list.  The decision uses the
 * positions and cell rounded to float (the precision the GPU kernel receives),
 * d = ((double)r_j - (double)r_i) + S.h in double without fused multiply-add,
 * rounded once to float, kept iff the float sum (dx*dx + dy*dy) + dz*dz < rc*rc.
 * d64 returns the displacement of the unrounded double inputs for the physics. */
static float pair_geometry(const double *pi, const double *pj, const double *h, int Sa, int Sb, int Sc,
                           double *d64) {
    float d32[3];
    for (int x = 0; x < 3; x++) {
        double rel = (double)(float)pj[x] - (double)(float)pi[x];
        double sh = ((double)Sa * (double)(float)h[x] + (double)Sb * (double)(float)h[3 + x]) +
                    (double)Sc * (double)(float)h[6 + x];
        d32[x] = (float)(rel + sh);
        d64[x] = (pj[x] - pi[x]) + ((Sa * h[x] + Sb * h[3 + x]) + Sc * h[6 + x]);
    }
    float xx = d32[0] * d32[0];
    float yy = d32[1] * d32[1];
    float zz = d32[2] * d32[2];
    return (xx + yy) + zz;
}

static int cell_geometry(const double *hf, double *inv, double *width) {
    double h[9];
    for (int k = 0; k < 9; k++) h[k] = hf[k];
    double c0[3] = {h[4] * h[8] - h[5] * h[7], h[5] * h[6] - h[3] * h[8], h[3] * h[7] - h[4] * h[6]}; /* b x c */
    double c1[3] = {h[7] * h[2] - h[8] * h[1], h[8] * h[0] - h[6] * h[2], h[6] * h[1] - h[7] * h[0]}; /* c x a */
    double c2[3] = {h[1] * h[5] - h[2] * h[4], h[2] * h[3] - h[0] * h[5], h[0] * h[4] - h[1] * h[3]}; /* a x b */
    double vol = h[0] * c0[0] + h[1] * c0[1] + h[2] * c0[2];
    if (!(fabs(vol) > 1e-12) || !isfinite(vol)) return 0;
    /* inverse of the row-vector cell: f = r h^-1, columns of h^-1 are (b x c)/V etc. */
    for (int x = 0; x < 3; x++) {
        inv[3 * x + 0] = c0[x] / vol;
        inv[3 * x + 1] = c1[x] / vol;
        inv[3 * x + 2] = c2[x] / vol;
    }
    width[0] = fabs(vol) / sqrt(dot3(c0, c0));
    width[1] = fabs(vol) / sqrt(dot3(c1, c1));
    width[2] = fabs(vol) / sqrt(dot3(c2, c2));
    return 1;
}

/* Brute-force enumeration of all (i, j, S) with d.d < rc^2 (float predicate),
 * j = i allowed for S != 0.  Returns the number of pairs (or -1 on a bad
 * cell); writes at most cap pairs. */
static int64_t brute_pairs(int n, const double *pos, const double *cell, float rcR, float rcA,
                           opair *out, int64_t cap) {
    double inv[9], w[3];
    if (!cell_geometry(cell, inv, w)) return -1;
    double fmin[3] = {1e300, 1e300, 1e300}, fmax[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < n; i++)
        for (int a = 0; a < 3; a++) {
            double f = 0.0;
            for (int x = 0; x < 3; x++) f += (double)pos[3 * i + x] * inv[3 * x + a];
            if (f < fmin[a]) fmin[a] = f;
            if (f > fmax[a]) fmax[a] = f;
        }
    int M[3];
    for (int a = 0; a < 3; a++) {
        double span = n > 0 ? fmax[a] - fmin[a] : 0.0;
        /* |f_j - f_i + S_a| <= rc / w_a is needed for |d| < rc, and |f_j - f_i| <= span */
        M[a] = (int)ceil((double)rcR / w[a] + span + 1e-9);
    }
    float rc2R = rcR * rcR, rc2A = rcA * rcA;
    int64_t cnt = 0;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int Sa = -M[0]; Sa <= M[0]; Sa++)
                for (int Sb = -M[1]; Sb <= M[1]; Sb++)
                    for (int Sc = -M[2]; Sc <= M[2]; Sc++) {
                        if (i == j && Sa == 0 && Sb == 0 && Sc == 0) continue;
                        double d64[3];
                        float r2 = pair_geometry(pos + 3 * i, pos + 3 * j, cell, Sa, Sb, Sc, d64);
                        if (!(r2 < rc2R)) continue;
                        if (cnt < cap && out) {
                            opair *p = out + cnt;
                            p->i = i;
                            p->j = j;
                            p->S[0] = Sa;
                            p->S[1] = Sb;
                            p->S[2] = Sc;
                            p->d[0] = d64[0];
                            p->d[1] = d64[1];
                            p->d[2] = d64[2];
                            p->ang = (r2 < rc2A) ? 1 : 0;
                        }
                        cnt++;
                    }
    return cnt;
}

/* Public brute-force neighbour list (bit-exact reference for the GPU cell list).
 * For every structure: all pairs with float d.d < rc_R^2; ang[p] = (d.d < rc_A^2).
 * Output atom indices are global (atom_off[s] + local).  Returns the total count,
 * -1 on a degenerate cell; writes at most cap entries. */
int64_t orc_neighbors(int64_t n_struct, const int64_t *atom_off, const double *pos, const double *cell,
                      float rc_R, float rc_A, int64_t cap, int64_t *out_i, int64_t *out_j, int32_t *out_S,
                      uint8_t *out_ang) {
    int64_t total = 0;
    for (int64_t s = 0; s < n_struct; s++) {
        int n = (int)(atom_off[s + 1] - atom_off[s]);
        const double *ps = pos + 3 * atom_off[s];
        int64_t c = brute_pairs(n, ps, cell + 9 * s, rc_R, rc_A, NULL, 0);
        if (c < 0) return -1;
        opair *buf = (opair *)malloc(sizeof(opair) * (size_t)(c > 0 ? c : 1));
        brute_pairs(n, ps, cell + 9 * s, rc_R, rc_A, buf, c);
        for (int64_t k = 0; k < c; k++) {
            int64_t o = total + k;
            if (o < cap) {
                out_i[o] = atom_off[s] + buf[k].i;
                out_j[o] = atom_off[s] + buf[k].j;
                out_S[3 * o + 0] = buf[k].S[0];
                out_S[3 * o + 1] = buf[k].S[1];
                out_S[3 * o + 2] = buf[k].S[2];
                out_ang[o] = (uint8_t)buf[k].ang;
            }
        }
        free(buf);
        total += c;
    }
    return total;
}

/* ------------------------------------------------------ per-atom workspace */
typedef struct {
    int cap;        /* pairs it can hold */
    dl *fR, *fA;    /* [p][K] */
    dl *gA;         /* [p][NA] */
    dl *Y;          /* [p][L3] */
    dl *Qm;         /* [p][9] */
    double *J;      /* [ND][p][3] Jacobian dq/dd_p */
    double *q, *qt, *e, *h, *A, *M;
} work;

static void work_alloc(work *w, const sizes *z, int cap) {
    w->cap = cap;
    w->fR = (dl *)calloc((size_t)cap * z->KR + 1, sizeof(dl));
    w->fA = (dl *)calloc((size_t)cap * z->KA + 1, sizeof(dl));
    w->gA = (dl *)calloc((size_t)cap * z->NA + 1, sizeof(dl));
    w->Y = (dl *)calloc((size_t)cap * 24 + 1, sizeof(dl));
    w->Qm = (dl *)calloc((size_t)cap * 9 + 1, sizeof(dl));
    w->J = (double *)calloc((size_t)z->ND * cap * 3 + 1, sizeof(double));
    w->q = (double *)calloc(z->ND, sizeof(double));
    w->qt = (double *)calloc(z->ND, sizeof(double));
    w->e = (double *)calloc(z->ND, sizeof(double));
    w->h = (double *)calloc(z->NN, sizeof(double));
    w->A = (double *)calloc((size_t)z->NA * 24 + 1, sizeof(double));
    w->M = (double *)calloc((size_t)z->NA * 9 + 1, sizeof(double));
}
static void work_free(work *w) {
    free(w->fR); free(w->fA); free(w->gA); free(w->Y); free(w->Qm); free(w->J);
    free(w->q); free(w->qt); free(w->e); free(w->h); free(w->A); free(w->M);
}

static int idx3(const sizes *z, int n, int l) { return z->NR + (l - 1) * z->NA + n; }
static int idx4(const sizes *z, int n) { return z->NR + z->L * z->NA + n; }
static int idx5(const sizes *z, int n) { return z->NR + (z->L + z->H4) * z->NA + n; }

/* Forward pass of one atom: descriptors (Methods), ANN (Eq. "ann"), e = dE_i/dq~,
 * and the Jacobian dq_nu/dd_p for each of its pairs.  Returns E_i. */
static double atom_forward(const orc_cfg *cfg, const sizes *z, const double *th, const double *qs,
                           int ti, const int32_t *type_s, const opair *pr, int np, work *w) {
    const double *cR = th + z->o_cR, *cA = th + z->o_cA;
    const int L3 = z->L3;
    memset(w->q, 0, sizeof(double) * z->ND);
    memset(w->A, 0, sizeof(double) * z->NA * 24);
    memset(w->M, 0, sizeof(double) * z->NA * 9);
    /* per-pair functions of d */
    for (int p = 0; p < np; p++) {
        dl dx = {pr[p].d[0], {1.0, 0.0, 0.0}};
        dl dy = {pr[p].d[1], {0.0, 1.0, 0.0}};
        dl dz = {pr[p].d[2], {0.0, 0.0, 1.0}};
        dl r = dsqrt(add(add(mul(dx, dx), mul(dy, dy)), mul(dz, dz)));
        int tj = type_s[pr[p].j];
        basis(r, cfg->rc_R, z->KR, w->fR + (size_t)p * z->KR);
        /* radial descriptor q_n = sum_j g_n(r_ij) */
        for (int n = 0; n < z->NR; n++) {
            double g = 0.0;
            for (int k = 0; k < z->KR; k++)
                g += cR[(((size_t)ti * z->T + tj) * z->NR + n) * z->KR + k] * w->fR[(size_t)p * z->KR + k].v;
            w->q[n] += g;
        }
        if (!pr[p].ang) continue;
        basis(r, cfg->rc_A, z->KA, w->fA + (size_t)p * z->KA);
        dl ux = ddiv(dx, r), uy = ddiv(dy, r), uz = ddiv(dz, r);
        dl *Y = w->Y + (size_t)p * 24;
        if (z->L > 0) real_ylm(ux, uy, uz, z->L, Y);
        dl u[3] = {ux, uy, uz};
        dl *Q = w->Qm + (size_t)p * 9;
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) Q[3 * a + b] = sub(mul(u[a], u[b]), D(a == b ? 1.0 / 3.0 : 0.0));
        for (int n = 0; n < z->NA; n++) {
            dl g = D(0.0);
            for (int k = 0; k < z->KA; k++)
                g = add(g, scl(w->fA[(size_t)p * z->KA + k],
                               cA[(((size_t)ti * z->T + tj) * z->NA + n) * z->KA + k]));
            w->gA[(size_t)p * z->NA + n] = g;
            for (int lm = 0; lm < L3; lm++) w->A[n * 24 + lm] += g.v * Y[lm].v;
            for (int ab = 0; ab < 9; ab++) w->M[n * 9 + ab] += g.v * Q[ab].v;
        }
    }
    /* angular invariants */
    double kap = kappa4();
    for (int n = 0; n < z->NA; n++) {
        for (int l = 1; l <= z->L; l++) {
            double s = 0.0;
            for (int m = -l; m <= l; m++) {
                double a = w->A[n * 24 + l * l - 1 + m + l];
                s += a * a;
            }
            w->q[idx3(z, n, l)] = s;
        }
        if (z->H4) {
            double M2[9], M3[9];
            mat_mul3(w->M + n * 9, w->M + n * 9, M2);
            mat_mul3(M2, w->M + n * 9, M3);
            w->q[idx4(z, n)] = kap * (M3[0] + M3[4] + M3[8]);
        }
        if (z->H5) {
            double q1 = w->q[idx3(z, n, 1)];
            w->q[idx5(z, n)] = q1 * q1;
        }
    }
    /* network, Eq. "ann" */
    const double *w0 = th + z->o_w0 + (size_t)ti * z->NN * z->ND;
    const double *b0 = th + z->o_b0 + (size_t)ti * z->NN;
    const double *w1 = th + z->o_w1 + (size_t)ti * z->NN;
    double b1 = th[z->o_b1];
    for (int v = 0; v < z->ND; v++) w->qt[v] = w->q[v] * qs[v];
    double Ei = -b1;
    for (int v = 0; v < z->ND; v++) w->e[v] = 0.0;
    for (int mu = 0; mu < z->NN; mu++) {
        double zz = -b0[mu];
        for (int v = 0; v < z->ND; v++) zz += w0[(size_t)mu * z->ND + v] * w->qt[v];
        double hh = tanh(zz);
        w->h[mu] = hh;
        Ei += w1[mu] * hh;
        double hp = 1.0 - hh * hh;
        for (int v = 0; v < z->ND; v++) w->e[v] += w1[mu] * hp * w0[(size_t)mu * z->ND + v];
    }
    /* Jacobian dq_nu / dd_p */
    memset(w->J, 0, sizeof(double) * (size_t)z->ND * np * 3);
    for (int p = 0; p < np; p++) {
        int tj = type_s[pr[p].j];
        for (int n = 0; n < z->NR; n++) {
            double g3[3] = {0.0, 0.0, 0.0};
            for (int k = 0; k < z->KR; k++) {
                double c = cR[(((size_t)ti * z->T + tj) * z->NR + n) * z->KR + k];
                for (int a = 0; a < 3; a++) g3[a] += c * w->fR[(size_t)p * z->KR + k].g[a];
            }
            for (int a = 0; a < 3; a++) w->J[((size_t)n * np + p) * 3 + a] = g3[a];
        }
        if (!pr[p].ang) continue;
        const dl *Y = w->Y + (size_t)p * 24;
        const dl *Q = w->Qm + (size_t)p * 9;
        for (int n = 0; n < z->NA; n++) {
            dl g = w->gA[(size_t)p * z->NA + n];
            for (int l = 1; l <= z->L; l++) {
                double j3[3] = {0.0, 0.0, 0.0};
                for (int m = -l; m <= l; m++) {
                    int lm = l * l - 1 + m + l;
                    dl gy = mul(g, Y[lm]);
                    for (int a = 0; a < 3; a++) j3[a] += 2.0 * w->A[n * 24 + lm] * gy.g[a];
                }
                for (int a = 0; a < 3; a++) w->J[((size_t)idx3(z, n, l) * np + p) * 3 + a] = j3[a];
            }
            if (z->H4) {
                double M2[9];
                mat_mul3(w->M + n * 9, w->M + n * 9, M2);
                for (int a = 0; a < 3; a++) {
                    double dM[9];
                    for (int ab = 0; ab < 9; ab++) dM[ab] = mul(g, Q[ab]).g[a];
                    w->J[((size_t)idx4(z, n) * np + p) * 3 + a] = 3.0 * kap * tr_mul(M2, dM);
                }
            }
            if (z->H5) {
                double q1 = w->q[idx3(z, n, 1)];
                for (int a = 0; a < 3; a++)
                    w->J[((size_t)idx5(z, n) * np + p) * 3 + a] =
                        2.0 * q1 * w->J[((size_t)idx3(z, n, 1) * np + p) * 3 + a];
            }
        }
    }
    return Ei;
}

/* G_p = dE_i/dd_p = sum_nu e_nu s_nu dq_nu/dd_p */
static void pair_gradient(const sizes *z, const double *qs, const work *w, int np, int p, double *G) {
    G[0] = G[1] = G[2] = 0.0;
    for (int v = 0; v < z->ND; v++) {
        double c = w->e[v] * qs[v];
        for (int a = 0; a < 3; a++) G[a] += c * w->J[((size_t)v * np + p) * 3 + a];
    }
}

/* ------------------------------------------------------- adjoint of one atom
 * Adds to grad the theta-derivative of  J_i = eb * E_i + e_i . (s * dq_i)
 * where dq_i = sum_p (dq/dd_p) lambda_p.  Requires atom_forward first. */
static void atom_adjoint(const orc_cfg *cfg, const sizes *z, const double *th, const double *qs,
                         int ti, const int32_t *type_s, const opair *pr, int np, work *w,
                         const double *lam /*[np][3]*/, double eb, double *grad) {
    (void)cfg;
    const double *cR = th + z->o_cR, *cA = th + z->o_cA;
    const int ND = z->ND, NN = z->NN, T = z->T;
    double *dq = (double *)calloc(ND, sizeof(double));
    double *dqt = (double *)calloc(ND, sizeof(double));
    double *abar = (double *)calloc(ND, sizeof(double));  /* dJ/dq */
    double *bbar = (double *)calloc(ND, sizeof(double));  /* dJ/d(dq) */
    for (int v = 0; v < ND; v++) {
        double s = 0.0;
        for (int p = 0; p < np; p++) s += dot3(w->J + ((size_t)v * np + p) * 3, lam + 3 * p);
        dq[v] = s;
        dqt[v] = s * qs[v];
    }
    /* reverse through the network */
    const double *w0 = th + z->o_w0 + (size_t)ti * NN * ND;
    const double *w1 = th + z->o_w1 + (size_t)ti * NN;
    double *gw0 = grad + z->o_w0 + (size_t)ti * NN * ND;
    double *gb0 = grad + z->o_b0 + (size_t)ti * NN;
    double *gw1 = grad + z->o_w1 + (size_t)ti * NN;
    grad[z->o_b1] += -eb;
    double *zeta = (double *)calloc(NN, sizeof(double));
    for (int mu = 0; mu < NN; mu++) {
        double hh = w->h[mu];
        double hp = 1.0 - hh * hh;
        double hpp = -2.0 * hh * hp;
        double vv = 0.0;
        for (int v = 0; v < ND; v++) vv += w0[(size_t)mu * ND + v] * dqt[v];
        gw1[mu] += eb * hh + hp * vv;
        double ze = eb * w1[mu] * hp + w1[mu] * hpp * vv;
        double uu = w1[mu] * hp;
        zeta[mu] = ze;
        gb0[mu] += -ze;
        for (int v = 0; v < ND; v++) gw0[(size_t)mu * ND + v] += ze * w->qt[v] + uu * dqt[v];
    }
    for (int v = 0; v < ND; v++) {
        double s = 0.0;
        for (int mu = 0; mu < NN; mu++) s += zeta[mu] * w0[(size_t)mu * ND + v];
        abar[v] = s * qs[v];
        bbar[v] = w->e[v] * qs[v];
    }
    /* moments per neighbour species b and basis index k */
    const int KR = z->KR, KA = z->KA, NR = z->NR, NA = z->NA, L3 = z->L3;
    double *R = (double *)calloc((size_t)T * KR, sizeof(double));
    double *dR = (double *)calloc((size_t)T * KR, sizeof(double));
    double *Am = (double *)calloc((size_t)T * KA * 24 + 1, sizeof(double));
    double *dAm = (double *)calloc((size_t)T * KA * 24 + 1, sizeof(double));
    double *Mm = (double *)calloc((size_t)T * KA * 9 + 1, sizeof(double));
    double *dMm = (double *)calloc((size_t)T * KA * 9 + 1, sizeof(double));
    double *dA = (double *)calloc((size_t)NA * 24 + 1, sizeof(double));
    double *dM = (double *)calloc((size_t)NA * 9 + 1, sizeof(double));
    for (int p = 0; p < np; p++) {
        int tj = type_s[pr[p].j];
        const double *lp = lam + 3 * p;
        for (int k = 0; k < KR; k++) {
            dl f = w->fR[(size_t)p * KR + k];
            R[tj * KR + k] += f.v;
            dR[tj * KR + k] += dot3(f.g, lp);
        }
        if (!pr[p].ang) continue;
        const dl *Y = w->Y + (size_t)p * 24;
        const dl *Q = w->Qm + (size_t)p * 9;
        for (int k = 0; k < KA; k++) {
            dl f = w->fA[(size_t)p * KA + k];
            for (int lm = 0; lm < L3; lm++) {
                dl fy = mul(f, Y[lm]);
                Am[((size_t)tj * KA + k) * 24 + lm] += fy.v;
                dAm[((size_t)tj * KA + k) * 24 + lm] += dot3(fy.g, lp);
            }
            for (int ab = 0; ab < 9; ab++) {
                dl fq = mul(f, Q[ab]);
                Mm[((size_t)tj * KA + k) * 9 + ab] += fq.v;
                dMm[((size_t)tj * KA + k) * 9 + ab] += dot3(fq.g, lp);
            }
        }
        for (int n = 0; n < NA; n++) {
            dl g = w->gA[(size_t)p * NA + n];
            for (int lm = 0; lm < L3; lm++) dA[n * 24 + lm] += dot3(mul(g, Y[lm]).g, lp);
            for (int ab = 0; ab < 9; ab++) dM[n * 9 + ab] += dot3(mul(g, Q[ab]).g, lp);
        }
    }
    double kap = kappa4();
    for (int b = 0; b < T; b++) {
        /* radial: q_n and dq_n are linear in c^{ti b}_{nk} */
        for (int n = 0; n < NR; n++)
            for (int k = 0; k < KR; k++)
                grad[z->o_cR + (((size_t)ti * T + b) * NR + n) * KR + k] += abar[n] * R[b * KR + k] + bbar[n] * dR[b * KR + k];
        /* angular */
        for (int n = 0; n < NA; n++)
            for (int k = 0; k < KA; k++) {
                const double *Ak = Am + ((size_t)b * KA + k) * 24;
                const double *dAk = dAm + ((size_t)b * KA + k) * 24;
                double gsum = 0.0;
                double dQdc = 0.0, ddQdc = 0.0;  /* l = 1 pieces for the 5-body term */
                for (int l = 1; l <= z->L; l++) {
                    double dqdc = 0.0, ddqdc = 0.0;
                    for (int m = -l; m <= l; m++) {
                        int lm = l * l - 1 + m + l;
                        dqdc += 2.0 * w->A[n * 24 + lm] * Ak[lm];
                        ddqdc += 2.0 * (Ak[lm] * dA[n * 24 + lm] + w->A[n * 24 + lm] * dAk[lm]);
                    }
                    int v = idx3(z, n, l);
                    gsum += abar[v] * dqdc + bbar[v] * ddqdc;
                    if (l == 1) { dQdc = dqdc; ddQdc = ddqdc; }
                }
                if (z->H4) {
                    const double *Mk = Mm + ((size_t)b * KA + k) * 9;
                    const double *dMk = dMm + ((size_t)b * KA + k) * 9;
                    const double *Mn = w->M + n * 9;
                    const double *dMn = dM + n * 9;
                    double M2[9], t1[9], t2[9];
                    mat_mul3(Mn, Mn, M2);
                    double dq4dc = 3.0 * kap * tr_mul(M2, Mk);
                    mat_mul3(Mk, Mn, t1);
                    mat_mul3(Mn, Mk, t2);
                    double dd4 = 3.0 * kap * (tr_mul(M2, dMk) + tr_mul(t1, dMn) + tr_mul(t2, dMn));
                    int v = idx4(z, n);
                    gsum += abar[v] * dq4dc + bbar[v] * dd4;
                }
                if (z->H5) {
                    double Qn = w->q[idx3(z, n, 1)];
                    double dQn = dq[idx3(z, n, 1)];
                    int v = idx5(z, n);
                    gsum += abar[v] * 2.0 * Qn * dQdc + bbar[v] * (2.0 * dQdc * dQn + 2.0 * Qn * ddQdc);
                }
                grad[z->o_cA + (((size_t)ti * T + b) * NA + n) * KA + k] += gsum;
            }
    }
    (void)cR; (void)cA;
    free(dq); free(dqt); free(abar); free(bbar); free(zeta);
    free(R); free(dR); free(Am); free(dAm); free(Mm); free(dMm); free(dA); free(dM);
}

/* ---------------------------------------------------------- ZBL short-range term
 * Sec. "Training" lets TorchNEP add, as NEP does, the Ziegler-Biersack-Littmark
 * screened Coulomb repulsion (the paper cites the ZBL treatise and prints no formula).
 * Taken from that treatise: the universal screening function
 *   phi(x) = 0.1818 e^{-3.2 x} + 0.5099 e^{-0.9423 x} + 0.2802 e^{-0.4029 x} + 0.02817 e^{-0.2016 x},
 *   x = r / a,  a = 0.8854 a_0 / (Z_i^0.23 + Z_j^0.23)  (a_0 the Bohr radius),
 *   V(r) = (e^2 / (4 pi eps_0)) Z_i Z_j phi(r / a) / r.
 * Reading of NEP's switch (not in the paper): V is multiplied by
 *   f_s = 1 (r < r1),  (1 + cos(pi (r - r1)/(r2 - r1)))/2 (r1 <= r < r2),  0 (r >= r2),
 * and every ordered neighbour pair (i, j) adds f_s V / 2 to E_i, so a pair of atoms
 * contributes f_s V in all.  Returns e = f_s V and de = d(f_s V)/dr. */
static void zbl_pair(const orc_cfg *cfg, int ti, int tj, double r, double *e, double *de) {
    const double ke = 14.399645;     /* e^2 / (4 pi eps_0) in eV A */
    const double a0 = 0.52917721;    /* Bohr radius in A */
    const double zi = cfg->zbl_Z[ti], zj = cfg->zbl_Z[tj];
    const double a = 0.8854 * a0 / (pow(zi, 0.23) + pow(zj, 0.23));
    const double c[4] = {0.1818, 0.5099, 0.2802, 0.02817}, d[4] = {3.2, 0.9423, 0.4029, 0.2016};
    double phi = 0.0, dphi = 0.0; /* phi(r/a) and its r-derivative */
    for (int k = 0; k < 4; k++) {
        double t = c[k] * exp(-d[k] * r / a);
        phi += t;
        dphi -= d[k] / a * t;
    }
    double v = ke * zi * zj * phi / r;
    double dv = ke * zi * zj * (dphi / r - phi / (r * r));
    double f = 0.0, fp = 0.0;
    if (r < cfg->zbl_r1) {
        f = 1.0;
    } else if (r < cfg->zbl_r2) {
        double w = cfg->zbl_r2 - cfg->zbl_r1, t = M_PI * (r - cfg->zbl_r1) / w;
        f = 0.5 * (1.0 + cos(t));
        fp = -0.5 * sin(t) * M_PI / w;
    }
    *e = f * v;
    *de = f * dv + fp * v;
}

/* ---------------------------------------------------------- structure pass
 * mode 0: E, F, W (and optionally q).  mode 1: also the adjoint with the loss
 * cotangents (eb_s, fb, Wb_s) given by the caller.  Returns 0 or -1 on a bad cell. */
static int structure_pass(const orc_cfg *cfg, const sizes *z, const double *th, const double *qs,
                          int n, const double *pos, const int32_t *type_s, const double *cell,
                          double *E, double *F, double *W, double *qout,
                          int mode, double eb, const double *fb, const double *Wb, double *grad) {
    int64_t c = brute_pairs(n, pos, cell, (float)cfg->rc_R, (float)cfg->rc_A, NULL, 0);
    if (c < 0) return -1;
    opair *pr = (opair *)malloc(sizeof(opair) * (size_t)(c > 0 ? c : 1));
    brute_pairs(n, pos, cell, (float)cfg->rc_R, (float)cfg->rc_A, pr, c);
    int64_t *beg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t p = 0; p < c; p++) beg[pr[p].i + 1]++;
    for (int i = 0; i < n; i++) beg[i + 1] += beg[i];
    int maxp = 1;
    for (int i = 0; i < n; i++) if (beg[i + 1] - beg[i] > maxp) maxp = (int)(beg[i + 1] - beg[i]);
    work w;
    work_alloc(&w, z, maxp);
    double Es = 0.0;
    for (int a = 0; a < 9; a++) W[a] = 0.0;
    for (int i = 0; i < 3 * n; i++) F[i] = 0.0;
    for (int i = 0; i < n; i++) {
        int np = (int)(beg[i + 1] - beg[i]);
        const opair *pi = pr + beg[i];
        double Ei = atom_forward(cfg, z, th, qs, type_s[i], type_s, pi, np, &w);
        Es += Ei;
        if (qout) for (int v = 0; v < z->ND; v++) qout[(size_t)i * z->ND + v] = w.q[v];
        for (int p = 0; p < np; p++) {
            double G[3];
            pair_gradient(z, qs, &w, np, p, G);
            int j = pi[p].j;
            if (cfg->zbl) {
                const double *d = pi[p].d;
                double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                if (r < cfg->zbl_r2) {
                    double e, de;
                    zbl_pair(cfg, type_s[i], type_s[j], r, &e, &de);
                    Es += 0.5 * e;
                    for (int a = 0; a < 3; a++) G[a] += 0.5 * de * d[a] / r;
                }
            }
            for (int a = 0; a < 3; a++) {
                F[3 * i + a] += G[a];
                F[3 * j + a] -= G[a];
            }
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) W[3 * a + b] -= G[a] * pi[p].d[b];
        }
        if (mode == 1) {
            double *lam = (double *)malloc(sizeof(double) * 3 * (size_t)(np > 0 ? np : 1));
            for (int p = 0; p < np; p++) {
                int j = pi[p].j;
                for (int a = 0; a < 3; a++) {
                    double wd = Wb[3 * a + 0] * pi[p].d[0] + Wb[3 * a + 1] * pi[p].d[1] + Wb[3 * a + 2] * pi[p].d[2];
                    lam[3 * p + a] = fb[3 * i + a] - fb[3 * j + a] - wd;
                }
            }
            atom_adjoint(cfg, z, th, qs, type_s[i], type_s, pi, np, &w, lam, eb, grad);
            free(lam);
        }
    }
    *E = Es;
    work_free(&w);
    free(beg);
    free(pr);
    return 0;
}

static int threads_used(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
int orc_threads(void) { return threads_used(); }

/* Threads for the following calls (timing single-core against all-core); n <= 0 restores
 * one per host core.  Changes no arithmetic. */
void orc_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
    (void)n;
#endif
}

/* E [Ns], F [Na*3], W [Ns*9], q [Na*ND] (optional) at theta (FP64). */
int orc_eval(const orc_cfg *cfg, const double *theta, const double *qscale, int64_t n_struct,
             const int64_t *atom_off, const double *pos, const int32_t *type, const double *cell,
             double *E, double *F, double *W, double *q) {
    if (!cfg_ok(cfg)) return -2;
    sizes z = get_sizes(cfg);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int64_t s = 0; s < n_struct; s++) {
        int n = (int)(atom_off[s + 1] - atom_off[s]);
        int64_t a0 = atom_off[s];
        if (structure_pass(cfg, &z, theta, qscale, n, pos + 3 * a0, type + a0, cell + 9 * s, E + s, F + 3 * a0,
                           W + 9 * s, q ? q + (size_t)a0 * z.ND : NULL, 0, 0.0, NULL, NULL, NULL) != 0)
            bad = 1;
    }
    return bad ? -1 : 0;
}

/* Parameter gradient of  sum_s dE_s E_s + sum_i dF_i . F_i + sum_s dW_s : W_s  (cotangents given). */
int orc_backward(const orc_cfg *cfg, const double *theta, const double *qscale, int64_t n_struct,
                 const int64_t *atom_off, const double *pos, const int32_t *type, const double *cell,
                 const double *dE, const double *dF, const double *dW, double *grad) {
    if (!cfg_ok(cfg)) return -2;
    sizes z = get_sizes(cfg);
    int nt = threads_used();
    double *part = (double *)calloc((size_t)nt * z.P, sizeof(double));
    int bad = 0;
#pragma omp parallel reduction(| : bad)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *g = part + (size_t)tid * z.P;
#pragma omp for schedule(static)
        for (int64_t s = 0; s < n_struct; s++) {
            int n = (int)(atom_off[s + 1] - atom_off[s]);
            int64_t a0 = atom_off[s];
            double Es, Wt[9];
            double *Ft = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
            if (structure_pass(cfg, &z, theta, qscale, n, pos + 3 * a0, type + a0, cell + 9 * s, &Es, Ft, Wt, NULL,
                               1, dE[s], dF + 3 * a0, dW + 9 * s, g) != 0)
                bad = 1;
            free(Ft);
        }
    }
    for (int64_t k = 0; k < z.P; k++) {
        double s = 0.0;
        for (int t = 0; t < nt; t++) s += part[(size_t)t * z.P + k];
        grad[k] = s;
    }
    free(part);
    return bad ? -1 : 0;
}

/* Eq. "loss": loss3 = (DE, DF, DV) and grad = dL/dtheta for L = lE DE + lF DF + lV DV.
 * norms (optional, may be NULL): (N_s, N_a, N_s^V) used as the normalisers, for a
 * batch that is one shard of a larger one.  E/F/W outputs optional (may be NULL). */
int orc_loss_grad(const orc_cfg *cfg, const double *theta, const double *qscale, int64_t n_struct,
                  const int64_t *atom_off, const double *pos, const int32_t *type, const double *cell,
                  const double *E_ref, const double *F_ref, const double *W_ref, const uint8_t *has_W,
                  double lamE, double lamF, double lamV, const double *norms,
                  double *loss3, double *grad, double *E_out, double *F_out, double *W_out) {
    if (!cfg_ok(cfg)) return -2;
    sizes z = get_sizes(cfg);
    int64_t Na = atom_off[n_struct];
    double Ns_d = (double)n_struct, Na_d = (double)Na, NsV_d = 0.0;
    for (int64_t s = 0; s < n_struct; s++) NsV_d += (has_W == NULL || has_W[s]) ? 1.0 : 0.0;
    if (norms) { Ns_d = norms[0]; Na_d = norms[1]; NsV_d = norms[2]; }
    double *E = (double *)malloc(sizeof(double) * (size_t)(n_struct > 0 ? n_struct : 1));
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)(Na > 0 ? Na : 1));
    double *W = (double *)malloc(sizeof(double) * 9 * (size_t)(n_struct > 0 ? n_struct : 1));
    int rc = orc_eval(cfg, theta, qscale, n_struct, atom_off, pos, type, cell, E, F, W, NULL);
    if (rc != 0) { free(E); free(F); free(W); return rc; }
    double *dE = (double *)calloc((size_t)(n_struct > 0 ? n_struct : 1), sizeof(double));
    double *dF = (double *)calloc(3 * (size_t)(Na > 0 ? Na : 1), sizeof(double));
    double *dW = (double *)calloc(9 * (size_t)(n_struct > 0 ? n_struct : 1), sizeof(double));
    double sE = 0.0, sF = 0.0, sV = 0.0;
    for (int64_t s = 0; s < n_struct; s++) {
        double na = (double)(atom_off[s + 1] - atom_off[s]);
        double r = (E[s] - E_ref[s]) / na;
        sE += r * r;
        dE[s] = lamE * 2.0 * (E[s] - E_ref[s]) / (na * na) / Ns_d;
        int hw = (has_W == NULL || has_W[s]);
        if (hw && NsV_d > 0) {
            for (int a = 0; a < 9; a++) {
                double rw = (W[9 * s + a] - W_ref[9 * s + a]) / na;
                sV += rw * rw;
                dW[9 * s + a] = lamV * 2.0 * (W[9 * s + a] - W_ref[9 * s + a]) / (na * na) / (9.0 * NsV_d);
            }
        }
    }
    for (int64_t i = 0; i < 3 * Na; i++) {
        double r = F[i] - F_ref[i];
        sF += r * r;
        dF[i] = lamF * 2.0 * r / (3.0 * Na_d);
    }
    loss3[0] = n_struct > 0 ? sE / Ns_d : 0.0;
    loss3[1] = Na > 0 ? sF / (3.0 * Na_d) : 0.0;
    loss3[2] = NsV_d > 0 ? sV / (9.0 * NsV_d) : 0.0;
    rc = orc_backward(cfg, theta, qscale, n_struct, atom_off, pos, type, cell, dE, dF, dW, grad);
    if (E_out) memcpy(E_out, E, sizeof(double) * (size_t)n_struct);
    if (F_out) memcpy(F_out, F, sizeof(double) * 3 * (size_t)Na);
    if (W_out) memcpy(W_out, W, sizeof(double) * 9 * (size_t)n_struct);
    free(E); free(F); free(W); free(dE); free(dF); free(dW);
    return rc;
}

/* Raw descriptors q (before scaling) for every atom, [Na*ND]. */
int orc_descriptors(const orc_cfg *cfg, const double *theta, int64_t n_struct, const int64_t *atom_off,
                    const double *pos, const int32_t *type, const double *cell, double *q) {
    if (!cfg_ok(cfg)) return -2;
    sizes z = get_sizes(cfg);
    double *ones = (double *)malloc(sizeof(double) * z.ND);
    for (int v = 0; v < z.ND; v++) ones[v] = 1.0;
    int64_t Na = atom_off[n_struct];
    double *E = (double *)malloc(sizeof(double) * (size_t)(n_struct > 0 ? n_struct : 1));
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)(Na > 0 ? Na : 1));
    double *W = (double *)malloc(sizeof(double) * 9 * (size_t)(n_struct > 0 ? n_struct : 1));
    int rc = orc_eval(cfg, theta, ones, n_struct, atom_off, pos, type, cell, E, F, W, q);
    free(ones); free(E); free(F); free(W);
    return rc;
}

/* Exposed for tests: real harmonics and the basis at one point (value and gradient). */
void orc_ylm(const double *d, int lmax, double *val /*[24]*/, double *grad /*[24*3]*/) {
    dl dx = {d[0], {1.0, 0.0, 0.0}}, dy = {d[1], {0.0, 1.0, 0.0}}, dz = {d[2], {0.0, 0.0, 1.0}};
    dl r = dsqrt(add(add(mul(dx, dx), mul(dy, dy)), mul(dz, dz)));
    dl Y[24];
    real_ylm(ddiv(dx, r), ddiv(dy, r), ddiv(dz, r), lmax, Y);
    int L3 = lmax * (lmax + 2);
    for (int k = 0; k < L3; k++) {
        val[k] = Y[k].v;
        for (int a = 0; a < 3; a++) grad[3 * k + a] = Y[k].g[a];
    }
}
void orc_basis(double r, double rc, int K, double *f, double *fp) {
    dl rr = {r, {1.0, 0.0, 0.0}};
    dl out[64];
    basis(rr, rc, K, out);
    for (int k = 0; k < K; k++) { f[k] = out[k].v; fp[k] = out[k].g[0]; }
}
double orc_kappa4(void) { return kappa4(); }

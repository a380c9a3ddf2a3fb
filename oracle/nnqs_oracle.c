/*
 * nnqs_oracle.c -- plain, slow, FP64 CPU oracle for the symmetry-projected
 * complex-RBM variational Monte Carlo path of
 * "Systematic improvement of neural network quantum states using a Lanczos
 * recursion" (Chen, Hendry, Weinberg, Feiguin).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the package's smoke check and the bench's
 * CPU-baseline leg do.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * Everything is evaluated from its definition, in double / double complex:
 *   - J1-J2 Hamiltonian, Sec. 2.1 Eq. 1 (S = s/2, s = +-1).
 *   - RBM amplitude, Sec. 3.1 Eq. 2, with spins s = +-1 (the paper's +-1/2
 *     rescales W and a by 2).  Bias-free form Eq. 3.
 *   - Momentum projection Eqs. 4-5 and C4v projection Eq. 6; spin inversion
 *     as an extra Z2 projection.
 *   - Local energy Eq. 10 by enumerating bonds and re-evaluating psi from
 *     scratch at every connected configuration (no incremental update).
 *   - (H^2 psi)/psi by explicit double enumeration (Sec. 3.3).
 *   - Moments <H^n>, n<=4, and the p=1 Lanczos energy, Eqs. 13-18, with the
 *     closed form re-derived from the 2x2 matrix in span{psi0, psi1}; the
 *     p=1 state's variance and the variance extrapolation (Sec. 4.3).
 *   - The p=2 step: (H^3 psi)/psi by triple enumeration, moments about a
 *     shift up to order 6, the 3x3 Krylov pencil (Cholesky + Jacobi).
 *   - Static spin structure factor S(q) (Sec. 4.1) as the double sum over
 *     site pairs.
 *   - Log-derivatives O_k and the SR system, Eq. 12.
 *   - Metropolis pair-exchange sampling, Sec. 3.2, driven by Philox4x32-10
 *     (Salmon, Moraes, Dror, Shaw, SC'11) written from its published
 *     definition.
 *   - Exact diagonalisation of the Sz=0 sector (Lanczos with full
 *     re-orthogonalisation, Sturm-sequence bisection, inverse iteration).
 *
 * Parity status of each function is stated at its definition; all of them
 * are pinned by the -m "not gpu" tests.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------------ */
/* Lattice: L x L periodic square lattice, site i = x + L*y (Sec. 3.4).       */
/* ------------------------------------------------------------------------ */

static int wrap(int v, int L) { v %= L; return v < 0 ? v + L : v; }
static int site_of(int L, int x, int y) { return wrap(x, L) + L * wrap(y, L); }

/* Bonds of Eq. 1.  For each site in increasing index: J1 (+x), J1 (+y),
 * J2 (+x+y), J2 (+x-y).  4N distinct bonds for L >= 3.  type 1 = J1, 2 = J2. */
int or_bonds(int L, int *bi, int *bj, int *btype)
{
    int nb = 0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            int i = site_of(L, x, y);
            bi[nb] = i; bj[nb] = site_of(L, x + 1, y);     btype[nb++] = 1;
            bi[nb] = i; bj[nb] = site_of(L, x, y + 1);     btype[nb++] = 1;
            bi[nb] = i; bj[nb] = site_of(L, x + 1, y + 1); btype[nb++] = 2;
            bi[nb] = i; bj[nb] = site_of(L, x + 1, y - 1); btype[nb++] = 2;
        }
    return nb;
}

/* C4v about site 0 (Eq. 6).  Element order: E, C4, C2, C4^3, sigma_x
 * (x -> -x), sigma_y (y -> -y), sigma_d (x <-> y), sigma_d' (x,y -> -y,-x). */
static void point_op(int l, int x, int y, int *xo, int *yo)
{
    switch (l) {
    case 0: *xo = x;  *yo = y;  break;
    case 1: *xo = -y; *yo = x;  break;
    case 2: *xo = -x; *yo = -y; break;
    case 3: *xo = y;  *yo = -x; break;
    case 4: *xo = -x; *yo = y;  break;
    case 5: *xo = x;  *yo = -y; break;
    case 6: *xo = y;  *yo = x;  break;
    default: *xo = -y; *yo = -x; break;
    }
}

/* Characters of the one-dimensional C4v irreps (textbook table; the paper's
 * own table is not part of the text).  Rows A1, A2, B1, B2; B1 is even under
 * the axis mirrors and odd under the diagonal ones. */
static const int c4v_char[4][8] = {
    {1, 1, 1, 1, 1, 1, 1, 1},
    {1, 1, 1, 1, -1, -1, -1, -1},
    {1, -1, 1, -1, 1, 1, -1, -1},
    {1, -1, 1, -1, -1, -1, 1, 1},
};

/* Group G = {T_R o L_l}.  perm[g*N + i] = image of site i under g; chi[g] =
 * exp(-i K.R) chi_I(L_l) (Eqs. 4 and 6; only real phases occur).
 * momentum: 0=(0,0) 1=(pi,pi) 2=(pi,0) 3=(0,pi).  For K=(pi,0),(0,pi) the
 * point group is restricted to the little group {E, C2, sigma_x, sigma_y}.
 * Returns |G|, or -1 for an invalid combination. */
int or_group(int L, int proj_t, int proj_p, int momentum, int irrep, int *perm, double *chi)
{
    int N = L * L;
    int ops[8], nops = 0;
    if (irrep < 0 || irrep > 3 || momentum < 0 || momentum > 3) return -1;
    if (!proj_p) ops[nops++] = 0;
    else if (momentum <= 1) for (int l = 0; l < 8; ++l) ops[nops++] = l;
    else { ops[0] = 0; ops[1] = 2; ops[2] = 4; ops[3] = 5; nops = 4; }
    int nt = proj_t ? N : 1;
    int g = 0;
    for (int a = 0; a < nops; ++a) {
        int l = ops[a];
        for (int r = 0; r < nt; ++r) {
            int m = r % L, n = r / L;
            double phase = 1.0;
            if (momentum == 1) phase = ((m + n) & 1) ? -1.0 : 1.0;
            if (momentum == 2) phase = (m & 1) ? -1.0 : 1.0;
            if (momentum == 3) phase = (n & 1) ? -1.0 : 1.0;
            chi[g] = phase * c4v_char[irrep][l];
            for (int i = 0; i < N; ++i) {
                int xo, yo;
                point_op(l, i % L, i / L, &xo, &yo);
                perm[g * N + i] = site_of(L, xo + m, yo + n);
            }
            ++g;
        }
    }
    return g;
}

/* ------------------------------------------------------------------------ */
/* Model                                                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
    int L, N, K, M, G, use_bias, spin_inv, P1, nb;
    double J1, J2;
    int *perm; double *chi;
    int *bi, *bj, *bt;
    cplx *par;     /* K blocks of [log c_r, a[N], b[M], W[M][N] row-major] */
} or_model;

/* Number of complex parameters per RBM. */
int or_params_per_rbm(int N, int M) { return 1 + N + M + M * N; }

void *or_model_new(int L, double J1, double J2, int K, int M, int proj_t, int proj_p,
                   int momentum, int irrep, int spin_inv, int use_bias, const double *params)
{
    if (L < 4 || (L & 1)) return NULL;
    if (spin_inv != 0 && spin_inv != 1 && spin_inv != -1) return NULL;
    /* without biases every RBM is even under s -> -s (Eq. 3), so an odd
     * spin-inversion projection would vanish identically */
    if (!use_bias && spin_inv < 0) return NULL;
    or_model *h = (or_model *)calloc(1, sizeof(or_model));
    int N = L * L;
    h->L = L; h->N = N; h->K = K; h->M = M; h->J1 = J1; h->J2 = J2;
    h->use_bias = use_bias; h->spin_inv = spin_inv; h->P1 = or_params_per_rbm(N, M);
    h->perm = (int *)malloc(sizeof(int) * 8 * N * N);
    h->chi = (double *)malloc(sizeof(double) * 8 * N);
    h->G = or_group(L, proj_t, proj_p, momentum, irrep, h->perm, h->chi);
    if (h->G < 0) { free(h->perm); free(h->chi); free(h); return NULL; }
    h->bi = (int *)malloc(sizeof(int) * 4 * N);
    h->bj = (int *)malloc(sizeof(int) * 4 * N);
    h->bt = (int *)malloc(sizeof(int) * 4 * N);
    h->nb = or_bonds(L, h->bi, h->bj, h->bt);
    h->par = (cplx *)malloc(sizeof(cplx) * (size_t)K * h->P1);
    for (size_t k = 0; k < (size_t)K * h->P1; ++k)
        h->par[k] = params[2 * k] + I * params[2 * k + 1];
    return h;
}

void or_model_free(void *hp)
{
    or_model *h = (or_model *)hp;
    if (!h) return;
    free(h->perm); free(h->chi); free(h->bi); free(h->bj); free(h->bt); free(h->par); free(h);
}

int or_model_G(void *hp) { return ((or_model *)hp)->G; }

/* log(2 cosh z), written with the larger exponential factored out so that it
 * stays finite for any Re z: 2cosh z = e^{z}(1 + e^{-2z}) for Re z >= 0. */
static cplx log2cosh(cplx z)
{
    if (creal(z) < 0) z = -z;
    return z + clog(1.0 + cexp(-2.0 * z));
}

/* log of the single-RBM amplitude of Eq. 2 at the (+-1) configuration t. */
static cplx log_rbm(const or_model *h, int r, const int8_t *t)
{
    const int N = h->N, M = h->M;
    const cplx *p = h->par + (size_t)r * h->P1;
    const cplx *a = p + 1, *b = p + 1 + N, *W = p + 1 + N + M;
    cplx acc = 0;
    if (h->use_bias)
        for (int j = 0; j < N; ++j) acc += a[j] * t[j];
    for (int m = 0; m < M; ++m) {
        cplx th = h->use_bias ? b[m] : 0;
        for (int j = 0; j < N; ++j) th += W[(size_t)m * N + j] * t[j];
        acc += log2cosh(th);
    }
    return acc;
}

static double wrap_phase(double ph)
{
    ph = fmod(ph, 2.0 * M_PI);
    if (ph <= -M_PI) ph += 2.0 * M_PI;
    if (ph > M_PI) ph -= 2.0 * M_PI;
    return ph;
}

/* Number of terms of the projected sum: K * |G| * (2 with spin inversion). */
static int n_terms(const or_model *h) { return h->K * h->G * (h->spin_inv ? 2 : 1); }

/* Log of every term c_r chi(g) chi_P psi_r(+-T_g s) of the projected sum
 * (Eq. 6 summed over RBMs r and the spin-inversion pair), in the order
 * (r, g, sign), together with the transformed configurations if wanted. */
static void log_terms(const or_model *h, const int8_t *s, cplx *terms, int8_t *tbuf)
{
    const int N = h->N;
    int nsg = h->spin_inv ? 2 : 1, k = 0;
    int8_t *t = tbuf;
    for (int r = 0; r < h->K; ++r) {
        cplx logc = h->par[(size_t)r * h->P1];
        for (int g = 0; g < h->G; ++g) {
            for (int sg = 0; sg < nsg; ++sg) {
                int sign = sg ? -1 : 1;
                for (int i = 0; i < N; ++i) t[h->perm[g * N + i]] = (int8_t)(sign * s[i]);
                cplx lt = logc + log_rbm(h, r, t);
                if (h->chi[g] < 0) lt += I * M_PI;
                if (sign < 0 && h->spin_inv < 0) lt += I * M_PI;
                terms[k++] = lt;
            }
        }
    }
}

/* log psi(s) = log sum_k exp(term_k), shifted by the largest real part. */
static cplx log_psi_one(const or_model *h, const int8_t *s)
{
    int nt = n_terms(h);
    cplx *terms = (cplx *)malloc(sizeof(cplx) * nt);
    int8_t *t = (int8_t *)malloc(h->N);
    log_terms(h, s, terms, t);
    double mx = -INFINITY;
    for (int k = 0; k < nt; ++k) if (creal(terms[k]) > mx) mx = creal(terms[k]);
    cplx sum = 0;
    for (int k = 0; k < nt; ++k) sum += cexp(terms[k] - mx);
    free(terms); free(t);
    cplx lp = mx + clog(sum);
    return creal(lp) + I * wrap_phase(cimag(lp));
}

/* Batched log psi.  spins: [n][N] int8 (+-1).  out: [n][2] (re, im), the
 * imaginary part in (-pi, pi]. */
void or_log_psi(void *hp, const int8_t *spins, int n, double *out)
{
    const or_model *h = (const or_model *)hp;
    #pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < n; ++k) {
        cplx lp = log_psi_one(h, spins + (size_t)k * h->N);
        out[2 * k] = creal(lp); out[2 * k + 1] = cimag(lp);
    }
}

/* Diagonal part of Eq. 1: sum_bonds J/4 s_i s_j. */
static double diag_energy(const or_model *h, const int8_t *s)
{
    double d = 0;
    for (int b = 0; b < h->nb; ++b) {
        double J = h->bt[b] == 1 ? h->J1 : h->J2;
        d += 0.25 * J * s[h->bi[b]] * s[h->bj[b]];
    }
    return d;
}

/* Local energy, Eq. 10: E_loc(s) = sum_s' H_{s s'} psi(s')/psi(s).  The
 * off-diagonal element of S_i.S_j is 1/2 between configurations that differ by
 * exchanging an anti-aligned pair.  Every psi(s') is evaluated from scratch. */
static cplx eloc_one(const or_model *h, const int8_t *s, cplx lp)
{
    int8_t *sp = (int8_t *)malloc(h->N);
    cplx off = 0;
    for (int b = 0; b < h->nb; ++b) {
        int i = h->bi[b], j = h->bj[b];
        if (s[i] == s[j]) continue;
        double J = h->bt[b] == 1 ? h->J1 : h->J2;
        memcpy(sp, s, h->N);
        sp[i] = s[j]; sp[j] = s[i];
        off += 0.5 * J * cexp(log_psi_one(h, sp) - lp);
    }
    free(sp);
    return diag_energy(h, s) + off;
}

void or_local_energy(void *hp, const int8_t *spins, int n, double *eloc)
{
    /* Same sums as eloc_one, with every (sample, bond) ratio evaluated in
     * parallel and then added in bond order. */
    const or_model *h = (const or_model *)hp;
    const int nb = h->nb;
    cplx *lp = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *ratio = (cplx *)calloc((size_t)n * nb, sizeof(cplx));
    #pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < n; ++k) lp[k] = log_psi_one(h, spins + (size_t)k * h->N);
    #pragma omp parallel for schedule(dynamic)
    for (long q = 0; q < (long)n * nb; ++q) {
        const int k = (int)(q / nb), b = (int)(q % nb);
        const int8_t *s = spins + (size_t)k * h->N;
        const int i = h->bi[b], j = h->bj[b];
        if (s[i] == s[j]) continue;
        int8_t *sp = (int8_t *)malloc(h->N);
        memcpy(sp, s, h->N);
        sp[i] = s[j]; sp[j] = s[i];
        ratio[q] = cexp(log_psi_one(h, sp) - lp[k]);
        free(sp);
    }
    for (int k = 0; k < n; ++k) {
        const int8_t *s = spins + (size_t)k * h->N;
        cplx off = 0;
        for (int b = 0; b < nb; ++b) {
            const int i = h->bi[b], j = h->bj[b];
            if (s[i] == s[j]) continue;
            const double J = h->bt[b] == 1 ? h->J1 : h->J2;
            off += 0.5 * J * ratio[(size_t)k * nb + b];
        }
        const cplx e = diag_energy(h, s) + off;
        eloc[2 * k] = creal(e); eloc[2 * k + 1] = cimag(e);
    }
    free(lp); free(ratio);
}

/* Lanczos-step quantities (Sec. 3.3): h1 = (H psi)(s)/psi(s) and
 * h2 = (H^2 psi)(s)/psi(s) = sum_s' H_{s s'} [psi(s')/psi(s)] h1(s'),
 * by explicit double enumeration.  The inner loop over first-level
 * neighbours runs in parallel. */
void or_lanczos_h(void *hp, const int8_t *spins, int n, double *h1out, double *h2out)
{
    const or_model *h = (const or_model *)hp;
    const int N = h->N;
    for (int k = 0; k < n; ++k) {
        const int8_t *s = spins + (size_t)k * N;
        cplx lp = log_psi_one(h, s);
        cplx h1 = eloc_one(h, s, lp);
        cplx acc = diag_energy(h, s) * h1;
        #pragma omp parallel
        {
            int8_t *sp = (int8_t *)malloc(N);
            cplx part = 0;
            #pragma omp for schedule(dynamic)
            for (int b = 0; b < h->nb; ++b) {
                int i = h->bi[b], j = h->bj[b];
                if (s[i] == s[j]) continue;
                double J = h->bt[b] == 1 ? h->J1 : h->J2;
                memcpy(sp, s, N);
                sp[i] = s[j]; sp[j] = s[i];
                cplx lpp = log_psi_one(h, sp);
                part += 0.5 * J * cexp(lpp - lp) * eloc_one(h, sp, lpp);
            }
            #pragma omp critical
            acc += part;
            free(sp);
        }
        h1out[2 * k] = creal(h1); h1out[2 * k + 1] = cimag(h1);
        h2out[2 * k] = creal(acc); h2out[2 * k + 1] = cimag(acc);
    }
}

/* (H^2 psi)(s)/psi(s) of one configuration by double enumeration, serial:
 * diag(s) h1(s) + sum_{s'} (J/2) [psi(s')/psi(s)] h1(s'), h1 = eloc_one. */
static cplx h2_one(const or_model *h, const int8_t *s, cplx lp, cplx h1)
{
    int8_t *sp = (int8_t *)malloc(h->N);
    cplx acc = diag_energy(h, s) * h1;
    for (int b = 0; b < h->nb; ++b) {
        int i = h->bi[b], j = h->bj[b];
        if (s[i] == s[j]) continue;
        double J = h->bt[b] == 1 ? h->J1 : h->J2;
        memcpy(sp, s, h->N);
        sp[i] = s[j]; sp[j] = s[i];
        cplx lpp = log_psi_one(h, sp);
        acc += 0.5 * J * cexp(lpp - lp) * eloc_one(h, sp, lpp);
    }
    free(sp);
    return acc;
}

/* The p = 2 quantities (Sec. 3.3, |Psi_2> = (1 + beta_1 H + beta_2 H^2)
 * |psi0>): h1, h2 and h3 = (H^3 psi)(s)/psi(s) = diag(s) h2(s) +
 * sum_{s'} (J/2) [psi(s')/psi(s)] h2(s') by explicit triple enumeration,
 * every psi from scratch.  The first-level neighbours run in parallel. */
void or_lanczos_h3(void *hp, const int8_t *spins, int n, double *h1out, double *h2out, double *h3out)
{
    const or_model *h = (const or_model *)hp;
    const int N = h->N;
    for (int k = 0; k < n; ++k) {
        const int8_t *s = spins + (size_t)k * N;
        const cplx lp = log_psi_one(h, s);
        const cplx h1 = eloc_one(h, s, lp);
        const cplx h2 = h2_one(h, s, lp, h1);
        cplx acc = diag_energy(h, s) * h2;
        #pragma omp parallel
        {
            int8_t *sp = (int8_t *)malloc(N);
            cplx part = 0;
            #pragma omp for schedule(dynamic)
            for (int b = 0; b < h->nb; ++b) {
                int i = h->bi[b], j = h->bj[b];
                if (s[i] == s[j]) continue;
                double J = h->bt[b] == 1 ? h->J1 : h->J2;
                memcpy(sp, s, N);
                sp[i] = s[j]; sp[j] = s[i];
                const cplx lpp = log_psi_one(h, sp);
                const cplx h1p = eloc_one(h, sp, lpp);
                part += 0.5 * J * cexp(lpp - lp) * h2_one(h, sp, lpp, h1p);
            }
            #pragma omp critical
            acc += part;
            free(sp);
        }
        h1out[2 * k] = creal(h1); h1out[2 * k + 1] = cimag(h1);
        h2out[2 * k] = creal(h2); h2out[2 * k + 1] = cimag(h2);
        h3out[2 * k] = creal(acc); h3out[2 * k + 1] = cimag(acc);
    }
}

/* ------------------------------------------------------------------------ */
/* Moments and the p = 1 Lanczos step (Eqs. 13-18)                           */
/* ------------------------------------------------------------------------ */

/* Estimators of <H^n> (n = 0..3) from per-sample h1, h2.  With weights == NULL
 * the samples are draws from |psi|^2 and every weight is 1; otherwise the
 * weights are |psi(s)|^2 (exact enumeration).  out[0..3] = m0..m3 with m0 = 1
 * (normalised); out[4] = sum of weights; out[5] = mean Im h1; out[6] = mean
 * Im(conj(h1) h2).  Sums are pairwise. */
static double pairwise(const double *v, int n)
{
    if (n <= 8) { double s = 0; for (int k = 0; k < n; ++k) s += v[k]; return s; }
    return pairwise(v, n / 2) + pairwise(v + n / 2, n - n / 2);
}

void or_moments(int n, const double *h1, const double *h2, const double *weights, double *out)
{
    double *c = (double *)malloc(sizeof(double) * 7 * (size_t)n);
    for (int k = 0; k < n; ++k) {
        double w = weights ? weights[k] : 1.0;
        cplx a = h1[2 * k] + I * h1[2 * k + 1];
        cplx b = h2 ? h2[2 * k] + I * h2[2 * k + 1] : 0;
        cplx ab = conj(a) * b;
        c[0 * (size_t)n + k] = w;
        c[1 * (size_t)n + k] = w * creal(a);
        c[2 * (size_t)n + k] = w * (creal(a) * creal(a) + cimag(a) * cimag(a));
        c[3 * (size_t)n + k] = w * creal(ab);
        c[4 * (size_t)n + k] = w * cimag(a);
        c[5 * (size_t)n + k] = w * cimag(ab);
        c[6 * (size_t)n + k] = w * (creal(b) * creal(b) + cimag(b) * cimag(b));
    }
    double z = pairwise(c, n);
    out[0] = 1.0;
    out[1] = pairwise(c + 1 * (size_t)n, n) / z;
    out[2] = pairwise(c + 2 * (size_t)n, n) / z;
    out[3] = pairwise(c + 3 * (size_t)n, n) / z;
    out[4] = z;
    out[5] = pairwise(c + 4 * (size_t)n, n) / z;
    out[6] = pairwise(c + 5 * (size_t)n, n) / z;
    out[7] = pairwise(c + 6 * (size_t)n, n) / z;   /* m4 = <H^4> = <|h2|^2> */
    free(c);
}

/* Lowest eigenpair of the 2x2 Hamiltonian in span{psi0, psi1}, psi1 =
 * (H - <H>) psi0 / v (Eq. 13): H00 = m1, H01 = v, H11 = (m3 - 2 m1 m2 +
 * m1^3)/v^2.  Its lowest eigenvalue is m1 + v*alpha with d = (H11 - m1)/(2v)
 * = (m3 - 3 m1 m2 + 2 m1^3)/(2 v^3) and alpha = d - sqrt(d^2 + 1); the
 * eigenvector is proportional to psi0 + alpha psi1.  (The printed r lacks the
 * factor 1/2, and Eq. 16's second psi0 is psi1.)  A vanishing variance
 * (v^2 <= 1e-14 m1^2) means psi0 is an eigenstate: E = m1, alpha = 0.
 * out = {E_p1, v, alpha}. */
void or_lanczos_step(const double *m, double *out)
{
    double m1 = m[1], m2 = m[2], m3 = m[3];
    double v2 = m2 - m1 * m1;
    if (v2 <= 1e-14 * m1 * m1 || v2 <= 0) { out[0] = m1; out[1] = v2 > 0 ? sqrt(v2) : 0; out[2] = 0; return; }
    double v = sqrt(v2);
    double d = (m3 - 3 * m1 * m2 + 2 * m1 * m1 * m1) / (2 * v2 * v);
    double alpha = d - sqrt(d * d + 1);
    out[0] = m1 + v * alpha; out[1] = v; out[2] = alpha;
}

/* Energy and variance of the p = 1 Lanczos state, and the variance
 * extrapolation (Sec. 3.3 Eq. 16; Sec. 4.3).  The state is phi = psi0 +
 * alpha psi1 with psi1 = (H - m1) psi0 / v, i.e. phi = a psi0 + b H psi0 with
 * b = alpha / v and a = 1 - alpha m1 / v.  With m_n = <H^n> (m4 = <H^4>),
 *   <phi|H^k|phi> / <psi0|psi0> = a^2 m_k + 2 a b m_{k+1} + b^2 m_{k+2},
 * so E1 = <H>_phi and var1 = <H^2>_phi - E1^2; the p = 0 point is (m1,
 * var0 = m2 - m1^2).  The straight line through (var0, m1) and (var1, E1)
 * is evaluated at zero variance (equal variances: E1).
 * m: m0..m4 (m0 = 1); lz: {E_p1, v, alpha}.  out = {var0, E1, var1, E_extrap}. */
void or_lanczos_variance(const double *m, const double *lz, double *out)
{
    const double m1 = m[1], m2 = m[2], m3 = m[3], m4 = m[4];
    const double v = lz[1], alpha = lz[2];
    const double var0 = m2 - m1 * m1;
    double a = 1.0, b = 0.0;
    if (v > 0.0) { b = alpha / v; a = 1.0 - alpha * m1 / v; }
    const double n0 = a * a + 2 * a * b * m1 + b * b * m2;
    const double n1 = a * a * m1 + 2 * a * b * m2 + b * b * m3;
    const double n2 = a * a * m2 + 2 * a * b * m3 + b * b * m4;
    const double E1 = n1 / n0, var1 = n2 / n0 - E1 * E1;
    out[0] = var0;
    out[1] = E1;
    out[2] = var1;
    out[3] = var0 != var1 ? E1 - var1 * (m1 - E1) / (var0 - var1) : E1;
}

/* Moments about a shift c, mu_k = <psi|(H - c)^k|psi>/<psi|psi> for k = 0..6,
 * from the local quantities a_0 = 1, a_1 = h1 - c, a_2 = h2 - 2c h1 + c^2,
 * a_3 = h3 - 3c h2 + 3c^2 h1 - c^3 (a_i = ((H - c)^i psi)(s)/psi(s)):
 * mu_{i+j} = <Re(conj(a_i) a_j)> with (i, j) = (0,0), (0,1), (1,1), (1,2),
 * (2,2), (2,3), (3,3).  Weighted means (weights NULL: plain means), summed
 * pairwise.  out[0..6] = mu_0..mu_6, out[7] = sum of weights. */
void or_shifted_moments(int n, const double *h1, const double *h2, const double *h3, double c,
                        const double *weights, double *out)
{
    double *col = (double *)malloc(sizeof(double) * 8 * (size_t)n);
    for (int k = 0; k < n; ++k) {
        const double w = weights ? weights[k] : 1.0;
        const cplx x1 = h1[2 * k] + I * h1[2 * k + 1];
        const cplx x2 = h2[2 * k] + I * h2[2 * k + 1];
        const cplx x3 = h3[2 * k] + I * h3[2 * k + 1];
        const cplx a1 = x1 - c;
        const cplx a2 = x2 - 2 * c * x1 + c * c;
        const cplx a3 = x3 - 3 * c * x2 + 3 * c * c * x1 - c * c * c;
        const double v[8] = {w, w * creal(a1), w * creal(conj(a1) * a1), w * creal(conj(a1) * a2),
                             w * creal(conj(a2) * a2), w * creal(conj(a2) * a3), w * creal(conj(a3) * a3), w};
        for (int q = 0; q < 8; ++q) col[(size_t)q * n + k] = v[q];
    }
    const double z = pairwise(col, n);
    for (int q = 0; q < 7; ++q) out[q] = pairwise(col + (size_t)q * n, n) / z;
    out[7] = z;
    free(col);
}

/* The p = 2 Lanczos step (Sec. 3.3): the lowest eigenpair of the pencil
 * A x = lambda B x with A_ij = mu_{i+j+1}, B_ij = mu_{i+j} (i, j = 0..2), the
 * Hamiltonian about c and the overlap in the Krylov basis {psi0, (H - c)psi0,
 * (H - c)^2 psi0} (the Krylov space, and so E, does not depend on c).
 * B = L L^T (Cholesky), C = L^{-1} A L^{-T}, cyclic Jacobi rotations on C,
 * x = L^{-T} y for the lowest eigenvector y, scaled so that x0 = 1.
 * out = {E_p2 = c + lambda, x0, x1, x2, var_p2} with
 * var_p2 = sum x_i x_j mu_{i+j+2} / sum x_i x_j mu_{i+j} - lambda^2. */
void or_krylov2(const double *mu, double c, double *out)
{
    double A[3][3], B[3][3], Lm[3][3] = {{0}}, Li[3][3] = {{0}}, C[3][3], T[3][3], V[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) { A[i][j] = mu[i + j + 1]; B[i][j] = mu[i + j]; }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j <= i; ++j) {
            double t = B[i][j];
            for (int k = 0; k < j; ++k) t -= Lm[i][k] * Lm[j][k];
            Lm[i][j] = i == j ? sqrt(t) : t / Lm[j][j];
        }
    for (int j = 0; j < 3; ++j) {            /* Li = L^{-1} by forward substitution */
        for (int i = 0; i < 3; ++i) {
            double t = i == j ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) t -= Lm[i][k] * Li[k][j];
            Li[i][j] = t / Lm[i][i];
        }
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double t = 0;
            for (int k = 0; k < 3; ++k) t += Li[i][k] * A[k][j];
            T[i][j] = t;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double t = 0;
            for (int k = 0; k < 3; ++k) t += T[i][k] * Li[j][k];
            C[i][j] = t;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = i == j;
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = fabs(C[0][1]) + fabs(C[0][2]) + fabs(C[1][2]);
        if (off < 1e-300) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (C[p][q] == 0.0) continue;
                const double th = (C[q][q] - C[p][p]) / (2 * C[p][q]);
                const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1));
                const double cs = 1 / sqrt(t * t + 1), sn = t * cs;
                for (int k = 0; k < 3; ++k) {      /* C <- J^T C J */
                    const double ckp = C[k][p], ckq = C[k][q];
                    C[k][p] = cs * ckp - sn * ckq;
                    C[k][q] = sn * ckp + cs * ckq;
                }
                for (int k = 0; k < 3; ++k) {
                    const double cpk = C[p][k], cqk = C[q][k];
                    C[p][k] = cs * cpk - sn * cqk;
                    C[q][k] = sn * cpk + cs * cqk;
                }
                for (int k = 0; k < 3; ++k) {
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = cs * vkp - sn * vkq;
                    V[k][q] = sn * vkp + cs * vkq;
                }
            }
    }
    int lo = 0;
    for (int i = 1; i < 3; ++i)
        if (C[i][i] < C[lo][lo]) lo = i;
    const double lam = C[lo][lo];
    double x[3];
    for (int i = 0; i < 3; ++i) {                 /* x = L^{-T} y */
        double t = 0;
        for (int k = 0; k < 3; ++k) t += Li[k][i] * V[k][lo];
        x[i] = t;
    }
    for (int i = 2; i >= 0; --i) x[i] /= x[0];
    double n0 = 0, n2 = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) { n0 += x[i] * x[j] * mu[i + j]; n2 += x[i] * x[j] * mu[i + j + 2]; }
    out[0] = c + lam;
    out[1] = x[0]; out[2] = x[1]; out[3] = x[2];
    out[4] = n2 / n0 - lam * lam;
}

/* ------------------------------------------------------------------------ */
/* Static spin structure factor (Sec. 4.1)                                    */
/* ------------------------------------------------------------------------ */

/* S(q) = (1/N^2) sum_{i,j} <sz_i sz_j> e^{i q.(r_i - r_j)}, sz = s/2, for
 * every q = 2 pi (qx, qy) / L (out index qx + L qy), as the weighted mean of
 * the diagonal estimator over the configurations (weights NULL: plain mean).
 * Written as the double sum over site pairs; the imaginary parts cancel
 * between (i, j) and (j, i), so only the cosine is summed. */
void or_structure_factor(int L, const int8_t *spins, int n, const double *weights, double *out)
{
    const int N = L * L;
    double *acc = (double *)calloc((size_t)N, sizeof(double));
    double z = 0;
    for (int k = 0; k < n; ++k) z += weights ? weights[k] : 1.0;
    #pragma omp parallel for schedule(static)
    for (int q = 0; q < N; ++q) {
        const int qx = q % L, qy = q / L;
        double sum = 0;
        for (int k = 0; k < n; ++k) {
            const int8_t *s = spins + (size_t)k * N;
            double t = 0;
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < N; ++j) {
                    const int dx = i % L - j % L, dy = i / L - j / L;
                    t += 0.25 * s[i] * s[j] * cos(2.0 * M_PI * (qx * dx + qy * dy) / L);
                }
            sum += (weights ? weights[k] : 1.0) * t;
        }
        acc[q] = sum;
    }
    for (int q = 0; q < N; ++q) out[q] = acc[q] / (z * (double)N * (double)N);
    free(acc);
}

/* ------------------------------------------------------------------------ */
/* Log-derivatives O_k = d log psi / d alpha_k (Sec. 3.2, after Eq. 12)       */
/* ------------------------------------------------------------------------ */

/* O per sample in parameter order [log c_r, a_r, b_r, W_r] for r = 0..K-1.
 * out: [n][K*P1][2].  With w_t = term_t / psi (normalised terms of the
 * projected sum) and u = +-T_g s the transformed configuration of term t:
 *   d/d log c_r = sum_{t in r} w_t
 *   d/d a_rj    = sum_{t in r} w_t u_j
 *   d/d b_rm    = sum_{t in r} w_t tanh(theta_tm)
 *   d/d W_rmj   = sum_{t in r} w_t tanh(theta_tm) u_j
 * (the bias entries are zero when the model has no biases). */
void or_grad_logpsi(void *hp, const int8_t *spins, int n, double *out)
{
    const or_model *h = (const or_model *)hp;
    const int N = h->N, M = h->M, P1 = h->P1;
    const int nsg = h->spin_inv ? 2 : 1;
    #pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < n; ++k) {
        const int8_t *s = spins + (size_t)k * N;
        int nt = n_terms(h);
        cplx *terms = (cplx *)malloc(sizeof(cplx) * nt);
        cplx *O = (cplx *)calloc((size_t)h->K * P1, sizeof(cplx));
        int8_t *t = (int8_t *)malloc(N);
        log_terms(h, s, terms, t);
        cplx lp = log_psi_one(h, s);
        int idx = 0;
        for (int r = 0; r < h->K; ++r) {
            const cplx *p = h->par + (size_t)r * P1;
            const cplx *b = p + 1 + N, *W = p + 1 + N + M;
            cplx *Or = O + (size_t)r * P1;
            for (int g = 0; g < h->G; ++g)
                for (int sg = 0; sg < nsg; ++sg, ++idx) {
                    int sign = sg ? -1 : 1;
                    for (int i = 0; i < N; ++i) t[h->perm[g * N + i]] = (int8_t)(sign * s[i]);
                    cplx w = cexp(terms[idx] - lp);
                    Or[0] += w;
                    if (h->use_bias)
                        for (int j = 0; j < N; ++j) Or[1 + j] += w * t[j];
                    for (int m = 0; m < M; ++m) {
                        cplx th = h->use_bias ? b[m] : 0;
                        for (int j = 0; j < N; ++j) th += W[(size_t)m * N + j] * t[j];
                        cplx wt = w * ctanh(th);
                        if (h->use_bias) Or[1 + N + m] += wt;
                        for (int j = 0; j < N; ++j) Or[1 + N + M + (size_t)m * N + j] += wt * t[j];
                    }
                }
        }
        double *o = out + (size_t)k * h->K * P1 * 2;
        for (size_t q = 0; q < (size_t)h->K * P1; ++q) { o[2 * q] = creal(O[q]); o[2 * q + 1] = cimag(O[q]); }
        free(terms); free(O); free(t);
    }
}

/* Energy gradient F_k = < conj(O_k) (E_loc - <E_loc>) > (right-hand side of
 * Eq. 12 without -dtau).  O: [n][P][2], eloc: [n][2].  weights == NULL: plain
 * sample means; otherwise weighted means with weights |psi|^2 (exact
 * enumeration). */
void or_energy_grad(int n, int P, const double *O, const double *eloc, const double *weights, double *F)
{
    cplx E = 0;
    double z = 0;
    for (int k = 0; k < n; ++k) {
        double w = weights ? weights[k] : 1.0;
        E += w * (eloc[2 * k] + I * eloc[2 * k + 1]);
        z += w;
    }
    E /= z;
    for (int q = 0; q < P; ++q) {
        cplx acc = 0;
        for (int k = 0; k < n; ++k) {
            double w = weights ? weights[k] : 1.0;
            cplx o = O[((size_t)k * P + q) * 2] + I * O[((size_t)k * P + q) * 2 + 1];
            cplx e = eloc[2 * k] + I * eloc[2 * k + 1];
            acc += w * conj(o) * (e - E);
        }
        acc /= z;
        F[2 * q] = creal(acc); F[2 * q + 1] = cimag(acc);
    }
}

/* Stochastic reconfiguration, Eq. 12: (S + lambda I) delta = -dtau F with
 * S_kk' = <conj(O_k) O_k'> - <conj(O_k)><O_k'>, solved densely by Gaussian
 * elimination with partial pivoting (small P only). */
int or_sr_solve(int n, int P, const double *O, const double *F, double lambda, double dtau, double *delta)
{
    cplx *S = (cplx *)calloc((size_t)P * P, sizeof(cplx));
    cplx *x = (cplx *)malloc(sizeof(cplx) * P);
    cplx *mean = (cplx *)calloc(P, sizeof(cplx));
    for (int k = 0; k < n; ++k)
        for (int q = 0; q < P; ++q)
            mean[q] += O[((size_t)k * P + q) * 2] + I * O[((size_t)k * P + q) * 2 + 1];
    for (int q = 0; q < P; ++q) mean[q] /= n;
    for (int k = 0; k < n; ++k)
        for (int a = 0; a < P; ++a) {
            cplx oa = O[((size_t)k * P + a) * 2] + I * O[((size_t)k * P + a) * 2 + 1];
            for (int b = 0; b < P; ++b) {
                cplx ob = O[((size_t)k * P + b) * 2] + I * O[((size_t)k * P + b) * 2 + 1];
                S[(size_t)a * P + b] += conj(oa) * ob;
            }
        }
    for (int a = 0; a < P; ++a)
        for (int b = 0; b < P; ++b)
            S[(size_t)a * P + b] = S[(size_t)a * P + b] / n - conj(mean[a]) * mean[b] + (a == b ? lambda : 0);
    for (int q = 0; q < P; ++q) x[q] = -dtau * (F[2 * q] + I * F[2 * q + 1]);
    for (int c = 0; c < P; ++c) {
        int piv = c;
        for (int r = c + 1; r < P; ++r) if (cabs(S[(size_t)r * P + c]) > cabs(S[(size_t)piv * P + c])) piv = r;
        if (cabs(S[(size_t)piv * P + c]) == 0) { free(S); free(x); free(mean); return -1; }
        if (piv != c) {
            for (int b = 0; b < P; ++b) { cplx tmp = S[(size_t)c * P + b]; S[(size_t)c * P + b] = S[(size_t)piv * P + b]; S[(size_t)piv * P + b] = tmp; }
            cplx tmp = x[c]; x[c] = x[piv]; x[piv] = tmp;
        }
        for (int r = c + 1; r < P; ++r) {
            cplx f = S[(size_t)r * P + c] / S[(size_t)c * P + c];
            if (f == 0) continue;
            for (int b = c; b < P; ++b) S[(size_t)r * P + b] -= f * S[(size_t)c * P + b];
            x[r] -= f * x[c];
        }
    }
    for (int c = P - 1; c >= 0; --c) {
        cplx acc = x[c];
        for (int b = c + 1; b < P; ++b) acc -= S[(size_t)c * P + b] * x[b];
        x[c] = acc / S[(size_t)c * P + c];
    }
    for (int q = 0; q < P; ++q) { delta[2 * q] = creal(x[q]); delta[2 * q + 1] = cimag(x[q]); }
    free(S); free(x); free(mean);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies, with a   */
/* Weyl-sequence key schedule.                                                */
/* ------------------------------------------------------------------------ */

void or_philox4x32_10(const uint32_t *ctr_in, const uint32_t *key_in, uint32_t *out)
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* Metropolis pair-exchange sampler (Sec. 3.2)                                */
/* ------------------------------------------------------------------------ */
/*
 * Conventions (the paper fixes none of them):
 *   key = (seed_lo, seed_hi ^ chain).
 *   Initial state: a Fisher-Yates shuffle of [+1]*N/2 + [-1]*N/2; for
 *   j = N-1 .. 1 the (N-1-j)-th random word x (counter (w/4, 1, 0, 0), word
 *   w%4) picks r = (x * (j+1)) >> 32 and swaps entries j and r.
 *   Step t uses counter (t, 0, 0, 0): words x0, x1 pick the up-rank
 *   ku = (x0 * N/2) >> 32 and the down-rank kd = (x1 * N/2) >> 32; the
 *   proposal exchanges the ku-th up site and the kd-th down site (in
 *   increasing site order).  u = (x2 >> 8) * 2^-24; accept iff
 *   u < |psi(s')/psi(s)|^2.
 *   n_burn steps are discarded, then a sample is kept after every n_skip
 *   steps.  acc_out = accepted / (n_per_chain * n_skip) after burn-in.
 */
static void philox_words(uint64_t seed, int chain, uint32_t c0, uint32_t c1, uint32_t *w)
{
    uint32_t ctr[4] = {c0, c1, 0, 0};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ (uint32_t)chain};
    or_philox4x32_10(ctr, key, w);
}

void or_init_config(uint64_t seed, int chain, int N, int8_t *s)
{
    for (int i = 0; i < N; ++i) s[i] = (int8_t)(i < N / 2 ? 1 : -1);
    uint32_t w[4];
    for (int j = N - 1, q = 0; j >= 1; --j, ++q) {
        if (q % 4 == 0) philox_words(seed, chain, (uint32_t)(q / 4), 1u, w);
        uint32_t x = w[q % 4];
        int r = (int)(((uint64_t)x * (uint64_t)(j + 1)) >> 32);
        int8_t tmp = s[j]; s[j] = s[r]; s[r] = tmp;
    }
}

/* The proposal of step t: sites (iu, id) holding +1 and -1. */
void or_proposal(uint64_t seed, int chain, uint32_t t, int N, const int8_t *s, int *iu, int *id, double *u)
{
    uint32_t w[4];
    philox_words(seed, chain, t, 0u, w);
    int ku = (int)(((uint64_t)w[0] * (uint64_t)(N / 2)) >> 32);
    int kd = (int)(((uint64_t)w[1] * (uint64_t)(N / 2)) >> 32);
    int cu = 0, cd = 0;
    *iu = -1; *id = -1;
    for (int i = 0; i < N; ++i) {
        if (s[i] > 0) { if (cu == ku) *iu = i; ++cu; }
        else { if (cd == kd) *id = i; ++cd; }
    }
    *u = (double)(w[2] >> 8) * (1.0 / 16777216.0);
}

void or_sample(void *hp, uint64_t seed, int n_chains, int n_per_chain, int n_skip, int n_burn,
               int8_t *out, double *acc_out)
{
    const or_model *h = (const or_model *)hp;
    const int N = h->N;
    #pragma omp parallel for schedule(dynamic)
    for (int c = 0; c < n_chains; ++c) {
        int8_t *s = (int8_t *)malloc(N), *sp = (int8_t *)malloc(N);
        or_init_config(seed, c, N, s);
        cplx lp = log_psi_one(h, s);
        long acc = 0;
        uint32_t t = 0;
        int total = n_burn + n_per_chain * n_skip;
        for (int step = 0; step < total; ++step, ++t) {
            int iu, id; double u;
            or_proposal(seed, c, t, N, s, &iu, &id, &u);
            memcpy(sp, s, N);
            sp[iu] = -1; sp[id] = 1;
            cplx lpp = log_psi_one(h, sp);
            double r2 = exp(2.0 * creal(lpp - lp));
            if (u < r2) { memcpy(s, sp, N); lp = lpp; if (step >= n_burn) ++acc; }
            if (step >= n_burn && (step - n_burn + 1) % n_skip == 0) {
                int kept = (step - n_burn + 1) / n_skip - 1;
                memcpy(out + ((size_t)c * n_per_chain + kept) * N, s, N);
            }
        }
        if (acc_out) acc_out[c] = n_per_chain * n_skip > 0 ? (double)acc / (n_per_chain * n_skip) : 0.0;
        free(s); free(sp);
    }
}

/* ------------------------------------------------------------------------ */
/* Exact diagonalisation of the Sz = 0 sector (Eq. 1), for the 4x4 pins       */
/* ------------------------------------------------------------------------ */

/* Sz = 0 basis: all N-bit patterns with N/2 set bits (bit i set <=> s_i = +1),
 * ascending.  Returns the dimension; fills states if non-NULL. */
long or_sz0_basis(int N, uint64_t *states)
{
    long d = 0;
    if (N > 30) return -1;
    for (uint64_t x = 0; x < (1ull << N); ++x)
        if (__builtin_popcountll(x) == N / 2) { if (states) states[d] = x; ++d; }
    return d;
}

static long find_state(const uint64_t *states, long d, uint64_t x)
{
    long lo = 0, hi = d - 1;
    while (lo <= hi) {
        long mid = (lo + hi) / 2;
        if (states[mid] == x) return mid;
        if (states[mid] < x) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* y = H x in the Sz=0 basis (real symmetric H). */
void or_apply_h(int L, double J1, double J2, const uint64_t *states, long d, const double *x, double *y)
{
    int N = L * L;
    int bi[4 * 64], bj[4 * 64], bt[4 * 64];
    int nb = or_bonds(L, bi, bj, bt);
    #pragma omp parallel for schedule(static)
    for (long k = 0; k < d; ++k) {
        uint64_t st = states[k];
        double acc = 0;
        for (int b = 0; b < nb; ++b) {
            double J = bt[b] == 1 ? J1 : J2;
            int si = (st >> bi[b]) & 1, sj = (st >> bj[b]) & 1;
            acc += 0.25 * J * (si == sj ? 1.0 : -1.0) * x[k];
            if (si != sj) {
                long k2 = find_state(states, d, st ^ ((1ull << bi[b]) | (1ull << bj[b])));
                acc += 0.5 * J * x[k2];
            }
        }
        y[k] = acc;
    }
    (void)N;
}

/* Number of eigenvalues of the symmetric tridiagonal (a, b) below x
 * (Sturm sequence count of the LDL^T pivots). */
static int sturm_count(int n, const double *a, const double *b, double x)
{
    int cnt = 0;
    double q = a[0] - x;
    if (q < 0) ++cnt;
    for (int k = 1; k < n; ++k) {
        double den = q != 0 ? q : 1e-300;
        q = a[k] - x - b[k - 1] * b[k - 1] / den;
        if (q < 0) ++cnt;
    }
    return cnt;
}

/* Ground state of the Sz=0 sector.  Lanczos with full re-orthogonalisation
 * (at most maxit vectors), lowest Ritz value by bisection on the Sturm
 * count, Ritz vector from inverse iteration on the tridiagonal matrix.
 * Returns the eigenvalue; vec (length d) receives the normalised vector. */
double or_ed_ground(int L, double J1, double J2, int maxit, double *vec)
{
    int N = L * L;
    long d = or_sz0_basis(N, NULL);
    uint64_t *states = (uint64_t *)malloc(sizeof(uint64_t) * d);
    or_sz0_basis(N, states);
    if (maxit > d) maxit = (int)d;
    double *V = (double *)malloc(sizeof(double) * (size_t)d * (maxit + 1));
    double *a = (double *)calloc(maxit + 1, sizeof(double));
    double *b = (double *)calloc(maxit + 1, sizeof(double));
    double *w = (double *)malloc(sizeof(double) * d);
    /* deterministic start vector with weight on every state */
    double nrm = 0;
    for (long k = 0; k < d; ++k) { V[k] = 1.0 + 0.5 * sin(0.37 * k + 0.1); nrm += V[k] * V[k]; }
    nrm = sqrt(nrm);
    for (long k = 0; k < d; ++k) V[k] /= nrm;
    int m = 0;
    for (int it = 0; it < maxit; ++it) {
        double *v = V + (size_t)it * d;
        or_apply_h(L, J1, J2, states, d, v, w);
        double al = 0;
        for (long k = 0; k < d; ++k) al += v[k] * w[k];
        a[it] = al;
        for (int pass = 0; pass < 2; ++pass)
            for (int j = 0; j <= it; ++j) {
                double *vj = V + (size_t)j * d, c = 0;
                for (long k = 0; k < d; ++k) c += vj[k] * w[k];
                for (long k = 0; k < d; ++k) w[k] -= c * vj[k];
            }
        double be = 0;
        for (long k = 0; k < d; ++k) be += w[k] * w[k];
        be = sqrt(be);
        m = it + 1;
        if (be < 1e-12 || it == maxit - 1) break;
        b[it] = be;
        double *vn = V + (size_t)(it + 1) * d;
        for (long k = 0; k < d; ++k) vn[k] = w[k] / be;
    }
    /* bisection for the lowest eigenvalue of T (m x m) */
    double lo = a[0], hi = a[0];
    for (int k = 0; k < m; ++k) {
        double r = (k > 0 ? fabs(b[k - 1]) : 0) + (k < m - 1 ? fabs(b[k]) : 0);
        if (a[k] - r < lo) lo = a[k] - r;
        if (a[k] + r > hi) hi = a[k] + r;
    }
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (sturm_count(m, a, b, mid) >= 1) hi = mid; else lo = mid;
        if (hi - lo < 1e-15 * (fabs(lo) + fabs(hi) + 1)) break;
    }
    double lam = 0.5 * (lo + hi);
    /* inverse iteration on T - (lam - eps) I, which is positive definite */
    double shift = lam - 1e-10 * (fabs(lam) + 1);
    double *y = (double *)malloc(sizeof(double) * m), *cp = (double *)malloc(sizeof(double) * m);
    double *dp = (double *)malloc(sizeof(double) * m);
    for (int k = 0; k < m; ++k) y[k] = 1.0;
    for (int rep = 0; rep < 4; ++rep) {
        /* Thomas algorithm */
        double den = a[0] - shift;
        cp[0] = (m > 1 ? b[0] : 0) / den; dp[0] = y[0] / den;
        for (int k = 1; k < m; ++k) {
            den = a[k] - shift - b[k - 1] * cp[k - 1];
            cp[k] = (k < m - 1 ? b[k] : 0) / den;
            dp[k] = (y[k] - b[k - 1] * dp[k - 1]) / den;
        }
        y[m - 1] = dp[m - 1];
        for (int k = m - 2; k >= 0; --k) y[k] = dp[k] - cp[k] * y[k + 1];
        double s = 0;
        for (int k = 0; k < m; ++k) s += y[k] * y[k];
        s = sqrt(s);
        for (int k = 0; k < m; ++k) y[k] /= s;
    }
    for (long k = 0; k < d; ++k) {
        double acc = 0;
        for (int j = 0; j < m; ++j) acc += V[(size_t)j * d + k] * y[j];
        vec[k] = acc;
    }
    nrm = 0;
    for (long k = 0; k < d; ++k) nrm += vec[k] * vec[k];
    nrm = sqrt(nrm);
    for (long k = 0; k < d; ++k) vec[k] /= nrm;
    free(states); free(V); free(a); free(b); free(w); free(y); free(cp); free(dp);
    return lam;
}

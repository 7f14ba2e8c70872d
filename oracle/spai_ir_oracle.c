/*
 * Plain, slow CPU oracle for SPAI-GMRES-IR (Carson & Khan, arXiv 2202.10204).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code, header, table or helper with the CUDA path; it is written from the
 * paper's definitions:
 *   - Section 2.2, eq. (fronormmin) and (redprob): column-wise Frobenius
 *     least squares on the shadow I_k of the pattern J_k;
 *   - Algorithm 1 (Grote-Huckle / Sedlacek variant): fixed or adaptive
 *     pattern, rho_jk scores, mean-acceptance, up to beta additions per step;
 *   - Section 4 (experimental set-up): SPAI is run on A^T D where D scales
 *     every column of A^T to max-abs 1, and P = M^T D;
 *   - Algorithm 3 (SPAI-GMRES-IR): x0 = P b in u_f, residual in u_r,
 *     left-preconditioned MGS-GMRES in u_g with products in u_p, update in u.
 *
 * Arithmetic model.  Double is native.  Quad is _Float128 (software, IEEE
 * binary128).  Single is obtained by rounding a double result to float, and
 * half by a hand-written round-to-nearest-even "chop" to 11 significant bits
 * with exponent range [-14, 15], gradual underflow to 2^-24 and overflow to
 * +-Inf (the paper simulates half with the chop library, Section 4).  A
 * double result of +,-,*,/,sqrt on operands of precision p (p = half or
 * single) rounded to p equals the correctly rounded p-result, because 53 >=
 * 2*24 + 2.  The file must be compiled with -ffp-contract=off.
 *
 * Inner products.  Section 4 runs single and double as the built-in
 * datatypes, whose vector reductions are library routines rather than one
 * left-to-right chain; the oracle takes pairwise summation, the textbook
 * model of such a reduction: sum(a[0..n)) = sum(a[0..n/2)) + sum(a[n/2..n)),
 * every product and every addition rounded to the precision (error bound
 * gamma_{ceil(log2 n)+1} sum |x_i y_i|).  Half (the chop simulation) keeps
 * the per-operation left-to-right chain.  With a strict chain of 262,144
 * single-precision additions the Arnoldi basis of the 64^3 system lost all
 * orthogonality within 60 steps, unlike any single-precision library.
 *
 * Two SPAI arithmetic modes:
 *   MODE_PEROP : every operation rounded to u_f (the paper's model);
 *   MODE_ACC32 : at u_f = half, stored values are rounded to half but every
 *                inner product / norm is accumulated in binary32 and rounded
 *                to half once (the FP16-storage / FP32-accumulate model).  At
 *                u_f = single or double the two modes coincide.
 *
 * The same two modes for the Krylov part (kmode) when u_g or u_p is half:
 *   MODE_PEROP : every GMRES operation rounded to u_g / u_p (the paper's chop
 *                model);
 *   MODE_ACC32 : (one-reduction MGS only) half is a storage format: the
 *                basis vectors, u_j and w are stored in half, every scalar,
 *                inner product, quotient and update is computed in binary32
 *                and the vectors are rounded to half once when stored; the
 *                sparse products take half matrix values and inputs,
 *                multiply and sum in binary32 and round the result to half.
 *                At u_g, u_p in {single, double} it is MODE_PEROP.
 *
 * Readings of points where the paper is silent or garbled (each one is a
 * parameter or a documented constant):
 *   R1  L_k = { l in I_k : s_l != 0 }, and I_k always contains k.
 *   R2  N_l = { j : b_lj != 0 } \ J_k (row l of B), J~_k = union of N_l.
 *   R3  rho_j^2 = max(0, ||s||^2 - (s^T b_j)^2 / ||b_j||^2) with b_j the full
 *       column j of B (rho_restricted=1: b_j restricted to I_k).  The
 *       selection statistics (rho^2, the mean) are accumulated in binary32
 *       at u_f = half, in u_f otherwise.
 *   R4  mean over J~_k; acceptable = rho_j <= mean; add the
 *       min(beta, max_fill - |J_k|) acceptable indices with smallest rho,
 *       ties broken by the smaller index.
 *   R5  at most alpha + 1 least-squares solves; no augmentation after the
 *       last one.
 *   R6  |J_k| <= max_fill; an initial pattern larger than the cap keeps k,
 *       then the indices nearest to k (ties: smaller index).
 *   R7  MGS-GMRES, x0 = 0, no restart, stop when |g_{j+1}| / beta <= tau;
 *       Givens rotations, H, g and y in double.  Options: classical
 *       Gram-Schmidt applied twice (CGS2) instead of MGS; and MGS in its
 *       inverse compact WY form with one reduction per iteration and lagged
 *       normalisation (Swirydowicz, Langou, Ananthan, Yang and Thomas, "Low
 *       synchronization Gram-Schmidt and GMRES algorithms", 2020), which
 *       equals MGS in exact arithmetic; see orc_gmres.
 *   R8  IR stop (the paper fixes only i_max), checked before step i in this
 *       order: BACKWARD rule: nbe_i = ||r_i||_inf / (||A||_inf ||x_i||_inf
 *       + ||b||_inf) <= stop_tol; CORRECTION rule: i >= 1 and
 *       q_i = ||d_{i-1}||_inf / ||x_i||_inf <= stop_tol (the relative size of
 *       the last correction); i = i_max; then, for both rules, stagnation:
 *       i >= 2 and q_i >= q_{i-1} / 2 (the correction did not halve), which
 *       stops without convergence.  The FIXED rule runs i_max solves.
 *   R10 pattern(A) / pattern(A^2) initial patterns: J_k = nonzero rows of
 *       column k of A (resp. A^2).
 *   R14 right preconditioning (the paper leaves it as future work at the
 *       end of Section 3): GMRES on (A P) u = r from u = 0, w = A (P v_j)
 *       with both products in u_p, the initial vector r rounded to u_p and
 *       u_g (as with P = I), and the correction d = P (V_k y) in u_p,
 *       stored in u_g.  The right SPAI (A P ~ I) is the transpose of the
 *       left SPAI of A^T (Algorithm 1 run on A D, D scaling the columns of A).
 *   R17 u_g or u_p = half (Algorithm 3 allows any precision there; the
 *       paper's runs use u_g = u_p = u): GMRES gets the residual scaled by
 *       the power of two 2^-e with ||r||_inf = m 2^e, m in [0.5, 1) (exact),
 *       and the correction is scaled back by 2^e; otherwise the residuals of
 *       a converging refinement fall below half's range.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PH 0 /* half,   u = 2^-11  */
#define PS 1 /* single, u = 2^-24  */
#define PD 2 /* double, u = 2^-53  */
#define PQ 3 /* quad,   u = 2^-113 */

#define MODE_PEROP 0
#define MODE_ACC32 1

#define PAT_IDENTITY 0
#define PAT_A 1
#define PAT_A2 2

/* column flags */
#define CF_CONVERGED 1   /* ||s|| <= eps reached                */
#define CF_FILLCAP 2     /* stopped because |J_k| hit max_fill  */
#define CF_ALPHA 4       /* stopped because alpha steps done    */
#define CF_NOCAND 8      /* no acceptable candidate to add      */
#define CF_SINGULAR 16   /* a zero pivot in R                   */
#define CF_NONFINITE 32  /* Inf/NaN appeared (overflow in u_f)  */

/* IR status flags */
#define IR_CONVERGED 1
#define IR_MAXSTEPS 2
#define IR_BREAKDOWN 4
#define IR_NONFINITE 8
#define IR_STAGNATED 16

/* IR stopping rules (reading R8) */
#define STOP_BACKWARD 0
#define STOP_FIXED 1
#define STOP_CORRECTION 2

/* ------------------------------------------------------------------ */
/* Rounding to a precision (Table 1)                                   */
/* ------------------------------------------------------------------ */

/* Round a double to IEEE binary16, round-to-nearest-even, written out from
 * the format's definition: 11 significant bits, normal exponents [-14, 15],
 * subnormal quantum 2^-24, largest finite 65504. */
double orc_chop_half(double x)
{
    if (isnan(x)) return x;
    double ax = fabs(x);
    if (ax == 0.0) return x;
    /* 65520 is the midpoint between 65504 and 2^16; ties go to the even
     * neighbour 2^16, which overflows. */
    if (ax >= 65520.0) return x > 0 ? INFINITY : -INFINITY;
    int e;
    frexp(ax, &e);          /* ax = f * 2^e, f in [0.5, 1) => leading bit 2^(e-1) */
    int lead = e - 1;
    if (lead < -14) lead = -14; /* subnormal range: fixed quantum 2^-24 */
    double quantum = ldexp(1.0, lead - 10);
    double q = rint(ax / quantum) * quantum; /* rint: nearest-even */
    return x < 0 ? -q : q;
}

/* x rounded to precision p (Table 1): half by chop, single by the IEEE
 * conversion to float (round-to-nearest-even), double and quad unchanged
 * (quad values are carried as _Float128 where they occur). */
static double rnd(double x, int p)
{
    switch (p) {
    case PH: return orc_chop_half(x);
    case PS: return (double)(float)x;
    default: return x;
    }
}

/* rnd, exported for the pins. */
double orc_round(double x, int p) { return rnd(x, p); }

/* out[i] = x[i] rounded to p, i < n */
void orc_round_array(int64_t n, const double* x, int p, double* out)
{
    for (int64_t i = 0; i < n; i++) out[i] = rnd(x[i], p);
}

/* ------------------------------------------------------------------ */
/* Inner products in a precision under a mode                          */
/* ------------------------------------------------------------------ */

/* Pairwise sum of the products x[i*sx] * y[i*sy], i in [0, len), each
 * product and each addition rounded to p. */
static double dot_pairwise(const double* x, int sx, const double* y, int sy, int len, int p)
{
    if (len <= 0) return 0.0;
    if (len == 1) return rnd(x[0] * y[0], p);
    int m = len / 2;
    double a = dot_pairwise(x, sx, y, sy, m, p);
    double b = dot_pairwise(x + (size_t)m * sx, sx, y + (size_t)m * sy, sy, len - m, p);
    return rnd(a + b, p);
}

/* sum_i x[i*sx] * y[i*sy] computed in precision p: pairwise in single and
 * double, a left-to-right chain in half (per operation, or accumulated in
 * binary32 and rounded once under MODE_ACC32). */
static double dot_p(const double* x, int sx, const double* y, int sy, int len, int p, int mode)
{
    if (p != PH) return dot_pairwise(x, sx, y, sy, len, p);
    if (mode == MODE_ACC32) {
        float acc = 0.0f;
        for (int i = 0; i < len; i++) {
            float t = (float)x[(size_t)i * sx] * (float)y[(size_t)i * sy];
            acc = acc + t;
        }
        return orc_chop_half((double)acc);
    }
    double acc = 0.0;
    for (int i = 0; i < len; i++) {
        double t = rnd(x[(size_t)i * sx] * y[(size_t)i * sy], p);
        acc = rnd(acc + t, p);
    }
    return acc;
}

/* ------------------------------------------------------------------ */
/* Dense least squares by Householder QR (Algorithm 1, QR + solve)     */
/* ------------------------------------------------------------------ */

/*
 * Solve min || ebar - Abar mbar ||_2 for Abar (m x nc, column-major, values
 * already in u_f) by Householder QR in precision p under mode, then
 * mbar = R^{-1} (Q^T ebar)(1:nc) by back substitution, then the explicit
 * residual sbar = Abar mbar - ebar and ||sbar||_2 (Algorithm 1, the QR,
 * solve and residual lines).  Reflector: v = x - alpha e_1 with
 * alpha = -sign(x_1) ||x||, sign(0) = +1; H = I - 2 v v^T / (v^T v).
 * Returns flags (CF_SINGULAR / CF_NONFINITE).  sbar may be NULL.
 */
int orc_dense_ls(int m, int nc, const double* Abar, const double* ebar, int p, int mode,
                 double* mbar, double* sbar, double* snorm)
{
    int flags = 0;
    double* W = (double*)malloc(sizeof(double) * (size_t)m * (nc + 1)); /* [Abar | ebar] */
    double* v = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double* s = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    memcpy(W, Abar, sizeof(double) * (size_t)m * nc);
    memcpy(W + (size_t)m * nc, ebar, sizeof(double) * (size_t)m);
    int steps = nc < m ? nc : m;
    for (int c = 0; c < steps; c++) {
        double* x = W + (size_t)c * m + c;
        int len = m - c;
        double sig2 = dot_p(x, 1, x, 1, len, p, mode);
        double nrm = rnd(sqrt(sig2), p);
        if (nrm == 0.0) continue; /* zero column: H = I, R(c,c) = 0 */
        double alpha = x[0] >= 0.0 ? -nrm : nrm;
        for (int i = 0; i < len; i++) v[i] = x[i];
        v[0] = rnd(x[0] - alpha, p);
        double vtv = dot_p(v, 1, v, 1, len, p, mode);
        for (int t = c + 1; t <= nc; t++) { /* trailing columns and ebar */
            double* a = W + (size_t)t * m + c;
            double sv = dot_p(v, 1, a, 1, len, p, mode);
            double f = rnd(rnd(2.0 * sv, p) / vtv, p);
            for (int i = 0; i < len; i++) a[i] = rnd(a[i] - rnd(f * v[i], p), p);
        }
        x[0] = alpha;
        for (int i = 1; i < len; i++) x[i] = 0.0;
    }
    /* back substitution R mbar = (Q^T ebar)(1:nc) */
    const double* y = W + (size_t)m * nc;
    for (int c = nc - 1; c >= 0; c--) {
        if (c >= m) { mbar[c] = 0.0; flags |= CF_SINGULAR; continue; }
        double acc = y[c];
        /* acc - sum_{t>c} R(c,t) mbar(t), accumulated per mode */
        double sum = 0.0;
        if (nc - 1 - c > 0) sum = dot_p(W + (size_t)(c + 1) * m + c, m, mbar + c + 1, 1, nc - 1 - c, p, mode);
        acc = rnd(acc - sum, p);
        double rcc = W[(size_t)c * m + c];
        if (rcc == 0.0) { mbar[c] = 0.0; flags |= CF_SINGULAR; continue; }
        mbar[c] = rnd(acc / rcc, p);
    }
    /* explicit residual sbar = Abar mbar - ebar with the original Abar */
    for (int i = 0; i < m; i++) {
        double am = dot_p(Abar + i, m, mbar, 1, nc, p, mode);
        s[i] = rnd(am - ebar[i], p);
    }
    *snorm = rnd(sqrt(dot_p(s, 1, s, 1, m, p, mode)), p);
    if (sbar) memcpy(sbar, s, sizeof(double) * (size_t)m);
    for (int c = 0; c < nc; c++) if (!isfinite(mbar[c])) flags |= CF_NONFINITE;
    if (!isfinite(*snorm)) flags |= CF_NONFINITE;
    free(W); free(v); free(s);
    return flags;
}

/* ------------------------------------------------------------------ */
/* Sparse helpers                                                      */
/* ------------------------------------------------------------------ */

static int cmp_int(const void* a, const void* b)
{
    int x = *(const int*)a, y = *(const int*)b;
    return (x > y) - (x < y);
}

/* sort ascending and drop duplicates; returns the new length */
static int sort_unique(int* v, int len)
{
    if (len <= 1) return len;
    qsort(v, (size_t)len, sizeof(int), cmp_int);
    int w = 1;
    for (int i = 1; i < len; i++) if (v[i] != v[w - 1]) v[w++] = v[i];
    return w;
}

/* Position of key in the ascending v[0..len), -1 if absent (binary search). */
static int find_sorted(const int* v, int len, int key)
{
    int lo = 0, hi = len - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (v[mid] == key) return mid;
        if (v[mid] < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* structure of A^T (column lists of A): colptr[n+1], rowidx[nnz] sorted */
static void transpose_structure(int n, const int64_t* rp, const int* ci, int64_t* cp, int* ri)
{
    for (int j = 0; j <= n; j++) cp[j] = 0;
    for (int i = 0; i < n; i++)
        for (int64_t q = rp[i]; q < rp[i + 1]; q++) cp[ci[q] + 1]++;
    for (int j = 0; j < n; j++) cp[j + 1] += cp[j];
    int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int j = 0; j < n; j++) cur[j] = cp[j];
    for (int i = 0; i < n; i++) /* rows in increasing order => sorted lists */
        for (int64_t q = rp[i]; q < rp[i + 1]; q++) ri[cur[ci[q]]++] = i;
    free(cur);
}

/* order for the fill cap (R6): k first, then by |j-k|, then by j */
static _Thread_local int g_cap_k; /* the column of the qsort in apply_cap (per thread) */
static int cmp_cap(const void* a, const void* b)
{
    int x = *(const int*)a, y = *(const int*)b;
    long dx = labs((long)x - g_cap_k), dy = labs((long)y - g_cap_k);
    if (dx != dy) return (dx > dy) - (dx < dy);
    return (x > y) - (x < y);
}

/* The fill cap of reading R6: a pattern longer than max_fill keeps the
 * max_fill indices nearest to k (k itself first, ties to the smaller
 * index), returned in ascending order. */
static int apply_cap(int* J, int len, int k, int max_fill)
{
    if (len <= max_fill) return len;
    g_cap_k = k;
    qsort(J, (size_t)len, sizeof(int), cmp_cap);
    len = max_fill;
    qsort(J, (size_t)len, sizeof(int), cmp_int);
    return len;
}

/* ------------------------------------------------------------------ */
/* SPAI (Algorithm 1 on B = A^T D, P = M^T D)                           */
/* ------------------------------------------------------------------ */

typedef struct {
    int init;            /* PAT_IDENTITY, PAT_A, PAT_A2 */
    int adaptive;        /* 0 fixed pattern, 1 Grote-Huckle augmentation */
    double eps;          /* column tolerance */
    int alpha, beta;     /* alpha < 0 => ceil(n / beta) */
    int max_fill;        /* cap on |J_k| */
    int uf;              /* precision of the construction */
    int mode;            /* MODE_PEROP / MODE_ACC32 */
    int rho_restricted;  /* R3 literal reading */
    int scale;           /* 1: run on A^T D (Section 4); 0: on A^T */
} orc_spai_opts;

/* Candidate scores rho_j (Algorithm 1, rho_jk line; reading R3).
 * s: residual on I (length m, in u_f); cand: candidate indices; B's column j
 * is row j of A times d_j.  Writes rho (length ncand). */
void orc_rho(int n, const int64_t* rp, const int* ci, const double* val, const double* d,
             int m, const int* I, const double* s, int ncand, const int* cand, int uf,
             int rho_restricted, double* rho)
{
    (void)n;
    int ps = (uf == PH) ? PS : uf; /* statistics precision (R3) */
    double s2 = 0.0;
    for (int i = 0; i < m; i++) s2 = rnd(s2 + rnd(s[i] * s[i], ps), ps);
    for (int c = 0; c < ncand; c++) {
        int j = cand[c];
        double num = 0.0, den = 0.0;
        for (int64_t q = rp[j]; q < rp[j + 1]; q++) {
            double bij = rnd(val[q] * d[j], uf); /* b_ij = a_ji d_j in u_f */
            int pos = find_sorted(I, m, ci[q]);
            if (pos >= 0) num = rnd(num + rnd(s[pos] * bij, ps), ps);
            if (!rho_restricted || pos >= 0) den = rnd(den + rnd(bij * bij, ps), ps);
        }
        double r2 = s2;
        if (den > 0.0) r2 = rnd(s2 - rnd(rnd(num * num, ps) / den, ps), ps);
        if (r2 < 0.0) r2 = 0.0;
        rho[c] = rnd(sqrt(r2), ps);
    }
}

/* Selection (Algorithm 1, mean and "add up to beta" lines; reading R4).
 * Returns the number selected; sel receives the chosen indices. */
int orc_select(int ncand, const int* cand, const double* rho, int uf, int nmax, int* sel)
{
    if (ncand <= 0 || nmax <= 0) return 0;
    int ps = (uf == PH) ? PS : uf;
    double sum = 0.0;
    for (int c = 0; c < ncand; c++) sum = rnd(sum + rho[c], ps);
    double mean = rnd(sum / (double)ncand, ps);
    int* used = (int*)calloc((size_t)ncand, sizeof(int));
    int nsel = 0;
    for (int t = 0; t < nmax; t++) {
        int best = -1;
        for (int c = 0; c < ncand; c++) {
            if (used[c] || !(rho[c] <= mean)) continue;
            if (best < 0 || rho[c] < rho[best] || (rho[c] == rho[best] && cand[c] < cand[best])) best = c;
        }
        if (best < 0) break;
        used[best] = 1;
        sel[nsel++] = cand[best];
    }
    free(used);
    return nsel;
}

/*
 * Build the SPAI preconditioner P = M^T D.
 * Inputs: CSR A (n, rp[n+1], ci[nnz], val[nnz]), options.
 * Outputs (caller-allocated):
 *   d[n]                 scaling (1 if !scale)
 *   Jcnt[n]              |J_k|
 *   Jidx[n*max_fill]     J_k (sorted), padded
 *   mval[n*max_fill]     mbar_k in u_f (padded)
 *   colres[n]            ||sbar_k|| as computed in u_f
 *   colres64[n]          ||e_k - B(:,J_k) mbar_k||_2 re-evaluated in double
 *   flags[n]             CF_* flags
 *   nsolve[n]            least-squares solves performed for column k
 *   Icnt[n]              |I_k| of the last solve
 * Column subset: if cols != NULL only those ncols columns are computed.
 */
int orc_spai(int n, const int64_t* rp, const int* ci, const double* val, const orc_spai_opts* o,
             int ncols, const int* cols, double* d, int* Jcnt, int* Jidx, double* mval,
             double* colres, double* colres64, int* flags, int* nsolve, int* Icnt)
{
    int64_t nnz = rp[n];
    int64_t* cp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int* ri = (int*)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    transpose_structure(n, rp, ci, cp, ri);
    /* scaling D: d_j = 1 / max_i |a_ji| (Section 4: every column of A^T,
     * i.e. every row of A, gets max-abs 1) */
    for (int j = 0; j < n; j++) {
        double mx = 0.0;
        for (int64_t q = rp[j]; q < rp[j + 1]; q++) if (fabs(val[q]) > mx) mx = fabs(val[q]);
        d[j] = o->scale ? (mx > 0.0 ? 1.0 / mx : 1.0) : 1.0;
    }
    int beta = o->beta;
    int alpha = o->alpha < 0 ? (n + beta - 1) / (beta > 0 ? beta : 1) : o->alpha;
    int F = o->max_fill;
    int total = ncols > 0 && cols ? ncols : n;
    /* scratch large enough for any single column */
    int maxrow = 0, maxcol = 0;
    for (int i = 0; i < n; i++) if (rp[i + 1] - rp[i] > maxrow) maxrow = (int)(rp[i + 1] - rp[i]);
    for (int j = 0; j < n; j++) if (cp[j + 1] - cp[j] > maxcol) maxcol = (int)(cp[j + 1] - cp[j]);
    size_t capI = (size_t)F * maxrow + 2;
    size_t capJ0 = (size_t)maxcol * maxcol + (size_t)F + 2;
    size_t capC = capI * (size_t)(maxcol + 1) + 2;
    /* the columns are independent (Section 2.2): with OpenMP they are shared
     * among threads, each with scratch of its own; no arithmetic changes */
#pragma omp parallel
    {
    int* J = (int*)malloc(sizeof(int) * (capJ0 > (size_t)F ? capJ0 : (size_t)F + 2));
    int* I = (int*)malloc(sizeof(int) * capI);
    int* cand = (int*)malloc(sizeof(int) * capC);
    double* rho = (double*)malloc(sizeof(double) * capC);
    int* sel = (int*)malloc(sizeof(int) * (size_t)(beta + 1));
    double* Abar = (double*)malloc(sizeof(double) * capI * (size_t)F);
    double* ebar = (double*)malloc(sizeof(double) * capI);
    double* mb = (double*)malloc(sizeof(double) * (size_t)F);
    double* sb = (double*)malloc(sizeof(double) * capI);
#pragma omp for schedule(dynamic, 64)
    for (int t = 0; t < total; t++) {
        int k = (cols && ncols > 0) ? cols[t] : t;
        /* initial pattern J_k (R10), capped (R6) */
        int nj = 0;
        if (o->init == PAT_IDENTITY) {
            J[nj++] = k;
        } else if (o->init == PAT_A) {
            for (int64_t q = cp[k]; q < cp[k + 1]; q++) J[nj++] = ri[q];
        } else {
            for (int64_t q = cp[k]; q < cp[k + 1]; q++) {
                int i = ri[q];
                for (int64_t q2 = cp[i]; q2 < cp[i + 1]; q2++) J[nj++] = ri[q2];
            }
        }
        nj = sort_unique(J, nj);
        nj = apply_cap(J, nj, k, F);
        int fl = 0, ns = 0, m = 0;
        double snorm = 0.0;
        for (int step = 0; step <= alpha; step++) {
            /* shadow I_k = union of nonzero columns of rows j in J_k, plus k */
            m = 0;
            for (int c = 0; c < nj; c++)
                for (int64_t q = rp[J[c]]; q < rp[J[c] + 1]; q++) if (val[q] != 0.0) I[m++] = ci[q];
            I[m++] = k;
            m = sort_unique(I, m);
            /* Abar = B(I_k, J_k) in u_f, ebar = e_k(I_k) */
            for (size_t z = 0; z < (size_t)m * nj; z++) Abar[z] = 0.0;
            for (int c = 0; c < nj; c++) {
                int j = J[c];
                for (int64_t q = rp[j]; q < rp[j + 1]; q++) {
                    if (val[q] == 0.0) continue;
                    int pos = find_sorted(I, m, ci[q]);
                    Abar[(size_t)c * m + pos] = rnd(val[q] * d[j], o->uf);
                }
            }
            for (int i = 0; i < m; i++) ebar[i] = (I[i] == k) ? 1.0 : 0.0;
            fl &= ~(CF_SINGULAR | CF_NONFINITE);
            fl |= orc_dense_ls(m, nj, Abar, ebar, o->uf, o->mode, mb, sb, &snorm);
            ns++;
            if (snorm <= o->eps) { fl |= CF_CONVERGED; break; }
            if (!o->adaptive) break;
            if (step == alpha) { fl |= CF_ALPHA; break; }
            if (nj >= F) { fl |= CF_FILLCAP; break; }
            /* L_k (R1) and the candidate set J~_k (R2) */
            int nc = 0;
            for (int i = 0; i < m; i++) {
                if (sb[i] == 0.0) continue;
                int l = I[i];
                for (int64_t q = cp[l]; q < cp[l + 1]; q++) {
                    int j = ri[q];
                    if (find_sorted(J, nj, j) < 0) cand[nc++] = j;
                }
            }
            nc = sort_unique(cand, nc);
            if (nc == 0) { fl |= CF_NOCAND; break; }
            orc_rho(n, rp, ci, val, d, m, I, sb, nc, cand, o->uf, o->rho_restricted, rho);
            int room = F - nj;
            int nadd = orc_select(nc, cand, rho, o->uf, beta < room ? beta : room, sel);
            if (nadd == 0) { fl |= CF_NOCAND; break; }
            for (int a = 0; a < nadd; a++) J[nj++] = sel[a];
            nj = sort_unique(J, nj);
        }
        Jcnt[k] = nj;
        for (int c = 0; c < F; c++) {
            Jidx[(size_t)k * F + c] = c < nj ? J[c] : -1;
            mval[(size_t)k * F + c] = c < nj ? mb[c] : 0.0;
        }
        colres[k] = snorm;
        flags[k] = fl;
        nsolve[k] = ns;
        Icnt[k] = m;
        /* true residual in double: || e_k - B(:,J) mbar || over I_k */
        double acc = 0.0;
        for (int i = 0; i < m; i++) {
            double bm = 0.0;
            for (int c = 0; c < nj; c++) {
                int j = J[c];
                for (int64_t q = rp[j]; q < rp[j + 1]; q++)
                    if (ci[q] == I[i]) bm += val[q] * d[j] * mb[c];
            }
            double e = (I[i] == k) ? 1.0 : 0.0;
            acc += (e - bm) * (e - bm);
        }
        colres64[k] = sqrt(acc);
    }
    free(J); free(I); free(cand); free(rho); free(sel);
    free(Abar); free(ebar); free(mb); free(sb);
    }
    free(cp); free(ri);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Sparse matrix-vector products in a precision                        */
/* ------------------------------------------------------------------ */

/* y = M x with M's values and x rounded to p, products and sums in p
 * (acc32 at p = half: products and sums in binary32), y rounded to p. */
static void spmv_p(int n, const int64_t* rp, const int* ci, const double* mv, const double* x,
                   int p, int mode, double* y)
{
    for (int i = 0; i < n; i++) {
        if (p == PH && mode == MODE_ACC32) {
            float acc = 0.0f;
            for (int64_t q = rp[i]; q < rp[i + 1]; q++) {
                float t = (float)orc_chop_half(mv[q]) * (float)orc_chop_half(x[ci[q]]);
                acc = acc + t;
            }
            y[i] = orc_chop_half((double)acc);
        } else {
            double acc = 0.0;
            for (int64_t q = rp[i]; q < rp[i + 1]; q++)
                acc = rnd(acc + rnd(rnd(mv[q], p) * rnd(x[ci[q]], p), p), p);
            y[i] = acc;
        }
    }
}

/* r = b - A x in precision ur, stored in precision u (Algorithm 3 residual) */
static void residual_ur(int n, const int64_t* rp, const int* ci, const double* av, const double* b,
                        const double* x, int ur, int u, double* r)
{
    for (int i = 0; i < n; i++) {
        if (ur == PQ) {
            _Float128 s = (_Float128)b[i];
            for (int64_t q = rp[i]; q < rp[i + 1]; q++) s = s - (_Float128)av[q] * (_Float128)x[ci[q]];
            r[i] = rnd((double)s, u);
        } else {
            double s = b[i];
            for (int64_t q = rp[i]; q < rp[i + 1]; q++) s = rnd(s - rnd(av[q] * x[ci[q]], ur), ur);
            r[i] = rnd(s, u);
        }
    }
}

/* ||x||_inf; a NaN entry makes it infinite (a non-finite iterate or residual
 * must not pass for a small one in the stopping rule) */
static double norm_inf(int n, const double* x)
{
    double m = 0.0;
    for (int i = 0; i < n; i++) {
        if (isnan(x[i])) return INFINITY;
        if (fabs(x[i]) > m) m = fabs(x[i]);
    }
    return m;
}

/* ------------------------------------------------------------------ */
/* Left-preconditioned MGS-GMRES (Algorithm 3, GMRES line; reading R7)  */
/* ------------------------------------------------------------------ */

typedef struct {
    int ug, up;      /* GMRES working precision, product precision */
    double tau;      /* relative tolerance on the preconditioned residual */
    int maxit;       /* iteration cap */
    int orth;        /* 0: modified Gram-Schmidt (the paper's MGS-GMRES);
                        1: classical Gram-Schmidt applied twice (CGS2);
                        2: MGS with one reduction per iteration (ICWY form) */
    int side;        /* 0: left preconditioning (Algorithm 3);
                        1: right preconditioning, the variant the paper leaves
                        as future work at the end of Section 3 */
    int kmode;       /* MODE_PEROP / MODE_ACC32 for u_g, u_p = half */
} orc_gmres_opts;

/*
 * Left (side 0): solve (P A) d = P r from d0 = 0.  Right (side 1): solve
 * (A P) u = r from u0 = 0 and return d = P u; the Givens estimate |g_k|/beta
 * is then the unpreconditioned relative residual ||r - A d|| / ||r|| of exact
 * arithmetic.  P may be NULL (P = I, both sides coincide).  The result d is
 * in u_g precision values.  Returns the number of iterations; *breakdown is
 * set when h_{j+1,j} = 0.  relres receives |g_k| / beta (or 0).
 */
/* The Arnoldi product w = fl_ug(P (A v)) (left) or fl_ug(A (P v)) (right),
 * each product in u_p; P = NULL: w = fl_ug(A v).  t: scratch. */
static void arnoldi_product(int n, const int64_t* arp, const int* aci, const double* av, const int64_t* prp,
                            const int* pci, const double* pv, int right, int up, int ug, int pmode,
                            const double* v, double* t, double* w)
{
    if (right && prp) {
        spmv_p(n, prp, pci, pv, v, up, pmode, t);
        spmv_p(n, arp, aci, av, t, up, pmode, w);
    } else {
        spmv_p(n, arp, aci, av, v, up, pmode, t);
        if (prp) spmv_p(n, prp, pci, pv, t, up, pmode, w);
        else for (int i = 0; i < n; i++) w[i] = t[i];
    }
    for (int i = 0; i < n; i++) w[i] = rnd(w[i], ug);
}

/*
 * One step of MGS in inverse compact WY form with lagged normalisation
 * (orth = 2).  With Q_j = [q_0 .. q_{j-1}] and the not yet normalised
 * u_j, one set of inner products gives everything iteration j needs:
 *   a = Q_j^T u_j,  nu = u_j^T u_j,  c = Q_j^T w,  delta = u_j^T w,
 * where w = op(u_j) is the Arnoldi product of u_j.  Then r = sqrt(nu) is
 * h_{j,j-1} (the subdiagonal of the previous column), q_j = u_j / r, row j
 * of the strictly lower triangular L = (q_i^T q_k)_{i>k} is a / r, and
 * b = Q_{j+1}^T (w / r) = [c / r ; delta / r^2].  The MGS coefficients of
 * column j are h = (I + L)^{-1} b (forward substitution: h_i = b_i -
 * sum_{k<i} l_ik h_k, which is what projecting against q_0, q_1, ... one
 * after another gives), and u_{j+1} = w / r - Q_{j+1} h.  In exact
 * arithmetic L = 0 and h, u_{j+1} are those of MGS.  Every inner product,
 * quotient and update is rounded to u_g; the subtractions of the update and
 * of the substitution run in index order, as in MGS.
 *   V: the basis (V[i] = q_i, allocated here for i <= j); U: u_j on entry,
 *   u_{j+1} on return; W: w; L: row i at L + i * ldl; h: the coefficients.
 *   ug: the storage precision of the vectors; ag: the precision of every
 *   operation (u_g, or binary32 for half storage under MODE_ACC32); each
 *   vector entry is rounded to ug once it is complete.
 * Returns r.  For j = 0 there is no previous column and no L row.
 */
static double icwy_step(int n, int j, double** V, double* U, const double* W, double* L, int ldl, double* a,
                        double* c, double* h, int ug, int ag, int with_product, double* rnorm_only)
{
    double nu = dot_p(U, 1, U, 1, n, ag, MODE_PEROP);
    double r = rnd(sqrt(nu), ag);
    if (rnorm_only || !with_product) {
        if (rnorm_only) *rnorm_only = r;
        return r;
    }
    for (int i = 0; i < j; i++) {
        a[i] = dot_p(V[i], 1, U, 1, n, ag, MODE_PEROP);
        c[i] = dot_p(V[i], 1, W, 1, n, ag, MODE_PEROP);
    }
    double delta = dot_p(U, 1, W, 1, n, ag, MODE_PEROP);
    if (r == 0.0) return r;
    if (!V[j]) V[j] = (double*)malloc(sizeof(double) * (size_t)n);
    for (int q = 0; q < n; q++) V[j][q] = rnd(rnd(U[q] / r, ag), ug);
    double* Lj = L + (size_t)j * ldl;
    for (int i = 0; i < j; i++) Lj[i] = rnd(a[i] / r, ag);
    for (int i = 0; i < j; i++) h[i] = rnd(c[i] / r, ag);
    h[j] = rnd(rnd(delta / r, ag) / r, ag);
    for (int i = 0; i <= j; i++) {
        const double* Li = L + (size_t)i * ldl;
        double acc = h[i];
        for (int k = 0; k < i; k++) acc = rnd(acc - rnd(Li[k] * h[k], ag), ag);
        h[i] = acc;
    }
    for (int q = 0; q < n; q++) {
        double acc = rnd(W[q] / r, ag);
        for (int i = 0; i <= j; i++) acc = rnd(acc - rnd(h[i] * V[i][q], ag), ag);
        U[q] = rnd(acc, ug);
    }
    return r;
}

/* Apply the rotations 0..j-2 to column j-1 (h[0..j-1], h[j] its subdiagonal),
 * form rotation j-1 and update g; H receives the rotated column. */
static void givens_column(int j, double* h, double* cs, double* sn, double* g, double* H, int K)
{
    const int c = j - 1;
    for (int i = 0; i < c; i++) {
        double tmp = cs[i] * h[i] + sn[i] * h[i + 1];
        h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
        h[i] = tmp;
    }
    double den = sqrt(h[c] * h[c] + h[c + 1] * h[c + 1]);
    if (den == 0.0) { cs[c] = 1.0; sn[c] = 0.0; }
    else { cs[c] = h[c] / den; sn[c] = h[c + 1] / den; }
    h[c] = den;
    h[c + 1] = 0.0;
    g[c + 1] = -sn[c] * g[c];
    g[c] = cs[c] * g[c];
    for (int i = 0; i <= c; i++) H[(size_t)i * K + c] = h[i];
}

/* GMRES with the one-reduction MGS (orth = 2); arguments as orc_gmres. */
static int gmres_icwy(int n, const int64_t* arp, const int* aci, const double* av, const int64_t* prp,
                      const int* pci, const double* pv, const double* r, const orc_gmres_opts* o, double* d,
                      int* breakdown, double* relres)
{
    int ug = o->ug, up = o->up, K = o->maxit;
    const int right = o->side == 1;
    /* MODE_ACC32: half is storage only; operations in binary32 */
    const int ag = (o->kmode == MODE_ACC32 && ug == PH) ? PS : ug;
    const int pmode = o->kmode == MODE_ACC32 ? MODE_ACC32 : MODE_PEROP;
    double* t = (double*)malloc(sizeof(double) * (size_t)n);
    double* U = (double*)malloc(sizeof(double) * (size_t)n);
    double* W = (double*)malloc(sizeof(double) * (size_t)n);
    double** V = (double**)calloc((size_t)K + 2, sizeof(double*));
    double* L = (double*)calloc((size_t)(K + 1) * (K + 1), sizeof(double));
    double* H = (double*)calloc((size_t)(K + 1) * (K + 1), sizeof(double));
    double* a = (double*)calloc((size_t)K + 2, sizeof(double));
    double* c = (double*)calloc((size_t)K + 2, sizeof(double));
    double* h = (double*)calloc((size_t)K + 2, sizeof(double));
    double* col = (double*)calloc((size_t)K + 2, sizeof(double));
    double* cs = (double*)calloc((size_t)K + 1, sizeof(double));
    double* sn = (double*)calloc((size_t)K + 1, sizeof(double));
    double* g = (double*)calloc((size_t)K + 2, sizeof(double));
    *breakdown = 0;
    *relres = 0.0;
    for (int i = 0; i < n; i++) d[i] = 0.0;
    /* u_0 = P r (left) or r (right), in u_p then u_g; beta = ||u_0|| comes
     * from the first reduction */
    if (prp && !right) spmv_p(n, prp, pci, pv, r, up, pmode, U);
    else for (int i = 0; i < n; i++) U[i] = rnd(r[i], up);
    for (int i = 0; i < n; i++) U[i] = rnd(U[i], ug);
    double beta = 0.0;
    int k = 0;
    for (int j = 0; K > 0; j++) {
        const int prod = j < K;
        if (prod) arnoldi_product(n, arp, aci, av, prp, pci, pv, right, up, ug, pmode, U, t, W);
        double rn = 0.0;
        /* the last pass (j = K) only needs ||u_K|| */
        double rj = icwy_step(n, j, V, U, W, L, K + 1, a, c, h, ug, ag, prod, prod ? NULL : &rn);
        if (j == 0) {
            beta = rj;
            g[0] = beta;
            if (beta == 0.0) break;
        } else {
            col[j] = rj; /* h_{j,j-1} completes column j-1 */
            givens_column(j, col, cs, sn, g, H, K + 1);
            k = j;
            *relres = fabs(g[j]) / beta;
            if (rj == 0.0) { *breakdown = 1; break; }
            if (*relres <= o->tau) break;
        }
        if (!prod) break;
        for (int i = 0; i <= j; i++) col[i] = h[i]; /* column j above its subdiagonal */
    }
    /* y = R^{-1} g(0:k) in double, d = V_k y in u_g */
    double* y = (double*)calloc((size_t)k + 1, sizeof(double));
    for (int i = k - 1; i >= 0; i--) {
        double acc = g[i];
        for (int l = i + 1; l < k; l++) acc -= H[(size_t)i * (K + 1) + l] * y[l];
        y[i] = H[(size_t)i * (K + 1) + i] != 0.0 ? acc / H[(size_t)i * (K + 1) + i] : 0.0;
    }
    for (int q = 0; q < n; q++) {
        double acc = 0.0;
        for (int i = 0; i < k; i++) acc = rnd(acc + rnd(V[i][q] * rnd(y[i], ag), ag), ag);
        d[q] = acc;
    }
    if (right && prp) {
        spmv_p(n, prp, pci, pv, d, up, pmode, t);
        for (int q = 0; q < n; q++) d[q] = rnd(t[q], ug);
    }
    for (int i = 0; i <= K + 1; i++) free(V[i]);
    free(V); free(y); free(t); free(U); free(W); free(L); free(H); free(a); free(c); free(h); free(col);
    free(cs); free(sn); free(g);
    return k;
}

/* One GMRES solve (Algorithm 3, GMRES line; reading R7) in the Arnoldi form
 * o->orth selects: MGS (0) and CGS2 (1) here, the one-reduction MGS (2) in
 * gmres_icwy.  Returns the iterations taken, or -1 for the half-storage
 * model outside the one-reduction form. */
int orc_gmres(int n, const int64_t* arp, const int* aci, const double* av,
              const int64_t* prp, const int* pci, const double* pv,
              const double* r, const orc_gmres_opts* o, double* d, int* breakdown, double* relres)
{
    if (o->orth == 2) return gmres_icwy(n, arp, aci, av, prp, pci, pv, r, o, d, breakdown, relres);
    if (o->kmode == MODE_ACC32 && (o->ug == PH || o->up == PH)) return -1; /* defined for orth 2 only */
    int ug = o->ug, up = o->up, K = o->maxit;
    double* t = (double*)malloc(sizeof(double) * (size_t)n);
    double* w = (double*)malloc(sizeof(double) * (size_t)n);
    double** V = (double**)calloc((size_t)K + 1, sizeof(double*));
    double* H = (double*)calloc((size_t)(K + 1) * (K + 1), sizeof(double)); /* H[i*(K)+j] row-major (K+1) x K */
    double* cs = (double*)calloc((size_t)K + 1, sizeof(double));
    double* sn = (double*)calloc((size_t)K + 1, sizeof(double));
    double* g = (double*)calloc((size_t)K + 2, sizeof(double));
    *breakdown = 0;
    const int right = o->side == 1;
    /* left: z = P r in u_p; right: z = r; stored in u_g */
    if (prp && !right) spmv_p(n, prp, pci, pv, r, up, MODE_PEROP, w);
    else for (int i = 0; i < n; i++) w[i] = rnd(r[i], up);
    for (int i = 0; i < n; i++) w[i] = rnd(w[i], ug);
    double beta = rnd(sqrt(dot_p(w, 1, w, 1, n, ug, MODE_PEROP)), ug);
    for (int i = 0; i < n; i++) d[i] = 0.0;
    *relres = 0.0;
    if (beta == 0.0 || K == 0) {
        free(t); free(w); free(V); free(H); free(cs); free(sn); free(g);
        return 0;
    }
    V[0] = (double*)malloc(sizeof(double) * (size_t)n);
    for (int i = 0; i < n; i++) V[0][i] = rnd(w[i] / beta, ug);
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < K; j++) {
        /* left: w = P (A v_j); right: w = A (P v_j); both products in u_p */
        if (right && prp) {
            spmv_p(n, prp, pci, pv, V[j], up, MODE_PEROP, t);
            spmv_p(n, arp, aci, av, t, up, MODE_PEROP, w);
        } else {
            spmv_p(n, arp, aci, av, V[j], up, MODE_PEROP, t);
            if (prp) spmv_p(n, prp, pci, pv, t, up, MODE_PEROP, w);
            else for (int i = 0; i < n; i++) w[i] = t[i];
        }
        for (int i = 0; i < n; i++) w[i] = rnd(w[i], ug);
        double* h = (double*)calloc((size_t)j + 2, sizeof(double));
        if (o->orth == 0) {
            /* modified Gram-Schmidt in u_g: project against v_i one at a time */
            for (int i = 0; i <= j; i++) {
                double hij = dot_p(V[i], 1, w, 1, n, ug, MODE_PEROP);
                h[i] = hij;
                for (int q = 0; q < n; q++) w[q] = rnd(w[q] - rnd(hij * V[i][q], ug), ug);
            }
        } else {
            /* classical Gram-Schmidt twice in u_g: all projections of a pass
             * use the same w; the second pass re-orthogonalises */
            double* c = (double*)calloc((size_t)j + 2, sizeof(double));
            for (int pass = 0; pass < 2; pass++) {
                for (int i = 0; i <= j; i++) c[i] = dot_p(V[i], 1, w, 1, n, ug, MODE_PEROP);
                for (int q = 0; q < n; q++) {
                    double acc = w[q];
                    for (int i = 0; i <= j; i++) acc = rnd(acc - rnd(c[i] * V[i][q], ug), ug);
                    w[q] = acc;
                }
                for (int i = 0; i <= j; i++) h[i] = rnd(h[i] + c[i], ug);
            }
            free(c);
        }
        h[j + 1] = rnd(sqrt(dot_p(w, 1, w, 1, n, ug, MODE_PEROP)), ug);
        double hnext = h[j + 1];
        /* Givens rotations in double */
        for (int i = 0; i < j; i++) {
            double tmp = cs[i] * h[i] + sn[i] * h[i + 1];
            h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
            h[i] = tmp;
        }
        double den = sqrt(h[j] * h[j] + h[j + 1] * h[j + 1]);
        if (den == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
        else { cs[j] = h[j] / den; sn[j] = h[j + 1] / den; }
        h[j] = den;
        h[j + 1] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        for (int i = 0; i <= j; i++) H[(size_t)i * K + j] = h[i];
        free(h);
        k = j + 1;
        *relres = fabs(g[j + 1]) / beta;
        if (hnext == 0.0) { *breakdown = 1; break; }
        V[j + 1] = (double*)malloc(sizeof(double) * (size_t)n);
        for (int i = 0; i < n; i++) V[j + 1][i] = rnd(w[i] / hnext, ug);
        if (*relres <= o->tau) break;
    }
    /* y = R^{-1} g(0:k) in double, d = V_k y in u_g */
    double* y = (double*)calloc((size_t)k + 1, sizeof(double));
    for (int i = k - 1; i >= 0; i--) {
        double acc = g[i];
        for (int l = i + 1; l < k; l++) acc -= H[(size_t)i * K + l] * y[l];
        y[i] = H[(size_t)i * K + i] != 0.0 ? acc / H[(size_t)i * K + i] : 0.0;
    }
    for (int q = 0; q < n; q++) {
        double acc = 0.0;
        for (int i = 0; i < k; i++) acc = rnd(acc + rnd(V[i][q] * rnd(y[i], ug), ug), ug);
        d[q] = acc;
    }
    if (right && prp) {
        /* right preconditioning: d = P (V_k y) in u_p, stored in u_g */
        spmv_p(n, prp, pci, pv, d, up, MODE_PEROP, t);
        for (int q = 0; q < n; q++) d[q] = rnd(t[q], ug);
    }
    for (int i = 0; i <= K; i++) free(V[i]);
    free(y); free(t); free(w); free(V); free(H); free(cs); free(sn); free(g);
    return k;
}

/* ------------------------------------------------------------------ */
/* SPAI-GMRES-IR (Algorithm 3)                                         */
/* ------------------------------------------------------------------ */

typedef struct {
    int uf, u, ug, up, ur;  /* the five precisions */
    int mode;               /* arithmetic mode of the u_f product x0 = P b */
    double tau;             /* GMRES tolerance */
    int gmres_maxit;        /* per GMRES solve */
    int imax;               /* maximum number of refinement steps */
    double stop_tol;        /* R8 threshold of the stopping rule */
    int orth;               /* 0 MGS, 1 CGS2, 2 one-reduction MGS */
    int side;               /* 0 left, 1 right preconditioning */
    int stop_rule;          /* STOP_BACKWARD, STOP_FIXED, STOP_CORRECTION */
    int kmode;              /* arithmetic mode of the Krylov part at u_g, u_p = half */
} orc_ir_opts;

/*
 * Inputs: CSR A (values double), CSR P (structure + values pv_up for u_p use,
 * pv_uf for the u_f product; P may be NULL for no preconditioner), b.
 * Outputs: x[n] (values in precision u), its[imax] GMRES iterations per
 * step, nbe[imax+1] backward error before each step, *steps, status flags.
 */
int orc_gmres_ir(int n, const int64_t* arp, const int* aci, const double* av,
                 const int64_t* prp, const int* pci, const double* pv_up, const double* pv_uf,
                 const double* b, const orc_ir_opts* o, double* x, int* its, double* nbe,
                 int* steps)
{
    int status = 0;
    double* r = (double*)malloc(sizeof(double) * (size_t)n);
    double* dd = (double*)malloc(sizeof(double) * (size_t)n);
    double* ur_b = (double*)malloc(sizeof(double) * (size_t)n);
    /* ||A||_inf */
    double anorm = 0.0;
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t q = arp[i]; q < arp[i + 1]; q++) s += fabs(av[q]);
        if (s > anorm) anorm = s;
    }
    double bnorm = norm_inf(n, b);
    /* x0 = P b in u_f, stored in u (P = I: x0 = b rounded) */
    if (prp) spmv_p(n, prp, pci, pv_uf, b, o->uf, o->mode, x);
    else for (int i = 0; i < n; i++) x[i] = rnd(b[i], o->uf);
    for (int i = 0; i < n; i++) x[i] = rnd(x[i], o->u);
    orc_gmres_opts go = { o->ug, o->up, o->tau, o->gmres_maxit, o->orth, o->side, o->kmode };
    int i;
    double dn = 0.0, qprev = 0.0; /* ||d_{i-1}||_inf and q_{i-1} (reading R8) */
    *steps = 0;
    for (i = 0; i <= o->imax; i++) {
        residual_ur(n, arp, aci, av, b, x, o->ur, o->u, r);
        double rn = norm_inf(n, r), xn = norm_inf(n, x);
        double den = anorm * xn + bnorm;
        nbe[i] = den > 0.0 ? rn / den : 0.0;
        if (!isfinite(nbe[i])) { status |= IR_NONFINITE; break; }
        double q = xn > 0.0 ? dn / xn : (dn > 0.0 ? INFINITY : 0.0);
        if (o->stop_rule == STOP_BACKWARD && nbe[i] <= o->stop_tol) { status |= IR_CONVERGED; break; }
        if (o->stop_rule == STOP_CORRECTION && i >= 1 && q <= o->stop_tol) { status |= IR_CONVERGED; break; }
        if (i == o->imax) { status |= IR_MAXSTEPS; break; }
        if (o->stop_rule != STOP_FIXED && i >= 2 && q >= 0.5 * qprev) { status |= IR_STAGNATED; break; }
        qprev = q;
        int bd = 0;
        double rr;
        /* reading R17: with u_g or u_p = half the residual is scaled by a
         * power of two, 2^-e with ||r||_inf = m 2^e, m in [0.5, 1), before
         * GMRES (exact; residuals of a converging refinement would otherwise
         * fall below half's range), and d is scaled back by 2^e */
        int e = 0;
        if ((o->ug == PH || o->up == PH) && rn > 0.0) {
            frexp(rn, &e);
            for (int q2 = 0; q2 < n; q2++) r[q2] = ldexp(r[q2], -e);
        }
        its[i] = orc_gmres(n, arp, aci, av, prp, pci, pv_up, r, &go, dd, &bd, &rr);
        if (its[i] < 0) { its[i] = 0; status |= IR_NONFINITE; break; } /* unsupported mode */
        if (e != 0)
            for (int q2 = 0; q2 < n; q2++) dd[q2] = ldexp(dd[q2], e);
        if (bd) status |= IR_BREAKDOWN;
        dn = 0.0;
        for (int q2 = 0; q2 < n; q2++) {
            double dq = rnd(dd[q2], o->u);
            if (fabs(dq) > dn) dn = fabs(dq);
            x[q2] = rnd(x[q2] + dq, o->u);
        }
        *steps = i + 1;
    }
    (void)ur_b;
    free(r); free(dd); free(ur_b);
    return status;
}

/* Threads of the SPAI column loop (OpenMP); returns the number in use. */
int orc_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* Exported single steps, used by the oracle's own pins. */
double orc_dot(int len, const double* x, const double* y, int p, int mode)
{
    return dot_p(x, 1, y, 1, len, p, mode);
}

void orc_spmv(int n, const int64_t* rp, const int* ci, const double* mv, const double* x, int p,
              int mode, double* y)
{
    spmv_p(n, rp, ci, mv, x, p, mode, y);
}

void orc_residual(int n, const int64_t* rp, const int* ci, const double* av, const double* b,
                  const double* x, int ur, int u, double* r)
{
    residual_ur(n, rp, ci, av, b, x, ur, u, r);
}

/* Arithmetic probes for the chop pin: op 0 add, 1 sub, 2 mul, 3 div, 4 sqrt,
 * each on half operands with the result chopped to half. */
void orc_half_ops(int cnt, const double* a, const double* b, int op, double* out)
{
    for (int i = 0; i < cnt; i++) {
        double x = orc_chop_half(a[i]), y = orc_chop_half(b[i]), z;
        switch (op) {
        case 0: z = x + y; break;
        case 1: z = x - y; break;
        case 2: z = x * y; break;
        case 3: z = x / y; break;
        default: z = sqrt(fabs(x)); break;
        }
        out[i] = orc_chop_half(z);
    }
}

/* Arnoldi only (for the oracle's pins): k steps of the Gram-Schmidt variant
 * on (P A) from v_1 = P r / ||P r||, in u_g / u_p.  Writes V (n x (k+1),
 * column-major) and H ((k+1) x k, column-major, unrotated).  Returns the
 * number of columns produced (less than k+1 on breakdown). */
int orc_arnoldi(int n, const int64_t* arp, const int* aci, const double* av,
                const int64_t* prp, const int* pci, const double* pv,
                const double* r, int ug, int up, int orth, int k, double* Vout, double* Hout)
{
    if (orth == 2) {
        /* one-reduction MGS: k + 1 passes, the last only for ||u_k|| */
        double* t = (double*)malloc(sizeof(double) * (size_t)n);
        double* U = (double*)malloc(sizeof(double) * (size_t)n);
        double* W = (double*)malloc(sizeof(double) * (size_t)n);
        double** V = (double**)calloc((size_t)k + 2, sizeof(double*));
        double* L = (double*)calloc((size_t)(k + 1) * (k + 1), sizeof(double));
        double* a = (double*)calloc((size_t)k + 2, sizeof(double));
        double* c = (double*)calloc((size_t)k + 2, sizeof(double));
        double* h = (double*)calloc((size_t)k + 2, sizeof(double));
        if (prp) spmv_p(n, prp, pci, pv, r, up, MODE_PEROP, U);
        else for (int i = 0; i < n; i++) U[i] = rnd(r[i], up);
        for (int i = 0; i < n; i++) U[i] = rnd(U[i], ug);
        for (int z = 0; z < (k + 1) * k; z++) Hout[z] = 0.0;
        int cols = 0;
        for (int j = 0; j <= k; j++) {
            const int prod = j < k;
            if (prod) arnoldi_product(n, arp, aci, av, prp, pci, pv, 0, up, ug, MODE_PEROP, U, t, W);
            double rn = 0.0;
            double rj = icwy_step(n, j, V, U, W, L, k + 1, a, c, h, ug, ug, prod, prod ? NULL : &rn);
            if (j > 0) Hout[(size_t)(j - 1) * (k + 1) + j] = rj;
            if (rj == 0.0) break;
            if (!prod) {
                V[j] = (double*)malloc(sizeof(double) * (size_t)n);
                for (int q = 0; q < n; q++) V[j][q] = rnd(U[q] / rj, ug);
            }
            for (int q = 0; q < n; q++) Vout[(size_t)j * n + q] = V[j][q];
            cols = j + 1;
            if (!prod) break;
            for (int i = 0; i <= j; i++) Hout[(size_t)j * (k + 1) + i] = h[i];
        }
        for (int i = 0; i <= k + 1; i++) free(V[i]);
        free(V); free(t); free(U); free(W); free(L); free(a); free(c); free(h);
        return cols;
    }
    double* t = (double*)malloc(sizeof(double) * (size_t)n);
    double* w = (double*)malloc(sizeof(double) * (size_t)n);
    double* c = (double*)malloc(sizeof(double) * (size_t)(k + 2));
    if (prp) spmv_p(n, prp, pci, pv, r, up, MODE_PEROP, w);
    else for (int i = 0; i < n; i++) w[i] = rnd(r[i], up);
    for (int i = 0; i < n; i++) w[i] = rnd(w[i], ug);
    double beta = rnd(sqrt(dot_p(w, 1, w, 1, n, ug, MODE_PEROP)), ug);
    int cols = 1;
    for (int i = 0; i < n; i++) Vout[i] = rnd(w[i] / beta, ug);
    for (int z = 0; z < (k + 1) * k; z++) Hout[z] = 0.0;
    for (int j = 0; j < k; j++) {
        const double* vj = Vout + (size_t)j * n;
        spmv_p(n, arp, aci, av, vj, up, MODE_PEROP, t);
        if (prp) spmv_p(n, prp, pci, pv, t, up, MODE_PEROP, w);
        else for (int i = 0; i < n; i++) w[i] = t[i];
        for (int i = 0; i < n; i++) w[i] = rnd(w[i], ug);
        double* h = Hout + (size_t)j * (k + 1);
        if (orth == 0) {
            for (int i = 0; i <= j; i++) {
                double hij = dot_p(Vout + (size_t)i * n, 1, w, 1, n, ug, MODE_PEROP);
                h[i] = hij;
                for (int q = 0; q < n; q++) w[q] = rnd(w[q] - rnd(hij * Vout[(size_t)i * n + q], ug), ug);
            }
        } else {
            for (int pass = 0; pass < 2; pass++) {
                for (int i = 0; i <= j; i++) c[i] = dot_p(Vout + (size_t)i * n, 1, w, 1, n, ug, MODE_PEROP);
                for (int q = 0; q < n; q++) {
                    double acc = w[q];
                    for (int i = 0; i <= j; i++) acc = rnd(acc - rnd(c[i] * Vout[(size_t)i * n + q], ug), ug);
                    w[q] = acc;
                }
                for (int i = 0; i <= j; i++) h[i] = rnd(h[i] + c[i], ug);
            }
        }
        double hn = rnd(sqrt(dot_p(w, 1, w, 1, n, ug, MODE_PEROP)), ug);
        h[j + 1] = hn;
        if (hn == 0.0) break;
        for (int i = 0; i < n; i++) Vout[(size_t)(j + 1) * n + i] = rnd(w[i] / hn, ug);
        cols = j + 2;
    }
    free(t); free(w); free(c);
    return cols;
}

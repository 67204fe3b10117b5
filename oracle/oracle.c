/* CPU oracle for Lottery BP (+ OSD-0).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark call this file.  It shares no code, header
 * or table with the CUDA decoder, and the decoder never calls it.
 *
 * A plain, slow restatement of the paper's algorithms, one shot at a time,
 * in the order the paper states them:
 *   Alg. 1  normalised min-sum BP (prior LLR, V2C, C2V, LLR update, hard
 *           decision, syndrome estimate, early termination);
 *   Alg. 3  the lottery sign flip (Sec. III-B);
 *   Alg. 2  OSD-0 (sort, permute, basis selection, LU, forward and
 *           backward substitution, zero padding, inverse permutation).
 * The check-node update computes each exclusive sign product and minimum
 * literally (a loop over V(c) \ {v} per edge), not via min1/min2.
 *
 * Arithmetic modes (prec):
 *   0  F64: every value a double, nothing rounded.
 *   1  F32: each arithmetic result rounded to binary32.  A double holds the
 *      exact sum / difference / product of two binary32 values rounded once
 *      to 53 bits, and 53 >= 2*24+2, so rounding that double to binary32
 *      gives the binary32-rounded result (double rounding is innocuous for
 *      +, -, *); this is IEEE binary32 arithmetic without FMA contraction.
 *   2  F16 messages: F32 arithmetic, each stored C2V message rounded to
 *      binary16 (round to nearest even).
 *   3  I8 messages: F32 arithmetic, each stored C2V message quantised to the
 *      8-bit fixed point Int3.4 (Sec. VI-C): q = clamp(rne(16 x), -127, 127),
 *      value q / 16.
 *   Channel LLRs mu and posteriors lambda stay binary32 in modes 1-3.
 *
 * Readings taken where the paper is silent:
 *   sign(x) = -1 iff x < 0 (so both zeros count as +1);
 *   e_v = 1 iff lambda_v <= 0 (Alg. 1 hard decision);
 *   the lottery at iteration i uses U from s_hat of iteration i-1, with
 *   s_hat(-1) = 0; it runs for lottery_skip <= i < I-1 (policy 5, an
 *   ablation outside the paper, takes U from s_hat of iteration i and
 *   otherwise follows policy 0);
 *   RandomSelect: u = low 32 bits of SplitMix64 at counter (g << 24) + i for
 *   global shot index g, k = floor(u * N / 2^32), c* = k-th unsatisfied
 *   check in ascending row order (a random column, for the baseline policies,
 *   uses the high 32 bits of the same output);
 *   ties: most unsatisfied checks, then least |lambda|, then lowest column;
 *   OSD sorts signed lambda ascending, ties by column index; if s is not in
 *   the column space, the BP estimate is kept and a flag is raised;
 *   a row of H with exactly one nonzero is rejected (its exclusive minimum
 *   would be over an empty set).
 *
 * Compile with -ffp-contract=off (no fused multiply-add).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { PREC_F64 = 0, PREC_F32 = 1, PREC_F16 = 2, PREC_I8 = 3 };
enum { RULE_MIN_SUM = 0, RULE_SUM_PRODUCT = 1 };

typedef struct {
    int32_t max_iter;
    int32_t scale_mode;   /* 0: constant scale_const; 1: 1 - 2^-(i+1) (Alg. 1 CN update) */
    double scale_const;
    int32_t lottery;      /* Alg. 3 on/off */
    int32_t lottery_skip; /* first iteration index at which the lottery may run */
    int32_t osd;          /* Alg. 2 on shots BP did not converge on */
    int32_t prec;
    int32_t early_exit;   /* 1: Alg. 1 early termination; 0: exactly max_iter iterations */
    int32_t rule;         /* 0: normalised min-sum (Alg. 1); 1: sum-product tanh rule */
    int32_t policy;       /* lottery policy, Sec. III-B: 0 proposed (Alg. 3), 1 worst CN +
                             unreliable VN, 2 worst CN + random VN, 3 random CN + unreliable VN,
                             4 random CN + random VN; 5 (an ablation, not in the paper) as 0
                             with U from this iteration's s_hat(i) */
    uint64_t seed;
    uint64_t shot_offset;
} oracle_params;

/* ---------------------------------------------------------------- RNG --- */

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): output k >= 1 of the stream
 * with state x is mix(x + k * 0x9E3779B97F4A7C15). */
uint64_t oracle_splitmix64_at(uint64_t seed, uint64_t counter) {
    uint64_t z = seed + (counter + 1ULL) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* ---------------------------------------------------------- rounding --- */

static double arith(int prec, double x) {
    return prec == PREC_F64 ? x : (double)(float)x;
}

/* Round to binary16, round-to-nearest-even, from the format's definition:
 * 11 significant bits, smallest normal 2^-14, subnormal spacing 2^-24,
 * largest finite 65504. */
double oracle_round_f16(double x) {
    if (x == 0.0 || isnan(x) || isinf(x)) return x;
    double a = fabs(x);
    int e;
    frexp(a, &e);              /* a in [2^(e-1), 2^e) */
    int q = e - 11;            /* spacing of binary16 in that binade */
    if (q < -24) q = -24;
    double r = ldexp(nearbyint(ldexp(a, -q)), q);
    if (r > 65504.0) r = INFINITY;
    return copysign(r, x);
}

/* Int3.4: 8-bit two's complement with 4 fraction bits, saturating,
 * symmetric range [-127, 127] / 16. */
double oracle_round_i8(double x) {
    double q = nearbyint(16.0 * x);
    if (q > 127.0) q = 127.0;
    if (q < -127.0) q = -127.0;
    return q / 16.0;
}

static double store_msg(int prec, double x) {
    switch (prec) {
        case PREC_F64: return x;
        case PREC_F32: return (double)(float)x;
        case PREC_F16: return oracle_round_f16((double)(float)x);
        default:       return oracle_round_i8((double)(float)x);
    }
}

/* ------------------------------------------------------------- graph --- */

typedef struct {
    int m, n, nnz;
    const int32_t *row_ptr, *col_idx;  /* CSR of H, as given */
    int32_t *col_ptr, *csc_row, *csc_edge; /* per column: rows ascending, CSR edge id */
} graph_t;

static int graph_init(graph_t *g, int m, int n, const int32_t *row_ptr, const int32_t *col_idx) {
    if (m < 0 || n < 0 || !row_ptr || (m > 0 && !col_idx)) return -1;
    g->m = m; g->n = n; g->row_ptr = row_ptr; g->col_idx = col_idx;
    g->nnz = row_ptr[m];
    for (int c = 0; c < m; ++c) {
        if (row_ptr[c + 1] < row_ptr[c]) return -1;
        if (row_ptr[c + 1] - row_ptr[c] == 1) return -2;
        for (int e = row_ptr[c]; e < row_ptr[c + 1]; ++e) {
            if (col_idx[e] < 0 || col_idx[e] >= n) return -1;
            if (e > row_ptr[c] && col_idx[e] <= col_idx[e - 1]) return -1;
        }
    }
    g->col_ptr = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    g->csc_row = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->nnz + 1));
    g->csc_edge = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->nnz + 1));
    for (int e = 0; e < g->nnz; ++e) g->col_ptr[col_idx[e] + 1]++;
    for (int v = 0; v < n; ++v) g->col_ptr[v + 1] += g->col_ptr[v];
    int32_t *fill = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    for (int c = 0; c < m; ++c)          /* rows visited ascending */
        for (int e = row_ptr[c]; e < row_ptr[c + 1]; ++e) {
            int v = col_idx[e];
            int k = g->col_ptr[v] + fill[v]++;
            g->csc_row[k] = c;
            g->csc_edge[k] = e;
        }
    free(fill);
    return 0;
}

static void graph_free(graph_t *g) {
    free(g->col_ptr); free(g->csc_row); free(g->csc_edge);
}

/* ------------------------------------------------- Alg. 3: lottery --- */

/* Lottery selection.  U: unsatisfied set (bytes per check); lam: current
 * posteriors; r: one 64-bit draw, whose low 32 bits pick the random check and
 * whose high 32 bits pick the random column (policies 2 and 4).
 * Policy 0 (Alg. 3): c* = the k-th member of U, k = floor(u |U| / 2^32); v* in
 * V(c*) with the most members of C(v) in U, then least |lambda_v|, then lowest
 * column.  Baselines of Sec. III-B: "worst CN" = the member of U with the most
 * columns estimated in error (lambda <= 0 now), lowest row on ties; "random
 * CN" = as in policy 0; "unreliable VN" = least |lambda| in V(c*), lowest
 * column on ties; "random VN" = column number floor(u2 deg(c*) / 2^32) of c*.
 * Returns v*, or -1 when U is empty. */
static int lottery_select(const graph_t *g, const uint8_t *U, const double *lam,
                          uint64_t r, int policy, int *cstar_out) {
    int N = 0;
    for (int c = 0; c < g->m; ++c) N += U[c] ? 1 : 0;
    if (N == 0) return -1;
    const uint32_t u = (uint32_t)r, u2 = (uint32_t)(r >> 32);
    const int worst_cn = policy == 1 || policy == 2;
    const int random_vn = policy == 2 || policy == 4;
    int cstar = -1;
    if (worst_cn) {
        int best_err = -1;
        for (int c = 0; c < g->m; ++c) {
            if (!U[c]) continue;
            int ne = 0;                                  /* columns of c estimated in error */
            for (int e = g->row_ptr[c]; e < g->row_ptr[c + 1]; ++e) ne += lam[g->col_idx[e]] <= 0.0 ? 1 : 0;
            if (ne > best_err) { best_err = ne; cstar = c; }
        }
    } else {
        int k = (int)(((uint64_t)u * (uint64_t)N) >> 32);  /* floor(r N), r = u / 2^32 */
        for (int c = 0, seen = 0; c < g->m; ++c)
            if (U[c]) { if (seen == k) { cstar = c; break; } seen++; }
    }
    if (cstar_out) *cstar_out = cstar;
    const int e0 = g->row_ptr[cstar], deg = g->row_ptr[cstar + 1] - e0;
    if (random_vn) return g->col_idx[e0 + (int)(((uint64_t)u2 * (uint64_t)deg) >> 32)];
    int best = -1, best_cnt = -1;
    double best_abs = 0.0;
    for (int e = e0; e < e0 + deg; ++e) {
        int v = g->col_idx[e];
        int cnt = 0;                                     /* |C(v) ∩ U|, policy 0 only */
        if (policy == 0)
            for (int k2 = g->col_ptr[v]; k2 < g->col_ptr[v + 1]; ++k2) cnt += U[g->csc_row[k2]] ? 1 : 0;
        double a = fabs(lam[v]);
        if (cnt > best_cnt || (cnt == best_cnt && (a < best_abs || (a == best_abs && v < best)))) {
            best = v; best_cnt = cnt; best_abs = a;
        }
    }
    return best;
}

int oracle_lottery_select(int m, int n, const int32_t *row_ptr, const int32_t *col_idx,
                          const uint8_t *U, const double *lam, uint64_t r, int policy,
                          int32_t *cstar, int32_t *vstar) {
    if (policy < 0 || policy > 4) return -1;
    graph_t g;
    int rc = graph_init(&g, m, n, row_ptr, col_idx);
    if (rc) return rc;
    int cs = -1;
    int v = lottery_select(&g, U, lam, r, policy, &cs);
    if (cstar) *cstar = cs;
    if (vstar) *vstar = v;
    graph_free(&g);
    return 0;
}

/* ------------------------------------------------------ Alg. 2: OSD-0 --- */

typedef struct { double key; int idx; } keyed_t;

static int cmp_keyed(const void *pa, const void *pb) {
    const keyed_t *a = (const keyed_t *)pa, *b = (const keyed_t *)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/* Returns 0 on success, 1 if s is not in the column space of H (e_out is
 * then untouched), negative on bad input.  rank_out / basis_out (nullable)
 * report rank(H) and the basis columns S (original column indices, in
 * permuted order). */
static int osd0(const graph_t *g, const double *lam, const uint8_t *s, uint8_t *e_out,
                int *rank_out, int32_t *basis_out) {
    const int m = g->m, n = g->n;
    /* LLR sorting: pi orders lambda ascending (ties: lower column first). */
    keyed_t *kv = (keyed_t *)malloc(sizeof(keyed_t) * (size_t)(n > 0 ? n : 1));
    for (int v = 0; v < n; ++v) { kv[v].key = lam[v]; kv[v].idx = v; }
    qsort(kv, (size_t)n, sizeof(keyed_t), cmp_keyed);
    int *pi = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int j = 0; j < n; ++j) pi[j] = kv[j].idx;
    free(kv);

    /* Column permutation: H_OSD = H P_pi, dense bytes, column j of H_OSD is column pi[j] of H. */
    int *inv = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int j = 0; j < n; ++j) inv[pi[j]] = j;
    uint8_t *Hp = (uint8_t *)calloc((size_t)m * (size_t)n + 1, 1);
    for (int c = 0; c < m; ++c)
        for (int e = g->row_ptr[c]; e < g->row_ptr[c + 1]; ++e)
            Hp[(size_t)c * n + inv[g->col_idx[e]]] = 1;

    /* Basis selection: S = first rank(H) independent columns of H_OSD (column-by-column
     * forward elimination on a copy; a column that yields a new pivot is
     * independent of the ones before it). */
    uint8_t *W = (uint8_t *)malloc((size_t)m * (size_t)n + 1);
    memcpy(W, Hp, (size_t)m * (size_t)n);
    int *S = (int *)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
    int r = 0;
    uint8_t *tmp = (uint8_t *)malloc((size_t)n + 1);
    for (int j = 0; j < n && r < m; ++j) {
        int p = -1;
        for (int i = r; i < m; ++i) if (W[(size_t)i * n + j]) { p = i; break; }
        if (p < 0) continue;
        if (p != r) {
            memcpy(tmp, W + (size_t)p * n, (size_t)n);
            memcpy(W + (size_t)p * n, W + (size_t)r * n, (size_t)n);
            memcpy(W + (size_t)r * n, tmp, (size_t)n);
        }
        for (int i = r + 1; i < m; ++i)
            if (W[(size_t)i * n + j])
                for (int k = j; k < n; ++k) W[(size_t)i * n + k] ^= W[(size_t)r * n + k];
        S[r++] = j;
    }
    free(W); free(tmp);

    /* H'_OSD: the m x r submatrix of the basis columns. */
    uint8_t *A = (uint8_t *)calloc((size_t)m * (size_t)(r ? r : 1), 1);
    for (int i = 0; i < m; ++i)
        for (int k = 0; k < r; ++k) A[(size_t)i * r + k] = Hp[(size_t)i * n + S[k]];
    free(Hp);

    /* LU decomposition with row pivoting, P H' = L U over GF(2);
     * L is m x m unit lower triangular, U (in A) upper trapezoidal. */
    uint8_t *L = (uint8_t *)calloc((size_t)m * (size_t)m + 1, 1);
    int *P = (int *)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
    for (int i = 0; i < m; ++i) { P[i] = i; L[(size_t)i * m + i] = 1; }
    for (int k = 0; k < r; ++k) {
        int p = -1;
        for (int i = k; i < m; ++i) if (A[(size_t)i * r + k]) { p = i; break; }
        if (p < 0) { /* impossible: the basis columns are independent */
            free(A); free(L); free(P); free(S); free(pi); free(inv);
            return -3;
        }
        if (p != k) {
            for (int t = 0; t < r; ++t) {
                uint8_t x = A[(size_t)k * r + t]; A[(size_t)k * r + t] = A[(size_t)p * r + t]; A[(size_t)p * r + t] = x;
            }
            for (int t = 0; t < k; ++t) {
                uint8_t x = L[(size_t)k * m + t]; L[(size_t)k * m + t] = L[(size_t)p * m + t]; L[(size_t)p * m + t] = x;
            }
            int x = P[k]; P[k] = P[p]; P[p] = x;
        }
        for (int i = k + 1; i < m; ++i)
            if (A[(size_t)i * r + k]) {
                L[(size_t)i * m + k] = 1;
                for (int t = k; t < r; ++t) A[(size_t)i * r + t] ^= A[(size_t)k * r + t];
            }
    }

    /* Forward substitution, L y = P s. */
    uint8_t *y = (uint8_t *)calloc((size_t)m + 1, 1);
    for (int i = 0; i < m; ++i) {
        uint8_t acc = s[P[i]] & 1;
        for (int j = 0; j < i; ++j) acc ^= (uint8_t)(L[(size_t)i * m + j] & y[j]);
        y[i] = acc;
    }
    int consistent = 1;
    for (int i = r; i < m; ++i) if (y[i]) consistent = 0;

    /* Backward substitution, U e_S = y (first r rows). */
    uint8_t *x = (uint8_t *)calloc((size_t)(r ? r : 1), 1);
    for (int k = r - 1; k >= 0; --k) {
        uint8_t acc = y[k];
        for (int j = k + 1; j < r; ++j) acc ^= (uint8_t)(A[(size_t)k * r + j] & x[j]);
        x[k] = acc;
    }

    /* Error vector construction and inverse mapping: e' = (e_S, 0) in permuted order, mapped back through pi. */
    if (rank_out) *rank_out = r;
    if (basis_out) for (int k = 0; k < r; ++k) basis_out[k] = pi[S[k]];
    if (consistent) {
        memset(e_out, 0, (size_t)n);
        for (int k = 0; k < r; ++k) e_out[pi[S[k]]] = x[k];
    }
    free(A); free(L); free(P); free(S); free(pi); free(inv); free(y); free(x);
    return consistent ? 0 : 1;
}

int oracle_osd0(int m, int n, const int32_t *row_ptr, const int32_t *col_idx,
                const double *lam, const uint8_t *s, uint8_t *e_out,
                int32_t *rank_out, int32_t *basis_out) {
    graph_t g;
    int rc = graph_init(&g, m, n, row_ptr, col_idx);
    if (rc) return rc;
    int r = 0;
    rc = osd0(&g, lam, s, e_out, &r, basis_out);
    if (rank_out) *rank_out = r;
    graph_free(&g);
    return rc;
}

/* ------------------------------------------------- Alg. 1 (+ Alg. 3) --- */

typedef struct {
    const graph_t *g;
    const oracle_params *prm;
    const double *mu;
    double *beta;          /* stored C2V messages, one per edge (CSR order) */
    double *lam;
    double *alpha;         /* scratch for one check's incoming V2C messages */
    uint8_t *ehat, *shat, *shat_prev, *U;
} shot_ws;

static double scale_at(const oracle_params *prm, int i) {
    double f = prm->scale_mode == 1 ? 1.0 - ldexp(1.0, -(i + 1)) : prm->scale_const;
    return arith(prm->prec, f);
}

/* One check-node update (Alg. 1, CN update) for check c at iteration i. */
static void cn_update(shot_ws *w, int c, int i, uint8_t s_c) {
    const graph_t *g = w->g;
    const int prec = w->prm->prec;
    const int e0 = g->row_ptr[c], deg = g->row_ptr[c + 1] - e0;
    /* V2C messages: Initialization (i = 0) or VN update (i > 0). */
    for (int k = 0; k < deg; ++k) {
        int v = g->col_idx[e0 + k];
        w->alpha[k] = (i == 0) ? w->mu[v] : arith(prec, w->lam[v] - w->beta[e0 + k]);
    }
    const double f = scale_at(w->prm, i);
    for (int k = 0; k < deg; ++k) {
        double out;
        if (w->prm->rule == RULE_MIN_SUM) {
            int neg = s_c ? 1 : 0;                       /* (-1)^{s_c} */
            double mn = INFINITY;
            for (int k2 = 0; k2 < deg; ++k2) {
                if (k2 == k) continue;                   /* v' in V(c) \ {v} */
                if (w->alpha[k2] < 0.0) neg ^= 1;
                double a = fabs(w->alpha[k2]);
                if (a < mn) mn = a;
            }
            double mag = arith(prec, f * mn);
            out = neg ? -mag : mag;
        } else {
            /* tanh rule: beta = (-1)^{s_c} 2 atanh(prod tanh(alpha/2)) (F64 only),
             * magnitude saturated at 25 (atanh(+-1) would be infinite). */
            double prod = s_c ? -1.0 : 1.0;
            for (int k2 = 0; k2 < deg; ++k2) if (k2 != k) prod *= tanh(w->alpha[k2] / 2.0);
            double mag = 2.0 * atanh(fabs(prod));
            if (!(mag <= 25.0)) mag = 25.0;
            out = prod < 0.0 ? -mag : mag;
        }
        w->beta[e0 + k] = store_msg(prec, out);
    }
}

static void decode_one(shot_ws *w, uint64_t gshot, const uint8_t *s, uint8_t *e_out,
                       uint8_t *conv_out, uint8_t *osd_used, uint8_t *osd_nosol,
                       int32_t *iters_out, double *llr_out) {
    const graph_t *g = w->g;
    const oracle_params *prm = w->prm;
    const int m = g->m, n = g->n, I = prm->max_iter;
    const int prec = prm->prec;
    int converged = 0, iters = I;
    memset(w->shat_prev, 0, (size_t)m);                  /* s_hat(-1) = 0 */
    for (int i = 0; i < I; ++i) {
        /* CN update for every check (reads lambda(i-1), beta(i-1)). */
        for (int c = 0; c < m; ++c) cn_update(w, c, i, s[c]);
        /* LLR update: lambda_v = mu_v + sum over C(v), rows ascending. */
        for (int v = 0; v < n; ++v) {
            double acc = w->mu[v];
            for (int k = g->col_ptr[v]; k < g->col_ptr[v + 1]; ++k)
                acc = arith(prec, acc + w->beta[g->csc_edge[k]]);
            w->lam[v] = acc;
        }
        /* Hard decision. */
        for (int v = 0; v < n; ++v) w->ehat[v] = w->lam[v] <= 0.0 ? 1 : 0;
        /* Syndrome estimation, s_hat = e_hat H^T mod 2. */
        for (int c = 0; c < m; ++c) {
            uint8_t acc = 0;
            for (int e = g->row_ptr[c]; e < g->row_ptr[c + 1]; ++e) acc ^= w->ehat[g->col_idx[e]];
            w->shat[c] = acc;
        }
        if (prm->early_exit) {
            int match = 1;
            for (int c = 0; c < m; ++c) if (w->shat[c] != (s[c] & 1)) { match = 0; break; }
            if (match) { converged = 1; iters = i + 1; break; }
            /* Alg. 3, from s_hat(i-1) (policy 5: from s_hat(i), otherwise policy 0). */
            if (prm->lottery && i >= prm->lottery_skip && i < I - 1) {
                const uint8_t *sh = prm->policy == 5 ? w->shat : w->shat_prev;
                for (int c = 0; c < m; ++c) w->U[c] = (uint8_t)(sh[c] ^ (s[c] & 1));
                uint64_t ctr = (gshot << 24) + (uint64_t)i;
                uint64_t r = oracle_splitmix64_at(prm->seed, ctr);
                int vstar = lottery_select(g, w->U, w->lam, r, prm->policy == 5 ? 0 : prm->policy, NULL);
                if (vstar >= 0) w->lam[vstar] = -w->lam[vstar];
            }
        }
        memcpy(w->shat_prev, w->shat, (size_t)m);
    }
    if (!prm->early_exit) {
        converged = 1;
        for (int c = 0; c < m; ++c) if (w->shat[c] != (s[c] & 1)) { converged = 0; break; }
    }
    for (int v = 0; v < n; ++v) e_out[v] = w->lam[v] <= 0.0 ? 1 : 0;
    if (llr_out) memcpy(llr_out, w->lam, sizeof(double) * (size_t)n);
    uint8_t used = 0, nosol = 0;
    if (!converged && prm->osd) {
        int rc = osd0(g, w->lam, s, e_out, NULL, NULL);
        if (rc == 0) used = 1; else nosol = 1;
    }
    if (conv_out) *conv_out = (uint8_t)converged;
    if (osd_used) *osd_used = used;
    if (osd_nosol) *osd_nosol = nosol;
    if (iters_out) *iters_out = iters;
}

typedef struct {
    const graph_t *g;
    const oracle_params *prm;
    const double *mu;
    const uint8_t *syn;
    uint8_t *err, *conv, *osd_used, *osd_nosol;
    int32_t *iters;
    double *llr;
    int64_t lo, hi;
} job_t;

static void *run_job(void *arg) {
    job_t *j = (job_t *)arg;
    const graph_t *g = j->g;
    int maxdeg = 1;
    for (int c = 0; c < g->m; ++c)
        if (g->row_ptr[c + 1] - g->row_ptr[c] > maxdeg) maxdeg = g->row_ptr[c + 1] - g->row_ptr[c];
    shot_ws w;
    w.g = g; w.prm = j->prm; w.mu = j->mu;
    w.beta = (double *)calloc((size_t)g->nnz + 1, sizeof(double));
    w.lam = (double *)calloc((size_t)g->n + 1, sizeof(double));
    w.alpha = (double *)calloc((size_t)maxdeg, sizeof(double));
    w.ehat = (uint8_t *)calloc((size_t)g->n + 1, 1);
    w.shat = (uint8_t *)calloc((size_t)g->m + 1, 1);
    w.shat_prev = (uint8_t *)calloc((size_t)g->m + 1, 1);
    w.U = (uint8_t *)calloc((size_t)g->m + 1, 1);
    for (int64_t b = j->lo; b < j->hi; ++b) {
        const uint64_t gshot = j->prm->shot_offset + (uint64_t)b;
        decode_one(&w, gshot, j->syn + (size_t)b * g->m, j->err + (size_t)b * g->n,
                   j->conv ? j->conv + b : NULL, j->osd_used ? j->osd_used + b : NULL,
                   j->osd_nosol ? j->osd_nosol + b : NULL, j->iters ? j->iters + b : NULL,
                   j->llr ? j->llr + (size_t)b * g->n : NULL);
    }
    free(w.beta); free(w.lam); free(w.alpha); free(w.ehat); free(w.shat);
    free(w.shat_prev); free(w.U);
    return NULL;
}

/* Decode num_shots syndromes (bytes, [B][m]) into error estimates (bytes,
 * [B][n]).  Per shot: converged flag, OSD-used flag, OSD no-solution flag,
 * iterations executed, final lambda (nullable outputs).  Shots are split
 * statically across nthreads threads; nothing is shared inside a shot.
 * Returns 0, or a negative code for a malformed H or parameters. */
int oracle_decode(int m, int n, const int32_t *row_ptr, const int32_t *col_idx,
                  const double *priors, const oracle_params *prm, int64_t num_shots,
                  const uint8_t *syndromes, uint8_t *err_out, uint8_t *converged,
                  uint8_t *osd_used, uint8_t *osd_nosol, int32_t *iters, double *llr_out,
                  int nthreads) {
    if (m < 0 || n < 0 || num_shots < 0 || !prm || prm->max_iter < 1) return -1;
    if (prm->prec < PREC_F64 || prm->prec > PREC_I8) return -1;
    if (prm->rule == RULE_SUM_PRODUCT && prm->prec != PREC_F64) return -1;
    if (prm->lottery_skip < 0 || prm->max_iter >= (1 << 24)) return -1;
    if (prm->policy < 0 || prm->policy > 5) return -1;
    graph_t g;
    int rc = graph_init(&g, m, n, row_ptr, col_idx);
    if (rc) return rc;
    /* Alg. 1 prior LLR: mu_v = ln((1 - p_v) / p_v). */
    double *mu = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int v = 0; v < n; ++v) {
        double p = priors[v];
        if (!(p > 0.0 && p < 1.0)) { free(mu); graph_free(&g); return -1; }
        mu[v] = arith(prm->prec, log((1.0 - p) / p));
    }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > num_shots) nthreads = num_shots > 0 ? (int)num_shots : 1;
    pthread_t th[256];
    job_t jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        job_t *j = &jobs[t];
        j->g = &g; j->prm = prm; j->mu = mu; j->syn = syndromes; j->err = err_out;
        j->conv = converged; j->osd_used = osd_used; j->osd_nosol = osd_nosol;
        j->iters = iters; j->llr = llr_out;
        j->lo = num_shots * t / nthreads;
        j->hi = num_shots * (t + 1) / nthreads;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, run_job, &jobs[t]);
    run_job(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(mu);
    graph_free(&g);
    return 0;
}
